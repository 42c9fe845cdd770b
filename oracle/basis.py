"""1-D quadrature and basis functions, and their tensor products (Sec. 3.1).

The expansion of Eq. (coeff) uses a tensor-product basis of degree P per
direction; which basis the paper's runs used is not stated ("various nodal or
modal" bases), so the modified basis of Karniadakis & Sherwin is the default
and a nodal Lagrange basis on Gauss-Lobatto points is kept for the
basis-invariance check.  Quadrature is Gauss-Legendre with Q points per
direction.
"""
import numpy as np


def gauss_legendre(Q):
    """Q-point Gauss-Legendre nodes and weights on [-1, 1] (exact to degree 2Q-1)."""
    x, w = np.polynomial.legendre.leggauss(Q)
    return np.asarray(x, dtype=np.float64), np.asarray(w, dtype=np.float64)


def jacobi(n, a, b, x):
    """Jacobi polynomial P_n^(a,b)(x) and its derivative, by the three-term
    recurrence."""
    x = np.asarray(x, dtype=np.float64)

    def val(n, a, b):
        p0 = np.ones_like(x)
        if n == 0:
            return p0
        p1 = 0.5 * ((a - b) + (a + b + 2.0) * x)
        for k in range(1, n):
            c = 2.0 * k + a + b
            a1 = 2.0 * (k + 1) * (k + a + b + 1) * c
            a2 = (c + 1) * (a * a - b * b)
            a3 = c * (c + 1) * (c + 2)
            a4 = 2.0 * (k + a) * (k + b) * (c + 2)
            p0, p1 = p1, ((a2 + a3 * x) * p1 - a4 * p0) / a1
        return p1

    p = val(n, a, b)
    dp = np.zeros_like(x) if n == 0 else 0.5 * (n + a + b + 1) * val(n - 1, a + 1, b + 1)
    return p, dp


def modified_basis(P, x):
    """Modified (boundary-adapted) basis: psi_0 = (1-x)/2, psi_P = (1+x)/2,
    psi_p = (1-x)/2 (1+x)/2 P_{p-1}^(1,1)(x) for 0 < p < P.
    Returns (phi, dphi), each [len(x)][P+1]."""
    x = np.asarray(x, dtype=np.float64)
    phi = np.zeros((x.size, P + 1))
    dphi = np.zeros((x.size, P + 1))
    phi[:, 0] = 0.5 * (1 - x)
    dphi[:, 0] = -0.5
    phi[:, P] = 0.5 * (1 + x)
    dphi[:, P] = 0.5
    for p in range(1, P):
        j, dj = jacobi(p - 1, 1.0, 1.0, x)
        b = 0.25 * (1 - x) * (1 + x)
        phi[:, p] = b * j
        dphi[:, p] = -0.5 * x * j + b * dj
    return phi, dphi


def gll_points(P):
    """P+1 Gauss-Lobatto-Legendre points: -1, the roots of P_P', +1."""
    if P == 1:
        return np.array([-1.0, 1.0])
    c = np.zeros(P + 1)
    c[P] = 1.0
    r = np.polynomial.legendre.legroots(np.polynomial.legendre.legder(c))
    return np.concatenate([[-1.0], np.sort(np.real(r)), [1.0]])


def lagrange_basis(nodes, x):
    """Lagrange cardinal polynomials on `nodes` and derivatives at x."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    n = nodes.size
    phi = np.ones((x.size, n))
    dphi = np.zeros((x.size, n))
    for a in range(n):
        for b in range(n):
            if b == a:
                continue
            term = (x - nodes[b]) / (nodes[a] - nodes[b])
            dterm = 1.0 / (nodes[a] - nodes[b])
            dphi[:, a] = dphi[:, a] * term + phi[:, a] * dterm
            phi[:, a] = phi[:, a] * term
    return phi, dphi


def basis_1d(P, x, kind="modal"):
    if kind == "modal":
        return modified_basis(P, x)
    if kind == "nodal":
        return lagrange_basis(gll_points(P), x)
    raise ValueError(kind)


def tensor_tables(phi1, dphi1, dim):
    """Tensor products over `dim` directions of 1-D tables given at the same 1-D
    points: returns B [Np][Nm] and D[r] [Np][Nm] (derivative along xi_r), point
    and mode indices with the first direction fastest."""
    npt, nm = phi1.shape
    B = np.ones((npt ** dim, nm ** dim))
    D = [np.ones((npt ** dim, nm ** dim)) for _ in range(dim)]
    pidx = np.indices((npt,) * dim).reshape(dim, -1)[::-1]   # pidx[r] = index along r
    midx = np.indices((nm,) * dim).reshape(dim, -1)[::-1]
    for r in range(dim):
        vals = phi1[pidx[r][:, None], midx[r][None, :]]
        dvals = dphi1[pidx[r][:, None], midx[r][None, :]]
        B *= vals
        for s in range(dim):
            D[s] *= dvals if s == r else vals
    return B, D


def face_tables(P, Q, dim, kind="modal"):
    """Basis values and reference derivatives at the face points of each local
    face lf (lf = 2r: xi_r = -1; lf = 2r+1: xi_r = +1).  Face points are the
    tensor product of the 1-D Gauss points over the remaining directions in
    increasing order.  Returns (xi_face [2d][Nf][d], Bf [2d][Nf][Nm],
    Df [2d][d][Nf][Nm])."""
    xq, _ = gauss_legendre(Q)
    n = P + 1
    nf = Q ** (dim - 1)
    xi_f, Bf, Df = [], [], []
    for lf in range(2 * dim):
        r, s = lf // 2, lf % 2
        tang = [t for t in range(dim) if t != r]
        fidx = np.indices((Q,) * (dim - 1)).reshape(dim - 1, -1)[::-1] if dim > 1 else None
        xi = np.zeros((nf, dim))
        xi[:, r] = -1.0 if s == 0 else 1.0
        for a, t in enumerate(tang):
            xi[:, t] = xq[fidx[a]]
        xi_f.append(xi)
        B = np.ones((nf, n ** dim))
        D = [np.ones((nf, n ** dim)) for _ in range(dim)]
        midx = np.indices((n,) * dim).reshape(dim, -1)[::-1]
        for t in range(dim):
            ph, dph = basis_1d(P, xi[:, t], kind)
            vals = ph[:, midx[t]]
            dvals = dph[:, midx[t]]
            B *= vals
            for s2 in range(dim):
                D[s2] *= dvals if s2 == t else vals
        Bf.append(B)
        Df.append(D)
    return np.array(xi_f), np.array(Bf), np.array(Df)
