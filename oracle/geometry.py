"""Isoparametric element geometry: coordinates, metrics, |J|, face normals
and surface Jacobians (the w_i J_i and w^G J^G of Eq. discrete-form-Equations).

Element nodes are equispaced on [-1, 1]^d with geometry order g (1 = affine,
2 = quadratic), first direction fastest.
"""
import numpy as np


def shape_1d(g, x):
    """Lagrange shape functions of order g on equispaced nodes of [-1, 1] and
    their derivatives at x: [len(x)][g+1]."""
    nodes = np.linspace(-1.0, 1.0, g + 1)
    x = np.asarray(x, dtype=np.float64)
    N = np.ones((x.size, g + 1))
    dN = np.zeros((x.size, g + 1))
    for a in range(g + 1):
        for b in range(g + 1):
            if b == a:
                continue
            t = (x - nodes[b]) / (nodes[a] - nodes[b])
            dN[:, a] = dN[:, a] * t + N[:, a] / (nodes[a] - nodes[b])
            N[:, a] = N[:, a] * t
    return N, dN


def map_points(nodes, g, xi):
    """Physical coordinates x [E][N][d] and Jacobian dx/dxi [E][N][d_x][d_xi]
    of every element at the reference points xi [N][d]."""
    E, na, dim = nodes.shape
    npt = xi.shape[0]
    aidx = np.indices((g + 1,) * dim).reshape(dim, -1)[::-1]  # aidx[r][a]
    S = np.ones((npt, na))
    dS = [np.ones((npt, na)) for _ in range(dim)]
    for r in range(dim):
        N, dN = shape_1d(g, xi[:, r])
        v = N[:, aidx[r]]
        dv = dN[:, aidx[r]]
        S *= v
        for s in range(dim):
            dS[s] *= dv if s == r else v
    x = np.einsum("pa,eax->epx", S, nodes)
    jac = np.stack([np.einsum("pa,eax->epx", dS[s], nodes) for s in range(dim)], axis=-1)
    return x, jac


def metrics(jac):
    """|det J| and the inverse metric ginv[..., r, j] = d xi_r / d x_j."""
    det = np.linalg.det(jac)
    ginv = np.linalg.inv(jac)   # (dx/dxi)^-1 = dxi/dx, rows r = xi_r
    return det, ginv


def face_normal(ginv, det, lf):
    """Outward unit normal and surface Jacobian at points of local face lf of an
    element (Nanson: n dA = |J| grad(xi_r) dA_ref)."""
    r, s = lf // 2, lf % 2
    gr = ginv[..., r, :]                    # grad xi_r
    mag = np.linalg.norm(gr, axis=-1)
    sign = -1.0 if s == 0 else 1.0
    n = sign * gr / mag[..., None]
    jf = np.abs(det) * mag
    return n, jf
