"""Pins of the oracle's 1-D rules and bases against closed forms and
independent library routines."""
import numpy as np
import pytest
import sympy as sp
from scipy.special import eval_jacobi

from oracle import basis as bs


@pytest.mark.parametrize("Q", [2, 3, 5, 8])
def test_gauss_exact_to_degree_2Q_minus_1(Q):
    x, w = bs.gauss_legendre(Q)
    for k in range(2 * Q):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(w * x ** k) - exact) < 1e-14
    k = 2 * Q
    assert abs(np.sum(w * x ** k) - 2.0 / (k + 1)) > 1e-6


@pytest.mark.parametrize("n,a,b", [(0, 1, 1), (1, 1, 1), (3, 1, 1), (5, 1, 1), (4, 2, 0.5)])
def test_jacobi_against_scipy(n, a, b):
    x = np.linspace(-1, 1, 17)
    p, dp = bs.jacobi(n, a, b, x)
    assert np.allclose(p, eval_jacobi(n, a, b, x), atol=1e-13)
    h = 1e-6
    fd = (eval_jacobi(n, a, b, x + h) - eval_jacobi(n, a, b, x - h)) / (2 * h)
    assert np.allclose(dp, fd, atol=1e-7)


def test_modified_basis_boundary_values():
    P = 5
    phi, _ = bs.modified_basis(P, np.array([-1.0, 1.0]))
    assert np.allclose(phi[0], np.eye(P + 1)[0])
    assert np.allclose(phi[1], np.eye(P + 1)[P])


@pytest.mark.parametrize("P", [1, 2, 4])
def test_modified_mass_matrix_closed_form(P):
    """1-D mass matrix by Gauss quadrature equals exact rational integrals of
    the Karniadakis-Sherwin modified basis computed symbolically."""
    X = sp.symbols("x")
    funcs = [(1 - X) / 2]
    for p in range(1, P):
        funcs.append((1 - X) / 2 * (1 + X) / 2 * sp.jacobi(p - 1, 1, 1, X))
    funcs.append((1 + X) / 2)
    exact = np.array([[float(sp.integrate(f * g, (X, -1, 1))) for g in funcs] for f in funcs])
    dexact = np.array([[float(sp.integrate(sp.diff(f, X) * sp.diff(g, X), (X, -1, 1))) for g in funcs]
                       for f in funcs])
    x, w = bs.gauss_legendre(P + 1)
    phi, dphi = bs.modified_basis(P, x)
    assert np.allclose(phi.T @ (w[:, None] * phi), exact, atol=1e-14)
    assert np.allclose(dphi.T @ (w[:, None] * dphi), dexact, atol=1e-13)


def test_lagrange_cardinal_and_derivative():
    nodes = bs.gll_points(4)
    phi, dphi = bs.lagrange_basis(nodes, nodes)
    assert np.allclose(phi, np.eye(5), atol=1e-14)
    # derivative of x^3 interpolated exactly
    x = np.linspace(-0.9, 0.9, 7)
    _, d = bs.lagrange_basis(nodes, x)
    assert np.allclose(d @ nodes ** 3, 3 * x ** 2, atol=1e-12)


def test_gll_points_are_legendre_derivative_roots():
    P = 6
    r = bs.gll_points(P)[1:-1]
    dP = np.polynomial.legendre.Legendre.basis(P).deriv()
    assert np.allclose(dP(r), 0, atol=1e-12)


def test_tensor_tables_match_direct_products():
    x, _ = bs.gauss_legendre(3)
    phi, dphi = bs.modified_basis(2, x)
    B, D = bs.tensor_tables(phi, dphi, 3)
    # point (q0,q1,q2) = (2,0,1), mode (m0,m1,m2) = (1,2,0)
    q = 2 + 3 * (0 + 3 * 1)
    m = 1 + 3 * (2 + 3 * 0)
    assert np.isclose(B[q, m], phi[2, 1] * phi[0, 2] * phi[1, 0])
    assert np.isclose(D[1][q, m], phi[2, 1] * dphi[0, 2] * phi[1, 0])


def test_face_tables_equal_volume_basis_at_face_points():
    P, Q, d = 2, 4, 3
    xi_f, Bf, Df = bs.face_tables(P, Q, d)
    for lf in range(6):
        pts = xi_f[lf]
        # evaluate the tensor basis at the face points from 1-D tables
        vals = np.ones((pts.shape[0], (P + 1) ** 3))
        midx = np.indices((P + 1,) * 3).reshape(3, -1)[::-1]
        for r in range(3):
            ph, _ = bs.modified_basis(P, pts[:, r])
            vals *= ph[:, midx[r]]
        assert np.allclose(Bf[lf], vals)
