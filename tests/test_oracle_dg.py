"""Pins of the oracle's residual R(u) = M^-1 L(u) (Sec. 3.1) against
invariants of the discretisation: free-stream preservation, discrete
conservation, basis independence, mirror/rotation symmetry, consistency
with exact solutions at the design rate, and the symmetry of the interior
penalty operator."""
import numpy as np
import pytest

import workloads as w
from workloads import Physics
from oracle.dg import DG
from oracle import physics as phy


def uniform_u(dg, rho=1.2, vel=(0.3, -0.2, 0.1), T=1.1):
    """Coefficients of an exactly constant state (the constant function has
    coefficients 1 on the vertex modes and 0 elsewhere in the modified basis,
    1 on every mode in a nodal basis)."""
    ph = dg.ph
    d = dg.dim
    p = rho * T / (ph.gamma * ph.Ma ** 2)
    U0 = phy.conservative(np.array(rho), np.array(vel[:d]), np.array(p), ph)
    one = np.round(dg.one_coeffs(), 10)
    return np.broadcast_to(U0[None, :, None] * one[None, None, :], (dg.E, d + 2, dg.nm)).copy()


def random_u(dg, seed=0, amp=0.02):
    """A smooth background state with seeded relative perturbations of every
    coefficient."""
    u = uniform_u(dg)
    rng = np.random.default_rng(seed)
    scale = np.abs(u).max(axis=(0, 2))
    return u + amp * rng.standard_normal(u.shape) * scale[None, :, None]


def volume_scale(dg, u):
    return np.abs(dg.apply_minv(dg.rhs(u, 0.0, faces=False))).max()


CASES = [
    ("2d_roe", lambda: w.vortex_case(n=4, P=2)),
    ("2d_hllc_P3", lambda: w.vortex_case(n=3, P=3, riemann=phy.RIEMANN_HLLC)),
    ("3d_P2", lambda: w.small_tgv_case((3, 2, 2), P=2)),
    ("3d_stretched", lambda: w.small_tgv_case((2, 3, 2), P=1, stretch=True)),
]


@pytest.mark.parametrize("name,mk", CASES)
def test_free_stream_preserved(name, mk):
    """L(const) = 0 (and so R = M^-1 L = 0) to rounding of the volume term."""
    c = mk()
    dg = DG(c.mesh, c.P, c.Q, c.phys)
    u = uniform_u(dg)
    assert np.abs(dg.rhs(u)).max() < 1e-13 * np.abs(dg.rhs(u, faces=False)).sum(axis=2).max()


def test_free_stream_with_dirichlet_and_wall_bcs():
    c = w.poiseuille_case(2, nx=3, ny=2)
    ph = c.phys
    ph.fid, ph.forcing = w.FIELD_UNIFORM, 0
    ph.bc = [w.BC_DIRICHLET, w.BC_DIRICHLET]
    dg = DG(c.mesh, c.P, c.Q, ph)
    u = dg.project_exact()
    assert np.abs(dg.rhs(u)).max() < 1e-13 * np.abs(dg.rhs(u, faces=False)).sum(axis=2).max()


@pytest.mark.parametrize("name,mk", CASES)
def test_discrete_conservation_periodic(name, mk):
    c = mk()
    dg = DG(c.mesh, c.P, c.Q, c.phys)
    u = random_u(dg)
    L = dg.rhs(u)
    total = dg.integral(L)
    scale = np.abs(dg.rhs(u, faces=False)).sum(axis=(0, 2))
    assert np.all(np.abs(total) < 1e-13 * scale)


@pytest.mark.parametrize("dim", [2, 3])
def test_basis_independence(dim):
    """R as a function (values at the quadrature points) does not depend on
    the basis of Q_P chosen (modal vs nodal Lagrange)."""
    c = w.vortex_case(n=3, P=3) if dim == 2 else w.small_tgv_case((2, 2, 2), P=2)
    dm = DG(c.mesh, c.P, c.Q, c.phys, kind="modal")
    dn = DG(c.mesh, c.P, c.Q, c.phys, kind="nodal")
    um = random_u(dm)
    vals = dm.values(um, dm.B)                         # same function in both bases
    un = np.einsum("mq,eqv->evm", np.linalg.pinv(dn.B), vals)
    Rm = dm.values(dm.residual(um), dm.B)
    Rn = dn.values(dn.residual(un), dn.B)
    assert np.abs(Rm - Rn).max() < 1e-10 * np.abs(Rm).max()


def permute(u, n, P, dim, perm):
    """Field on an n^dim periodic uniform box mapped by the axis permutation
    x'_r = x_perm[r] (element and mode tensor indices permuted, momentum
    components permuted)."""
    E, nv, nm = u.shape
    out = np.empty_like(u)
    for e in range(E):
        c = np.unravel_index(e, (n,) * dim, order="F")
        e2 = np.ravel_multi_index(tuple(c[perm[r]] for r in range(dim)), (n,) * dim, order="F")
        for m in range(nm):
            a = np.unravel_index(m, (P + 1,) * dim, order="F")
            m2 = np.ravel_multi_index(tuple(a[perm[r]] for r in range(dim)), (P + 1,) * dim, order="F")
            out[e2, 0, m2] = u[e, 0, m]
            out[e2, -1, m2] = u[e, -1, m]
            for r in range(dim):
                out[e2, 1 + r, m2] = u[e, 1 + perm[r], m]
    return out


@pytest.mark.parametrize("dim,perm", [(2, [1, 0]), (3, [2, 0, 1]), (3, [1, 0, 2])])
def test_axis_permutation_symmetry(dim, perm):
    n, P = 3, 2
    lines = [np.linspace(0.0, 1.0, n + 1)] * dim
    mesh = w.box_mesh(lines, (True,) * dim)
    ph = Physics(Ma=0.3, Re=20.0)
    dg = DG(mesh, P, P + 2, ph)
    u = random_u(dg, seed=3, amp=0.05)
    R = dg.residual(u)
    R2 = dg.residual(permute(u, n, P, dim, perm))
    assert np.abs(R2 - permute(R, n, P, dim, perm)).max() < 1e-11 * np.abs(R).max()


def test_vortex_residual_consistent_at_design_rate():
    """Euler residual of the projected vortex approaches the projected exact
    time derivative at rate h^P (L2)."""
    errs = []
    P = 2
    for n in (16, 32, 64):
        c = w.vortex_case(n=n, P=P, viscous=False)
        dg = DG(c.mesh, c.P, c.Q, c.phys)
        R = dg.residual(dg.project_exact())
        h = 1e-6
        ref = dg.project(lambda x: (phy.exact_state(c.phys, x, h) - phy.exact_state(c.phys, x, -h)) / (2 * h))
        e = dg.l2_error(R - ref, lambda x: np.zeros(x.shape[:-1] + (4,)))
        errs.append(np.linalg.norm(e / np.array([1, 1, 1, 100.0])))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > P - 0.2), rates


def momentum_jacobian_at_rest(beta_s):
    n, P = 3, 1
    mesh = w.box_mesh([np.linspace(0, 1, n + 1)] * 2, (True, True))
    ph = Physics(Ma=0.3, Re=10.0, beta_s=beta_s)
    dg = DG(mesh, P, P + 2, ph)
    u = uniform_u(dg, rho=1.0, vel=(0.0, 0.0), T=1.0)
    idx = [(e, v, m) for e in range(dg.E) for v in (1, 2) for m in range(dg.nm)]
    J = np.zeros((len(idx), len(idx)))
    h = 1e-6
    for k, (e, v, m) in enumerate(idx):
        du = np.zeros_like(u)
        du[e, v, m] = h
        dR = (dg.residual(u + du) - dg.residual(u - du)) / (2 * h)
        J[:, k] = [dR[a, b, c] for (a, b, c) in idx]
    M = np.linalg.inv(dg.Minv[0])
    Mb = np.kron(np.eye(dg.E * 2), M)
    return Mb @ J


def test_interior_penalty_symmetric_at_rest():
    A1 = momentum_jacobian_at_rest(1.0)
    A0 = momentum_jacobian_at_rest(0.0)
    s1 = np.abs(A1 - A1.T).max() / np.abs(A1).max()
    s0 = np.abs(A0 - A0.T).max() / np.abs(A0).max()
    assert s1 < 1e-6, s1
    assert s0 > 1e-3, s0
    # the symmetric operator is negative semi-definite (dissipative penalty)
    ev = np.linalg.eigvalsh(0.5 * (A1 + A1.T))
    assert ev.max() < 1e-6 * np.abs(ev).max()
