"""Pins of the oracle on curved and rotated elements and on the far-field and
adiabatic-wall boundary conditions (the cylinder workload of Sec. 6.4):
closed-form metrics of an exactly quadratic map, free-stream preservation
on curved meshes (metric identities, exact for Q >= ceil(3(P+1)/2)),
equivariance of R under a rigid rotation of mesh and field, equality of the
affine and the 27-node description of the same elements, the characteristic
invariants of the far-field state, and zero mass and energy flux through an
adiabatic wall."""
import numpy as np
import pytest

import workloads as w
from workloads import Physics
from oracle.dg import DG
from oracle import geometry as geo
from oracle import physics as phy


def uniform_u(dg, rho=1.2, vel=(0.3, -0.2, 0.1), T=1.1):
    ph = dg.ph
    d = dg.dim
    p = rho * T / (ph.gamma * ph.Ma ** 2)
    U0 = phy.conservative(np.array(rho), np.array(vel[:d]), np.array(p), ph)
    one = np.round(dg.one_coeffs(), 10)
    return np.broadcast_to(U0[None, :, None] * one[None, None, :], (dg.E, d + 2, dg.nm)).copy()


def flux_scale(dg, u):
    return np.abs(dg.rhs(u, faces=False)).sum(axis=2).max()


def test_quadratic_map_metrics_closed_form():
    """x = X + a Y^2, y = Y + b X Z, z = Z (exactly quadratic): the 27-node
    element reproduces x, dx/dxi and |J| at arbitrary points."""
    a, b = 0.3, -0.2
    fn = lambda X: np.stack([X[..., 0] + a * X[..., 1] ** 2, X[..., 1] + b * X[..., 0] * X[..., 2],
                             X[..., 2]], -1)
    m = w.mapped_box_mesh([np.array([0.0, 1.0]), np.array([0.5, 1.5]), np.array([-1.0, 0.0])],
                          (False,) * 3, fn, order=2)
    rng = np.random.default_rng(0)
    xi = rng.uniform(-1, 1, (20, 3))
    x, jac = geo.map_points(m.nodes, 2, xi)
    X = np.stack([0.5 + 0.5 * xi[:, 0], 1.0 + 0.5 * xi[:, 1], -0.5 + 0.5 * xi[:, 2]], -1)
    assert np.allclose(x[0], fn(X), atol=1e-14)
    # dx/dX by hand, times dX/dxi = 1/2
    J = np.zeros((20, 3, 3))
    J[:, 0, 0] = 1
    J[:, 0, 1] = 2 * a * X[:, 1]
    J[:, 1, 0] = b * X[:, 2]
    J[:, 1, 1] = 1
    J[:, 1, 2] = b * X[:, 0]
    J[:, 2, 2] = 1
    assert np.allclose(jac[0], 0.5 * J, atol=1e-14)
    det, ginv = geo.metrics(jac)
    assert np.allclose(det[0], 0.125 * np.linalg.det(J), atol=1e-14)
    assert np.allclose(np.einsum("prj,pjs->prs", ginv[0], jac[0]), np.eye(3), atol=1e-13)


CURVED = [
    ("wavy_P2", lambda: w.wavy_box_case((3, 2, 2), P=2)),
    ("wavy_P3", lambda: w.wavy_box_case((2, 2, 2), P=3)),
    ("rotated_g1", lambda: w.rotated_box_case((3, 2, 2), P=2, order=1)),
    ("rotated_2d", lambda: w.rotated_box_case((3, 4), P=3, order=2)),
]


@pytest.mark.parametrize("name,mk", CURVED)
def test_free_stream_preserved_curved(name, mk):
    c = mk()
    dg = DG(c.mesh, c.P, c.Q, c.phys)
    u = uniform_u(dg)
    assert np.abs(dg.rhs(u)).max() < 1e-13 * flux_scale(dg, u)


def test_free_stream_on_ogrid_with_far_field():
    """A uniform stream through the O-grid with far-field conditions on both
    radial boundaries: R = 0 (curved metrics and the characteristic state both
    return the free stream)."""
    c = w.small_cylinder_case(n_r=2, n_theta=6, n_z=1, P=2, bc=(w.BC_FARFIELD, w.BC_FARFIELD))
    dg = DG(c.mesh, c.P, c.Q, c.phys)
    u = dg.project_exact()
    assert np.abs(dg.rhs(u)).max() < 1e-12 * flux_scale(dg, u)


def test_fluid_at_rest_with_walls_and_far_field():
    """Uniform fluid at rest (far-field state at rest too) is a steady state of
    the cylinder case's boundary conditions: adiabatic wall and far field."""
    c = w.small_cylinder_case(n_r=2, n_theta=6, n_z=1, P=2)
    c.phys.fid = w.FIELD_UNIFORM
    c.phys.fpar = (1.0, 0.0, 0.0, 0.0, 1.0)
    dg = DG(c.mesh, c.P, c.Q, c.phys)
    u = dg.project_exact()
    scale = np.abs(dg.rhs(u, faces=False)).sum(axis=2).max()
    assert np.abs(dg.rhs(u)).max() < 1e-12 * scale


def test_affine_and_quadratic_descriptions_agree():
    """The same rotated straight-sided elements given by 8 or 27 nodes: the
    isoparametric maps coincide, so R does too (to rounding)."""
    c1 = w.rotated_box_case((3, 2, 2), P=2, order=1)
    c2 = w.rotated_box_case((3, 2, 2), P=2, order=2)
    d1 = DG(c1.mesh, c1.P, c1.Q, c1.phys)
    d2 = DG(c2.mesh, c2.P, c2.Q, c2.phys)
    u = d1.project_exact()
    r1, r2 = d1.residual(u), d2.residual(u)
    assert np.linalg.norm(r1 - r2) < 1e-12 * np.linalg.norm(r1)


def rotate_momentum(u, R):
    d = R.shape[0]
    out = u.copy()
    out[:, 1:1 + d] = np.einsum("ij,ejm->eim", R, u[:, 1:1 + d])
    return out


@pytest.mark.parametrize("riemann", [phy.RIEMANN_ROE, phy.RIEMANN_HLLC])
def test_rotation_equivariance(riemann):
    """Rotating mesh and field together rotates R: R_rot(Rot u) = Rot R(u),
    with Rot acting on the momentum coefficients (the reference coordinates
    of every element are unchanged, so are the mode coefficients)."""
    c0 = w.small_tgv_case((3, 2, 2), P=2, riemann=riemann)
    cr = w.rotated_box_case((3, 2, 2), P=2, order=1, riemann=riemann)
    R = cr.mesh.meta["rotation"]
    d0 = DG(c0.mesh, c0.P, c0.Q, c0.phys)
    dr = DG(cr.mesh, cr.P, cr.Q, cr.phys)
    u = d0.project_exact() + 0.01 * w.random_direction(d0.project_exact(), 1)
    r0 = d0.residual(u)
    rr = dr.residual(rotate_momentum(u, R))
    # rounding floor: relative change of R under a one-ulp perturbation of u
    # (rotating u already rounds every momentum coefficient once)
    rng = np.random.default_rng(1)
    floor = max(np.linalg.norm(d0.residual(u * (1 + 2.0 ** -52 * rng.standard_normal(u.shape))) - r0)
                for _ in range(3)) / np.linalg.norm(r0)
    assert floor < 1e-12
    assert np.linalg.norm(rr - rotate_momentum(r0, R)) < 16 * floor * np.linalg.norm(r0)


# ---------------------------------------------------------------- far field

def ph_ff(Ma=0.3):
    return Physics(Ma=Ma, Re=100.0)


def states(rng, n, ph, mach):
    rho = 0.6 + rng.random(n)
    vel = mach / ph.Ma * rng.standard_normal((n, 3)) / np.sqrt(3)
    p = (0.6 + rng.random(n)) / (ph.gamma * ph.Ma ** 2)
    return phy.conservative(rho, vel, p, ph)


def unit(rng, n):
    v = rng.standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def invariants(U, n, ph):
    rho, vel, p, _ = phy.primitives(U, ph)
    c = np.sqrt(ph.gamma * p / rho)
    un = np.sum(vel * n, -1)
    g1 = ph.gamma - 1
    return un + 2 * c / g1, un - 2 * c / g1, p / rho ** ph.gamma, vel - un[:, None] * n


def test_far_field_returns_free_stream():
    ph = ph_ff()
    rng = np.random.default_rng(3)
    for mach in (0.2, 2.0):
        Ui = states(rng, 200, ph, mach)
        n = unit(rng, 200)
        assert np.allclose(phy.farfield_state(ph, Ui, Ui, n), Ui, rtol=1e-12, atol=1e-12)


def test_far_field_characteristics_subsonic():
    ph = ph_ff()
    rng = np.random.default_rng(4)
    UL = states(rng, 400, ph, 0.3)
    Ui = states(rng, 400, ph, 0.3)
    n = unit(rng, 400)
    Ub = phy.farfield_state(ph, UL, Ui, n)
    RpL, _, sL, tL = invariants(UL, n, ph)
    _, Rmi, si, ti = invariants(Ui, n, ph)
    Rpb, Rmb, sb, tb = invariants(Ub, n, ph)
    _, vL, _, _ = phy.primitives(UL, ph)
    sub = np.abs(np.sum(vL * n, -1)) < np.sqrt(ph.gamma * phy.primitives(UL, ph)[2] / UL[:, 0])
    assert sub.sum() > 300
    assert np.allclose(Rpb[sub], RpL[sub], rtol=1e-12)
    assert np.allclose(Rmb[sub], Rmi[sub], rtol=1e-12)
    out = (0.5 * (Rpb + Rmb) > 0) & sub
    inn = (0.5 * (Rpb + Rmb) <= 0) & sub
    assert out.sum() > 50 and inn.sum() > 50
    assert np.allclose(sb[out], sL[out], rtol=1e-12) and np.allclose(sb[inn], si[inn], rtol=1e-12)
    assert np.allclose(tb[out], tL[out], atol=1e-12) and np.allclose(tb[inn], ti[inn], atol=1e-12)


def test_far_field_supersonic_takes_upwind_state():
    ph = ph_ff()
    rng = np.random.default_rng(5)
    UL = states(rng, 100, ph, 0.3)
    Ui = states(rng, 100, ph, 0.3)
    rho, vel, p, _ = phy.primitives(UL, ph)
    n = unit(rng, 100)
    c = np.sqrt(ph.gamma * p / rho)
    fast = vel + 3.0 * c[:, None] * n          # supersonic outflow
    Uo = phy.conservative(rho, fast, p, ph)
    assert np.array_equal(phy.farfield_state(ph, Uo, Ui, n), Uo)
    slow = vel - 3.0 * c[:, None] * n          # supersonic inflow
    Uin = phy.conservative(rho, slow, p, ph)
    assert np.array_equal(phy.farfield_state(ph, Uin, Ui, n), Ui)


# ---------------------------------------------------------------- adiabatic wall

@pytest.mark.parametrize("riemann", [phy.RIEMANN_ROE, phy.RIEMANN_HLLC])
def test_adiabatic_wall_inviscid_flux_is_pure_pressure(riemann):
    """Against the mirror state, the Riemann flux carries no mass, no energy
    and no tangential momentum: F = (0, p* n, 0)."""
    ph = Physics(Ma=0.3, Re=100.0, riemann=riemann)
    rng = np.random.default_rng(6)
    UL = states(rng, 300, ph, 0.4)
    n = unit(rng, 300)
    Ur, Ub, adi = phy.boundary_states(ph, phy.BC_ADIA_WALL, np.zeros((300, 3)), 0.0, UL, n)
    assert adi
    F = phy.riemann_flux(UL, Ur, n, ph)
    scale = np.abs(F).max()
    assert np.abs(F[:, 0]).max() < 1e-13 * scale and np.abs(F[:, -1]).max() < 1e-13 * scale
    mom = F[:, 1:4]
    tang = mom - np.sum(mom * n, -1)[:, None] * n
    assert np.abs(tang).max() < 1e-12 * scale
    # the viscous state: interior density and temperature, zero velocity
    rL, _, _, TL = phy.primitives(UL, ph)
    rb, vb, _, Tb = phy.primitives(Ub, ph)
    assert np.allclose(rb, rL) and np.allclose(Tb, TL) and np.abs(vb).max() == 0


def test_adiabatic_wall_carries_no_mass_or_energy_discretely():
    """On the O-grid with a non-uniform state, the numerical normal flux of
    the wall face points has zero mass and energy components."""
    c = w.small_cylinder_case(n_r=2, n_theta=6, n_z=1, P=2)
    dg = DG(c.mesh, c.P, c.Q, c.phys)
    u = dg.project_exact() + 0.02 * w.random_direction(dg.project_exact(), 2)
    wall = [g for g in dg.groups if g["bctype"] == phy.BC_ADIA_WALL]
    assert wall
    for g in wall:
        QL, QR, Qa, dQa, _, _ = dg.face_states(g, u, 0.0)
        Hh, S = dg.face_flux(g, QL, QR, Qa, dQa, 0.0)
        scale = np.abs(Hh).max()
        assert np.abs(Hh[..., 0]).max() < 1e-13 * scale
        assert np.abs(Hh[..., -1]).max() < 1e-13 * scale
        assert np.abs(S[..., -1]).max() == 0.0


def test_cylinder_wall_layer_field():
    """The cylinder's initial stream with a wall layer: at rest on the wall,
    the undisturbed stream far away, monotone in between."""
    ph = Physics(Ma=0.2, Re=3900.0, fid=phy.FIELD_CYLINDER, fpar=(0.5, 0.1))
    th = np.linspace(0, 2 * np.pi, 7)
    for r, expect in ((0.5, 0.0), (20.0, 1.0)):
        x = np.stack([r * np.cos(th), r * np.sin(th), np.zeros_like(th)], -1)
        U = phy.exact_state(ph, x, 0.0)
        assert np.allclose(U[:, 1] / U[:, 0], expect, atol=1e-15) and np.all(U[:, 2:4] == 0)
    r = np.linspace(0.5, 2.0, 50)
    x = np.stack([r, np.zeros_like(r), np.zeros_like(r)], -1)
    u = phy.exact_state(ph, x, 0.0)[:, 1]
    assert np.all(np.diff(u) > 0)
    assert np.allclose(u, 1 - np.exp(-(r - 0.5) / 0.1), atol=1e-15)

