"""Pins of the oracle's shock capturing (Sec. 3.1.2) and of the oblique-shock
field of the SWBLI-like workload (Sec. 6.5): Rankine-Hugoniot conservation
across the shock and the textbook theta-beta-Mach deflection; the modal
sensor's projection, scale invariance, limits and ramp; artificial viscosity
entering the diffusion flux as extra viscosity and conductivity; free stream,
conservation and the smooth-field case where it must vanish."""
import numpy as np
import pytest

import workloads as w
from oracle import physics as phy
from oracle.dg import DG
from oracle import basis as bs


def test_oblique_shock_state_conserves_fluxes_and_deflects_by_theta_beta_mach():
    ph = w.Physics(Ma=2.15)
    g = ph.gamma
    for beta_deg in (30.8, 40.0, 55.0):
        beta = np.radians(beta_deg)
        r2, v2, p2 = phy.oblique_shock_state(beta, ph)
        U1 = phy.conservative(np.array([1.0]), np.array([[1.0, 0.0]]), np.array([1 / (g * ph.Ma ** 2)]), ph)
        U2 = phy.conservative(np.array([r2]), np.array([v2]), np.array([p2]), ph)
        n = np.array([[np.sin(beta), np.cos(beta)]])
        F1 = np.einsum("kiv,ki->kv", phy.euler_flux(U1, ph), n)
        F2 = np.einsum("kiv,ki->kv", phy.euler_flux(U2, ph), n)
        assert np.allclose(F1, F2, rtol=1e-13, atol=1e-13)          # mass, momentum, energy
        assert r2 > 1.0 and p2 > 1 / (g * ph.Ma ** 2)                # a compression
        # flow turned toward the shock by the theta-beta-Mach angle
        M = ph.Ma
        tan_t = 2 / np.tan(beta) * (M ** 2 * np.sin(beta) ** 2 - 1) / (M ** 2 * (g + np.cos(2 * beta)) + 2)
        assert abs(-v2[1] / v2[0] - tan_t) < 1e-13
        # the normal Mach number behind the shock is subsonic
        c2 = np.sqrt(g * p2 / r2)
        assert v2 @ n[0] / c2 < 1.0


def test_shock_field_states_on_both_sides_of_the_line():
    ph = w.Physics(Ma=2.15, fid=phy.FIELD_SHOCK, fpar=(30.8, 1.0))
    x = np.array([[0.5, 0.1], [0.5, 0.5], [1.5, 0.01]])
    U = phy.exact_state(ph, x, 0.0)
    r2, v2, _ = phy.oblique_shock_state(np.radians(30.8), ph)
    assert np.allclose(U[0, :3], [1.0, 1.0, 0.0])                     # below the line: stream
    assert np.allclose(U[1, :3], [r2, r2 * v2[0], r2 * v2[1]])        # above
    assert np.allclose(U[2, :3], [r2, r2 * v2[0], r2 * v2[1]])        # behind the foot


def test_smoothed_shock_field_limits():
    """width w > 0: the sharp states a few w away from the line, the mean of
    the two primitive states on it; wall layer l > 0: velocity zero at y = 0
    and within 1e-12 of the layer-free field at y = 30 l."""
    sharp = w.Physics(Ma=2.15, fid=phy.FIELD_SHOCK, fpar=(30.8, 1.0))
    smooth = w.Physics(Ma=2.15, fid=phy.FIELD_SHOCK, fpar=(30.8, 1.0, 0.01, 0.0))
    beta = np.radians(30.8)
    nrm = np.array([np.sin(beta), np.cos(beta)])          # unit normal, post side
    foot = np.array([1.0, 0.0])
    for sgn in (-1.0, 1.0):
        x = (foot + np.array([-0.5, 0.3]) + sgn * 0.2 * nrm)[None, :]
        assert np.allclose(phy.exact_state(smooth, x, 0.0), phy.exact_state(sharp, x, 0.0),
                           rtol=1e-12, atol=1e-12)
    on = (foot + np.array([-0.5, 0.3]))                    # a point of the line y = (1-x) tan b
    on[1] = (1.0 - on[0]) * np.tan(beta)
    rho, vel, p, _ = phy.primitives(phy.exact_state(smooth, on[None, :], 0.0), smooth)
    r2, v2, p2 = phy.oblique_shock_state(beta, smooth)
    p1 = 1.0 / (smooth.gamma * smooth.Ma ** 2)
    assert np.allclose([rho[0], vel[0, 0], vel[0, 1], p[0]],
                       [(1 + r2) / 2, (1 + v2[0]) / 2, v2[1] / 2, (p1 + p2) / 2], rtol=1e-13)
    layer = w.Physics(Ma=2.15, fid=phy.FIELD_SHOCK, fpar=(30.8, 1.0, 0.01, 0.02))
    xw = np.array([[1.5, 0.0], [0.5, 0.0], [1.5, 0.6]])
    U = phy.exact_state(layer, xw, 0.0)
    _, vel, _, _ = phy.primitives(U, layer)
    assert np.all(vel[:2] == 0.0)
    U0 = phy.exact_state(smooth, xw[2:], 0.0)
    assert np.allclose(U[2:], U0, rtol=1e-12, atol=1e-12)


def sensor_case(P=3, n=2):
    c = w.vortex_case(n=n, P=P, Q=P + 2)
    c.phys.av = 1
    return c, DG(c.mesh, c.P, c.Q, c.phys)


@pytest.mark.parametrize("P", [2, 3, 4])
def test_sensor_projection_limits_and_scale(P):
    """Density in Q_{P-1}: nothing left after the projection (S = 0); the
    degree-P Legendre polynomial in one direction: the projection removes all
    of it (ratio 1, s = 0 > s0 + kappa, S = 1); a mix whose ratio is 10^s0
    sits in the middle of the ramp (S = 1/2), also after rho -> 7 rho."""
    c, dg = sensor_case(P)
    xq, _ = bs.gauss_legendre(c.Q)
    n = c.P + 1
    B = dg.B
    rng = np.random.default_rng(P)
    # coefficients of a random polynomial of degree <= P-1 per direction, by
    # least squares on the Gauss grid (exact: the space is contained in Q_P)
    xi = dg.xi
    def fit(vals):
        return np.linalg.lstsq(B, vals, rcond=None)[0]
    low = sum(rng.standard_normal() * np.prod([xi[:, r] ** a[r] for r in range(2)], axis=0)
              for a in np.ndindex(*(P,) * 2))
    u = np.zeros((dg.E, dg.nv, dg.nm))
    u[:, 0, :] = fit(1.0 + 0.1 * low)
    assert np.all(dg.sensor(u) == 0.0)
    LP = bs.jacobi(P, 0.0, 0.0, xi[:, 0])[0]
    u[:, 0, :] = fit(LP)
    rq = dg.values(u[:, :1], dg.B)[..., 0]
    num = np.einsum("q,eq->e", dg.w, (rq - rq @ dg.sensor_proj.T) ** 2)
    den = np.einsum("q,eq->e", dg.w, rq ** 2)
    assert np.allclose(num / den, 1.0, rtol=1e-12)
    assert np.all(dg.sensor(u) == 1.0)
    # scale invariance and the ramp at s0: mix so that the ratio is 10^s0
    s0 = np.log10(1.0 / P ** 4)
    a = np.sqrt(10 ** s0 / (1 - 10 ** s0))
    mix = 1.0 + 0.0 * xi[:, 0]
    c0 = np.sqrt(np.sum(dg.w * mix ** 2) / np.sum(dg.w * LP ** 2))
    u[:, 0, :] = fit(mix + a * c0 * LP)
    assert np.allclose(dg.sensor(u), 0.5, atol=1e-9)
    u[:, 0, :] *= 7.0
    assert np.allclose(dg.sensor(u), 0.5, atol=1e-9)


@pytest.mark.parametrize("d", [2, 3])
def test_artificial_viscosity_raises_viscosity_and_conductivity(d):
    """G with mu_av equals G with constant mu times (mu + mu_av)/mu, point by
    point: the artificial conductivity mu_av C_p/Pr carries the same factor
    as the physical one."""
    rng = np.random.default_rng(40 + d)
    ph = w.Physics(Ma=0.3, Re=50.0)
    rho = 0.5 + rng.random(7)
    vel = rng.random((7, d)) - 0.5
    p = (0.5 + rng.random(7)) / (ph.gamma * ph.Ma ** 2)
    U = phy.conservative(rho, vel, p, ph)
    dU = rng.standard_normal((7, d, d + 2))
    mu_av = rng.random(7)
    G0 = phy.viscous_flux(U, dU, ph)
    G1 = phy.viscous_flux(U, dU, ph, mu_av)
    assert np.allclose(G1, G0 * ((1 / ph.Re + mu_av) * ph.Re)[:, None, None], rtol=1e-13, atol=1e-14)
    # mu_av = mu_0 rho (h/P)(c + |u|) S with the factor mu_0 S h/P given
    c = np.sqrt(ph.gamma * p / rho)
    assert np.allclose(phy.artificial_viscosity(U, 0.3, ph),
                       0.3 * rho * (c + np.linalg.norm(vel, axis=1)), rtol=1e-14)


def test_shock_capturing_vanishes_on_smooth_fields_and_keeps_free_stream():
    c, dg = sensor_case(P=3, n=3)
    u = dg.project_exact()              # a smooth vortex: sensor below the ramp
    assert np.all(dg.sensor(u) == 0.0)
    c.phys.av = 0
    R0 = dg.residual(u)
    c.phys.av = 1
    assert np.array_equal(dg.residual(u), R0)
    one = dg.one_coeffs()
    U0 = phy.exact_state(c.phys, np.array([[0.3, 0.3]]), 0.0)[0]
    uc = U0[None, :, None] * one[None, None, :] * np.ones((dg.E, 1, 1))
    assert np.abs(dg.rhs(uc)).max() < 1e-10 * np.abs(U0).max()


def test_shock_capturing_conserves_on_a_periodic_mesh():
    """A density jump inside an element (sensor active) on the periodic vortex mesh: the
    element sums of L still vanish for every conserved variable."""
    c, dg = sensor_case(P=3, n=4)
    u = dg.project(lambda x: phy.conservative(np.where(x[..., 0] < 0.4, 1.0, 0.6),
                                              np.stack([1.0 + 0 * x[..., 0], 0.3 + 0 * x[..., 0]], -1),
                                              1.0 / (1.4 * 0.01) + 0 * x[..., 0], c.phys))
    assert dg.sensor(u).max() > 0.0
    L = dg.rhs(u)
    tot = dg.integral(L)
    assert np.all(np.abs(tot) < 1e-11 * np.abs(L).sum(axis=(0, 2)))
    c.phys.av = 0
    assert not np.allclose(dg.rhs(u), L)


def _state_and_gradient(vel, grad_vel, rho=1.3, drho=None, p=5.0, d=2):
    """Conservative U and its gradient dU[j][v] at one point from the velocity,
    its gradient grad_vel[j][k] = d u_k / d x_j and the density gradient."""
    ph = w.Physics(Ma=0.3)
    vel = np.asarray(vel, float)
    G = np.asarray(grad_vel, float)
    drho = np.zeros(d) if drho is None else np.asarray(drho, float)
    U = phy.conservative(np.array([rho]), vel[None], np.array([p]), ph)[0]
    dU = np.zeros((d, d + 2))
    dU[:, 0] = drho
    dU[:, 1:1 + d] = rho * G + np.outer(drho, vel)        # d(rho u_k)/dx_j
    return ph, U, dU


def test_ducros_sensor_limits_and_invariance():
    """(div u)^2 / ((div u)^2 + |curl u|^2 + eps): 1 for a pure compression (up
    to eps), 0 for a rigid rotation, 1/2 where (div u)^2 = |curl u|^2 (up to
    eps); the velocity gradient alone counts (a density gradient changes
    nothing); 3-D: each curl component counts (u = (0, 0, y) is a shear: 0);
    gradients far below the floor sqrt(eps) count as uniform flow (0)."""
    eps = phy.DUCROS_EPS
    ph, U, dU = _state_and_gradient([0.4, -0.2], [[-1.0, 0.0], [0.0, -1.0]])
    assert abs(phy.ducros(U, dU, ph) - 4.0 / (4.0 + eps)) < 1e-15
    ph, U, dU = _state_and_gradient([0.4, -0.2], [[0.0, 1.0], [-1.0, 0.0]])
    assert phy.ducros(U, dU, ph) == 0.0
    # u = (-x - y, x - y): div = -2, curl = 2
    ph, U, dU = _state_and_gradient([0.1, 0.7], [[-1.0, 1.0], [-1.0, -1.0]], drho=[0.3, -0.8])
    assert abs(phy.ducros(U, dU, ph) - 4.0 / (8.0 + eps)) < 1e-15
    ph, U2, dU2 = _state_and_gradient([0.1 * 7, 0.7 * 7], [[-7.0, 7.0], [-7.0, -7.0]])
    assert abs(phy.ducros(U2, dU2, ph) - 196.0 / (392.0 + eps)) < 1e-15
    ph, U, dU = _state_and_gradient([0.0, 0.0, 0.3], [[0, 0, 0], [0, 0, 1.0], [0, 0, 0]], d=3)
    assert phy.ducros(U, dU, ph) == 0.0
    ph, U, dU = _state_and_gradient([0.0, 0.0, 0.3], [[2.0, 0, 0], [0, 0, 1.0], [0, 0, 0]], d=3)
    assert abs(phy.ducros(U, dU, ph) - 4.0 / (5.0 + eps)) < 1e-15     # div^2 = 4, curl^2 = 1
    ph, U, dU = _state_and_gradient([0.4, -0.2], [[-1e-9, 0.0], [0.0, -1e-9]])
    assert phy.ducros(U, dU, ph) < 1e-11
    rng = np.random.default_rng(3)
    for _ in range(20):
        ph, U, dU = _state_and_gradient(rng.standard_normal(3), rng.standard_normal((3, 3)),
                                        drho=rng.standard_normal(3), d=3)
        assert 0.0 <= phy.ducros(U, dU, ph) <= 1.0


def test_ducros_option_scales_the_artificial_viscosity_and_conserves():
    """av = 2 multiplies the modal sensor's viscosity by Ducros' sensor at each
    point.  A density jump (modal sensor active) carried by a compressing
    stream u = (1 - x/2, 0.3) (no curl: Ducros 1) gives the residual of av = 1;
    carried by a rotating stream u = (1 - y/2, 0.3 + x/2) (no divergence:
    Ducros 0) the residual without artificial viscosity; on the uniform stream
    too (its gradients are below the floor); and the residual stays
    conservative on the periodic mesh with the option acting."""
    c, dg = sensor_case(P=3, n=4)

    def field(velf):
        return lambda x: phy.conservative(np.where(x[..., 0] < 0.4, 1.0, 0.6), velf(x),
                                          1.0 / (1.4 * 0.01) + 0 * x[..., 0], c.phys)

    def residuals(u):
        out = []
        for av in (0, 1, 2):
            c.phys.av = av
            out.append(dg.rhs(u))
        return out

    n = np.linalg.norm
    u = dg.project(field(lambda x: np.stack([1.0 - 0.5 * x[..., 0], 0.3 + 0 * x[..., 0]], -1)))
    assert dg.sensor(u).max() > 0.0
    L0, L1, L2 = residuals(u)
    assert n(L1 - L0) > 1e-6 * n(L1)
    assert n(L2 - L1) < 1e-5 * n(L1 - L0)     # div^2 = 1/4: Ducros = 1 - 4 eps
    u = dg.project(field(lambda x: np.stack([1.0 - 0.5 * x[..., 1], 0.3 + 0.5 * x[..., 0]], -1)))
    L0, L1, L2 = residuals(u)
    assert n(L2 - L0) < 1e-12 * n(L1 - L0)
    # a uniform stream: the projection leaves velocity gradients far below the
    # floor, so the flow counts as uniform and no viscosity is added
    u = dg.project(field(lambda x: np.stack([1.0 + 0 * x[..., 0], 0.3 + 0 * x[..., 0]], -1)))
    L0, L1, L2 = residuals(u)
    assert n(L2 - L0) < 1e-12 * n(L1 - L0)
    # conservation with the option on, where it acts
    u = dg.project(field(lambda x: np.stack([1.0 - 0.5 * x[..., 0], 0.3 + 0.2 * x[..., 1]], -1)))
    L0, L1, L2 = residuals(u)
    assert n(L2 - L0) > 1e-6 * n(L2)
    tot = dg.integral(L2)
    assert np.all(np.abs(tot) < 1e-11 * np.abs(L2).sum(axis=(0, 2)))
