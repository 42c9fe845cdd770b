"""Pins of the oracle's fluxes and analytic fields against properties fixed
by the governing equations (Sec. 2.1) and by the verification cases
(Sec. 6.1, App. B)."""
import numpy as np
import pytest
import sympy as sp

from oracle import physics as phy
from workloads import Physics, FIELD_VORTEX, FIELD_POISEUILLE, FIELD_TGV, FORCING_POISEUILLE


def ph3(**kw):
    return Physics(Ma=0.3, Re=50.0, **kw)


def random_state(rng, d, n=6, ph=None, mach=0.4):
    ph = ph or ph3()
    rho = 0.5 + rng.random(n)
    vel = mach / ph.Ma * (rng.random((n, d)) - 0.5)
    p = (0.5 + rng.random(n)) / (ph.gamma * ph.Ma ** 2)
    return phy.conservative(rho, vel, p, ph)


def flux_jacobian(U, n, ph):
    """d(F.n)/dU by complex step (exact to rounding)."""
    nv = U.shape[-1]
    A = np.zeros(U.shape[:-1] + (nv, nv))
    for l in range(nv):
        Uc = U.astype(complex)
        Uc[..., l] += 1e-30j
        A[..., :, l] = np.einsum("...iv,...i->...v", phy.euler_flux(Uc, ph), n).imag / 1e-30
    return A


@pytest.mark.parametrize("d", [2, 3])
def test_euler_flux_homogeneous_and_eigenvalues(d):
    ph = ph3()
    rng = np.random.default_rng(1)
    U = random_state(rng, d, ph=ph)
    n = rng.standard_normal((U.shape[0], d))
    n /= np.linalg.norm(n, axis=-1, keepdims=True)
    A = flux_jacobian(U, n, ph)
    Fn = np.einsum("...iv,...i->...v", phy.euler_flux(U, ph), n)
    # Euler flux is homogeneous of degree one: A(U) U = F(U).n
    assert np.allclose(np.einsum("...kl,...l->...k", A, U), Fn, rtol=1e-12, atol=1e-10)
    rho, vel, p, _ = phy.primitives(U, ph)
    c = np.sqrt(ph.gamma * p / rho)
    un = np.sum(vel * n, -1)
    for k in range(U.shape[0]):
        ev = np.sort(np.linalg.eigvals(A[k]).real)
        ref = np.sort(np.concatenate([[un[k] - c[k]], [un[k]] * d, [un[k] + c[k]]]))
        assert np.allclose(ev, ref, rtol=1e-8, atol=1e-8)


def test_euler_flux_rotation_invariance():
    ph = ph3()
    rng = np.random.default_rng(2)
    U = random_state(rng, 2, ph=ph)
    th = 0.7
    Rm = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    n = np.array([np.cos(th), np.sin(th)])
    Fn = phy.euler_flux(U, ph) @ np.zeros(0) if False else np.einsum("kiv,i->kv", phy.euler_flux(U, ph), n)
    Ur = U.copy()
    Ur[:, 1:3] = U[:, 1:3] @ Rm      # momentum in the rotated frame (x' along n)
    Fx = phy.euler_flux(Ur, ph)[:, 0, :]
    back = Fx.copy()
    back[:, 1:3] = Fx[:, 1:3] @ Rm.T
    assert np.allclose(Fn, back, rtol=1e-13)


def test_viscous_flux_against_symbolic_primitive_derivatives():
    """G from conservative gradients (chain rule in the oracle) equals the
    stress and heat flux computed symbolically from primitive fields."""
    ph = ph3()
    g, Ma, Pr, mu = ph.gamma, ph.Ma, ph.Pr, 1.0 / ph.Re
    X = sp.symbols("x0:3")
    rng = np.random.default_rng(3)

    def poly():
        c = rng.standard_normal(4) * 0.3
        return 1 + c[0] * X[0] + c[1] * X[1] * X[2] + c[2] * X[2] ** 2 + c[3] * X[0] * X[1]

    rho = poly()
    vel = [poly() - 1 for _ in range(3)]
    T = poly()
    p = rho * T / (g * Ma ** 2)
    E = p / (g - 1) + rho * sum(v * v for v in vel) / 2
    Usym = [rho] + [rho * v for v in vel] + [E]
    kappa = mu / (Ma ** 2 * Pr * (g - 1))
    div = sum(sp.diff(vel[k], X[k]) for k in range(3))
    pt = {X[0]: 0.3, X[1]: -0.2, X[2]: 0.4}
    Gref = np.zeros((3, 5))
    for i in range(3):
        for k in range(3):
            tau = mu * (sp.diff(vel[i], X[k]) + sp.diff(vel[k], X[i])) - (sp.Rational(2, 3) * mu * div if i == k else 0)
            Gref[i, 1 + k] = float(tau.subs(pt))
        Gref[i, 4] = float((sum(vel[k] * Gref[i, 1 + k] for k in range(3)) + kappa * sp.diff(T, X[i])).subs(pt))
    U = np.array([float(s.subs(pt)) for s in Usym])
    dU = np.array([[float(sp.diff(s, X[j]).subs(pt)) for s in Usym] for j in range(3)])
    G = phy.viscous_flux(U, dU, ph)
    assert np.allclose(G, Gref, rtol=1e-12, atol=1e-13)


def test_viscous_flux_vanishes_for_rigid_rotation():
    ph = ph3()
    U = phy.conservative(np.array(1.3), np.array([0.2, -0.1, 0.05]), np.array(4.0), ph)
    rho, vel, p, T = phy.primitives(U, ph)
    w = np.array([0.3, -0.2, 0.5])
    # u = v0 + w x x has grad u antisymmetric; with rho, T uniform grad E = rho u . grad u
    W = np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])   # du_k/dx_j = W[k, j]
    dU = np.zeros((3, 5))
    dU[:, 1:4] = rho * W.T
    dU[:, 4] = rho * (W.T @ vel)
    assert np.allclose(phy.viscous_flux(U, dU, ph), 0, atol=1e-13)


ALL_FLUXES = [phy.RIEMANN_ROE, phy.RIEMANN_HLLC, phy.RIEMANN_HLL, phy.RIEMANN_LF, phy.RIEMANN_AUSM]


@pytest.mark.parametrize("riemann", ALL_FLUXES)
@pytest.mark.parametrize("d", [2, 3])
def test_riemann_consistency_and_conservation(riemann, d):
    ph = ph3(riemann=riemann)
    rng = np.random.default_rng(4)
    UL = random_state(rng, d, ph=ph)
    UR = random_state(rng, d, ph=ph)
    n = rng.standard_normal((UL.shape[0], d))
    n /= np.linalg.norm(n, axis=-1, keepdims=True)
    Fn = np.einsum("kiv,ki->kv", phy.euler_flux(UL, ph), n)
    assert np.allclose(phy.riemann_flux(UL, UL, n, ph), Fn, rtol=1e-13, atol=1e-12)
    assert np.allclose(phy.riemann_flux(UL, UR, n, ph), -phy.riemann_flux(UR, UL, -n, ph),
                       rtol=1e-12, atol=1e-11)


@pytest.mark.parametrize("riemann", [phy.RIEMANN_ROE, phy.RIEMANN_HLLC, phy.RIEMANN_HLL,
                                     phy.RIEMANN_AUSM])
def test_riemann_supersonic_upwind_and_contact(riemann):
    ph = ph3(riemann=riemann)
    g = ph.gamma
    n = np.array([[1.0, 0.0]])
    pL, pR = 1.0 / (g * ph.Ma ** 2), 1.1 / (g * ph.Ma ** 2)
    cL = np.sqrt(g * pL / 1.0)
    UL = phy.conservative(np.array([1.0]), np.array([[3.0 * cL, 0.1]]), np.array([pL]), ph)
    UR = phy.conservative(np.array([0.8]), np.array([[3.1 * cL, 0.0]]), np.array([pR]), ph)
    assert np.allclose(phy.riemann_flux(UL, UR, n, ph), phy.euler_flux(UL, ph)[:, 0], rtol=1e-12)
    # supersonic flow from the right: the right state's flux
    UL2 = phy.conservative(np.array([1.0]), np.array([[-3.0 * cL, 0.1]]), np.array([pL]), ph)
    UR2 = phy.conservative(np.array([0.8]), np.array([[-3.1 * cL, 0.0]]), np.array([pR]), ph)
    assert np.allclose(phy.riemann_flux(UL2, UR2, n, ph), phy.euler_flux(UR2, ph)[:, 0],
                       rtol=1e-12)
    if riemann == phy.RIEMANN_HLL:
        return    # HLL smears contacts (one intermediate state)
    # stationary contact: same pressure, zero velocity, different density
    UL = phy.conservative(np.array([1.0]), np.array([[0.0, 0.0]]), np.array([pL]), ph)
    UR = phy.conservative(np.array([0.3]), np.array([[0.0, 0.0]]), np.array([pL]), ph)
    assert np.allclose(phy.riemann_flux(UL, UR, n, ph), [[0.0, pL, 0.0, 0.0]], atol=1e-12)


@pytest.mark.parametrize("riemann", ALL_FLUXES)
def test_riemann_flux_dissipates_linear_waves(riemann):
    """Every flux adds dissipation, none adds energy: the DG Euler operator
    linearised about a uniform subsonic stream on a periodic 2x2 mesh (P = 1)
    has no eigenvalue with a positive real part beyond finite-difference
    noise, while its most damped mode decays at a rate of the order of the
    acoustic speed over the element size (a dissipation term of the wrong
    sign would turn it into growth; a central flux without it would leave
    every eigenvalue on the imaginary axis)."""
    from oracle.dg import DG
    import workloads as w
    c = w.vortex_case(n=2, P=1, viscous=False, riemann=riemann)
    c.phys.fid = phy.FIELD_UNIFORM
    c.phys.fpar = (1.0, 3.0, 2.0, 0.0, 1.0)      # rho, u, v, w, T (|u| / c = 0.36)
    dg = DG(c.mesh, c.P, c.Q, c.phys)
    u0 = dg.project_exact()
    n = u0.size
    J = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1e-6 * max(1.0, abs(u0.ravel()[k]))
        J[:, k] = (dg.residual(u0 + e.reshape(u0.shape)) - dg.residual(u0 - e.reshape(u0.shape))).ravel() / (2 * e[k])
    lam = np.linalg.eigvals(J)
    scale = np.abs(lam).max()
    assert lam.real.max() < 1e-6 * scale, lam.real.max() / scale
    assert lam.real.min() < -1e-2 * scale


def _fd_grad(fn, x, h):
    d = x.shape[-1]
    out = []
    for j in range(d):
        e = np.zeros(d)
        e[j] = h
        out.append((fn(x + e) - fn(x - e)) / (2 * h))
    return np.stack(out, axis=-2)          # [..., j, v]


def test_vortex_is_steady_in_moving_frame():
    """dU/dt + div F(U) = 0 for the (sign-corrected) isentropic vortex; the
    sign printed in Sec. 6.1 violates it."""
    ph = Physics(Ma=0.1, viscous=False, fid=FIELD_VORTEX, fpar=(1.0, 0.5, 5.0, 0.5, 0.5, 10.0))
    rng = np.random.default_rng(5)
    x = 0.5 + 0.15 * (rng.random((40, 2)) - 0.5)
    t, h = 0.01, 1e-6

    def resid(exact):
        dUdt = (exact(x, t + h) - exact(x, t - h)) / (2 * h)
        dF = _fd_grad(lambda y: phy.euler_flux(exact(y, t), ph).reshape(y.shape[0], -1), x, h)
        dF = dF.reshape(x.shape[0], 2, 2, 4)
        return dUdt + dF[:, 0, 0] + dF[:, 1, 1], np.abs(dUdt).max()

    r, scale = resid(lambda y, tt: phy.exact_state(ph, y, tt))
    assert np.abs(r).max() < 1e-6 * scale

    def printed(y, tt):   # u = u0 + phi (y - yc) e / 2pi as printed
        U = phy.exact_state(ph, y, tt)
        rho, vel, p, _ = phy.primitives(U, ph)
        vel = vel.copy()
        vel[:, 0] = 2 * 1.0 - vel[:, 0]
        return phy.conservative(rho, vel, p, ph)

    r, scale = resid(printed)
    assert np.abs(r).max() > 1e-2 * scale


def _poiseuille_ns_residual(ph, x, h=1e-4):
    """div(F - G)(U) - f at points x for the steady exact solution (nested
    central differences)."""
    ex = lambda y: phy.exact_state(ph, y, 0.0)

    def H(y):
        U = ex(y)
        dU = _fd_grad(ex, y, 1e-5)
        return (phy.euler_flux(U, ph) - phy.viscous_flux(U, dU, ph)).reshape(y.shape[0], -1)

    dH = _fd_grad(H, x, h).reshape(x.shape[0], 2, 2, 4)
    return dH[:, 0, 0] + dH[:, 1, 1] - phy.forcing(ph, x, 0.0)


def test_poiseuille_forcing_balances_exact_solution():
    ph = Physics(Ma=0.2, Re=100.0, fid=FIELD_POISEUILLE, forcing=FORCING_POISEUILLE,
                 fpar=(0.01, 1.0, -8.0 / 100.0))
    rng = np.random.default_rng(6)
    x = np.stack([2 * rng.random(30), rng.random(30)], -1)
    r = _poiseuille_ns_residual(ph, x)
    f = phy.forcing(ph, x, 0.0)
    assert np.abs(r).max() < 1e-5 * max(np.abs(f).max(), 1.0)
    # the f_4 printed in App. B (h(y) replaced by y(L-y)) leaves an O(1) residual
    theta, L, dpdx = ph.fpar
    mu = 1 / ph.Re
    y = x[:, 1]
    c = L * L - 6 * y * L + 6 * y * y
    h = y * (L - y) + theta * y * y * (L - y) ** 2
    delta = dpdx ** 2 / (2 * mu) * (h - y * (L - y)) * (1 - theta * c - ph.gamma / (ph.gamma - 1))
    assert np.abs(delta).max() > 50 * np.abs(r).max()


def test_tgv_velocity_divergence_free():
    ph = Physics(Ma=0.1, fid=FIELD_TGV)
    rng = np.random.default_rng(7)
    x = np.pi * (2 * rng.random((20, 3)) - 1)
    vel = lambda y: phy.primitives(phy.exact_state(ph, y, 0.0), ph)[1]
    dv = _fd_grad(vel, x, 1e-5)
    assert np.abs(np.einsum("kjj->k", dv)).max() < 1e-9
    _, _, _, T = phy.primitives(phy.exact_state(ph, x, 0.0), ph)
    assert np.allclose(T, 1.0)


# ------------------------------------------------------------------ Sutherland's law

def sutherland_dimensional(T_kelvin, mu0=1.716e-5, T0=273.15, S=110.0):
    """Sutherland's law in kelvin, mu = mu0 (T/T0)^(3/2) (T0 + S)/(T + S)
    (the textbook dimensional form; mu0 and T0 cancel in any ratio)."""
    return mu0 * (T_kelvin / T0) ** 1.5 * (T0 + S) / (T_kelvin + S)


@pytest.mark.parametrize("T_inf", [288.15, 120.0, 1000.0])
def test_sutherland_viscosity_pins(T_inf):
    """Sec. 2.1 non-dimensionalises mu by its free-stream value, mu = 1/Re at
    T = 1.  With Sutherland's law the non-dimensional mu(T) is the dimensional
    law's ratio mu(T T_inf) / mu(T_inf) over Re; it grows like T^(1/2) for
    T >> S/T_inf and like T^(3/2) for T << S/T_inf."""
    ph = Physics(Re=250.0, mu_law=1, T_inf_K=T_inf)
    assert phy.viscosity(np.array([1.0]), ph)[0] == pytest.approx(1.0 / ph.Re, rel=1e-15)
    T = np.array([0.3, 0.8, 1.7, 4.0])
    ref = sutherland_dimensional(T * T_inf) / sutherland_dimensional(T_inf) / ph.Re
    assert np.allclose(phy.viscosity(T, ph), ref, rtol=1e-13, atol=0)
    # the same ratio for another reference pair (mu0, T0): they cancel
    ref2 = sutherland_dimensional(T * T_inf, 3.0, 100.0) / sutherland_dimensional(T_inf, 3.0, 100.0)
    assert np.allclose(phy.viscosity(T, ph) * ph.Re, ref2, rtol=1e-13)
    s = 110.0 / T_inf
    big, small = np.array([1e8]), np.array([1e-8])
    assert phy.viscosity(big, ph)[0] / np.sqrt(big[0]) == pytest.approx((1 + s) / ph.Re, rel=1e-6)
    assert phy.viscosity(small, ph)[0] / small[0] ** 1.5 == pytest.approx((1 + s) / (s * ph.Re),
                                                                         rel=1e-6)
    # constant law: 1/Re at every temperature
    assert np.all(phy.viscosity(T, Physics(Re=250.0)) == 1.0 / 250.0)


@pytest.mark.parametrize("d", [2, 3])
def test_viscous_flux_scales_with_sutherland_viscosity(d):
    """The diffusion flux is linear in mu (stress and heat flux both carry it,
    kappa = mu/(Ma^2 Pr (gamma-1))), so the Sutherland flux equals the
    constant-mu flux times mu(T) Re, point by point."""
    rng = np.random.default_rng(17 + d)
    ph0 = Physics(Ma=0.3, Re=50.0)
    ph1 = Physics(Ma=0.3, Re=50.0, mu_law=1, T_inf_K=200.0)
    U = random_state(rng, d, n=7, ph=ph0)
    dU = rng.standard_normal((7, d, d + 2))
    _, _, _, T = phy.primitives(U, ph0)
    G0 = phy.viscous_flux(U, dU, ph0)
    G1 = phy.viscous_flux(U, dU, ph1)
    scale = (phy.viscosity(T, ph1) * ph1.Re)[:, None, None]
    assert np.allclose(G1, G0 * scale, rtol=1e-13, atol=1e-13 * np.abs(G0).max())
    assert not np.allclose(G1, G0, rtol=1e-3)     # temperatures differ from 1
