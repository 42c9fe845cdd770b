"""Shock capturing on the device (Sec. 3.1.2) against the oracle: the modal
sensor's per-element factor mu_0 S_e h_e / P, the residual with the
artificial viscosity and conductivity in the volume and face diffusion
fluxes, the JFNK product (which differentiates the sensor too), the BRJ
preconditioner that holds mu_av at its linearisation state (Sec. 4.2.2 drops
d mu_av / du from the preconditioning matrices), and SDIRK2 steps of the
SWBLI-like workload (Sec. 6.5: Dirichlet inflow with the Rankine-Hugoniot
state, far field on top, adiabatic wall below).

Test states: (a) on the 12 x 6 wall-clustered SWBLI mesh, the L2
projection of a contact discontinuity along the shock line (density 1
below, R above; the oracle projects it), whose elements on the line have
the sensor in its ramp and, for R = 8 at P = 3 with a ramp of half-width
0.5, at 1 (the projection's overshoots leave negative densities at some
points, so this state serves the sensor alone); (b) the projected oblique
shock at 50 degrees with the SWBLI boundaries; (c) "bubble" states: the
projected vortex (2-D) or Taylor-Green (3-D, affine and curved) field whose
density gets, per element, a seeded amplitude a_e from 1e-2 to 150..1000 of
the highest interior mode (the only one of degree P) plus a_e max|mode| on
the vertex modes, so the density stays positive while the sensor spans 0,
its ramp and 1 over the elements.

Bounds: factors to 1e-10 of the largest (the sensor's log10 of an energy
ratio is computed from modal coefficients on the device and from Gauss-point
values in the oracle); the residual is the method's residual plus the AV
diffusion term dR, each held to the rule of the other residual parity tests,
max(1e-12, 16 s) with s its own rounding floor at u (the oracle's relative
change under a one-ulp perturbation of u), so that ||R_gpu - R_or|| <=
max(1e-12, 16 s) ||R|| + max(1e-12, 16 s_av) ||dR||; with Ducros' sensor
(av = 2) s_av also covers the rounding of the velocity gradients the ratio
receives, at the level of the device's route to them (collocation derivative
on the Gauss grid, then extrapolation to the faces);
JFNK product by the residual difference at u + eps v over eps; BRJ apply
1e-6 (FP64 blocks); SDIRK with equal Newton and GMRES counts and u^{n+1} to
1e-9."""
import copy
import itertools

import numpy as np
import pytest
import torch

import workloads as w
from oracle.dg import DG
from oracle import implicit as im
from oracle import physics as phy

pytestmark = pytest.mark.gpu

R_TOL = 1e-12
JVP_TOL = 1e-6


@pytest.fixture(scope="module")
def dgl():
    import paper_2002_04222_gb300 as dgl
    return dgl


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def contact(ph, R, beta=30.8, xsh=1.0):
    """Density 1 below the line y = (xsh - x) tan(beta) and R above it, the
    stream velocity (1, 0) and pressure 1/(gamma Ma^2) on both sides."""
    def field(x):
        up = x[..., 1] > (xsh - x[..., 0]) * np.tan(np.radians(beta))
        rho = np.where(up, R, 1.0)
        vel = np.zeros(x.shape[:-1] + (2,))
        vel[..., 0] = 1.0
        p = np.full(x.shape[:-1], 1.0 / (ph.gamma * ph.Ma ** 2))
        return phy.conservative(rho, vel, p, ph)
    return field


def contact_state(P, R, kappa):
    c = w.swbli_case(nx=12, ny=6, P=P)
    c.phys.av_kappa = kappa
    dg = DG(c.mesh, c.P, c.Q, c.phys)
    return c, dg, dg.project(contact(c.phys, R))


def shock_state(P=3, beta=50.0):
    c = w.swbli_case(nx=12, ny=6, P=P)
    c.phys.fpar = (beta, 1.0)
    dg = DG(c.mesh, c.P, c.Q, c.phys)
    return c, dg, dg.project_exact()


def bubble_state(c, kappa, amax, seed=5):
    c.phys.av = 1
    c.phys.av_kappa = kappa
    dg = DG(c.mesh, c.P, c.Q, c.phys)
    u = dg.project_exact()
    P, N, d = c.P, c.P + 1, dg.dim
    amp = np.geomspace(1e-2, amax, dg.E)
    np.random.default_rng(seed).shuffle(amp)
    top = sum((P - 1) * N ** k for k in range(d))     # psi_{P-1} in every direction
    K = np.abs(dg.B[:, top]).max()
    for idx in itertools.product((0, P), repeat=d):    # the vertex modes sum to 1
        u[:, 0, sum(i * N ** k for k, i in enumerate(idx))] += amp * K
    u[:, 0, top] += amp
    return c, dg, u


STATES = {
    "contact_P3_R8_k0.5": lambda: contact_state(3, 8.0, 0.5),
    "contact_P2_R4_k1": lambda: contact_state(2, 4.0, 1.0),
    "shock50_P3": lambda: shock_state(3, 50.0),
    "bubble_vortex_P3_k0.5": lambda: bubble_state(w.vortex_case(n=6, P=3), 0.5, 150.0),
    "bubble_vortex_P2_k0.25": lambda: bubble_state(w.vortex_case(n=6, P=2), 0.25, 150.0),
    "bubble_box_P3_k0.5": lambda: bubble_state(w.small_tgv_case((3, 2, 2), P=3), 0.5, 1000.0),
    "bubble_wavy_P2_Q5_k0.5": lambda: bubble_state(w.wavy_box_case((2, 2, 2), P=2), 0.5, 1000.0),
}
PHYSICAL = sorted(k for k in STATES if not k.startswith("contact"))
DUCROS = ["bubble_box_P3_k0.5", "bubble_vortex_P3_k0.5", "bubble_wavy_P2_Q5_k0.5", "shock50_P3"]


def state(name, mode=1):
    """A test state with the modal sensor alone (mode 1) or times Ducros'
    sensor at each point (mode 2)."""
    c, dg, u = STATES[name]()
    c.phys.av = mode
    return c, dg, u


def tag(name, mode):
    return name if mode == 1 else name + "_ducros"


def gradient_rounding_gain(Q):
    """Sum |l_k(1)| of the Lagrange extrapolation from the Q Gauss points to
    the end point times the row-sum norm of the Gauss-point collocation
    derivative: the factor by which the device's route to a face gradient
    (collocation derivative, then extrapolation) can scale rounding."""
    x, _ = np.polynomial.legendre.leggauss(Q)
    lam = sum(abs(np.prod([(1.0 - x[j]) / (x[k] - x[j]) for j in range(Q) if j != k]))
              for k in range(Q))
    V = np.polynomial.legendre.legvander(x, Q - 1)
    dV = np.stack([np.polynomial.legendre.legval(x, np.polynomial.legendre.legder(np.eye(Q)[k]))
                   for k in range(Q)], 1)
    return lam * np.abs(dV @ np.linalg.inv(V)).sum(axis=1).max()


def ducros_floor(dg, u, R, dR, monkeypatch):
    """Relative change of the AV term dR when the velocity gradients that
    Ducros' ratio receives carry rounding at the level of the device's gradient
    route (2^-52 x gradient_rounding_gain(Q) x the largest gradient entry of the
    point): the ratio is non-linear in the gradient, so this rounding reaches R
    through it and not only through the linear diffusion flux."""
    gain = gradient_rounding_gain(dg.Q)
    orig = phy.ducros
    rng = np.random.default_rng(7)
    out = 0.0
    for _ in range(3):
        def perturbed(U, dU, ph):
            scale = np.abs(dU).max(axis=(-2, -1), keepdims=True)
            return orig(U, dU + 2.0 ** -52 * gain * scale * rng.standard_normal(dU.shape), ph)
        monkeypatch.setattr(phy, "ducros", perturbed)
        out = max(out, np.linalg.norm(dg.residual(u) - R) / np.linalg.norm(dR))
        monkeypatch.setattr(phy, "ducros", orig)
    return out


@pytest.mark.parametrize("beta,smooth", [(30.8, False), (50.0, False), (30.8, True)])
def test_shock_field_projection_parity(dgl, beta, smooth):
    """The device's oblique-shock field (both sides of the line; sharp, or
    smoothed over 0.02 with the wall layer 0.01 of the SWBLI workload)
    projected like the oracle's: mass-weighted relative difference 1e-13, as
    for the other analytic fields."""
    if smooth:
        c = w.swbli_case(nx=12, ny=6, P=3)
        dg = DG(c.mesh, c.P, c.Q, c.phys)
        ref = dg.project_exact()
    else:
        c, dg, ref = shock_state(3, beta)
    m = dgl.Mesh.from_case(c)
    got = m.project(0.0).cpu().numpy()
    Mx = np.linalg.inv(dg.Minv)
    mass = lambda x: np.einsum("emn,evn->evm", Mx, x)
    assert rel(mass(got), mass(ref)) < 1e-13


@pytest.mark.parametrize("name", sorted(STATES))
def test_sensor_factor_parity(dgl, name, parity_record):
    c, dg, u = STATES[name]()
    m = dgl.Mesh.from_case(c)
    ref = dg.av_factor(u)
    S = dg.sensor(u)
    got = m.av_factor(to_dev(u)).cpu().numpy()
    err = float(np.abs(got - ref).max() / ref.max())
    parity_record("av_factor", name, "max|f_gpu-f_or|/max f_or", err, 1e-10,
                  ramp=int(((S > 0) & (S < 1)).sum()), full=int((S == 1).sum()),
                  zero=int((S == 0).sum()))
    assert ((S > 0) & (S < 1)).sum() > 0              # the ramp is exercised
    assert err < 1e-10, err
    assert np.all(got[ref == 0.0] == 0.0)            # smooth elements: no viscosity
    if name in ("contact_P3_R8_k0.5", "bubble_vortex_P3_k0.5", "bubble_box_P3_k0.5"):
        assert (S == 1).sum() > 0
        h = dg.h_elem
        assert np.allclose(got[S == 1], c.phys.av_mu0 * h[S == 1] / c.P, rtol=1e-14)


@pytest.mark.parametrize("name,mode", [(n, 1) for n in PHYSICAL] + [(n, 2) for n in DUCROS])
def test_residual_parity_with_artificial_viscosity(dgl, name, mode, parity_record, monkeypatch):
    c, dg, u = state(name, mode)
    m = dgl.Mesh.from_case(c)
    R_ref = dg.residual(u, 0.0)
    R = m.residual(to_dev(u)).cpu().numpy()
    ph0 = copy.copy(c.phys)                    # dg keeps c.phys: change a copy
    ph0.av = 0
    dg0 = DG(c.mesh, c.P, c.Q, ph0)
    R_plain = dg0.residual(u, 0.0)
    dR = R_ref - R_plain                       # the artificial-viscosity contribution
    rng = np.random.default_rng(123)
    s = s_av = 0.0
    for _ in range(3):
        up = u * (1 + 2.0 ** -52 * rng.standard_normal(u.shape))
        Rp, R0p = dg.residual(up), dg0.residual(up)
        s = max(s, rel(Rp, R_ref))
        s_av = max(s_av, rel(Rp - R0p, dR))
    # with Ducros' sensor the AV term's floor also carries the gradient rounding
    # the ratio amplifies
    s_grad = ducros_floor(dg, u, R_ref, dR, monkeypatch) if mode == 2 else 0.0
    # R is the method's residual plus the AV diffusion term; each operator is
    # held to the residual rule max(1e-12, 16 s) with its own floor, and the
    # bound on R is the sum of the two parts' bounds
    tol = (max(R_TOL, 16.0 * s) * np.linalg.norm(R_ref)
           + max(R_TOL, 16.0 * max(s_av, s_grad)) * np.linalg.norm(dR)) / np.linalg.norm(R_ref)
    parity_record("residual_av", tag(name, mode), "||R_gpu-R_or||/||R_or||", rel(R, R_ref), tol, floor_s=s,
                  floor_s_av=s_av, floor_s_grad=s_grad, av_effect=rel(R_plain, R_ref))
    assert rel(R_plain, R_ref) > 1e-6          # the test is not vacuous
    assert s < 1e-10 and s_av < 1e-10          # floors of FP64 evaluations
    assert rel(R, R_ref) < tol, (rel(R, R_ref), tol)


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("name", ["bubble_vortex_P3_k0.5", "bubble_box_P3_k0.5", "shock50_P3"])
def test_jvp_parity_with_artificial_viscosity(dgl, name, mode, parity_record):
    c, dg, u = state(name, mode)
    m = dgl.Mesh.from_case(c)
    v = w.random_direction(u, 7)
    R = dg.residual(u)
    ud, Rd, vd = to_dev(u), to_dev(R), to_dev(v)
    eps = im.jfnk_eps(u, v)
    wv = u + eps * v
    dR = np.linalg.norm(m.residual(to_dev(wv)).cpu().numpy() - dg.residual(wv))
    for alpha, beta in ((0.0, 1.0), (1.0, -0.002)):
        ref = im.jvp(dg, u, R, 0.0, v, alpha, beta)
        got = m.jvp(ud, Rd, vd, 0.0, alpha, beta).cpu().numpy()
        bound = max(JVP_TOL, 4 * abs(beta) * dR / eps / np.linalg.norm(ref))
        parity_record("jvp_av", f"{tag(name, mode)}_alpha{alpha:g}", "||Jv_gpu-Jv_or||/||Jv_or||",
                      rel(got, ref), bound)
        assert rel(got, ref) < bound, (rel(got, ref), bound)


@pytest.mark.parametrize("name,full,mode", [("bubble_vortex_P3_k0.5", False, 1), ("shock50_P3", False, 1),
                                            ("bubble_box_P3_k0.5", False, 1),
                                            ("bubble_vortex_P2_k0.25", True, 1),
                                            ("bubble_vortex_P3_k0.5", False, 2),
                                            ("bubble_box_P3_k0.5", False, 2), ("shock50_P3", False, 2)])
def test_brj_apply_parity_with_frozen_artificial_viscosity(dgl, name, full, mode, parity_record):
    c, dg, u = state(name, mode)
    m = dgl.Mesh.from_case(c)
    dt_a = 0.002
    q = w.random_direction(u, 3)
    ref_pc = im.BRJ(dg, u, 0.0, dt_a, J=7, full=full)
    ref = ref_pc.apply(q)
    pc = dgl.Precond(m).build(to_dev(u), 0.0, dt_a, J=7, full_jacobian=full)
    got = pc.apply(to_dev(q)).cpu().numpy()
    ph0 = copy.copy(c.phys)
    ph0.av = 0
    plain = im.BRJ(DG(c.mesh, c.P, c.Q, ph0), u, 0.0, dt_a, J=7, full=full).apply(q)
    parity_record("brj_apply_av", f"{tag(name, mode)}{'_full' if full else ''}",
                  "||P^-1q_gpu-P^-1q_or||/||P^-1q_or||", rel(got, ref), 1e-6,
                  av_effect=rel(plain, ref))
    assert rel(plain, ref) > 1e-5                   # mu_av is in the blocks
    assert rel(got, ref) < 1e-6


def test_sdirk2_steps_on_the_oblique_shock(dgl, parity_record):
    """Two SDIRK2 steps (dt = 0.005, BRJ(7) rebuilt each step, GMRES(20)) of
    the 50-degree shock at P = 3: equal Newton and GMRES counts per stage and
    the same state."""
    c, dg, u0 = shock_state(3, 50.0)
    m = dgl.Mesh.from_case(c)
    dt, lam = 0.005, 1 - np.sqrt(2) / 2
    cfg = im.NewtonConfig(alpha=1e-3, gmres=im.GmresConfig(restart=20))
    u_ref, ud = u0, to_dev(u0)
    pc = dgl.Precond(m)
    for k in range(2):
        pc_ref = im.BRJ(dg, u_ref, k * dt, dt * lam, J=7)
        u_ref, st_ref = im.sdirk_step(dg, u_ref, k * dt, dt, "sdirk2", pc_ref.apply, cfg)
        st = m.sdirk_step(ud, k * dt, dt, precond=pc, rebuild=True, restart=20, J=7)
        assert st["converged"]
        assert st["stage_newton"] == [s.iters for s in st_ref.stages], (k, st, st_ref)
        assert st["stage_gmres"] == [s.gmres_iters for s in st_ref.stages], (k, st, st_ref)
    err = rel(ud.cpu().numpy(), u_ref)
    parity_record("sdirk2_shock", "shock50_P3_2steps", "||u2_gpu-u2_or||/||u2_or||", err, 1e-9,
                  newton=st["stage_newton"], gmres=st["stage_gmres"])
    assert err < 1e-9


def test_zero_coefficient_leaves_the_residual_unchanged(dgl):
    """av = 1 with mu_0 = 0: every factor is zero and the residual equals the
    one without shock capturing bit for bit."""
    c, dg, u = STATES["shock50_P3"]()
    c.phys.av_mu0 = 0.0
    m0 = dgl.Mesh.from_case(c)
    assert torch.all(m0.av_factor(to_dev(u)) == 0)
    c.phys.av = 0
    m1 = dgl.Mesh.from_case(c)
    assert torch.equal(m0.residual(to_dev(u)), m1.residual(to_dev(u)))


def test_shock_capturing_needs_the_diffusion_flux(dgl):
    from paper_2002_04222_gb300 import _lib
    c, _, _ = STATES["shock50_P3"]()
    c.phys.viscous = False
    with pytest.raises(_lib.DGError) as ei:
        dgl.Mesh.from_case(c)
    assert ei.value.code == -1
    c.phys.viscous, c.phys.av = True, 0
    m = dgl.Mesh.from_case(c)
    with pytest.raises(_lib.DGError) as ei:
        m.av_factor(m.project(0.0))
    assert ei.value.code == -6


def test_ducros_option_refuses_the_trace_gradient_terms(dgl):
    """Terms 4-5 (full_jacobian) are not built with Ducros' sensor: the build
    says so instead of holding a viscosity it cannot form."""
    from paper_2002_04222_gb300 import _lib
    c, dg, u = state("bubble_vortex_P2_k0.25", 2)
    m = dgl.Mesh.from_case(c)
    with pytest.raises(_lib.DGError) as ei:
        dgl.Precond(m).build(to_dev(u), 0.0, 0.002, J=7, full_jacobian=True)
    assert ei.value.code == -6
