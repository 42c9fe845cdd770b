"""Pins of the oracle's implicit machinery (Sec. 3.2, Sec. 4.2.2, App. A):
GMRES against direct solves, the JFNK product against central differences,
the BRJ Jacobian against dense finite-difference Jacobians, JFNK-Newton
against brute-force dense Newton, SDIRK against its closed-form stability
function and order, the memory table of Sec. 5.2, and the manufactured
Poiseuille order of accuracy (Sec. 6.1)."""
import os
import numpy as np
import pytest

import workloads as w
from oracle.dg import DG
from oracle import physics as phy
from oracle import implicit as im

HERE = os.path.dirname(os.path.abspath(__file__))


def perturbed_exact(dg, seed=0, amp=0.01):
    u = dg.project_exact()
    rng = np.random.default_rng(seed)
    return u * (1 + amp * rng.standard_normal(u.shape))


# ------------------------------------------------------------------ GMRES

@pytest.mark.parametrize("ortho", ["cgs2", "mgs"])
def test_gmres_solves_dense_system(ortho):
    rng = np.random.default_rng(0)
    n = 40
    A = np.eye(n) * 3 + rng.standard_normal((n, n)) / np.sqrt(n)
    b = rng.standard_normal(n)
    x, st = im.gmres(lambda v: A @ v, b, None, im.GmresConfig(restart=15, rtol=1e-12, max_cycles=50, ortho=ortho))
    assert st.converged
    assert np.allclose(x, np.linalg.solve(A, b), rtol=1e-10, atol=1e-10)


def test_gmres_cgs2_and_mgs_same_iterations_with_preconditioner():
    rng = np.random.default_rng(1)
    n = 60
    A = np.eye(n) * 2 + rng.standard_normal((n, n)) / np.sqrt(n)
    Pinv = np.linalg.inv(np.diag(np.diag(A)) + np.triu(A, 1) * 0.5)
    b = rng.standard_normal(n)
    its = []
    for ortho in ("cgs2", "mgs"):
        x, st = im.gmres(lambda v: A @ v, b, lambda v: Pinv @ v,
                         im.GmresConfig(restart=10, rtol=1e-8, max_cycles=30, ortho=ortho))
        its.append(st.iters)
        assert np.linalg.norm(A @ x - b) <= 1e-8 * np.linalg.norm(b) * 1.0001
    assert its[0] == its[1]


# ------------------------------------------------------------------ JFNK

def test_jvp_matches_central_difference_and_is_linear():
    c = w.vortex_case(n=3, P=2)
    dg = DG(c.mesh, c.P, c.Q, c.phys)
    u = perturbed_exact(dg)
    R = dg.residual(u)
    v1 = w.random_direction(u, 1)
    v2 = w.random_direction(u, 2)
    j1 = im.jvp(dg, u, R, 0.0, v1, 0.0, 1.0)
    h = 1e-4 * np.linalg.norm(u) / np.linalg.norm(v1)
    cd = (dg.residual(u + h * v1) - dg.residual(u - h * v1)) / (2 * h)
    assert np.linalg.norm(j1 - cd) < 1e-6 * np.linalg.norm(cd)
    j2 = im.jvp(dg, u, R, 0.0, v2, 0.0, 1.0)
    j12 = im.jvp(dg, u, R, 0.0, v1 + v2, 0.0, 1.0)
    assert np.linalg.norm(j12 - j1 - j2) < 1e-6 * np.linalg.norm(j12)
    # alpha/beta combination used by Newton: dN/du v = v - dt_a dR/du v
    jn = im.jvp(dg, u, R, 0.0, v1, 1.0, -0.01)
    assert np.allclose(jn, v1 - 0.01 * j1, rtol=1e-12, atol=1e-12 * np.abs(jn).max())


def dense_jacobian(fn, u, h=1e-6):
    n = u.size
    J = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = h * max(1.0, abs(u.ravel()[k]))
        J[:, k] = (fn(u + e.reshape(u.shape)) - fn(u - e.reshape(u.shape))).ravel() / (2 * e[k])
    return J


def assemble_brj(pc, shape):
    n = int(np.prod(shape))
    Pm = np.zeros((n, n))
    nb = pc.nb
    for e in range(pc.dg.E):
        Pm[e * nb:(e + 1) * nb, e * nb:(e + 1) * nb] = pc.D[e]
    for k in range(n):
        ek = np.zeros(n)
        ek[k] = 1.0
        Pm[:, k] += pc.offdiag(ek.reshape(shape)).ravel()
    return Pm


@pytest.mark.parametrize("mk", [lambda: w.vortex_case(n=3, P=1, viscous=False),
                                lambda: w.vortex_case(n=2, P=2, viscous=False, riemann=phy.RIEMANN_HLLC),
                                lambda: w.small_tgv_case((2, 2, 1), P=1)])
def test_brj_equals_true_jacobian_when_inviscid(mk):
    """Without viscosity the two neglected terms vanish, so the kept-term
    block matrix D + (L + U) equals dN/du = I - dt_a dR/du."""
    c = mk()
    c.phys.viscous = False
    dg = DG(c.mesh, c.P, c.Q, c.phys)
    # additive noise keeps every normal velocity away from 0, where the Roe
    # flux's |u_n| has a kink (one-sided and central differences disagree)
    u = perturbed_exact(dg) + 0.02 * w.random_direction(dg.project_exact(), 5)
    dt_a = 0.01
    Nj = np.eye(u.size) - dt_a * dense_jacobian(lambda x: dg.residual(x), u)
    pc = im.BRJ(dg, u, 0.0, dt_a, J=7)
    Pm = assemble_brj(pc, u.shape)
    # tolerance: the one-sided trace difference with chi = sqrt(eps) ||u_k|| has a
    # rounding error ~ eps |H| / chi, large where a variable's norm is small
    # next to the flux (the w-momentum of the 3-D case); sign or assembly
    # mistakes give O(1) differences
    assert np.abs(Pm - Nj).max() < 1e-4 * np.abs(Nj - np.eye(u.size)).max()


@pytest.mark.parametrize("mu_law", [0, 1])
def test_brj_volume_terms_exact_with_viscosity(mu_law):
    """Terms 1-2 of Eq. Jacobian-matrix-form2 equal the Jacobian of the volume
    integral alone (viscous, including the grad-Q dependence), with constant
    mu and with Sutherland's law (whose mu(T) the complex step differentiates
    through the temperature)."""
    c = w.vortex_case(n=2, P=2, Re=5.0)
    c.phys.mu_law = mu_law
    c.phys.T_inf_K = 120.0
    dg = DG(c.mesh, c.P, c.Q, c.phys)
    u = perturbed_exact(dg)
    Jv = dense_jacobian(lambda x: dg.rhs(x, 0.0, faces=False), u)
    pc = im.BRJ.__new__(im.BRJ)
    pc.dg = dg
    T = pc._volume_jacobian(u)
    nb = dg.nv * dg.nm
    for e in range(dg.E):
        blk = Jv[e * nb:(e + 1) * nb, e * nb:(e + 1) * nb]
        assert np.abs(T[e] - blk).max() < 1e-7 * np.abs(blk).max()


def test_brj_iteration_converges_to_kept_term_solve():
    c = w.vortex_case(n=3, P=1, Re=20.0)
    dg = DG(c.mesh, c.P, c.Q, c.phys)
    u = perturbed_exact(dg)
    pc = im.BRJ(dg, u, 0.0, 0.005, J=80)
    Pm = assemble_brj(pc, u.shape)
    q = w.random_direction(u, 4)
    ref = np.linalg.solve(Pm, q.ravel())
    assert np.linalg.norm(pc.apply(q).ravel() - ref) < 1e-10 * np.linalg.norm(ref)
    # J = 1 is plain block Jacobi
    pc.J = 1
    assert np.allclose(pc.apply(q), pc.diag_solve(q))


def test_brj_memory_table():
    """Per-element storage in the paper's accounting reproduces Tab.
    BRJ-Memory-consumption with Q = ceil(3(P+1)/2) face points per direction
    (single-precision blocks), and Jacobian-Dense = 7 blocks in double."""
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "brj_memory_table.txt"))
            if l.strip() and not l.startswith("#")]
    for P, diag, off, tot, dense in ([int(v) for v in r] for r in rows):
        Q = int(np.ceil(3 * (P + 1) / 2))
        nb = 5 * (P + 1) ** 3
        pc = im.BRJ.__new__(im.BRJ)
        pc.nb = nb
        pc.dg = type("G", (), {"dim": 3, "nf": Q * Q, "nv": 5})()
        dsz, osz = pc.memory_bytes_paper_layout(4)
        assert (dsz, osz, dsz + osz) == (diag, off, tot)
        assert 7 * nb * nb * 8 == dense


# ------------------------------------------------------------------ Newton

def test_jfnk_newton_matches_dense_newton():
    c = w.vortex_case(n=2, P=1, Re=50.0)
    dg = DG(c.mesh, c.P, c.Q, c.phys)
    u0 = perturbed_exact(dg, amp=0.02)
    dt_a = 0.02
    S = u0.copy()
    cfg = im.NewtonConfig(abs_tol=1e-11, max_iters=30,
                          gmres=im.GmresConfig(restart=80, rtol=1e-10, max_cycles=5))
    pc = im.BRJ(dg, u0, 0.0, dt_a, J=3)
    uj, _, st = im.newton(dg, S, 0.0, dt_a, S, pc.apply, cfg)
    assert st.converged
    # brute force: dense FD Jacobian + LU at every Newton step
    N = lambda x: x - S - dt_a * dg.residual(x)
    ud = S.copy()
    for _ in range(10):
        J = dense_jacobian(N, ud)
        ud = ud - np.linalg.solve(J, N(ud).ravel()).reshape(ud.shape)
    assert np.linalg.norm(uj - ud) < 1e-10 * np.linalg.norm(ud)


# ------------------------------------------------------------------ SDIRK

class ScalarODE:
    """y' = f(y, t) posed as a 1-coefficient 'mesh' for the oracle's
    Newton/SDIRK drivers."""
    def __init__(self, f):
        self.f = f

    def residual(self, u, t):
        return self.f(u, t)


@pytest.mark.parametrize("name", ["sdirk2", "sdirk3", "esdirk4", "be"])
def test_sdirk_stability_function(name):
    A, b, c = im.sdirk_tableau(name)
    cfg = im.NewtonConfig(abs_tol=1e-15, gmres=im.GmresConfig(restart=2, rtol=1e-14))
    for z in (-0.5, -3.0, -40.0, 0.3):
        ode = ScalarODE(lambda u, t: z * u)
        y1, _ = im.sdirk_step(ode, np.ones((1, 1, 1)), 0.0, 1.0, name, None, cfg)
        Rz = 1 + z * b @ np.linalg.solve(np.eye(len(b)) - z * A, np.ones(len(b)))
        assert abs(y1.item() - Rz) < 1e-13 * max(1, abs(Rz))


def test_butcher_order_conditions():
    A, b, c = im.sdirk_tableau("sdirk2")
    assert abs(b.sum() - 1) < 1e-15 and abs(b @ c - 0.5) < 1e-15
    A, b, c = im.sdirk_tableau("sdirk3")
    assert abs(b.sum() - 1) < 1e-10 and abs(b @ c - 0.5) < 1e-10
    assert abs(b @ c ** 2 - 1 / 3) < 1e-10 and abs(b @ A @ c - 1 / 6) < 1e-10
    lam = A[0, 0]
    assert abs(lam ** 3 - 3 * lam ** 2 + 1.5 * lam - 1 / 6) < 1e-10


def test_esdirk4_order_conditions_and_l_stability():
    """The fourth-order table (App. A, first column read as a^{i0} = a^{i1}):
    all eight order conditions up to order 4 hold, the weights are the last
    row (stiffly accurate), the nodes are the row sums with the printed
    1/2, 5/8, 26/25, 1, and the stability function vanishes at infinity
    (L-stable)."""
    A, b, c = im.sdirk_tableau("esdirk4")
    assert np.allclose(np.diag(A)[1:], 0.25) and A[0, 0] == 0.0
    assert np.array_equal(b, A[-1])
    assert np.allclose(c[[1, 3, 4, 5]], [0.5, 5 / 8, 26 / 25, 1.0], rtol=1e-14)
    conds = [(b.sum(), 1.0), (b @ c, 1 / 2), (b @ c ** 2, 1 / 3), (b @ A @ c, 1 / 6),
             (b @ c ** 3, 1 / 4), (b @ (c * (A @ c)), 1 / 8), (b @ A @ c ** 2, 1 / 12),
             (b @ A @ A @ c, 1 / 24)]
    for got, want in conds:
        assert abs(got - want) < 1e-14
    z = -1e8
    Rz = 1 + z * b @ np.linalg.solve(np.eye(6) - z * A, np.ones(6))
    assert abs(Rz) < 1e-6


def test_bdf2_step_closed_form_and_order():
    """BDF2 on y' = z y: one step gives (4 y_n - y_{n-1}) / (3 - 2 z); on the
    nonlinear ODE of the SDIRK order test its error falls at rate 2."""
    cfg = im.NewtonConfig(abs_tol=1e-15, gmres=im.GmresConfig(restart=2, rtol=1e-14))
    for z in (-0.5, -30.0, 0.2):
        ode = ScalarODE(lambda u, t: z * u)
        y1, _ = im.bdf2_step(ode, np.full((1, 1, 1), 0.9), np.ones((1, 1, 1)), 0.0, 1.0, None, cfg)
        assert abs(y1.item() - (4 * 0.9 - 1.0) / (3 - 2 * z)) < 1e-13
    f = lambda u, t: -u * u + np.cos(t)
    cfg = im.NewtonConfig(abs_tol=1e-15, max_iters=30, gmres=im.GmresConfig(restart=2, rtol=1e-14))
    ode = ScalarODE(f)

    def run(n):
        dt = 1.0 / n
        y0 = np.full((1, 1, 1), 0.5)
        y1, _ = im.sdirk_step(ode, y0, 0.0, dt, "esdirk4", None, cfg)   # start-up step
        for k in range(1, n):
            y0, (y1, _) = y1, im.bdf2_step(ode, y1, y0, k * dt, dt, None, cfg)
        return y1.item()

    ref = run(1024)
    e1, e2 = abs(run(32) - ref), abs(run(64) - ref)
    assert np.log2(e1 / e2) > 2 - 0.3


@pytest.mark.parametrize("name,order", [("sdirk2", 2), ("sdirk3", 3), ("esdirk4", 4), ("be", 1)])
def test_sdirk_order_on_nonlinear_ode(name, order):
    f = lambda u, t: -u * u + np.cos(t)
    cfg = im.NewtonConfig(abs_tol=1e-15, max_iters=30, gmres=im.GmresConfig(restart=2, rtol=1e-14))
    ode = ScalarODE(f)

    def run(n):
        y, dt = np.full((1, 1, 1), 0.5), 1.0 / n
        for k in range(n):
            y, _ = im.sdirk_step(ode, y, k * dt, dt, name, None, cfg)
        return y.item()

    ref = run(512)
    e1, e2 = abs(run(16) - ref), abs(run(32) - ref)
    assert np.log2(e1 / e2) > order - 0.3


# ------------------------------------------------------------------ order of accuracy

def steady_state(dg, u, max_steps=16):
    """Pseudo-transient continuation to R(u) = 0: each step is one Newton step
    of backward Euler from u (solve (I - dt dR/du) x = dt R(u) by BRJ(7)
    preconditioned JFNK GMRES, u += x), dt growing tenfold per step; stops
    when ||R|| has not halved over two steps (its rounding floor)."""
    dt, hist = 1.0, []
    for _ in range(max_steps):
        R = dg.residual(u)
        hist.append(np.linalg.norm(R))
        if len(hist) > 2 and hist[-1] > 0.5 * min(hist[:-2]):
            break
        pc = im.BRJ(dg, u, 0.0, dt, J=7)
        A = lambda v, u=u, R=R, dt=dt: im.jvp(dg, u, R, 0.0, v, 1.0, -dt)
        x, _ = im.gmres(A, dt * R, pc.apply, im.GmresConfig(restart=40, rtol=1e-4, max_cycles=5))
        u = u + x
        dt = min(10.0 * dt, 1e12)
    return u, hist


def poiseuille_error(P, nx, ny):
    c = w.poiseuille_case(P, nx=nx, ny=ny)
    dg = DG(c.mesh, c.P, c.Q, c.phys)
    u, hist = steady_state(dg, dg.project_exact())
    e = dg.l2_error(u, lambda x: phy.exact_state(c.phys, x, 0.0))
    return float(np.linalg.norm(e)), hist


@pytest.mark.slow
@pytest.mark.parametrize("P,ny", [(1, 4), (2, 4), (3, 2), (4, 2), (5, 2), (6, 2)])
def test_poiseuille_steady_order_of_accuracy(P, ny):
    """Steady solves of the manufactured Poiseuille flow (weak Dirichlet
    inflow/outflow, isothermal walls, App. B forcing) converge at the design
    order P+1 in L2 (Sec. 6.1: all four variables), h-refining the
    wall-clustered y-spacing of the channel family (ratio 1.1 from each wall)
    from ny to 2 ny cells: the exact solution is linear in x (p and E) or
    independent of x, which two elements in x represent exactly, so the
    x-resolution does not enter the error.  The device runs the same check on
    the 4x2, 8x4, 16x8 family itself."""
    e1, _ = poiseuille_error(P, 2, ny)
    e2, h2 = poiseuille_error(P, 2, 2 * ny)
    assert h2[-1] < 1e-6
    assert np.log2(e1 / e2) > P + 1 - 0.3, (P, e1, e2)


# ------------------------------------------------------------------ JFNK epsilon

def test_jfnk_eps_is_the_paper_formula_for_unit_directions():
    """Eq. eps-JF: eps = ||u||_2 sqrt(eps_hat) with eps_hat the double-precision
    machine epsilon 2.22e-16 (Krylov directions have unit norm).  For other
    directions the perturbation eps v keeps the norm sqrt(eps_hat) ||u||, so
    eps scales as 1/||v||; u = 0 takes sqrt(eps_hat) / ||v||."""
    rng = np.random.default_rng(3)
    u = rng.standard_normal((4, 3, 5))
    v = rng.standard_normal((4, 3, 5))
    v1 = v / np.sqrt(np.sum(v * v))
    eps_hat = np.finfo(np.float64).eps
    assert eps_hat == pytest.approx(2.22e-16, rel=2e-3)
    assert im.jfnk_eps(u, v1) == pytest.approx(np.sqrt(eps_hat) * np.sqrt(np.sum(u * u)), rel=1e-14)
    for c in (1e-6, 3.0, 1e6):
        assert im.jfnk_eps(u, c * v1) == pytest.approx(im.jfnk_eps(u, v1) / c, rel=1e-14)
    assert im.jfnk_eps(np.zeros_like(u), 5 * v1) == pytest.approx(np.sqrt(eps_hat) / 5, rel=1e-14)


def test_jvp_is_homogeneous_in_the_direction():
    """With eps ~ 1/||v|| the perturbed state u + eps v does not depend on the
    scale of v, so J(c v) = c J(v) to rounding for any c; without the 1/||v||
    factor a direction of norm 1e6 ||u|| would perturb u by 1e-2 ||u|| and the
    finite difference would carry an O(1e-2) nonlinear error."""
    c = w.vortex_case(n=3, P=2)
    dg = DG(c.mesh, c.P, c.Q, c.phys)
    u = perturbed_exact(dg)
    R = dg.residual(u)
    v = w.random_direction(u, 8)
    j1 = im.jvp(dg, u, R, 0.0, v, 0.0, 1.0)
    for s in (1e-6, 1e6):
        js = im.jvp(dg, u, R, 0.0, s * v, 0.0, 1.0)
        assert np.linalg.norm(js / s - j1) < 1e-9 * np.linalg.norm(j1)


# ------------------------------------------------------------------ terms 4-5 of the Jacobian

@pytest.mark.parametrize("mk", [lambda: w.vortex_case(n=3, P=1, Re=20.0),
                                lambda: w.poiseuille_case(2, nx=2, ny=2, Re=10.0),
                                lambda: w.small_tgv_case((2, 2, 1), P=1, Re=20.0)])
def test_brj_with_all_five_terms_equals_the_viscous_jacobian(mk):
    """With viscosity, the kept-term block matrix D + (L + U) misses the
    trace-gradient and symmetric-flux terms 4-5 of Eq. Jacobian-matrix-form2;
    with them it equals dN/du = I - dt_a dR/du (dense central differences),
    to the rounding of the one-sided trace differences; without them it
    does not (periodic, Dirichlet and wall faces)."""
    c = mk()
    dg = DG(c.mesh, c.P, c.Q, c.phys)
    u = perturbed_exact(dg) + 0.02 * w.random_direction(dg.project_exact(), 5)
    dt_a = 0.01
    Nj = np.eye(u.size) - dt_a * dense_jacobian(lambda x: dg.residual(x), u)
    scale = np.abs(Nj - np.eye(u.size)).max()
    full = assemble_brj(im.BRJ(dg, u, 0.0, dt_a, J=7, full=True), u.shape)
    kept = assemble_brj(im.BRJ(dg, u, 0.0, dt_a, J=7), u.shape)
    assert np.abs(full - Nj).max() < 1e-4 * scale
    assert np.abs(kept - Nj).max() > 1e-2 * scale
