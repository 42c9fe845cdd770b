"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle on
the same seeded inputs: residual (1e-12 relative), projection, JFNK product
(1e-6 relative: the difference quotient amplifies rounding of R by 1/eps),
BRJ apply, GMRES and SDIRK (equal Newton and GMRES iteration counts)."""
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
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def perturbed(dg, seed=0, amp=0.01):
    u = dg.project_exact()
    return u + amp * w.random_direction(u, seed)


def sutherland(c, T_inf=120.0):
    """The case with Sutherland's law (T_inf = 120 K: S/T_inf = 0.92, so mu
    moves with T by about as much as T does)."""
    c.phys.mu_law = 1
    c.phys.T_inf_K = T_inf
    return c


CASES = {
    "vortex8_P2": lambda: w.vortex_case(n=8, P=2),
    "vortex_sutherland_P2": lambda: sutherland(w.vortex_case(n=5, P=2)),
    "box_sutherland_P3_Q6": lambda: sutherland(w.small_tgv_case((3, 2, 2), P=3)),
    "vortex_hllc_P3": lambda: w.vortex_case(n=5, P=3, Q=5, riemann=phy.RIEMANN_HLLC),
    "vortex_euler_P2": lambda: w.vortex_case(n=4, P=2, viscous=False),
    "poiseuille_P1": lambda: w.poiseuille_case(1),
    "poiseuille_P3": lambda: w.poiseuille_case(3, nx=6, ny=4),
    "poiseuille_P6": lambda: w.poiseuille_case(6, nx=4, ny=2),
    "box_P1": lambda: w.small_tgv_case((3, 2, 2), P=1),
    "box_P2_Q4": lambda: w.small_tgv_case((3, 3, 2), P=2, Q=4, stretch=True),
    "box_P3_Q6": lambda: w.small_tgv_case((3, 2, 3), P=3),
    "box_P4_Q8": lambda: w.small_tgv_case((2, 2, 2), P=4, riemann=phy.RIEMANN_HLLC),
}


def mass(dg, x):
    """M x per element (the weak-form vector of a modal field)."""
    return np.einsum("emn,evn->evm", np.linalg.inv(dg.Minv), x)


def rounding_floor(dg, u, R, trials=3, weak=False):
    """Relative change of the oracle's R (or of L = M R) under a one-ulp random
    relative perturbation of u: the FP64 rounding floor of the operator at u
    (two correct FP64 evaluations in different orders differ by a small
    multiple of it)."""
    rng = np.random.default_rng(123)
    out = 0.0
    for _ in range(trials):
        up = u * (1 + 2.0 ** -52 * rng.standard_normal(u.shape))
        if weak:
            out = max(out, rel(dg.rhs(up), dg.rhs(u)))
        else:
            out = max(out, rel(dg.residual(up), R))
    return out


@pytest.mark.parametrize("name", sorted(CASES))
def test_residual_parity(dgl, name, parity_record):
    """||R_gpu - R_oracle|| / ||R_oracle|| <= max(1e-12, 16 s), s = the
    oracle's rounding floor at u (its relative change under a one-ulp
    perturbation of u); the achieved error is recorded beside s."""
    c = CASES[name]()
    dg = DG(c.mesh, c.P, c.Q, c.phys)
    m = dgl.Mesh.from_case(c)
    u = perturbed(dg)
    R_ref = dg.residual(u, 0.0)
    R = m.residual(to_dev(u)).cpu().numpy()
    s = rounding_floor(dg, u, R_ref)
    tol = max(R_TOL, 16.0 * s)
    err = rel(R, R_ref)
    parity_record("residual", name, "||R_gpu-R_or||/||R_or||", err, tol, floor_s=s,
                  meets_1e12=bool(err < 1e-12))
    assert err < tol, (err, tol)
    assert np.abs(R - R_ref).max() < 10 * tol * np.abs(R_ref).max()
    # the weak form L = M R (no mass-matrix amplification); the kernels
    # differentiate by collocation on the Q-point Gauss grid, whose matrix norm
    # (~Q^2/2) multiplies their rounding, hence the wider factor
    L, L_ref = mass(dg, R), mass(dg, R_ref)
    sL = rounding_floor(dg, u, R_ref, weak=True)
    tolL = max(R_TOL, 64.0 * sL)
    parity_record("residual_weak_form", name, "||L_gpu-L_or||/||L_or||", rel(L, L_ref), tolL,
                  floor_s=sL)
    assert rel(L, L_ref) < tolL, rel(L, L_ref)


@pytest.mark.parametrize("name", ["vortex8_P2", "poiseuille_P3", "box_P3_Q6"])
def test_projection_parity(dgl, name):
    c = CASES[name]()
    dg = DG(c.mesh, c.P, c.Q, c.phys)
    m = dgl.Mesh.from_case(c)
    ref = dg.project_exact(0.0)
    got = m.project(0.0).cpu().numpy()
    # mass-weighted (backward) error: both sides solve M u = B^T W U(x); the
    # forward error carries cond(M) ~ 1e5 of the 3-D modal mass matrix
    assert rel(mass(dg, got), mass(dg, ref)) < 1e-13
    assert rel(got, ref) < 1e-10


def test_residual_repeats_bitwise(dgl):
    c = CASES["box_P3_Q6"]()
    m = dgl.Mesh.from_case(c)
    u = to_dev(perturbed(DG(c.mesh, c.P, c.Q, c.phys)))
    a = m.residual(u)
    b = m.residual(u)
    assert torch.equal(a, b)


@pytest.mark.parametrize("name", ["vortex8_P2", "poiseuille_P3", "box_P2_Q4", "box_P3_Q6",
                                  "vortex_sutherland_P2", "box_sutherland_P3_Q6"])
def test_jvp_parity(dgl, name, parity_record):
    c = CASES[name]()
    dg = DG(c.mesh, c.P, c.Q, c.phys)
    m = dgl.Mesh.from_case(c)
    u = perturbed(dg)
    v = w.random_direction(u, 7)
    R = dg.residual(u)
    ud, Rd, vd = to_dev(u), to_dev(R), to_dev(v)
    # the difference quotient divides the residual's GPU/oracle difference at
    # u + eps v by eps: measure that difference and bound the product by it
    eps = im.jfnk_eps(u, v)
    wv = u + eps * v
    dR = np.linalg.norm(m.residual(to_dev(wv)).cpu().numpy() - dg.residual(wv))
    for alpha, beta in ((0.0, 1.0), (1.0, -0.013)):
        ref = im.jvp(dg, u, R, 0.0, v, alpha, beta)
        got = m.jvp(ud, Rd, vd, 0.0, alpha, beta).cpu().numpy()
        bound = max(JVP_TOL, 4 * abs(beta) * dR / eps / np.linalg.norm(ref))
        parity_record("jvp", f"{name}_alpha{alpha:g}", "||Jv_gpu-Jv_or||/||Jv_or||",
                      rel(got, ref), bound)
        assert rel(got, ref) < bound, (rel(got, ref), bound)
    zero = m.jvp(ud, Rd, torch.zeros_like(vd), 0.0, 1.0, -0.1).cpu().numpy()
    assert np.all(zero == 0.0)


@pytest.mark.parametrize("name", ["vortex8_P2", "box_P3_Q6"])
def test_jvp_homogeneous_in_the_direction(dgl, name, parity_record):
    """Eq. eps-JF scaled by 1/||v||: the perturbed state u + eps v does not
    depend on the scale of v, so the device's J(c v) equals c J(v) to rounding
    for c = 1e-6 and 1e6 (a missing 1/||v|| would perturb u by 1e-2 ||u|| at
    c = 1e6 and change the product by O(1e-2))."""
    c = CASES[name]()
    dg = DG(c.mesh, c.P, c.Q, c.phys)
    m = dgl.Mesh.from_case(c)
    u = to_dev(perturbed(dg))
    R = m.residual(u)
    v = to_dev(w.random_direction(u.cpu().numpy(), 9))
    j1 = m.jvp(u, R, v, 0.0, 0.0, 1.0)
    for sc in (1e-6, 1e6):
        js = m.jvp(u, R, v * sc, 0.0, 0.0, 1.0)
        err = (torch.linalg.norm(js / sc - j1) / torch.linalg.norm(j1)).item()
        parity_record("jvp_homogeneity", f"{name}_c{sc:g}", "||J(cv)/c-J(v)||/||J(v)||", err, 1e-9)
        assert err < 1e-9, (sc, err)


def test_free_stream_and_conservation_on_gpu(dgl):
    c = w.small_tgv_case((3, 2, 2), P=3)
    dg = DG(c.mesh, c.P, c.Q, c.phys)
    m = dgl.Mesh.from_case(c)
    one = np.round(dg.one_coeffs(), 10)
    U0 = phy.exact_state(c.phys, np.zeros((1, 3)), 0.0)[0]
    u = U0[None, :, None] * one[None, None, :] * np.ones((dg.E, 1, 1))
    R = m.residual(to_dev(u)).cpu().numpy()
    Mx = np.linalg.inv(dg.Minv)
    L = np.einsum("emn,evn->evm", Mx, R)
    scale = np.abs(np.einsum("emn,evn->evm", Mx, dg.apply_minv(dg.rhs(u, faces=False)))).sum(axis=2).max()
    assert np.abs(L).max() < 1e-12 * scale
    ur = perturbed(dg, amp=0.05)
    R = m.residual(to_dev(ur)).cpu().numpy()
    L = np.einsum("emn,evn->evm", Mx, R)
    tot = np.einsum("evm,m->v", L, dg.one_coeffs())
    assert np.all(np.abs(tot) < 1e-12 * np.abs(L).sum(axis=(0, 2)))


@pytest.mark.parametrize("name,precision,tol", [("vortex8_P2", "fp64", 1e-6),
                                                ("poiseuille_P3", "fp64", 1e-6),
                                                ("box_P2_Q4", "fp64", 1e-6),
                                                ("box_P2_Q4", "fp32", 1e-4),
                                                ("box_P3_Q6", "bf16", 3e-2),
                                                ("box_P4_Q8", "fp32", 1e-4),
                                                ("box_P3_Q6", "fp32-tc", 1e-4),
                                                ("box_P4_Q8", "fp32-tc", 1e-4),
                                                ("vortex_sutherland_P2", "fp64", 1e-6),
                                                ("box_sutherland_P3_Q6", "fp32", 1e-4)])
def test_precond_apply_parity(dgl, name, precision, tol, parity_record):
    c = CASES[name]()
    dg = DG(c.mesh, c.P, c.Q, c.phys)
    m = dgl.Mesh.from_case(c)
    u = perturbed(dg)
    dt_a = 0.02
    ref_pc = im.BRJ(dg, u, 0.0, dt_a, J=7)
    q = w.random_direction(u, 3)
    # "fp32-tc": FP32 blocks inverted with the tensor-core trailing updates
    tc = precision.endswith("-tc")
    precision = precision.replace("-tc", "")
    if precision == "fp32":
        # the device assembles FP32 blocks: at high order its rounding, after
        # cancellation in the volume sums, exceeds 1e-4; bound by 4x the
        # oracle's own float32-assembly difference
        ref32 = im.BRJ(dg, u, 0.0, dt_a, J=7, assembly_dtype=np.float32).apply(q)
        tol = max(tol, 4 * rel(ref32, ref_pc.apply(q)))
    ref = ref_pc.apply(q)
    pc = dgl.Precond(m).build(to_dev(u), 0.0, dt_a, J=7, precision=precision, tc_invert=tc)
    got = pc.apply(to_dev(q)).cpu().numpy()
    tag = f"{name}_{precision}{'_tc' if tc else ''}"
    parity_record("brj_apply_J7", tag, "||P^-1q_gpu-P^-1q_or||/||P^-1q_or||", rel(got, ref), tol)
    assert rel(got, ref) < tol
    # J = 1 is plain block Jacobi
    ref_pc.J = 1
    pc1 = dgl.Precond(m).build(to_dev(u), 0.0, dt_a, J=1, precision=precision, tc_invert=tc)
    err1 = rel(pc1.apply(to_dev(q)).cpu().numpy(), ref_pc.apply(q))
    parity_record("brj_apply_J1", tag, "||D^-1q_gpu-D^-1q_or||/||D^-1q_or||", err1, tol)
    assert err1 < tol


@pytest.mark.parametrize("name", ["vortex8_P2", "box_P2_Q4", "box_P3_Q6", "poiseuille_P3",
                                  "vortex_hllc_P3", "box_sutherland_P3_Q6"])
def test_gmres_parity(dgl, name, parity_record):
    c = CASES[name]()
    dg = DG(c.mesh, c.P, c.Q, c.phys)
    m = dgl.Mesh.from_case(c)
    u = perturbed(dg)
    R = dg.residual(u)
    dt_a = 0.05
    b = w.random_direction(u, 11)
    pc_ref = im.BRJ(dg, u, 0.0, dt_a, J=7)
    A = lambda v: im.jvp(dg, u, R, 0.0, v, 1.0, -dt_a)
    cfg = im.GmresConfig(restart=20, rtol=1e-3, max_cycles=5)
    x_ref, st_ref = im.gmres(A, b, pc_ref.apply, cfg)
    pc = dgl.Precond(m).build(to_dev(u), 0.0, dt_a, J=7)
    x, st = m.gmres(to_dev(u), to_dev(R), to_dev(b), 0.0, dt_a, pc, restart=20, max_cycles=5, rtol=1e-3)
    parity_record("gmres", name, "||x_gpu-x_or||/||x_or||", rel(x.cpu().numpy(), x_ref), 1e-4,
                  iters=st["iters"], oracle_iters=st_ref.iters)
    assert st["iters"] == st_ref.iters
    assert rel(x.cpu().numpy(), x_ref) < 1e-4


def test_sdirk_step_parity_vortex_cfg(dgl, parity_record):
    """One SDIRK2 step of the 8x8 P=2 vortex at dt = 0.01 (BRJ(7), restart 20):
    equal Newton and GMRES counts per stage and the same u^{n+1}."""
    c = w.vortex_case(n=8, P=2)
    dg = DG(c.mesh, c.P, c.Q, c.phys)
    m = dgl.Mesh.from_case(c)
    u0 = dg.project_exact()
    dt = 0.01
    lam = 1 - np.sqrt(2) / 2
    pc_ref = im.BRJ(dg, u0, 0.0, dt * lam, J=7)
    cfg = im.NewtonConfig(alpha=1e-3, gmres=im.GmresConfig(restart=20))
    u1_ref, st_ref = im.sdirk_step(dg, u0, 0.0, dt, "sdirk2", pc_ref.apply, cfg)
    ud = to_dev(u0)
    st = m.sdirk_step(ud, 0.0, dt, restart=20, J=7)
    assert st["converged"]
    parity_record("sdirk2_vortex8", "vortex8_P2", "||u1_gpu-u1_or||/||u1_or||",
                  rel(ud.cpu().numpy(), u1_ref), 1e-9, newton=st["stage_newton"],
                  gmres=st["stage_gmres"])
    assert st["stage_newton"] == [s.iters for s in st_ref.stages]
    assert st["stage_gmres"] == [s.gmres_iters for s in st_ref.stages]
    assert rel(ud.cpu().numpy(), u1_ref) < 1e-9
