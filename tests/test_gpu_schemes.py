"""Parity of the further schemes of Sec. 4.3 through the C ABI: the HLL,
local Lax-Friedrichs and AUSM advection fluxes (residual, Jacobian-free
product and BRJ apply, whose trace Jacobians difference the flux), and the
backward Euler, fourth-order ESDIRK (App. A) and BDF2 time steps on the
8 x 8, P = 2 vortex of the first configuration (equal Newton and GMRES
counts per stage, the same u^{n+1})."""
import numpy as np
import pytest
import torch

import workloads as w
from oracle.dg import DG
from oracle import implicit as im

pytestmark = pytest.mark.gpu

R_TOL = 1e-12


@pytest.fixture(scope="module")
def dgl():
    import paper_2002_04222_gb300 as dgl
    return dgl


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


FLUX_CASES = {
    "vortex_hll_P2": lambda: w.vortex_case(n=5, P=2, riemann=w.RIEMANN_HLL),
    "vortex_lf_P3": lambda: w.vortex_case(n=4, P=3, Q=5, riemann=w.RIEMANN_LF),
    "vortex_ausm_P2": lambda: w.vortex_case(n=5, P=2, riemann=w.RIEMANN_AUSM),
    "box_hll_P3_Q6": lambda: w.small_tgv_case((3, 2, 2), P=3, riemann=w.RIEMANN_HLL),
    "box_lf_P2_Q4": lambda: w.small_tgv_case((3, 3, 2), P=2, Q=4, riemann=w.RIEMANN_LF),
    "box_ausm_P3_Q6": lambda: w.small_tgv_case((2, 3, 2), P=3, riemann=w.RIEMANN_AUSM),
}


def perturbed(dg, seed=0, amp=0.01):
    u = dg.project_exact()
    return u + amp * w.random_direction(u, seed)


def floor(dg, u, R):
    rng = np.random.default_rng(123)
    return max(rel(dg.residual(u * (1 + 2.0 ** -52 * rng.standard_normal(u.shape))), R)
               for _ in range(3))


@pytest.mark.parametrize("name", sorted(FLUX_CASES))
def test_flux_residual_jvp_and_brj_parity(dgl, name, parity_record):
    c = FLUX_CASES[name]()
    dg = DG(c.mesh, c.P, c.Q, c.phys)
    m = dgl.Mesh.from_case(c)
    u = perturbed(dg)
    R_ref = dg.residual(u)
    ud = to_dev(u)
    R = m.residual(ud).cpu().numpy()
    s = floor(dg, u, R_ref)
    tol = max(R_TOL, 16.0 * s)
    parity_record("residual_flux", name, "||R_gpu-R_or||/||R_or||", rel(R, R_ref), tol, floor_s=s)
    assert rel(R, R_ref) < tol
    # Jacobian-free product, bounded by the residual difference at u + eps v over eps
    v = w.random_direction(u, 7)
    eps = im.jfnk_eps(u, v)
    wv = u + eps * v
    dR = np.linalg.norm(m.residual(to_dev(wv)).cpu().numpy() - dg.residual(wv))
    ref = im.jvp(dg, u, R_ref, 0.0, v, 1.0, -0.013)
    got = m.jvp(ud, to_dev(R_ref), to_dev(v), 0.0, 1.0, -0.013).cpu().numpy()
    bound = max(1e-6, 4 * 0.013 * dR / eps / np.linalg.norm(ref))
    parity_record("jvp_flux", name, "||Jv_gpu-Jv_or||/||Jv_or||", rel(got, ref), bound)
    assert rel(got, ref) < bound
    # BRJ(7) apply with FP64 blocks
    dt_a = 0.02
    q = w.random_direction(u, 3)
    refq = im.BRJ(dg, u, 0.0, dt_a, J=7).apply(q)
    pc = dgl.Precond(m).build(ud, 0.0, dt_a, J=7, precision="fp64")
    gotq = pc.apply(to_dev(q)).cpu().numpy()
    parity_record("brj_apply_flux", name, "||P^-1q_gpu-P^-1q_or||/||P^-1q_or||", rel(gotq, refq), 1e-6)
    assert rel(gotq, refq) < 1e-6


@pytest.mark.parametrize("tableau", ["be", "esdirk4", "sdirk3"])
def test_rk_step_parity_vortex_cfg(dgl, tableau, parity_record):
    c = w.vortex_case(n=8, P=2)
    dg = DG(c.mesh, c.P, c.Q, c.phys)
    m = dgl.Mesh.from_case(c)
    u0 = dg.project_exact()
    dt = 0.01
    A, b, cc = im.sdirk_tableau(tableau)
    gdiag = next(a for a in np.diag(A) if a != 0.0)
    pc_ref = im.BRJ(dg, u0, 0.0, dt * gdiag, J=7)
    cfg = im.NewtonConfig(alpha=1e-3, gmres=im.GmresConfig(restart=20))
    u1_ref, st_ref = im.sdirk_step(dg, u0, 0.0, dt, tableau, pc_ref.apply, cfg)
    ud = to_dev(u0)
    st = m.sdirk_step(ud, 0.0, dt, tableau=tableau, restart=20, J=7)
    assert st["converged"]
    err = rel(ud.cpu().numpy() - u0, u1_ref - u0)
    parity_record("rk_step", f"vortex8_P2_{tableau}", "||du_gpu-du_or||/||du_or||", err, 1e-6,
                  newton=st["stage_newton"], gmres=st["stage_gmres"])
    assert st["stage_newton"] == [s.iters for s in st_ref.stages]
    assert st["stage_gmres"] == [s.gmres_iters for s in st_ref.stages]
    assert err < 1e-6


def test_bdf2_steps_parity_vortex_cfg(dgl, parity_record):
    """A backward-Euler start-up step, then two BDF2 steps: equal counts and
    the same states."""
    c = w.vortex_case(n=8, P=2)
    dg = DG(c.mesh, c.P, c.Q, c.phys)
    m = dgl.Mesh.from_case(c)
    u0 = dg.project_exact()
    dt = 0.01
    cfg = im.NewtonConfig(alpha=1e-3, gmres=im.GmresConfig(restart=20))
    pc_be = im.BRJ(dg, u0, 0.0, dt, J=7)
    u1, _ = im.sdirk_step(dg, u0, 0.0, dt, "be", pc_be.apply, cfg)
    pc_ref = im.BRJ(dg, u1, dt, 2 * dt / 3, J=7)
    refs = []
    prev, cur = u0, u1
    for k in (1, 2):
        nxt, st = im.bdf2_step(dg, cur, prev, k * dt, dt, pc_ref.apply, cfg)
        refs.append((nxt, st))
        prev, cur = cur, nxt
    ud = to_dev(u0)
    m.sdirk_step(ud, 0.0, dt, tableau="be", restart=20, J=7)
    up = to_dev(u0)
    pc = dgl.Precond(m)
    for i, k in enumerate((1, 2)):
        st = m.bdf2_step(ud, up, k * dt, dt, precond=pc, rebuild=(k == 1), restart=20, J=7)
        nxt, st_ref = refs[i]
        assert st["converged"]
        err = rel(ud.cpu().numpy() - up.cpu().numpy(), nxt - refs[i - 1][0] if i else nxt - u1)
        parity_record("bdf2_step", f"vortex8_P2_step{k}", "||du_gpu-du_or||/||du_or||", err, 1e-6,
                      newton=st["stage_newton"], gmres=st["stage_gmres"])
        assert st["stage_newton"] == [s.iters for s in st_ref.stages]
        assert st["stage_gmres"] == [s.gmres_iters for s in st_ref.stages]
        assert err < 1e-6


def test_learned_guess_refuses_explicit_first_stage(dgl):
    from paper_2002_04222_gb300 import _lib
    c = w.vortex_case(n=4, P=2)
    m = dgl.Mesh.from_case(c)
    u = m.project(0.0)
    g = dgl.Guess(m, None, stages=4)
    with pytest.raises(_lib.DGError) as ei:
        m.sdirk_step(u, 0.0, 0.01, tableau="esdirk4", guess=g)
    assert ei.value.code == -6
