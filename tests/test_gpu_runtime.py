"""Runtime features with no counterpart in the paper, through the C ABI:
CUDA-graph replay of the BRJ apply and autotuned launch shapes of the
sum-factorisation kernels.  Both change how the same kernels are launched,
never their arithmetic, so results must match the plain launches bit for bit
(and the plain launches match the oracle in test_gpu_parity)."""
import ctypes

import numpy as np
import pytest
import torch

import workloads as w
from oracle.dg import DG

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dgl():
    import paper_2002_04222_gb300 as dgl
    return dgl


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def perturbed(c, seed=0, amp=0.01):
    dg = DG(c.mesh, c.P, c.Q, c.phys)
    u = dg.project_exact()
    return u + amp * w.random_direction(u, seed)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16"])
def test_graph_apply_bitwise(dgl, precision):
    c = w.small_tgv_case((3, 2, 3), P=2, Q=4)
    m = dgl.Mesh.from_case(c)
    u = to_dev(perturbed(c))
    qs = [to_dev(w.random_direction(u.cpu().numpy(), s)) for s in range(3)]
    plain = dgl.Precond(m).build(u, 0.0, 0.02, J=5, precision=precision, omega=0.9)
    graph = dgl.Precond(m).build(u, 0.0, 0.02, J=5, precision=precision, omega=0.9, graphs=True)
    outs = [m.empty() for _ in qs]
    for rep in range(3):                       # capture, then replays
        for q, o in zip(qs, outs):
            n0 = dgl.kernel_launches()
            graph.apply(q, o)
            n_graph = dgl.kernel_launches() - n0
            n0 = dgl.kernel_launches()
            ref = plain.apply(q)
            assert dgl.kernel_launches() - n0 == n_graph   # replays are counted
            torch.cuda.synchronize()
            assert torch.equal(o, ref), (rep, precision)
    # a rebuild at another state and dt_a drops the captured graphs
    u2 = to_dev(perturbed(c, seed=4))
    plain.build(u2, 0.1, 0.05, J=3, precision=precision)
    graph.build(u2, 0.1, 0.05, J=3, precision=precision, graphs=True)
    for q, o in zip(qs, outs):
        graph.apply(q, o)
        assert torch.equal(o, plain.apply(q))


def test_graph_sdirk_bitwise(dgl):
    """Three SDIRK2 steps of the 8x8 P=2 vortex with the preconditioner frozen
    after the first: the graph-replayed BRJ gives the same iterates and counts."""
    c = w.vortex_case(n=8, P=2)
    m = dgl.Mesh.from_case(c)
    u0 = m.project()
    res = []
    for graphs in (False, True):
        u = u0.clone()
        pc = dgl.Precond(m)
        stats = []
        for k in range(3):
            st = m.sdirk_step(u, 0.02 * k, 0.02, precond=pc, rebuild=(k == 0), restart=20, J=7,
                              graphs=graphs)
            assert st["converged"]
            stats.append((st["stage_newton"], st["stage_gmres"]))
        res.append((u, stats))
    assert res[0][1] == res[1][1]
    assert torch.equal(res[0][0], res[1][0])


def test_graph_bypassed_while_profiling(dgl):
    c = w.small_tgv_case((2, 2, 2), P=1)
    m = dgl.Mesh.from_case(c)
    u = m.project()
    pc = dgl.Precond(m).build(u, 0.0, 0.02, J=3, graphs=True)
    q = m.residual(u)
    dgl.profile_enable(True)
    try:
        dgl.profile_read()                         # clear
        out = pc.apply(q)
        names = set(dgl.profile_read())
    finally:
        dgl.profile_enable(False)
    assert "brj_diag" in names and "brj_offdiag" in names
    assert torch.equal(out, pc.apply(q))


@pytest.mark.parametrize("case", ["vortex", "box_P3"])
def test_autotune_shape_does_not_change_results(dgl, case):
    c = w.vortex_case(n=8, P=2) if case == "vortex" else w.small_tgv_case((3, 3, 2), P=3)
    m = dgl.Mesh.from_case(c)
    u = to_dev(perturbed(c))
    r_default = m.residual(u)
    r = dgl.autotune(m, reps=2)
    assert r["vol_ms"] <= r["vol_ms_default"] * 1.5 and r["lift_ms"] <= r["lift_ms_default"] * 1.5
    r_tuned = m.residual(u)
    assert torch.equal(r_default, r_tuned)
    v = to_dev(w.random_direction(u.cpu().numpy(), 9))
    assert torch.equal(m.jvp(u, r_tuned, v), m.jvp(u, r_default, v))


def test_set_tune_rejects_non_candidates(dgl):
    from paper_2002_04222_gb300 import _lib
    DG_ERR_ARG = -1
    c = w.vortex_case(n=4, P=2)
    m = dgl.Mesh.from_case(c)
    bad = _lib.TuneResult(0, 0, 0, 0, 0.0, 0.0, 0.0, 0.0)
    assert dgl.lib().dg_set_tune(m.handle, ctypes.byref(bad)) == DG_ERR_ARG
    bad = _lib.TuneResult(1, 7, 1, 64, 0.0, 0.0, 0.0, 0.0)
    assert dgl.lib().dg_set_tune(m.handle, ctypes.byref(bad)) == DG_ERR_ARG
