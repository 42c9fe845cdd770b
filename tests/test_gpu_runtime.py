"""Runtime features with no counterpart in the paper, through the C ABI:
CUDA-graph replay of the BRJ apply and of the GMRES Arnoldi steps, and
autotuned launch shapes of the sum-factorisation kernels.  They change how the
same kernels are launched, never their arithmetic, so results must match the
plain launches bit for bit (and the plain launches match the oracle in
test_gpu_parity)."""
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


def dirichlet_vortex_case(n=6, P=2):
    """The advected isentropic vortex on the unit square with weak Dirichlet
    data from the exact solution on all four sides: the boundary fluxes depend
    on t, so a graph that kept the t of its capture would be caught."""
    from workloads.configs import Case
    lines = [np.linspace(0.0, 1.0, n + 1)] * 2
    mesh = w.box_mesh(lines, (False, False), side_bc=[0, 0, 0, 0])
    ph = w.Physics(Re=100.0, fid=w.FIELD_VORTEX, fpar=(1.0, 0.5, 5.0, 0.5, 0.5, 10.0),
                   bc=[w.BC_DIRICHLET])
    return Case(f"vortex_dirichlet{n}_P{P}", mesh, P, P + 2, ph)


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


@pytest.mark.parametrize("precision", [None, "fp32", "bf16"])
def test_gmres_graph_bitwise(dgl, precision):
    """GMRES with every Arnoldi step replayed as one graph: the same iterate and
    statistics as the plain launches, bit for bit, across calls at other t and
    dt_a (read by the graph from device scalars), with restarts, and with the
    replayed kernels counted."""
    c = dirichlet_vortex_case()
    m = dgl.Mesh.from_case(c)
    u = to_dev(perturbed(c))
    b = to_dev(w.random_direction(u.cpu().numpy(), 3))
    pc = None
    if precision:
        pc = dgl.Precond(m).build(u, 0.0, 0.03, J=4, precision=precision)
    kw = dict(precond=pc, restart=4, max_cycles=12, rtol=1e-6)
    for t, dta in [(0.0, 0.03), (0.37, 0.05), (0.0, 0.03), (0.37, 0.05)]:
        r_u = m.residual(u, t)
        n0 = dgl.kernel_launches()
        x_plain, st_plain = m.gmres(u, r_u, b, t, dta, graphs=False, **kw)
        n_plain = dgl.kernel_launches() - n0
        n0 = dgl.kernel_launches()
        x_graph, st_graph = m.gmres(u, r_u, b, t, dta, graphs=True, **kw)
        n_graph = dgl.kernel_launches() - n0
        torch.cuda.synchronize()
        assert st_plain["cycles"] > 1, st_plain    # restarts exercised
        assert st_graph == st_plain, (t, dta)
        assert torch.equal(x_graph, x_plain), (t, dta, precision)
        # the graph path adds one launch per solve (the device scalars)
        assert n_graph == n_plain + 1, (n_graph, n_plain)


def test_gmres_graph_follows_a_new_preconditioner(dgl):
    """A rebuild with another J, omega or dt_a gives the apply another launch
    sequence (they are kernel arguments): the Arnoldi graphs captured with the
    old one are not replayed.  A rebuild at the same (J, omega, dt_a) refills
    the blocks in place and the graphs stay valid."""
    c = dirichlet_vortex_case(n=4)
    m = dgl.Mesh.from_case(c)
    u = to_dev(perturbed(c))
    b = to_dev(w.random_direction(u.cpu().numpy(), 5))
    r_u = m.residual(u, 0.1)
    pc = dgl.Precond(m).build(u, 0.1, 0.04, J=2, precision="fp32")
    u2 = to_dev(perturbed(c, seed=7))
    for J, omega, dta, state in [(2, 1.0, 0.04, u), (5, 1.0, 0.04, u), (5, 1.0, 0.01, u),
                                 (5, 0.8, 0.01, u), (5, 0.8, 0.01, u2), (2, 1.0, 0.04, u)]:
        pc.build(state, 0.1, dta, J=J, omega=omega, precision="fp32")
        x_plain, st_plain = m.gmres(u, r_u, b, 0.1, dta, precond=pc, restart=10, rtol=1e-6)
        x_graph, st_graph = m.gmres(u, r_u, b, 0.1, dta, precond=pc, restart=10, rtol=1e-6,
                                    graphs=True)
        assert st_graph == st_plain and torch.equal(x_graph, x_plain), (J, omega, dta)


@pytest.mark.parametrize("case", ["vortex", "vortex_dirichlet", "vortex_ramp"])
def test_graph_sdirk_bitwise(dgl, case):
    """Three SDIRK2 steps with the preconditioner frozen after the first (or,
    for vortex_ramp, rebuilt every step at a growing step size): the
    graph-replayed BRJ applies and Arnoldi steps give the same iterates and
    counts (on the Dirichlet vortex every stage has another t)."""
    c = dirichlet_vortex_case(n=6) if case == "vortex_dirichlet" else w.vortex_case(n=8, P=2)
    ramp = case == "vortex_ramp"
    dts = [0.005, 0.01, 0.02] if ramp else [0.02] * 3
    m = dgl.Mesh.from_case(c)
    u0 = m.project()
    res = []
    for graphs in (False, True):
        u = u0.clone()
        pc = dgl.Precond(m)
        stats = []
        for k in range(3):
            st = m.sdirk_step(u, sum(dts[:k]), dts[k], precond=pc, rebuild=(k == 0 or ramp),
                              restart=20, J=7, graphs=graphs)
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
    # GMRES with graphs requested launches plainly while profiling
    r_u = m.residual(u)
    dgl.profile_enable(True)
    try:
        dgl.profile_read()
        x, _ = m.gmres(u, r_u, q, 0.0, 0.02, precond=pc, restart=4, max_cycles=1, graphs=True)
        names = set(dgl.profile_read())
    finally:
        dgl.profile_enable(False)
    assert {"dg_vol", "dg_face", "dg_lift", "multi_dot"} <= names
    x2, _ = m.gmres(u, r_u, q, 0.0, 0.02, precond=pc, restart=4, max_cycles=1, graphs=True)
    assert torch.equal(x, x2)


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


@pytest.mark.parametrize("case,precision", [("vortex", "fp64"), ("vortex", "bf16"),
                                            ("box_P3", "fp32"), ("box_P3", "bf16"),
                                            ("box_P3", "fp64"), ("wavy_P2", "fp32")])
def test_fused_sweeps_bitwise(dgl, case, precision):
    """The fused sweep (off-diagonal product and block product of an element in
    one kernel) forms the same y_e in the same order and multiplies it by the
    same block: BRJ(J) applies equal the separate kernels' bit for bit, for
    several J and omega, with graphs and inside GMRES."""
    if case == "vortex":
        c = w.vortex_case(n=6, P=2)
    elif case == "box_P3":
        c = w.small_tgv_case((3, 3, 2), P=3, Q=6)
    else:
        c = w.wavy_box_case((3, 2, 2), P=2)
    m = dgl.Mesh.from_case(c)
    u = to_dev(perturbed(c))
    qs = [to_dev(w.random_direction(u.cpu().numpy(), s)) for s in range(2)]
    for J, omega in [(1, 1.0), (2, 1.0), (3, 0.8), (7, 1.0)]:
        plain = dgl.Precond(m).build(u, 0.0, 0.03, J=J, precision=precision, omega=omega)
        fused = dgl.Precond(m).build(u, 0.0, 0.03, J=J, precision=precision, omega=omega,
                                     fused=True)
        for q in qs:
            n0 = dgl.kernel_launches()
            ref = plain.apply(q)
            n_plain = dgl.kernel_launches() - n0
            n0 = dgl.kernel_launches()
            out = fused.apply(q)
            n_fused = dgl.kernel_launches() - n0
            torch.cuda.synchronize()
            assert torch.equal(out, ref), (J, omega)
            assert n_fused == n_plain - (J - 1), (n_fused, n_plain)
        graph = dgl.Precond(m).build(u, 0.0, 0.03, J=J, precision=precision, omega=omega,
                                     fused=True, graphs=True)
        o = m.empty()
        for _ in range(2):
            graph.apply(qs[0], o)
            assert torch.equal(o, plain.apply(qs[0]))
    # the plain handle switched to fused and back: GMRES (with Arnoldi graphs) agrees
    r_u = m.residual(u)
    pc = dgl.Precond(m).build(u, 0.0, 0.03, J=4, precision=precision)
    x0, s0 = m.gmres(u, r_u, qs[1], 0.0, 0.03, precond=pc, restart=8, rtol=1e-6, graphs=True)
    pc.build(u, 0.0, 0.03, J=4, precision=precision, fused=True)
    x1, s1 = m.gmres(u, r_u, qs[1], 0.0, 0.03, precond=pc, restart=8, rtol=1e-6, graphs=True)
    assert s0 == s1 and torch.equal(x0, x1)


def test_fused_sweeps_sdirk_bitwise(dgl):
    c = w.vortex_case(n=8, P=2)
    m = dgl.Mesh.from_case(c)
    u0 = m.project()
    res = []
    for fused in (False, True):
        u = u0.clone()
        pc = dgl.Precond(m)
        stats = []
        for k in range(2):
            st = m.sdirk_step(u, 0.02 * k, 0.02, precond=pc, rebuild=(k == 0), restart=20, J=7,
                              precision="fp32", graphs=True, fused=fused)
            assert st["converged"]
            stats.append((st["stage_newton"], st["stage_gmres"]))
        res.append((u, stats))
    assert res[0][1] == res[1][1]
    assert torch.equal(res[0][0], res[1][0])


def test_results_do_not_depend_on_earlier_allocations(dgl):
    """Two SDIRK2 steps on a fresh mesh and preconditioner give the same bits
    whether the device memory they get was never used or held NaNs just
    before (a 1 GiB NaN-filled tensor freed back to the driver): no kernel may
    read a workspace before writing it (0 * NaN is NaN)."""
    c = w.vortex_case(n=8, P=2)
    runs = []
    for poison in (False, True):
        if poison:
            junk = torch.full((1 << 27,), float("nan"), dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            del junk
            torch.cuda.empty_cache()
        m = dgl.Mesh.from_case(c)
        u = m.project()
        pc = dgl.Precond(m)
        for k in range(2):
            st = m.sdirk_step(u, 0.02 * k, 0.02, precond=pc, rebuild=(k == 0), restart=20, J=7,
                              precision="fp32", fused=True)
            assert st["converged"]
        runs.append(u.clone())
        pc.close()
        m.close()
    assert torch.isfinite(runs[1]).all()
    assert torch.equal(runs[0], runs[1])
