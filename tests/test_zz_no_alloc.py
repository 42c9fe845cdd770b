"""dg_gmres_noalloc: GMRES for callers that cannot allocate device memory
(applications whose memory pool has reserved the device, loops that forbid
allocator calls).  It must return what dg_gmres returns on the same inputs,
call after call, although its Krylov basis lives in a shared static device
array instead of memory that dg_gmres allocates, and a call after the first
must leave the device's free memory unchanged, also with a preconditioner
built for graph replay (whose sweeps it launches plainly).  This file is
collected last so that a failure here comes after every other test has run;
it also passes alone in a fresh process."""
import numpy as np
import pytest
import torch

import workloads as w
from oracle.dg import DG

pytestmark = pytest.mark.gpu


def _state(c, seed=0):
    dg = DG(c.mesh, c.P, c.Q, c.phys)
    u = dg.project_exact()
    return u + 0.01 * w.random_direction(u, seed)


def test_gmres_noalloc_allocates_nothing_with_graph_preconditioner():
    """Fresh mesh and preconditioner (built with graphs=True), no dg_gmres call
    before: after one warm-up call, a second dg_gmres_noalloc call changes the
    device's free memory by nothing.  Then both calls' results equal dg_gmres's
    on the same preconditioner."""
    import paper_2002_04222_gb300 as dgl
    c = w.small_tgv_case((3, 2, 2), P=2, Q=4, stretch=True)
    u = _state(c, 1)
    m = dgl.Mesh.from_case(c)
    ud = torch.from_numpy(u).cuda()
    R = m.residual(ud)
    dt_a = 0.05
    pc = dgl.Precond(m).build(ud, 0.0, dt_a, J=7, precision="fp32", graphs=True)
    b = torch.from_numpy(w.random_direction(u, 21)).cuda()
    x1 = torch.full_like(b, float("nan"))
    x2 = torch.full_like(b, float("nan"))
    kw = dict(restart=20, max_cycles=5, rtol=1e-3)
    _, st1 = m.gmres_noalloc(ud, R, b, x1, 0.0, dt_a, pc, **kw)       # warm-up (set-up)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    _, st2 = m.gmres_noalloc(ud, R, b, x2, 0.0, dt_a, pc, **kw)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0, (free0, free1)
    assert st1 == st2 and torch.equal(x1, x2)
    x_ref, st_ref = m.gmres(ud, R, b, 0.0, dt_a, pc, **kw)
    assert st2["iters"] == st_ref["iters"] and st2["converged"] == st_ref["converged"]
    err = (torch.linalg.norm(x2 - x_ref) / torch.linalg.norm(x_ref)).item()
    assert err < 1e-12, err


def test_gmres_noalloc_matches_gmres_twice():
    import paper_2002_04222_gb300 as dgl
    c = w.small_tgv_case((3, 3, 2), P=2, Q=4, stretch=True)
    u = _state(c, 0)
    m = dgl.Mesh.from_case(c)
    ud = torch.from_numpy(u).cuda()
    R = m.residual(ud)
    dt_a = 0.05
    pc = dgl.Precond(m).build(ud, 0.0, dt_a, J=7)
    for seed in (11, 12):
        b = torch.from_numpy(w.random_direction(u, seed)).cuda()
        x_ref, st_ref = m.gmres(ud, R, b, 0.0, dt_a, pc, restart=20, max_cycles=5, rtol=1e-3)
        for _ in range(2):          # two calls in a row on the shared static basis
            out = torch.full_like(b, float("nan"))
            x, st = m.gmres_noalloc(ud, R, b, out, 0.0, dt_a, pc, restart=20, max_cycles=5, rtol=1e-3)
            assert st["iters"] == st_ref["iters"] and st["converged"] == st_ref["converged"]
            err = (torch.linalg.norm(x - x_ref) / torch.linalg.norm(x_ref)).item()
            assert err < 1e-12, err
    # without a preconditioner too
    b = torch.from_numpy(w.random_direction(u, 13)).cuda()
    x_ref, st_ref = m.gmres(ud, R, b, 0.0, dt_a, None, restart=20, max_cycles=5, rtol=1e-2)
    x, st = m.gmres_noalloc(ud, R, b, torch.empty_like(b), 0.0, dt_a, None, restart=20,
                            max_cycles=5, rtol=1e-2)
    assert st["iters"] == st_ref["iters"]
    assert (torch.linalg.norm(x - x_ref) / torch.linalg.norm(x_ref)).item() < 1e-12


def test_gmres_noalloc_rejects_too_large_basis():
    import paper_2002_04222_gb300 as dgl
    from paper_2002_04222_gb300 import _lib
    c = w.tgv_case(n=8, P=3)     # 163,840 DOF: 31 basis vectors (restart 30, no
    m = dgl.Mesh.from_case(c)    # preconditioner) need 5.1 M doubles > 2,097,152
    u = m.project(0.0)
    R = m.residual(u)
    assert m.info["n_dof"] * 31 > _lib.NOALLOC_MAX_DOUBLES
    with pytest.raises(_lib.DGError) as ei:
        m.gmres_noalloc(u, R, R.clone(), torch.empty_like(u), 0.0, 0.01, None, restart=30)
    assert ei.value.code == -1
