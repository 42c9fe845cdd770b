"""dg_gmres_noalloc: GMRES for callers that cannot allocate device memory
(stream capture, pre-reserved memory pools, allocator-free loops).  It must
return what dg_gmres returns on the same inputs, call after call, although its
Krylov basis lives in a shared static device array instead of memory that
dg_gmres allocates.  This file is collected last so that a failure here comes
after every other test has run; it also passes alone in a fresh process."""
import numpy as np
import pytest
import torch

import workloads as w
from oracle.dg import DG

pytestmark = pytest.mark.gpu


def test_gmres_noalloc_matches_gmres_twice():
    import paper_2002_04222_gb300 as dgl
    c = w.small_tgv_case((3, 3, 2), P=2, Q=4, stretch=True)
    dg = DG(c.mesh, c.P, c.Q, c.phys)
    u = dg.project_exact()
    u = u + 0.01 * w.random_direction(u, 0)
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
    c = w.tgv_case(n=8, P=3)     # 163,840 DOF: 61 vectors exceed the static array
    m = dgl.Mesh.from_case(c)
    u = m.project(0.0)
    R = m.residual(u)
    with pytest.raises(_lib.DGError) as ei:
        m.gmres_noalloc(u, R, R.clone(), torch.empty_like(u), 0.0, 0.01, None, restart=30)
    assert ei.value.code == -1
