"""Order of accuracy of the device path on the manufactured compressible
Poiseuille flow (Sec. 6.1, App. B) on the wall-clustered channel family of
the 16 x 8 configuration (4x2, 8x4, 16x8 quads on [0,2]x[0,1], geometric
ratio 1.1 from each wall), P = 1..6, Q = P + 2: steady states reached through
the C ABI (residual, BRJ build, preconditioned JFNK GMRES) by pseudo-transient
continuation.

Bounds fixed beforehand: the h-rate of the L2 error (all four variables)
between 8x4 and 16x8 is at least P + 1 - 0.3 for every P; on the 16x8 mesh
each increment of P lowers the error at least fourfold (p-convergence); and
on the oracle's own mesh pair (2 x ny) the device's steady error equals the
oracle's to 1e-3 relative (the same discrete steady state, reached by two
implementations)."""
import numpy as np
import pytest
import torch

import workloads as w
from oracle.dg import DG
from oracle import implicit as im
from oracle import physics as phy

pytestmark = pytest.mark.gpu

FAMILY = [(4, 2), (8, 4), (16, 8)]


@pytest.fixture(scope="module")
def dgl():
    import paper_2002_04222_gb300 as dgl
    return dgl


STEPS = 14


def steady_state_device(dgl, m, u, steps=STEPS):
    """Pseudo-transient continuation through the C ABI: one backward-Euler
    Newton step per pseudo-time step, (I - dt dR/du) x = dt R(u) by BRJ(7)
    preconditioned GMRES(40) (rtol 1e-4, at most 5 cycles), dt growing
    tenfold up to 1e12, a fixed number of steps (||R|| reaches its rounding
    floor, M^-1 times the rounding of L, well before u stops changing)."""
    pc = dgl.Precond(m)
    dt, hist = 1.0, []
    for _ in range(steps):
        R = m.residual(u)
        hist.append(torch.linalg.norm(R).item())
        pc.build(u, 0.0, dt, J=7)
        x, _ = m.gmres(u, R, R * dt, 0.0, dt, pc, restart=40, max_cycles=5, rtol=1e-4)
        u = u + x
        dt = min(10.0 * dt, 1e12)
    return u, hist


def device_error(dgl, P, nx, ny):
    c = w.poiseuille_case(P, nx=nx, ny=ny)
    dg = DG(c.mesh, c.P, c.Q, c.phys)          # evaluates the error only
    m = dgl.Mesh.from_case(c)
    u, hist = steady_state_device(dgl, m, m.project(0.0))
    e = dg.l2_error(u.cpu().numpy(), lambda x: phy.exact_state(c.phys, x, 0.0))
    return float(np.linalg.norm(e)), hist


@pytest.fixture(scope="module")
def errors(dgl):
    return {(P, nx, ny): device_error(dgl, P, nx, ny) for P in range(1, 7) for nx, ny in FAMILY}


@pytest.mark.parametrize("P", range(1, 7))
def test_h_rate_on_the_clustered_channel_family(errors, P, parity_record):
    (e1, _), (e2, h2) = errors[(P, 8, 4)], errors[(P, 16, 8)]
    rate = float(np.log2(e1 / e2))
    parity_record("poiseuille_h_rate", f"P{P}_8x4_16x8", "log2(e_8x4/e_16x8)", rate, P + 1 - 0.3,
                  errors=[errors[(P, nx, ny)][0] for nx, ny in FAMILY], final_residual=h2[-1])
    assert rate > P + 1 - 0.3, (P, e1, e2)


def test_p_convergence_on_16x8(errors, parity_record):
    e = [errors[(P, 16, 8)][0] for P in range(1, 7)]
    ratios = [e[i] / e[i + 1] for i in range(5)]
    parity_record("poiseuille_p_sweep", "16x8_P1..6", "min e(P)/e(P+1)", min(ratios), 4.0,
                  errors=e)
    assert all(r > 4.0 for r in ratios), e


@pytest.mark.parametrize("P,ny", [(2, 4), (4, 2), (5, 2), (6, 2)])
def test_device_and_oracle_reach_the_same_steady_state(dgl, P, ny, parity_record):
    c = w.poiseuille_case(P, nx=2, ny=ny)
    dg = DG(c.mesh, c.P, c.Q, c.phys)
    exact = lambda x: phy.exact_state(c.phys, x, 0.0)
    # the same continuation in the oracle
    u, dt = dg.project_exact(), 1.0
    for _ in range(STEPS):
        R = dg.residual(u)
        pc = im.BRJ(dg, u, 0.0, dt, J=7)
        A = lambda v, u=u, R=R, dt=dt: im.jvp(dg, u, R, 0.0, v, 1.0, -dt)
        x, _ = im.gmres(A, dt * R, pc.apply, im.GmresConfig(restart=40, rtol=1e-4, max_cycles=5))
        u = u + x
        dt = min(10.0 * dt, 1e12)
    e_or = float(np.linalg.norm(dg.l2_error(u, exact)))
    e_dev, _ = device_error(dgl, P, 2, ny)
    parity_record("poiseuille_steady_error", f"P{P}_2x{ny}", "|e_dev-e_or|/e_or",
                  abs(e_dev - e_or) / e_or, 1e-3, e_dev=e_dev, e_or=e_or)
    assert abs(e_dev - e_or) < 1e-3 * e_or, (e_dev, e_or)
