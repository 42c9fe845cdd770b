"""Parity of the general-geometry path (curved quadratic hexes, rotated
straight-sided elements, the O-grid of the cylinder workload of Sec. 6.4)
and of the far-field / adiabatic-wall boundary conditions with the FP64 CPU
oracle, through the C ABI: residual, projection, JFNK product, BRJ apply,
GMRES and an SDIRK3 step.  Tolerances as in the affine parity tests: R to
max(1e-12, 16 x the oracle's one-ulp rounding floor), the JVP to the
residual difference divided by eps, the BRJ apply to the block precision."""
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


def mass(dg, x):
    return np.einsum("emn,evn->evm", np.linalg.inv(dg.Minv), x)


def rounding_floor(dg, u, R, trials=3, weak=False):
    rng = np.random.default_rng(123)
    out = 0.0
    for _ in range(trials):
        up = u * (1 + 2.0 ** -52 * rng.standard_normal(u.shape))
        if weak:
            out = max(out, rel(dg.rhs(up), dg.rhs(u)))
        else:
            out = max(out, rel(dg.residual(up), R))
    return out


def channel_with_new_bcs():
    """2-D affine channel: far field at x = 0, 2 and adiabatic walls at y = 0, 1
    (the axis-aligned kernels with the cylinder's boundary types)."""
    c = w.poiseuille_case(2, nx=4, ny=2, x_bc=w.BC_FARFIELD, y_bc=w.BC_ADIA_WALL)
    c.phys.forcing = 0
    c.phys.fid = w.FIELD_UNIFORM
    c.phys.fpar = (1.0, 0.8, 0.1, 0.0, 1.0)
    return c


CASES = {
    "wavy_P2": lambda: w.wavy_box_case((3, 2, 2), P=2),
    "wavy_P3": lambda: w.wavy_box_case((2, 2, 2), P=3),
    "rotated_g1_P2": lambda: w.rotated_box_case((3, 2, 2), P=2, order=1),
    "rotated_2d_P3": lambda: w.rotated_box_case((3, 4), P=3, Q=5, order=2),
    "cylinder_P2": lambda: w.small_cylinder_case(3, 8, 2, P=2),
    "cylinder_P3_hllc": lambda: w.small_cylinder_case(2, 6, 2, P=3),
    "cylinder_far_far": lambda: w.small_cylinder_case(2, 6, 1, P=2,
                                                      bc=(w.BC_FARFIELD, w.BC_FARFIELD)),
    "channel_ff_adiabatic": channel_with_new_bcs,
    "cylinder_wall_layer": lambda: w.small_cylinder_case(3, 8, 2, P=2, wall_layer=0.1),
}


def case(name):
    c = CASES[name]()
    if name == "cylinder_P3_hllc":
        c.phys.riemann = phy.RIEMANN_HLLC
    return c


@pytest.mark.parametrize("name", sorted(CASES))
def test_residual_parity_general(dgl, name):
    c = case(name)
    dg = DG(c.mesh, c.P, c.Q, c.phys)
    m = dgl.Mesh.from_case(c)
    u = perturbed(dg, amp=0.02)
    R_ref = dg.residual(u, 0.0)
    R = m.residual(to_dev(u)).cpu().numpy()
    tol = max(R_TOL, 16.0 * rounding_floor(dg, u, R_ref))
    assert rel(R, R_ref) < tol, (rel(R, R_ref), tol)
    L, L_ref = mass(dg, R), mass(dg, R_ref)
    assert rel(L, L_ref) < max(R_TOL, 64.0 * rounding_floor(dg, u, R_ref, weak=True)), rel(L, L_ref)


@pytest.mark.parametrize("name", ["wavy_P3", "cylinder_P2", "rotated_2d_P3", "cylinder_wall_layer"])
def test_projection_parity_general(dgl, name):
    c = case(name)
    dg = DG(c.mesh, c.P, c.Q, c.phys)
    m = dgl.Mesh.from_case(c)
    ref = dg.project_exact(0.0)
    got = m.project(0.0).cpu().numpy()
    # both sides apply an explicit inverse of the element mass matrix (cond up
    # to ~1e6 on these meshes): bound the mass-weighted difference by the
    # oracle's own backward residual |M x_ref - b| / |b| (the GPU's is of the
    # same size, the difference at most their sum)
    U = phy.exact_state(dg.ph, dg.x, 0.0)
    b = np.einsum("qm,eqv->evm", dg.B, U * dg.wJ[..., None])
    M = np.einsum("qm,eq,qn->emn", dg.B, dg.wJ, dg.B)
    floor = rel(np.einsum("emn,evn->evm", M, ref), b)
    assert rel(mass(dg, got), mass(dg, ref)) < max(1e-13, 4 * floor), (rel(mass(dg, got), mass(dg, ref)), floor)
    assert rel(got, ref) < 1e-10


def test_free_stream_on_curved_gpu(dgl):
    """R(const) = 0 on the wavy mesh and on the O-grid with far field on both
    sides (the metric identities hold for the device's metrics too)."""
    for name in ("wavy_P3", "cylinder_far_far"):
        c = case(name)
        dg = DG(c.mesh, c.P, c.Q, c.phys)
        m = dgl.Mesh.from_case(c)
        one = np.round(dg.one_coeffs(), 10)
        U0 = phy.exact_state(c.phys, np.zeros((1, 3)), 0.0)[0]
        if name == "wavy_P3":
            U0 = phy.conservative(np.array(1.1), np.array([0.3, -0.2, 0.1]), np.array(60.0), c.phys)
        u = U0[None, :, None] * one[None, None, :] * np.ones((dg.E, 1, 1))
        L = mass(dg, m.residual(to_dev(u)).cpu().numpy())
        scale = np.abs(dg.rhs(u, faces=False)).sum(axis=2).max()
        assert np.abs(L).max() < 1e-12 * scale, name


@pytest.mark.parametrize("name", ["wavy_P2", "cylinder_P2", "channel_ff_adiabatic"])
def test_jvp_parity_general(dgl, name):
    c = case(name)
    dg = DG(c.mesh, c.P, c.Q, c.phys)
    m = dgl.Mesh.from_case(c)
    u = perturbed(dg, amp=0.02)
    v = w.random_direction(u, 7)
    R = dg.residual(u)
    ud, Rd, vd = to_dev(u), to_dev(R), to_dev(v)
    eps = im.jfnk_eps(u, v)
    wv = u + eps * v
    dR = np.linalg.norm(m.residual(to_dev(wv)).cpu().numpy() - dg.residual(wv))
    for alpha, beta in ((0.0, 1.0), (1.0, -0.013)):
        ref = im.jvp(dg, u, R, 0.0, v, alpha, beta)
        got = m.jvp(ud, Rd, vd, 0.0, alpha, beta).cpu().numpy()
        bound = 4 * abs(beta) * dR / eps / np.linalg.norm(ref)
        assert rel(got, ref) < max(JVP_TOL, bound), (rel(got, ref), bound)


@pytest.mark.parametrize("name,precision,tol", [("wavy_P2", "fp64", 1e-6),
                                                ("cylinder_P2", "fp64", 1e-6),
                                                ("cylinder_P2", "fp32", 1e-4),
                                                ("channel_ff_adiabatic", "fp64", 1e-6),
                                                ("cylinder_P3_hllc", "bf16", 3e-2)])
def test_precond_apply_parity_general(dgl, name, precision, tol):
    c = case(name)
    dg = DG(c.mesh, c.P, c.Q, c.phys)
    m = dgl.Mesh.from_case(c)
    u = perturbed(dg, amp=0.02)
    dt_a = 0.02
    ref_pc = im.BRJ(dg, u, 0.0, dt_a, J=7)
    q = w.random_direction(u, 3)
    if precision == "fp32":
        # the device assembles FP32 blocks: at high order its rounding, after
        # cancellation in the volume sums, exceeds 1e-4; bound by 4x the
        # oracle's own float32-assembly difference
        ref32 = im.BRJ(dg, u, 0.0, dt_a, J=7, assembly_dtype=np.float32).apply(q)
        tol = max(tol, 4 * rel(ref32, ref_pc.apply(q)))
    pc = dgl.Precond(m).build(to_dev(u), 0.0, dt_a, J=7, precision=precision)
    assert rel(pc.apply(to_dev(q)).cpu().numpy(), ref_pc.apply(q)) < tol
    ref_pc.J = 1
    pc1 = dgl.Precond(m).build(to_dev(u), 0.0, dt_a, J=1, precision=precision)
    assert rel(pc1.apply(to_dev(q)).cpu().numpy(), ref_pc.apply(q)) < tol


def test_gmres_parity_cylinder(dgl):
    c = case("cylinder_P2")
    dg = DG(c.mesh, c.P, c.Q, c.phys)
    m = dgl.Mesh.from_case(c)
    u = perturbed(dg, amp=0.02)
    R = dg.residual(u)
    dt_a = 0.05
    b = w.random_direction(u, 11)
    pc_ref = im.BRJ(dg, u, 0.0, dt_a, J=7)
    A = lambda v: im.jvp(dg, u, R, 0.0, v, 1.0, -dt_a)
    cfg = im.GmresConfig(restart=20, rtol=1e-3, max_cycles=5)
    x_ref, st_ref = im.gmres(A, b, pc_ref.apply, cfg)
    pc = dgl.Precond(m).build(to_dev(u), 0.0, dt_a, J=7)
    x, st = m.gmres(to_dev(u), to_dev(R), to_dev(b), 0.0, dt_a, pc, restart=20, max_cycles=5,
                    rtol=1e-3)
    assert st["iters"] == st_ref.iters
    assert rel(x.cpu().numpy(), x_ref) < 1e-4


def test_sdirk3_step_parity_cylinder(dgl):
    """One SDIRK3 step (the cylinder workload's scheme) on the coarse O-grid:
    equal Newton and GMRES counts per stage and the same u^{n+1}."""
    c = case("cylinder_P2")
    dg = DG(c.mesh, c.P, c.Q, c.phys)
    m = dgl.Mesh.from_case(c)
    u0 = perturbed(dg, seed=5, amp=0.01)
    dt = 0.05
    lam = 0.4358665215
    pc_ref = im.BRJ(dg, u0, 0.0, dt * lam, J=7)
    cfg = im.NewtonConfig(alpha=1e-3, gmres=im.GmresConfig(restart=20))
    u1_ref, st_ref = im.sdirk_step(dg, u0, 0.0, dt, "sdirk3", pc_ref.apply, cfg)
    ud = to_dev(u0)
    st = m.sdirk_step(ud, 0.0, dt, tableau=3, restart=20, J=7)
    assert st["converged"]
    assert st["stage_newton"] == [s.iters for s in st_ref.stages]
    assert st["stage_gmres"] == [s.gmres_iters for s in st_ref.stages]
    # every Newton update comes from Krylov solves on JFNK products that agree
    # to JVP_TOL: the step's increment agrees to that relative accuracy
    inc = np.linalg.norm(u1_ref - u0) / np.linalg.norm(u1_ref)
    assert rel(ud.cpu().numpy(), u1_ref) < max(1e-9, JVP_TOL * inc), (rel(ud.cpu().numpy(), u1_ref), inc)


def test_fp64_blocks_on_curved_p3_not_offered(dgl):
    """FP64 BRJ blocks on general elements stop at P = 2 (the build returns
    unsupported before launching anything); FP32 blocks cover P = 3."""
    from paper_2002_04222_gb300 import _lib
    c = case("cylinder_P3_hllc")
    m = dgl.Mesh.from_case(c)
    u = m.project(0.0)
    with pytest.raises(_lib.DGError) as ei:
        dgl.Precond(m).build(u, 0.0, 0.02, J=7, precision="fp64")
    assert ei.value.code == -6
    dgl.Precond(m).build(u, 0.0, 0.02, J=7, precision="fp32")

