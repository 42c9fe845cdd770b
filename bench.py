#!/usr/bin/env python
"""Benchmark of the implicit DG hot path on one GB300 (or N replicas).

A step is one SDIRK2 step (Sec. 3.2, App. A) of the 3-D Taylor-Green vortex on
16^3 periodic hexahedra, P = 3, Q = 6 Gauss points per direction (the
over-integration rule ceil(3(P+1)/2)), Re = 1600, Ma = 0.1, at 10x the explicit
time step (CFL 0.10): each stage runs Newton (alpha = 1e-3 relative
tolerance) with right-preconditioned restarted GMRES(30, rtol 5e-2), the
Jacobian-free product and BRJ(7), the preconditioner rebuilt every 10 steps
(frozen in between).  All arithmetic of the residual, the JFNK difference, the
Krylov vectors and Newton is FP64; the BRJ blocks are stored in the chosen
precision (default FP32, as in the paper).

Output: one JSON line (rank 0).  `value` = DOF-steps per second over all
ranks (n_dof x steps / time); `e2e` repeats the measurement through host
buffers (host->device copy of u before and device->host copy after every
step); `roofline` describes the kernel with the largest device time in the
step; `cpu_baseline` times the CPU oracle on a bounded sample.

--impl reference runs the CPU oracle as the reference arm (rank 0 only).
"""
import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = {"n": 16, "P": 3, "Q": 6, "Re": 1600.0, "Ma": 0.1, "cfl": 0.10, "dt_factor": 10.0}
# turbulent cylinder of Sec. 6.4 on a curved O-grid (quadratic hexes): SDIRK3,
# BF16 BRJ blocks, learned Newton guess.  Time step from the convective CFL of
# Tab. Efficiency-comparison-3900CYLINDER at P = 3 (CFL_c = 1.7, Eq. CFLc) on
# the first radial cell; a short untimed ramp (1/4, 1/2 of it) from the
# synthetic start-up field
CYLINDER = {"n_r": 64, "n_theta": 96, "n_z": 12, "P": 3, "Q": 6, "Re": 3900.0, "Ma": 0.2,
            "cfl_c": 1.7, "seed": 5, "wall_layer": 0.1, "ramp": (0.25, 0.5)}
# the same flow at P = 4 on 24^3 hexes (over-integration Q = 8)
TGV24 = {"n": 24, "P": 4, "Q": 8, "Re": 1600.0, "Ma": 0.1, "cfl": 0.10, "dt_factor": 10.0}
# supersonic shock-wave / boundary-layer interaction of Sec. 6.5 (119 x 39 quads,
# P = 3, Ma 2.15, Re 1e5 on the shock's foot distance, shock at 30.8 degrees),
# artificial-viscosity shock capturing (Sec. 3.1.2), SDIRK2; time step from
# Eq. CFL on the first cell at the wall with c + |u| = 1/Ma + 1
SWBLI = {"nx": 119, "ny": 39, "P": 3, "Q": 5, "Ma": 2.15, "Re": 1.0e5, "beta": 30.8, "cfl": 100.0,
         "ramp": (0.1,), "kappa": 1.0}
SAMPLE_N = 3          # CPU sample: the same case on 3^3 elements (same P, Q, CFL)
FREEZE = 10
# DRAM bytes (read + write) per element and launch from one ncu capture of the
# kernel as it stands (profiles/); a kernel changed since then has no entry
TRAFFIC_PER_ELEM = {("brj_diag", "fp32", 3, 6): 418_400.0, ("brj_diag", "bf16", 3, 6): 209_770.0,
                    ("brj_sweep", "fp32", 3, 6): 439_400.0}


def max_over_ranks(x, world, device="cuda"):
    """The largest of the ranks' values of x (a duration): the job lasts as long
    as its slowest replica.  world = 1 returns x without a process group."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier_all(world):
    """Barrier over the ranks (none for one process)."""
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def job_throughput(units_per_rank, world, seconds):
    """Whole-job throughput of `world` replicas that each processed
    units_per_rank units in `seconds` (the max over ranks)."""
    return world * units_per_rank / seconds


def tgv_dt(n, P, Ma, cfl=0.10, factor=10.0):
    """dt = factor x the explicit step of Eq. CFL on the Taylor-Green box (the
    workload's own rule)."""
    import workloads as w
    return w.tgv_dt(n, P, Ma, cfl, factor)


def cylinder_dt(wl, frac=1.0):
    """dt = CFL_c h_min / (P |u|) (Eq. CFLc, |u| = 1, h_min = the first radial
    cell at the wall), times frac."""
    h = 1.08 ** (wl["n_r"] - 1 - __import__("numpy").arange(wl["n_r"]))
    dr = (20.0 - 0.5) * 1.0 / h.sum()            # first cell (geometric growth 1.08)
    return frac * wl["cfl_c"] * dr / wl["P"]


def swbli_dt(case, wl):
    """dt of Eq. CFL: CFL d_RK dx / (c_lambda (c + |u|) P^2), c_lambda = 0.2,
    d_RK = 2, c + |u| = 1/Ma + 1, dx = the smallest element edge (the first
    cell at the wall)."""
    import numpy as np
    ys = np.unique(case.mesh.nodes[..., 1])
    dx = float(np.diff(ys).min())
    return wl["cfl"] * 2.0 * dx / (0.2 * (1.0 / wl["Ma"] + 1.0) * wl["P"] ** 2)


def cylinder_initial(m, wl):
    """Uniform stream (1, 0, 0) at T = 1, brought to rest at the wall over the
    wall-layer length, plus a piecewise-constant 1% velocity perturbation
    N(0, 1) x 0.01 per element (numpy PCG64, seed 5)."""
    import numpy as np
    import torch
    import workloads as w
    u = m.project(0.0)
    E, nv, nm = m.shape
    n = wl["P"] + 1
    idx = np.indices((n,) * 3).reshape(3, -1)
    one = np.all((idx == 0) | (idx == n - 1), axis=0).astype(np.float64)  # vertex modes
    du = np.zeros((E, nv, nm))
    du[:, 1:4, :] = w.perturbation((E, 3), wl["seed"])[:, :, None] * one[None, None, :]
    u += torch.from_numpy(du).to(u.device)
    return u


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(path)), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# ------------------------------------------------------------------ clocks
class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9 and f[1].isdigit():
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        mhz = sorted(int(r[1]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": mhz[len(mhz) // 2], "sm_max_mhz": int(rows[0][2]), "reasons": reasons,
                "samples": len(rows)}


# ------------------------------------------------------------------ work model
def residual_flops_per_elem(P, Q, d=3):
    """Algorithmic FP64 flops (FMA = 2) of one residual per element, as the
    three kernels implement it; c_F / c_T = flops of the volume flux per Gauss
    point and of the face flux per face point (counted from the flux code)."""
    n, nv = P + 1, d + 2
    c_F, c_T = 190, 420
    bwd = 2 * nv * (n ** 3 * Q + n * n * Q * Q + n * Q ** 3)
    grad = 2 * d * nv * Q ** 4
    trace = 2 * (2 * d) * (1 + d) * nv * Q ** 2 * Q
    vol = bwd + grad + c_F * Q ** 3 + trace
    face = d * Q ** 2 * c_T                   # d faces per element
    spread = 2 * 2 * d * (1 + d) * nv * Q ** 3
    lift = spread + grad + bwd + 2 * d * nv * n ** 4
    return {"dg_vol": vol, "dg_face": face, "dg_lift": lift}


def kernel_work(name, launches, E, nb, prec_bytes, P, Q, d=3):
    """(bound, algorithmic units per launch, unit) of a kernel family.  The
    residual kernels' flop counts are those of the 3-D kernels."""
    f = residual_flops_per_elem(P, Q)
    if name in f:
        return ("alu", f[name] * E, "flop") if d == 3 else (None, None, None)
    if name == "brj_diag":
        return "hbm", E * (nb * nb * prec_bytes + 2 * nb * 8), "byte"
    if name == "brj_sweep":
        # the block, the element's 6 neighbour trace Jacobians (5x5 per face
        # point), q, the own previous iterate and the output, the neighbours'
        # face-slice coefficients (3-D workloads)
        sj = 8 if prec_bytes == 8 else 4
        nv = d + 2
        per = (nb * nb * prec_bytes + 2 * d * nv * nv * Q ** (d - 1) * sj + 3 * nb * 8
               + 2 * d * nv * (P + 1) ** (d - 1) * 8)
        return "hbm", E * per, "byte"
    if name in ("multi_dot", "multi_axpy", "dot", "vector"):
        return "hbm", None, "byte"
    return None, None, None


# ------------------------------------------------------------------ variants
VARIANTS = [("fp64", "plain", True), ("fp32", "plain", False), ("fp32", "plain", True),
            ("bf16", "plain", True), ("bf16", "extrap", True), ("bf16", "learned", True)]


def time_variant(m, u0, dt, precision, guess, fused, steps, warmup, tableau=2):
    """One form of the step (block precision, Newton initial guess, fused BRJ
    sweeps) from the same initial field at the same Newton criterion: each
    stage stops at alpha ||N(S_m)|| (alpha = 1e-3, an absolute number per
    stage that every form computes from its own S_m).  W untimed steps (at
    least 6 for the guess forms, whose network and extrapolation need a
    history), then K steps timed with CUDA events on the launch stream; the
    preconditioner is rebuilt every FREEZE steps in every form."""
    import torch
    import workloads as w
    import paper_2002_04222_gb300 as dgl
    u = u0.clone()
    pc = dgl.Precond(m)
    kw = dict(restart=30, rtol=5e-2, alpha=1e-3, J=7, precision=precision, tableau=tableau,
              graphs=True, fused=fused)
    g = None
    if guess != "plain":
        nb = m.info["n_var"] * m.info["n_mode"]
        params = None
        if guess == "learned":
            params = []
            for st in range(tableau):
                params += w.mlp_params(3 * nb, 256, nb, seed=101 + st, zero_last=True)
        g = dgl.Guess(m, params, stages=tableau, hidden=256, lr=1e-3)
        kw["guess"] = g
        kw["guess_train_iters"] = 4
        warmup = max(warmup, 6)
    state = {"k": 0, "t": 0.0}
    stats = []

    def step():
        st = m.sdirk_step(u, state["t"], dt, precond=pc, rebuild=state["k"] % FREEZE == 0, **kw)
        state["k"] += 1
        state["t"] += dt
        stats.append(st)

    for _ in range(warmup):
        step()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    stats.clear()
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    out = {"blocks": precision, "guess": guess, "fused": fused, "ms_per_step": round(ms, 3),
           "newton_per_step": sum(s["newton_iters"] for s in stats) / steps,
           "gmres_per_step": sum(s["gmres_iters"] for s in stats) / steps,
           "converged": all(s["converged"] for s in stats),
           "guess_used_per_step": sum(s["guess_used"] for s in stats) / steps}
    pc.close()
    if g is not None:
        g.close()
    return out


# ------------------------------------------------------------------ our arm
def run_ours(args, rank, world):
    import torch
    import workloads as w
    import paper_2002_04222_gb300 as dgl

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    cyl = args.workload == "cylinder"
    sw = args.workload == "swbli"
    wl = {"cylinder": CYLINDER, "tgv24": TGV24, "swbli": SWBLI}.get(args.workload, WORKLOAD)
    if cyl:
        case = w.cylinder_case(wl["n_r"], wl["n_theta"], wl["n_z"], P=wl["P"], Q=wl["Q"],
                               Re=wl["Re"], Ma=wl["Ma"], wall_layer=wl["wall_layer"])
        dt = cylinder_dt(wl)
    elif sw:
        wl["cfl"] = args.cfl if args.cfl is not None else wl["cfl"]
        wl["beta"] = args.shock_angle if args.shock_angle is not None else wl["beta"]
        wl["kappa"] = args.av_kappa if args.av_kappa is not None else wl["kappa"]
        case = w.swbli_case(nx=wl["nx"], ny=wl["ny"], P=wl["P"], Q=wl["Q"], Ma=wl["Ma"],
                            Re=wl["Re"], beta_deg=wl["beta"])
        case.phys.av_kappa = wl["kappa"]
        dt = swbli_dt(case, wl)
    else:
        case = w.tgv_case(n=wl["n"], P=wl["P"], Q=wl["Q"], Re=wl["Re"], Ma=wl["Ma"])
        dt = tgv_dt(wl["n"], wl["P"], wl["Ma"], wl["cfl"], wl["dt_factor"])
    m = dgl.Mesh.from_case(case)
    tuning = dgl.apply_tuning(m)          # stored autotuning choice for this (dim, P, Q)
    ndof = m.info["n_dof"]
    E = m.info["n_elem"]
    nb = m.info["n_var"] * m.info["n_mode"]
    u = cylinder_initial(m, wl) if cyl else m.project(0.0)
    pc = dgl.Precond(m)
    tableau = 3 if cyl else 2
    nstage = tableau
    kw = dict(restart=30, rtol=5e-2, alpha=1e-3, J=7, precision=args.precision, tableau=tableau,
              graphs=True, fused=args.fused)
    if args.guess != "plain":
        # initial guess S_m + previous stage increment (+ learned MLP correction, one
        # per stage, 2 x 256 hidden, seeded weights with a zero output layer,
        # trained online during the warm-up and the timed steps)
        nb = m.info["n_var"] * m.info["n_mode"]
        params = None
        if args.guess == "learned":
            params = []
            for st in range(nstage):
                params += w.mlp_params(3 * nb, 256, nb, seed=101 + st, zero_last=True)
        kw["guess"] = dgl.Guess(m, params, stages=nstage, hidden=256, lr=1e-3)
        kw["guess_train_iters"] = 4
        args.warmup = max(args.warmup, 6)
    state = {"k": 0, "t": 0.0}
    stats = []

    def step(uu, dt_step=dt, rebuild=None):
        rb = (state["k"] % FREEZE == 0) if rebuild is None else rebuild
        st = m.sdirk_step(uu, state["t"], dt_step, precond=pc, rebuild=rb, **kw)
        state["k"] += 1
        state["t"] += dt_step
        stats.append(st)
        return st

    if cyl or sw:
        # start-up (untimed): steps at fractions of dt from the synthetic field
        # (cylinder: dt/4, dt/2; SWBLI: dt/10), preconditioner rebuilt at every
        # step size, then the step counter restarts so that the timed steps see
        # the regular rebuild cadence
        for f in wl["ramp"]:
            step(u, dt * f, rebuild=True)
        state["k"] = 0

    def barrier():
        barrier_all(world)

    for _ in range(args.warmup):
        step(u)
    torch.cuda.synchronize()
    clocks = Clocks(dev)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = dgl.kernel_launches()
    stats.clear()
    e0.record(stream)
    for _ in range(args.steps):
        step(u)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = dgl.kernel_launches() - l0
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    timed_stats = list(stats)
    ms = max_over_ranks(ms, world)
    value = job_throughput(ndof * args.steps, world, ms / 1e3)

    # per-kernel device time over the same number of further steps (CUDA events
    # on the launch stream, recorded by the library)
    dgl.profile_enable(True)
    dgl.profile_read()
    for _ in range(args.steps):
        step(u)
    prof = dgl.profile_read()
    dgl.profile_enable(False)
    # measured FP64 FMA throughput of this GPU (the residual kernels' pipe)
    fp64_peak = dgl.peak_fp64(20)
    total_k = sum(v[1] for v in prof.values())
    dom = max(prof, key=lambda k: prof[k][1])
    pk, how = peaks()
    prec_bytes = {"fp64": 8, "fp32": 4, "bf16": 2}[args.precision]
    dim = m.info["dim"]
    bound, work, unit = kernel_work(dom, prof[dom][0], E, nb, prec_bytes, wl["P"], wl["Q"], dim)
    avg_ms = prof[dom][1] / prof[dom][0]
    roof = {"kernel": dom, "launches": prof[dom][0], "avg_ms": avg_ms,
            "share": prof[dom][1] / total_k, "traffic": None}
    tkey = (dom, args.precision, wl["P"], wl["Q"])
    if tkey in TRAFFIC_PER_ELEM:
        roof["traffic"] = TRAFFIC_PER_ELEM[tkey] * E
        roof["traffic_source"] = "ncu dram bytes of a small-case capture scaled by elements"
    if bound == "hbm":
        roof.update(bound="hbm", achieved=work / (avg_ms / 1e3) / 1e9, peak=pk["hbm_gbs"], unit="GB/s",
                    peak_source=how)
    elif bound == "alu":
        roof.update(bound="alu", achieved=work / (avg_ms / 1e3) / 1e12, peak=fp64_peak,
                    unit="TFLOP/s",
                    peak_source="measured in this run: dg_peak_fp64 (FP64 FMA chains)")
    else:
        roof.update(bound=None, achieved=None, peak=None, unit=None)
    if roof.get("achieved") is not None:
        roof["frac"] = roof["achieved"] / roof["peak"]
    kernels = {k: {"launches": v[0], "ms": round(v[1], 3), "share": round(v[1] / total_k, 4)}
               for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])}

    # residual throughput (GDOF/s) on the same mesh and state
    r = m.residual(u)
    torch.cuda.synchronize()
    e0.record(stream)
    nres = 20
    for _ in range(nres):
        m.residual(u, out=r)
    e1.record(stream)
    torch.cuda.synchronize()
    res_ms = e0.elapsed_time(e1) / nres
    # the residual's roofline: algorithmic FP64 flops (the kernels' own count)
    # over the measured FP64 FMA throughput of this GPU, taken in this run
    rflops = sum(residual_flops_per_elem(wl["P"], wl["Q"]).values()) * E
    res_roof = {"bound": "alu", "achieved": rflops / (res_ms / 1e3) / 1e12, "peak": fp64_peak,
                "unit": "TFLOP/s", "frac": rflops / (res_ms / 1e3) / 1e12 / fp64_peak,
                "flops_per_launch": rflops, "avg_ms": res_ms,
                "peak_source": "measured in this run: dg_peak_fp64 (FP64 FMA chains at full "
                               "occupancy, CUDA events)"}
    if dim != 3:
        res_roof = {"bound": "alu", "achieved": None, "peak": fp64_peak, "unit": "TFLOP/s",
                    "avg_ms": res_ms, "note": "flop counts are those of the 3-D kernels"}
    for kname in ("dg_vol", "dg_face", "dg_lift"):
        if kname in prof and not cyl and dim == 3:
            kf = residual_flops_per_elem(wl["P"], wl["Q"])[kname] * E
            kms = prof[kname][1] / prof[kname][0]
            res_roof[kname] = {"avg_ms": round(kms, 4),
                               "frac": round(kf / (kms / 1e3) / 1e12 / fp64_peak, 3)}

    # end to end through host buffers
    e2e = None
    if not args.no_e2e:
        host = torch.empty(u.shape, dtype=torch.float64, pin_memory=True)
        host.copy_(u)
        dev_u = torch.empty_like(u)
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            dev_u.copy_(host, non_blocking=True)
            step(dev_u)
            host.copy_(dev_u, non_blocking=True)
            torch.cuda.synchronize()
        el = max_over_ranks(time.perf_counter() - t0, world)
        nbytes = ndof * 8
        e2e = {"value": job_throughput(ndof * args.steps, world, el), "unit": "DOF*step/s",
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes}

    variants = None
    if args.variants and not cyl and not sw:
        u0 = m.project(0.0)
        variants = [time_variant(m, u0, dt, p_, g_, f_, args.steps, args.warmup)
                    for p_, g_, f_ in VARIANTS]
    av_elements = int((m.av_factor(u) > 0).sum().item()) if sw else None
    newton = [s["newton_iters"] for s in timed_stats]
    gm = [s["gmres_iters"] for s in timed_stats]
    if sw:
        metric = ("SDIRK2 step throughput at fixed Newton tolerance (DOF-steps/s); SWBLI "
                  f"{wl['nx']}x{wl['ny']} quads P={wl['P']}, Ma {wl['Ma']:g}, shock {wl['beta']:g} deg, "
                  f"artificial viscosity, CFL {wl['cfl']:g}")
        wname = (f"swbli{wl['nx']}x{wl['ny']}_P{wl['P']}_Q{wl['Q']}_Ma{wl['Ma']:g}_beta{wl['beta']:g}"
                 f"_av_k{wl['kappa']:g}_sdirk2_cfl{wl['cfl']:g}")
        data = ("synthetic (the projected oblique-shock field: uniform stream below the shock "
                "line, Rankine-Hugoniot state above)")
    elif cyl:
        metric = ("SDIRK3 step throughput at fixed Newton tolerance (DOF-steps/s); curved O-grid "
                  f"{wl['n_r']}x{wl['n_theta']}x{wl['n_z']} quadratic hexes P=3, CFL_c {wl['cfl_c']:g}")
        wname = (f"cylinder_ogrid{wl['n_r']}x{wl['n_theta']}x{wl['n_z']}_P{wl['P']}_Q{wl['Q']}"
                 f"_sdirk3_cflc{wl['cfl_c']:g}")
        data = ("synthetic (uniform stream at rest on the wall over 0.1 D + seeded 1% velocity "
                "perturbation; start-up ramp dt/4, dt/2 before the warm-up)")
    else:
        metric = ("SDIRK2 step throughput at fixed Newton tolerance (DOF-steps/s); "
                  f"TGV {wl['n']}^3 hexes P={wl['P']}, 10x explicit dt")
        wname = f"tgv{wl['n']}^3_P{wl['P']}_Q{wl['Q']}_sdirk2_dt{wl['dt_factor']:g}xexplicit"
        data = "synthetic (analytic Taylor-Green initial field)"
    out = {
        "metric": metric,
        "value": value,
        "unit": "DOF*step/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": data,
        "config": {"workload": wname,
                   "n_dof": ndof, "dt": dt, "newton_alpha": 1e-3, "gmres": "restart 30, rtol 5e-2",
                   "precond": f"BRJ(7) {args.precision} blocks, rebuilt every {FREEZE} steps"
                              + (", fused sweeps" if args.fused else ""),
                   "initial_guess": {"plain": "S_m (plain)",
                                     "extrap": "S_m + previous stage increment",
                                     "learned": "S_m + previous stage increment + per-element "
                                                "MLP correction (2x256, BF16, online Adam)"}[args.guess],
                   "l2": "working set > L2 (BRJ blocks %.2f GB read per sweep)" % (E * nb * nb * prec_bytes / 1e9),
                   "parallelism": f"replicas x{world}",
                   "launch_shapes": ({k: tuning[k] for k in ("vol_epb", "vol_threads", "lift_epb",
                                                             "lift_threads")}
                                     if tuning else "built-in defaults")},
        "newton_per_step": sum(newton) / len(newton),
        "av_elements": av_elements,
        "gmres_per_step": sum(gm) / len(gm),
        "residual_gdofs": ndof / (res_ms / 1e3) / 1e9,
        "residual_ms": res_ms,
        # the preconditioner build inside the profiled steps (one per FREEZE steps):
        # its kernels' time, and the step time with the build taken out
        "rebuild_kernels_ms": round(sum(prof[k][1] for k in ("brj_weights", "brj_tracejac",
                                                             "brj_block", "brj_invert") if k in prof), 3),
        "ms_per_step_frozen": ms / args.steps - sum(prof[k][1] for k in ("brj_weights", "brj_tracejac",
                                                                         "brj_block", "brj_invert")
                                                    if k in prof) / args.steps,
        "gpu_launches": launches,
        "clocks": clk,
        "roofline": roof,
        "residual_roofline": res_roof,
        "variants": variants,
        "kernels": kernels,
        "e2e": e2e,
    }
    return out


# ------------------------------------------------------------------ CPU oracle
def oracle_sample(steps, warmup):
    """The CPU oracle (as it stands) on the bounded sample: same P, Q and CFL on
    SAMPLE_N^3 elements; BRJ built every FREEZE steps."""
    import numpy as np
    import workloads as w
    from oracle.dg import DG
    from oracle import implicit as im
    wl = WORKLOAD
    c = w.tgv_case(n=SAMPLE_N, P=wl["P"], Q=wl["Q"], Re=wl["Re"], Ma=wl["Ma"])
    dg = DG(c.mesh, c.P, c.Q, c.phys)
    u = dg.project_exact()
    dt = tgv_dt(SAMPLE_N, wl["P"], wl["Ma"], wl["cfl"], wl["dt_factor"])
    lam = 1 - math.sqrt(2) / 2
    cfg = im.NewtonConfig(alpha=1e-3, gmres=im.GmresConfig(restart=30, rtol=5e-2))
    pc = None
    t = 0.0
    times = []
    for k in range(warmup + steps):
        t0 = time.perf_counter()
        if k % FREEZE == 0:
            pc = im.BRJ(dg, u, t, dt * lam, J=7)
        u, _ = im.sdirk_step(dg, u, t, dt, "sdirk2", pc.apply, cfg)
        t += dt
        times.append(time.perf_counter() - t0)
    timed = times[warmup:]
    return u.size, sum(timed), len(timed)


def cpu_baseline_sample():
    """One build + one step of the oracle on the sample, amortised like the
    GPU run (build every FREEZE steps)."""
    import workloads as w
    from oracle.dg import DG
    from oracle import implicit as im
    wl = WORKLOAD
    c = w.tgv_case(n=SAMPLE_N, P=wl["P"], Q=wl["Q"], Re=wl["Re"], Ma=wl["Ma"])
    dg = DG(c.mesh, c.P, c.Q, c.phys)
    u = dg.project_exact()
    dt = tgv_dt(SAMPLE_N, wl["P"], wl["Ma"], wl["cfl"], wl["dt_factor"])
    lam = 1 - math.sqrt(2) / 2
    cfg = im.NewtonConfig(alpha=1e-3, gmres=im.GmresConfig(restart=30, rtol=5e-2))
    t0 = time.perf_counter()
    pc = im.BRJ(dg, u, 0.0, dt * lam, J=7)
    tb = time.perf_counter() - t0
    t0 = time.perf_counter()
    im.sdirk_step(dg, u, 0.0, dt, "sdirk2", pc.apply, cfg)
    ts = time.perf_counter() - t0
    per_step = ts + tb / FREEZE
    return {"value": u.size / per_step, "unit": "DOF*step/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"TGV {SAMPLE_N}^3 hexes P={wl['P']} Q={wl['Q']} ({u.size} DOF), same CFL: one BRJ "
                      f"build ({tb:.1f} s, amortised over {FREEZE} steps) + one SDIRK2 step ({ts:.1f} s), "
                      f"numpy FP64"}


def run_reference(args):
    ndof, secs, k = oracle_sample(args.steps, args.warmup)
    value = ndof * k / secs
    return {
        "impl": "reference",
        "metric": "SDIRK2 step throughput at fixed Newton tolerance (DOF-steps/s); "
                  "TGV 16^3 hexes P=3, 10x explicit dt",
        "value": value, "unit": "DOF*step/s", "n_gpus": 1, "steps": k, "warmup": args.warmup,
        "ms_per_step": secs / k * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (analytic Taylor-Green initial field)",
        "config": {"workload": f"tgv{WORKLOAD['n']}^3_P{WORKLOAD['P']}_Q{WORKLOAD['Q']}_sdirk2_dt10xexplicit",
                   "sample": f"{SAMPLE_N}^3 elements, same P, Q, CFL"},
        "cpu_baseline": {"value": value, "unit": "DOF*step/s", "cores": os.cpu_count(), "kind": "oracle",
                         "sample": f"TGV {SAMPLE_N}^3 hexes, {ndof} DOF, {k} steps after {args.warmup} "
                                   f"warm-up, BRJ rebuilt every {FREEZE} steps"},
        "e2e": {"value": value, "unit": "DOF*step/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp64", "fp32", "bf16"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--guess", default="plain", choices=["plain", "extrap", "learned"],
                    help="Newton initial guess: S_m, S_m + previous stage increment, or that plus "
                         "the learned MLP correction")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--variants", action=argparse.BooleanOptionalAction, default=True,
                    help="also time the step's forms (FP64/FP32/BF16 blocks, fused sweeps, "
                         "extrapolated and learned guesses) in the same run")
    ap.add_argument("--fused", action=argparse.BooleanOptionalAction, default=True,
                    help="BRJ sweeps after the first as one off-diagonal + block kernel each "
                         "(default; --no-fused: separate off-diagonal and block launches)")
    ap.add_argument("--workload", default="tgv", choices=["tgv", "tgv24", "cylinder", "swbli"],
                    help="tgv: the Taylor-Green benchmark (default, 16^3 P=3); tgv24: 24^3 P=4 "
                         "Q=8; cylinder: the curved O-grid workload (SDIRK3, BF16 blocks, learned "
                         "guess unless overridden); swbli: the supersonic shock / boundary-layer "
                         "workload with artificial viscosity (SDIRK2, 119x39 P=3)")
    ap.add_argument("--cfl", type=float, default=None,
                    help="swbli only: CFL of Eq. CFL (default 100)")
    ap.add_argument("--shock-angle", type=float, default=None,
                    help="swbli only: shock angle in degrees (default 30.8)")
    ap.add_argument("--av-kappa", type=float, default=None,
                    help="swbli only: half-width of the sensor's ramp in decades (default 1)")
    ap.add_argument("--elems", type=int, default=WORKLOAD["n"],
                    help="elements per direction (16 = the benchmark; smaller only for profiler captures)")
    args = ap.parse_args()
    WORKLOAD["n"] = args.elems
    if args.workload != "tgv":
        args.no_cpu_baseline = True    # the oracle sample is the 16^3 P=3 Taylor-Green case
    if args.workload == "cylinder":
        if "--precision" not in sys.argv:
            args.precision = "bf16"
        if "--guess" not in sys.argv:
            args.guess = "learned"
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    out = run_ours(args, rank, world)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline_sample()
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
