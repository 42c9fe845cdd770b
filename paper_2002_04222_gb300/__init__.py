"""GB300 (sm_103a) implementation of the implicit spectral/hp DG compressible
Navier-Stokes hot path: DG residual, Jacobian-free Newton-Krylov product,
restarted GMRES, block relaxed Jacobi preconditioner, Newton and SDIRK
(arXiv 2002.04222, Sec. 3-4).

The compute path is the CUDA library libdgjfnk.so behind the C ABI of
include/dg.h; this module only marshals torch CUDA tensors and host
descriptors into it.  There is no CPU path.
"""
import ctypes

import torch

from . import _lib

_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        _LIB = _lib.load()
    return _LIB


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    if t is None:
        return None
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA float64 tensor")
    return ctypes.c_void_p(t.data_ptr())


def _check(name, code, ok=(0,)):
    if code not in ok:
        raise _lib.DGError(name, code)
    return code


class Mesh:
    """A mesh handle (dg_mesh_t) built from a workloads mesh, P, Q and
    Physics record."""

    def __init__(self, mesh, P, Q, phys, stream=None):
        self._lib = lib()
        self._desc = _lib.mesh_desc(mesh, P, Q)
        self._phys = _lib.physics(phys)
        h = ctypes.c_void_p()
        _check("dg_mesh_create", self._lib.dg_mesh_create(ctypes.byref(self._desc),
                                                          ctypes.byref(self._phys),
                                                          _stream(stream), ctypes.byref(h)))
        self.handle = h
        info = _lib.MeshInfo()
        _check("dg_mesh_info", self._lib.dg_mesh_info(h, ctypes.byref(info)))
        self.info = {f: getattr(info, f) for f, _ in _lib.MeshInfo._fields_}
        self.shape = (info.n_elem, info.n_var, info.n_mode)

    @classmethod
    def from_case(cls, case, stream=None):
        return cls(case.mesh, case.P, case.Q, case.phys, stream)

    def close(self):
        if self.handle:
            self._lib.dg_mesh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def empty(self):
        return torch.empty(self.shape, dtype=torch.float64, device="cuda")

    def project(self, t=0.0, out=None, stream=None):
        out = self.empty() if out is None else out
        _check("dg_project", self._lib.dg_project(self.handle, t, _ptr(out), _stream(stream)))
        return out

    def residual(self, u, t=0.0, out=None, stream=None):
        out = self.empty() if out is None else out
        _check("dg_residual", self._lib.dg_residual(self.handle, _ptr(u), t, _ptr(out),
                                                    _stream(stream)))
        return out

    def av_factor(self, u, out=None, stream=None):
        """Per-element artificial-viscosity factor mu_0 S_e h_e / P at u
        (shock capturing, Sec. 3.1.2): a float64 tensor of n_elem values."""
        out = torch.empty(self.shape[0], dtype=torch.float64, device=u.device) if out is None else out
        _check("dg_av_factor", self._lib.dg_av_factor(self.handle, _ptr(u), _ptr(out),
                                                      _stream(stream)))
        return out

    def jvp(self, u, r_u, v, t=0.0, alpha=0.0, beta=1.0, out=None, stream=None):
        out = self.empty() if out is None else out
        _check("dg_jvp", self._lib.dg_jvp(self.handle, _ptr(u), _ptr(r_u), t, _ptr(v), alpha, beta,
                                          _ptr(out), _stream(stream)))
        return out

    def gmres(self, u, r_u, b, t=0.0, dt_a=0.0, precond=None, restart=30, max_cycles=10,
              rtol=5e-2, graphs=False, out=None, stream=None):
        """dg_gmres; graphs=True replays each Arnoldi step as one CUDA graph."""
        out = self.empty() if out is None else out
        cfg = _lib.GmresCfg(restart, max_cycles, rtol, int(graphs))
        st = _lib.GmresStats()
        code = self._lib.dg_gmres(self.handle, precond.handle if precond else None, _ptr(u),
                                  _ptr(r_u), t, dt_a, _ptr(b), _ptr(out), ctypes.byref(cfg),
                                  ctypes.byref(st), _stream(stream))
        _check("dg_gmres", code, ok=(0, _lib.DG_ERR_NOT_CONVERGED))
        return out, {f: getattr(st, f) for f, _ in _lib.GmresStats._fields_}

    def gmres_noalloc(self, u, r_u, b, out, t=0.0, dt_a=0.0, precond=None, restart=30,
                      max_cycles=10, rtol=5e-2, stream=None):
        """dg_gmres_noalloc: the same solve as gmres() for callers that cannot
        allocate device memory; the Krylov basis lives in the library's fixed
        static device array and `out` must be supplied by the caller."""
        cfg = _lib.GmresCfg(restart, max_cycles, rtol)
        st = _lib.GmresStats()
        code = self._lib.dg_gmres_noalloc(self.handle, precond.handle if precond else None,
                                          _ptr(u), _ptr(r_u), t, dt_a, _ptr(b), _ptr(out),
                                          ctypes.byref(cfg), ctypes.byref(st), _stream(stream))
        _check("dg_gmres_noalloc", code, ok=(0, _lib.DG_ERR_NOT_CONVERGED))
        return out, {f: getattr(st, f) for f, _ in _lib.GmresStats._fields_}

    @staticmethod
    def _step_cfg(tableau, alpha, abs_tol, max_newton, rebuild, use_precond, restart, max_cycles,
                  rtol, J, precision, omega, guess, guess_train_iters, graphs, fused,
                  full_jacobian=False):
        tab = _lib.TABLEAU[tableau] if isinstance(tableau, str) else tableau
        return _lib.SdirkCfg(tab, alpha, abs_tol, max_newton, int(rebuild), int(use_precond),
                             _lib.GmresCfg(restart, max_cycles, rtol, int(graphs)),
                             _lib.PrecCfg(J, _lib.PREC[precision], omega, int(graphs), 0,
                                          int(fused), int(full_jacobian)),
                             guess.handle if guess is not None else None, guess_train_iters)

    def sdirk_step(self, u, t, dt, precond=None, tableau=2, alpha=1e-3, abs_tol=0.0,
                   max_newton=20, rebuild=False, restart=30, max_cycles=10, rtol=5e-2,
                   J=7, precision="fp64", omega=1.0, use_precond=True, guess=None,
                   guess_train_iters=4, graphs=False, fused=False, full_jacobian=False,
                   stream=None):
        """One implicit Runge-Kutta step in place on u (tableau: 1/"be",
        2/"sdirk2", 3/"sdirk3", 4/"esdirk4"); `precond` is a Precond holder
        whose handle is built (or reused, frozen) by the library; `guess` an
        optional Guess (learned initial guess, trained on the converged
        stages); graphs=True replays the BRJ applies and the GMRES Arnoldi
        steps as CUDA graphs; fused=True runs each BRJ sweep after the first
        as one kernel."""
        cfg = self._step_cfg(tableau, alpha, abs_tol, max_newton, rebuild, use_precond, restart,
                             max_cycles, rtol, J, precision, omega, guess, guess_train_iters,
                             graphs, fused, full_jacobian)
        st = _lib.StepStats()
        holder = precond if precond is not None else Precond(self)
        code = self._lib.sdirk_step(self.handle, ctypes.byref(cfg), _ptr(u), t, dt,
                                    ctypes.byref(holder.handle), ctypes.byref(st), _stream(stream))
        return self._step_out("sdirk_step", code, st)

    def bdf2_step(self, u, u_prev, t, dt, precond=None, alpha=1e-3, abs_tol=0.0, max_newton=20,
                  rebuild=False, restart=30, max_cycles=10, rtol=5e-2, J=7, precision="fp64",
                  omega=1.0, use_precond=True, graphs=False, fused=False, stream=None):
        """One BDF2 step: u (u^n) becomes u^{n+1} and u_prev (u^{n-1}) becomes u^n."""
        cfg = self._step_cfg(2, alpha, abs_tol, max_newton, rebuild, use_precond, restart,
                             max_cycles, rtol, J, precision, omega, None, 0, graphs, fused)
        st = _lib.StepStats()
        holder = precond if precond is not None else Precond(self)
        code = self._lib.bdf2_step(self.handle, ctypes.byref(cfg), _ptr(u), _ptr(u_prev), t, dt,
                                   ctypes.byref(holder.handle), ctypes.byref(st), _stream(stream))
        return self._step_out("bdf2_step", code, st)

    @staticmethod
    def _step_out(name, code, st):
        _check(name, code, ok=(0, _lib.DG_ERR_NOT_CONVERGED))
        out = {f: getattr(st, f) for f, _ in _lib.StepStats._fields_}
        for k in ("stage_newton", "stage_gmres", "stage_res0", "stage_res"):
            out[k] = list(out[k])[: st.stages]
        out["converged"] = code == 0
        return out


class Precond:
    """Holder of a BRJ preconditioner handle (dg_precond_t)."""

    def __init__(self, mesh):
        self.mesh = mesh
        self.handle = ctypes.c_void_p()
        self._lib = lib()

    def build(self, u, t=0.0, dt_a=0.0, J=7, precision="fp64", omega=1.0, graphs=False,
              tc_invert=False, fused=False, full_jacobian=False, stream=None):
        """dg_precond_build; full_jacobian=True keeps terms 4-5 of the element
        Jacobian (the paper neglects them)."""
        cfg = _lib.PrecCfg(J, _lib.PREC[precision], omega, int(graphs), int(tc_invert), int(fused),
                           int(full_jacobian))
        _check("dg_precond_build", self._lib.dg_precond_build(
            self.mesh.handle, _ptr(u), t, dt_a, ctypes.byref(cfg), ctypes.byref(self.handle),
            _stream(stream)))
        return self

    def apply(self, q, out=None, stream=None):
        out = self.mesh.empty() if out is None else out
        _check("dg_precond_apply", self._lib.dg_precond_apply(self.handle, _ptr(q), _ptr(out),
                                                              _stream(stream)))
        return out

    def close(self):
        if self.handle:
            self._lib.dg_precond_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def kernel_launches():
    """Number of CUDA kernels the library has launched since it was loaded."""
    return int(lib().dg_kernel_launches())


def peak_fp64(reps=20, stream=None):
    """Measured FP64 FMA throughput (TFLOP/s) of the current GPU (dg_peak_fp64)."""
    out = ctypes.c_double()
    _check("dg_peak_fp64", lib().dg_peak_fp64(reps, ctypes.byref(out), _stream(stream)))
    return out.value


def profile_enable(on=True):
    _check("dg_profile_enable", lib().dg_profile_enable(int(on)))


def profile_read(cap=32):
    """{kernel family: (launches, total ms)} since the previous read."""
    arr = (_lib.KernelTime * cap)()
    n = ctypes.c_int()
    _check("dg_profile_read", lib().dg_profile_read(arr, cap, ctypes.byref(n)))
    return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].ms)) for i in range(n.value)}


class Guess:
    """Holder of a learned-initial-guess handle (dg_guess_t): the previous
    step's stage increment plus, when `params` is given, one MLP correction per
    SDIRK stage (`params`: the 6*stages FP32 host arrays W1, b1, W2, b2, W3, b3
    of each stage, initial values); params=None keeps the extrapolation only."""

    def __init__(self, mesh, params=None, stages=2, hidden=256, lr=1e-3, beta1=0.9,
                 beta2=0.999, eps=1e-8, gate=0.2):
        import numpy as np
        self.mesh = mesh
        self._lib = lib()
        self._arrs = [np.ascontiguousarray(p, dtype=np.float32) for p in (params or [])]
        ptrs = (ctypes.c_void_p * max(1, len(self._arrs)))(*[a.ctypes.data for a in self._arrs])
        cfg = _lib.GuessCfg(stages, hidden if params else 0, 1 if params else 0, lr, beta1, beta2,
                            eps, gate)
        self.handle = ctypes.c_void_p()
        _check("dg_guess_create", self._lib.dg_guess_create(mesh.handle, ctypes.byref(cfg), ptrs,
                                                            ctypes.byref(self.handle)))
        self.shapes = [a.shape for a in self._arrs[:6]]

    def push(self, u, stream=None):
        _check("dg_guess_push", self._lib.dg_guess_push(self.handle, _ptr(u), _stream(stream)))

    def ready(self, stage):
        r = ctypes.c_int()
        _check("dg_guess_ready", self._lib.dg_guess_ready(self.handle, stage, ctypes.byref(r)))
        return bool(r.value)

    def predict(self, stage, S, out=None, stream=None):
        out = self.mesh.empty() if out is None else out
        _check("dg_guess_predict", self._lib.dg_guess_predict(self.handle, stage, _ptr(S),
                                                              _ptr(out), _stream(stream)))
        return out

    def train(self, stage, S, u, iters=1, grads=False, stream=None):
        """Adam steps on target u - S; returns (loss before, loss after, grads at
        entry or None)."""
        import numpy as np
        l0, l1 = ctypes.c_double(), ctypes.c_double()
        g = [np.zeros(s, dtype=np.float32) for s in self.shapes] if grads else None
        gp = (ctypes.c_void_p * 6)(*[a.ctypes.data for a in g]) if grads else None
        _check("dg_guess_train", self._lib.dg_guess_train(
            self.handle, stage, _ptr(S), _ptr(u), iters, ctypes.byref(l0), ctypes.byref(l1), gp,
            _stream(stream)))
        return l0.value, l1.value, g

    def params(self, stage):
        import numpy as np
        out = [np.zeros(s, dtype=np.float32) for s in self.shapes]
        ptrs = (ctypes.c_void_p * 6)(*[a.ctypes.data for a in out])
        _check("dg_guess_params", self._lib.dg_guess_params(self.handle, stage, ptrs))
        return out

    def close(self):
        if self.handle:
            self._lib.dg_guess_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


TUNING_TABLE = __import__("os").path.join(__import__("os").path.dirname(__file__), "tuning.json")


def autotune(mesh, reps=5, stream=None):
    """Time the launch shapes of the sum-factorisation kernels on `mesh`, keep
    the fastest, and return the choice (a dict) with its timings."""
    r = _lib.TuneResult()
    _check("dg_autotune", lib().dg_autotune(mesh.handle, reps, ctypes.byref(r), _stream(stream)))
    return {f: getattr(r, f) for f, _ in _lib.TuneResult._fields_}


def apply_tuning(mesh, table_path=TUNING_TABLE):
    """Apply the stored tuning-table entry of this mesh's (dim, P, Q), if any."""
    import json
    import os
    if not os.path.exists(table_path):
        return None
    key = f"{mesh.info['dim']}d_P{mesh.info['P']}_Q{mesh.info['Q']}"
    entry = json.load(open(table_path)).get(key)
    if entry is None:
        return None
    r = _lib.TuneResult(entry["vol_epb"], entry["vol_threads"], entry["lift_epb"],
                        entry["lift_threads"], 0.0, 0.0, 0.0, 0.0)
    _check("dg_set_tune", lib().dg_set_tune(mesh.handle, ctypes.byref(r)))
    return entry
