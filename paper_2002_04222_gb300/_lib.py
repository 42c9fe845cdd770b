"""ctypes binding of libdgjfnk.so (include/dg.h): argument marshalling only.

Device vectors are torch CUDA float64 tensors (contiguous, layout
[n_elem][n_var][n_mode]); their data pointers and the current CUDA stream are
handed to the C ABI.  There is no fallback: if the library is missing the
import fails.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdgjfnk.so")

DG_OK = 0
STATUS = {0: "ok", -1: "invalid argument", -2: "CUDA error", -3: "out of device memory",
          -4: "non-finite norm", -5: "not converged", -6: "unsupported", -7: "timeout"}
DG_ERR_NOT_CONVERGED = -5
PREC = {"fp64": 0, "fp32": 1, "bf16": 2}
NOALLOC_MAX_DOUBLES = 2097152   # DG_GMRES_NOALLOC_MAX_DOUBLES of include/dg.h


class DGError(RuntimeError):
    def __init__(self, fn, code):
        super().__init__(f"{fn} failed: {STATUS.get(code, code)} ({code})")
        self.code = code


class MeshDesc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("P", ctypes.c_int), ("Q", ctypes.c_int),
                ("n_elem", ctypes.c_int), ("geom_order", ctypes.c_int), ("n_faces", ctypes.c_int),
                ("nodes", ctypes.POINTER(ctypes.c_double)),
                ("faces", ctypes.POINTER(ctypes.c_int32))]


class Physics(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("Pr", ctypes.c_double), ("Ma", ctypes.c_double),
                ("Re", ctypes.c_double), ("T_inf_K", ctypes.c_double), ("beta_s", ctypes.c_double),
                ("viscous", ctypes.c_int), ("mu_law", ctypes.c_int), ("riemann", ctypes.c_int),
                ("forcing", ctypes.c_int), ("field", ctypes.c_int),
                ("fpar", ctypes.c_double * 8), ("n_bc", ctypes.c_int), ("bc", ctypes.c_int * 8),
                ("av", ctypes.c_int), ("av_mu0", ctypes.c_double), ("av_kappa", ctypes.c_double)]


class MeshInfo(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("P", ctypes.c_int), ("Q", ctypes.c_int),
                ("n_elem", ctypes.c_int), ("n_var", ctypes.c_int), ("n_mode", ctypes.c_int),
                ("n_quad", ctypes.c_int), ("n_faces", ctypes.c_int), ("n_dof", ctypes.c_longlong)]


class PrecCfg(ctypes.Structure):
    _fields_ = [("J", ctypes.c_int), ("precision", ctypes.c_int), ("omega", ctypes.c_double),
                ("graphs", ctypes.c_int), ("tc_invert", ctypes.c_int), ("fused", ctypes.c_int),
                ("full_jacobian", ctypes.c_int)]


class GmresCfg(ctypes.Structure):
    _fields_ = [("restart", ctypes.c_int), ("max_cycles", ctypes.c_int), ("rtol", ctypes.c_double),
                ("graphs", ctypes.c_int)]


class GmresStats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("cycles", ctypes.c_int), ("converged", ctypes.c_int),
                ("res0", ctypes.c_double), ("res", ctypes.c_double)]


class SdirkCfg(ctypes.Structure):
    _fields_ = [("tableau", ctypes.c_int), ("alpha", ctypes.c_double), ("abs_tol", ctypes.c_double),
                ("max_newton", ctypes.c_int), ("rebuild", ctypes.c_int), ("use_precond", ctypes.c_int),
                ("gmres", GmresCfg), ("prec", PrecCfg), ("guess", ctypes.c_void_p),
                ("guess_train_iters", ctypes.c_int)]


MAX_STAGES = 6   # DG_MAX_STAGES of include/dg.h
TABLEAU = {"be": 1, "sdirk2": 2, "sdirk3": 3, "esdirk4": 4}


class StepStats(ctypes.Structure):
    _fields_ = [("newton_iters", ctypes.c_int), ("gmres_iters", ctypes.c_int), ("stages", ctypes.c_int),
                ("precond_built", ctypes.c_int), ("stage_newton", ctypes.c_int * MAX_STAGES),
                ("stage_gmres", ctypes.c_int * MAX_STAGES), ("stage_res0", ctypes.c_double * MAX_STAGES),
                ("stage_res", ctypes.c_double * MAX_STAGES), ("guess_used", ctypes.c_int)]


class GuessCfg(ctypes.Structure):
    _fields_ = [("stages", ctypes.c_int), ("hidden", ctypes.c_int), ("mlp", ctypes.c_int),
                ("lr", ctypes.c_float),
                ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("eps", ctypes.c_float),
                ("gate", ctypes.c_float)]


class TuneResult(ctypes.Structure):
    _fields_ = [("vol_epb", ctypes.c_int), ("vol_threads", ctypes.c_int), ("lift_epb", ctypes.c_int),
                ("lift_threads", ctypes.c_int), ("vol_ms", ctypes.c_double),
                ("lift_ms", ctypes.c_double), ("vol_ms_default", ctypes.c_double),
                ("lift_ms_default", ctypes.c_double)]


class KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("launches", ctypes.c_longlong), ("ms", ctypes.c_double)]


# exported symbols and their argument types (mirrors include/dg.h)
VP, D, I = ctypes.c_void_p, ctypes.c_double, ctypes.c_int
SIGNATURES = {
    "dg_mesh_create": [ctypes.POINTER(MeshDesc), ctypes.POINTER(Physics), VP, ctypes.POINTER(VP)],
    "dg_mesh_destroy": [VP],
    "dg_mesh_info": [VP, ctypes.POINTER(MeshInfo)],
    "dg_project": [VP, D, VP, VP],
    "dg_residual": [VP, VP, D, VP, VP],
    "dg_av_factor": [VP, VP, VP, VP],
    "dg_jvp": [VP, VP, VP, D, VP, D, D, VP, VP],
    "dg_precond_build": [VP, VP, D, D, ctypes.POINTER(PrecCfg), ctypes.POINTER(VP), VP],
    "dg_precond_apply": [VP, VP, VP, VP],
    "dg_precond_destroy": [VP],
    "dg_gmres": [VP, VP, VP, VP, D, D, VP, VP, ctypes.POINTER(GmresCfg), ctypes.POINTER(GmresStats), VP],
    "dg_gmres_noalloc": [VP, VP, VP, VP, D, D, VP, VP, ctypes.POINTER(GmresCfg),
                         ctypes.POINTER(GmresStats), VP],
    "sdirk_step": [VP, ctypes.POINTER(SdirkCfg), VP, D, D, ctypes.POINTER(VP), ctypes.POINTER(StepStats), VP],
    "bdf2_step": [VP, ctypes.POINTER(SdirkCfg), VP, VP, D, D, ctypes.POINTER(VP),
                  ctypes.POINTER(StepStats), VP],
    "dg_status_string": [I],
    "dg_kernel_launches": [],
    "dg_autotune": [VP, I, ctypes.POINTER(TuneResult), VP],
    "dg_set_tune": [VP, ctypes.POINTER(TuneResult)],
    "dg_guess_create": [VP, ctypes.POINTER(GuessCfg), ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(VP)],
    "dg_guess_destroy": [VP],
    "dg_guess_push": [VP, VP, VP],
    "dg_guess_ready": [VP, I, ctypes.POINTER(I)],
    "dg_guess_predict": [VP, I, VP, VP, VP],
    "dg_guess_train": [VP, I, VP, VP, I, ctypes.POINTER(D), ctypes.POINTER(D),
                       ctypes.POINTER(ctypes.c_void_p), VP],
    "dg_guess_params": [VP, I, ctypes.POINTER(ctypes.c_void_p)],
    "dg_profile_enable": [I],
    "dg_profile_read": [ctypes.POINTER(KernelTime), I, ctypes.POINTER(I)],
    "dg_peak_fp64": [I, ctypes.POINTER(D), VP],
}


def load(path=LIB_PATH):
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_2002_04222_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, args in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = {"dg_status_string": ctypes.c_char_p,
                      "dg_kernel_launches": ctypes.c_longlong}.get(name, ctypes.c_int)
    return lib


def mesh_desc(mesh, P, Q):
    """ctypes descriptor of a workloads.Mesh (keeps the numpy buffers alive)."""
    nodes = np.ascontiguousarray(mesh.nodes, dtype=np.float64)
    faces = np.ascontiguousarray(mesh.faces, dtype=np.int32)
    d = MeshDesc(mesh.dim, P, Q, mesh.n_elem, mesh.geom_order, mesh.n_faces,
                 nodes.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                 faces.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    d._keep = (nodes, faces)
    return d


def physics(ph):
    p = Physics()
    p.gamma, p.Pr, p.Ma, p.Re = ph.gamma, ph.Pr, ph.Ma, ph.Re
    p.T_inf_K, p.beta_s = ph.T_inf_K, ph.beta_s
    p.viscous, p.mu_law, p.riemann = int(ph.viscous), ph.mu_law, ph.riemann
    p.forcing, p.field = ph.forcing, ph.fid
    for i, v in enumerate(ph.fpar):
        p.fpar[i] = v
    p.n_bc = len(ph.bc)
    for i, v in enumerate(ph.bc):
        p.bc[i] = v
    p.av = int(getattr(ph, "av", 0))
    p.av_mu0 = float(getattr(ph, "av_mu0", 0.0))
    p.av_kappa = float(getattr(ph, "av_kappa", 1.0))
    return p
