"""Host-side argument checks of the C ABI, without a GPU: every entry point
rejects missing handles and pointers (and the invalid settings it checks
before touching the device) with DG_ERR_ARG, before any CUDA call, and every
status code has its own message.  (Nothing here initialises CUDA.)"""
import ctypes

import pytest

DG_ERR_ARG = -1
NULL = None


@pytest.fixture(scope="module")
def lib():
    from paper_2002_04222_gb300 import _lib, build
    import os
    if not os.path.exists(_lib.LIB_PATH):
        build.build()
    return _lib.load(_lib.LIB_PATH)


def test_status_strings_are_distinct(lib):
    msgs = [lib.dg_status_string(c) for c in range(0, -8, -1)]
    assert msgs[0] == b"ok"
    assert all(m for m in msgs) and len(set(msgs)) == len(msgs)
    assert lib.dg_status_string(-99)        # unknown codes still get a message


def test_null_handles_and_pointers_are_rejected(lib):
    from paper_2002_04222_gb300 import _lib
    d = ctypes.c_double
    out = ctypes.c_void_p()
    gcfg = _lib.GmresCfg(10, 2, 1e-2, 0)
    pcfg = _lib.PrecCfg(7, 1, 1.0, 0, 0, 0)
    calls = {
        "dg_mesh_create": (NULL, NULL, NULL, ctypes.byref(out)),
        "dg_mesh_destroy": (NULL,),
        "dg_mesh_info": (NULL, NULL),
        "dg_project": (NULL, d(0.0), NULL, NULL),
        "dg_residual": (NULL, NULL, d(0.0), NULL, NULL),
        "dg_av_factor": (NULL, NULL, NULL, NULL),
        "dg_jvp": (NULL, NULL, NULL, d(0.0), NULL, d(0.0), d(1.0), NULL, NULL),
        "dg_precond_build": (NULL, NULL, d(0.0), d(0.1), ctypes.byref(pcfg), ctypes.byref(out),
                             NULL),
        "dg_precond_apply": (NULL, NULL, NULL, NULL),
        "dg_precond_destroy": (NULL,),
        "dg_gmres": (NULL, NULL, NULL, NULL, d(0.0), d(0.1), NULL, NULL, ctypes.byref(gcfg),
                     NULL, NULL),
        "dg_gmres_noalloc": (NULL, NULL, NULL, NULL, d(0.0), d(0.1), NULL, NULL,
                             ctypes.byref(gcfg), NULL, NULL),
        "sdirk_step": (NULL, NULL, NULL, d(0.0), d(0.1), NULL, NULL, NULL),
        "bdf2_step": (NULL, NULL, NULL, NULL, d(0.0), d(0.1), NULL, NULL, NULL),
        "dg_peak_fp64": (0, NULL, NULL),
        "dg_autotune": (NULL, 1, NULL, NULL),
        "dg_set_tune": (NULL, NULL),
        "dg_guess_create": (NULL, NULL, NULL, ctypes.byref(out)),
        "dg_guess_destroy": (NULL,),
        "dg_guess_push": (NULL, NULL, NULL),
        "dg_guess_ready": (NULL, 0, NULL),
        "dg_guess_predict": (NULL, 0, NULL, NULL, NULL),
        "dg_guess_train": (NULL, 0, NULL, NULL, 1, NULL, NULL, NULL, NULL),
        "dg_guess_params": (NULL, 0, NULL),
        "dg_profile_read": (NULL, 4, NULL),
    }
    missing = set(_lib.SIGNATURES) - set(calls) - {"dg_status_string", "dg_kernel_launches",
                                                   "dg_profile_enable"}
    assert not missing, missing
    for name, args in calls.items():
        assert getattr(lib, name)(*args) == DG_ERR_ARG, name


def test_counters_and_profiling_switch_need_no_device(lib):
    n0 = lib.dg_kernel_launches()
    assert n0 >= 0
    assert lib.dg_profile_enable(1) == 0
    assert lib.dg_profile_enable(0) == 0
    assert lib.dg_kernel_launches() == n0
