"""ctypes view of libfmm2d.so: the C ABI declared in include/fmm2d.h, under the
same names.  Argument marshalling only; every step of the method runs in the
library's CUDA kernels.  Loading fails loudly when the library is missing."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfmm2d.so")

FMM_OK = 0
FMM_ERR_INVALID_ARG = 1
FMM_ERR_CUDA = 2
FMM_ERR_OOM = 3
FMM_ERR_TIMEOUT = 4
FMM_ERR_NONFINITE = 5

FMM_PATH_FP32 = 0
FMM_PATH_FP64 = 1

FMM_FLAG_NO_GRAPH = 1
FMM_FLAG_SERIAL = 2
FMM_FLAG_TIMING = 4
FMM_FLAG_GRAPH = 8
FMM_FLAG_PERSISTENT = 16

FMM_P_MAX = 32

EXPORT = dict(perm=0, bstart=1, bcount=2, center=3, radius=4, nstrong=5, strong=6, nweak=7, weak=8,
              mpole=9, local=10, near=11, inst=12, rho=13, soff=14, woff=15, m2l_items=16, m2l_rows=17,
              p2p_items=18, p2p_rows=19)


class FMMParams(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int), ("theta", ctypes.c_double), ("nlevels", ctypes.c_int),
                ("path", ctypes.c_int), ("flags", ctypes.c_int)]


class FMMTreeInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("ninst", ctypes.c_int), ("nlevels_max", ctypes.c_int),
                ("p", ctypes.c_int), ("path", ctypes.c_int), ("theta", ctypes.c_double),
                ("nboxes", ctypes.c_int64), ("nleaves", ctypes.c_int64), ("n_strong", ctypes.c_int64),
                ("n_weak", ctypes.c_int64), ("n_strong_leaf", ctypes.c_int64), ("p2p_pairs", ctypes.c_int64),
                ("p2p_items", ctypes.c_int64), ("m2l_items", ctypes.c_int64), ("autotune_nlevels", ctypes.c_int),
                ("launches_build", ctypes.c_int), ("launches_eval", ctypes.c_int),
                ("autotune_theta", ctypes.c_double)]


class FMMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


_lib = None
_VP = ctypes.c_void_p
_PP = ctypes.POINTER(ctypes.c_void_p)


def load() -> ctypes.CDLL:
    """Load libfmm2d.so (raises when it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libfmm2d.so not found at {LIB_PATH}; build it with "
                          "`python -m paper_1311_1006_b300.build`")
    lib = ctypes.CDLL(LIB_PATH)
    S = ctypes.c_int
    sig = {
        "fmm_build_tree": (S, [_VP, ctypes.c_int64, ctypes.POINTER(FMMParams), _VP, _PP]),
        "fmm_tree_rebuild": (S, [_VP, _VP, ctypes.POINTER(FMMParams), _VP]),
        "fmm_build_tree_batched": (S, [_VP, ctypes.POINTER(ctypes.c_int64), ctypes.c_int,
                                       ctypes.POINTER(FMMParams), ctypes.POINTER(ctypes.c_int), _VP, _PP]),
        "fmm_eval": (S, [_VP, _VP, _VP, _VP]),
        "fmm_build_tree_targets": (S, [_VP, ctypes.c_int64, _VP, ctypes.c_int64, ctypes.POINTER(FMMParams), _VP,
                                       _PP]),
        "fmm_tree_rebuild_targets": (S, [_VP, _VP, _VP, ctypes.POINTER(FMMParams), _VP]),
        "fmm_eval_targets": (S, [_VP, _VP, _VP, _VP]),
        "fmm_eval_batched": (S, [_VP, _VP, _VP, _VP]),
        "fmm_eval_log": (S, [_VP, _VP, _VP, _VP]),
        "fmm_step": (S, [_VP, _VP, _VP, _VP, _VP]),
        "fmm_selftest_bounded_wait": (S, [ctypes.c_int, _VP]),
        "fmm_eval_status": (S, [_VP, _VP]),
        "fmm_selftest_rcp64": (S, [_VP, _VP, ctypes.c_int64, _VP]),
        "fmm_eval_targets_log": (S, [_VP, _VP, _VP, _VP]),
        "fmm_eval_backward": (S, [_VP, _VP, _VP, _VP, _VP, _VP]),
        "fmm_autotune_step": (S, [_VP, ctypes.c_double, ctypes.POINTER(FMMParams)]),
        "fmm_autotune_config": (S, [_VP, ctypes.c_double, ctypes.c_int, ctypes.c_int]),
        "fmm_autotuner_create": (S, [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                     _PP]),
        "fmm_autotuner_step": (S, [_VP, ctypes.c_double, ctypes.POINTER(ctypes.c_int)]),
        "fmm_autotuner_stats": (S, [_VP, ctypes.POINTER(ctypes.c_double), ctypes.c_int]),
        "fmm_autotuner_destroy": (None, [_VP]),
        "fmm_autotune_theta": (S, [_VP, ctypes.c_double, ctypes.c_double, ctypes.c_double]),
        "fmm_p_for_tolerance": (ctypes.c_int, [ctypes.c_double, ctypes.c_double]),
        "fmm_autotuner_theta": (S, [_VP, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double]),
        "fmm_autotuner_step_params": (S, [_VP, ctypes.c_double, ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]),
        "fmm_default_nlevels": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int, ctypes.c_int]),
        "fmm_seed_nlevels": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_double]),
        "fmm_cost_model_calibrate": (S, [_VP, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
        "fmm_cost_model_get": (S, [ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
        "fmm_cost_model_set": (S, [ctypes.c_int, ctypes.c_double, ctypes.c_double]),
        "fmm_phase_times": (S, [_VP, ctypes.POINTER(ctypes.c_double), ctypes.c_int]),
        "fmm_get_tree_info": (S, [_VP, ctypes.POINTER(FMMTreeInfo)]),
        "fmm_tree_export": (S, [_VP, ctypes.c_int, _VP, ctypes.c_int64, _VP]),
        "fmm_tree_destroy": (None, [_VP]),
        "fmm_direct_eval_noalloc": (S, [_VP, _VP, ctypes.c_int64, _VP, _VP]),
        "fmm_status_string": (ctypes.c_char_p, [ctypes.c_int]),
        "fmm_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def check(status: int) -> None:
    if status != FMM_OK:
        lib = load()
        msg = (lib.fmm_status_string(status) or b"").decode() + ": " + (lib.fmm_last_error() or b"").decode()
        raise FMMError(status, msg)
