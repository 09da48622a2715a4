"""ctypes declarations of include/maclab.h and include/maclab_ws.h
(argument marshalling only)."""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

c_int, c_double, c_int64, c_size_t, c_void_p = (ctypes.c_int, ctypes.c_double, ctypes.c_int64,
                                                ctypes.c_size_t, ctypes.c_void_p)
P = ctypes.POINTER


class Grid(ctypes.Structure):
    _fields_ = [("nx", c_int), ("ny", c_int), ("dx", c_double)]


class Params(ctypes.Structure):
    _fields_ = [("precision", c_int), ("nu", c_double), ("e", c_double), ("g", c_double),
                ("rho_w", c_double), ("rho_a", c_double), ("Cw", c_double),
                ("wind_u", c_double), ("wind_v", c_double), ("Cb", c_double),
                ("Omega", c_double), ("h_ref", c_double)]


class Wave(ctypes.Structure):
    _fields_ = [("mean", c_double), ("amp", c_double), ("omega", c_double), ("phase", c_double)]


class BC(ctypes.Structure):
    _fields_ = [("edge", c_int * 4), ("h", Wave * 4), ("qx", Wave * 4), ("qy", Wave * 4)]


ALLOC_FN = ctypes.CFUNCTYPE(c_void_p, c_size_t, c_void_p)
RELEASE_FN = ctypes.CFUNCTYPE(None, c_void_p, c_void_p)


class Allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("release", RELEASE_FN), ("ctx", c_void_p)]


class Info(ctypes.Structure):
    _fields_ = [("nx", c_int), ("ny", c_int), ("pitch", c_int), ("precision", c_int),
                ("dx", c_double), ("e", c_double), ("dt", c_double), ("nu", c_double),
                ("n_dirichlet", c_int64), ("n_fluid", c_int64), ("n_fast", c_int64),
                ("device_bytes", c_size_t), ("tile_rows", c_int), ("step_kernel", c_int),
                ("dirichlet_fused", c_int), ("temporal_block", c_int), ("clean_tiles", c_int64),
                ("tau", c_double), ("hbar_level", c_int), ("two_step_blocks", c_int64)]


class WSConfig(ctypes.Structure):
    _fields_ = [("res", c_int), ("channels", c_int), ("blocks", c_int), ("dilation", c_int * 64),
                ("max_batch", c_int), ("seed", ctypes.c_uint64), ("tensor_path", c_int)]


c_float = ctypes.c_float

# (name, restype, argtypes) of every exported entry point of include/*.h
PROTOTYPES = [
    ("maclab_abi_version", c_int, []),
    ("maclab_create", c_int, [P(Grid), P(Params), P(BC), P(c_double), P(ctypes.c_uint8),
                              P(c_double), P(c_double), P(c_double), P(Allocator), c_void_p,
                              P(c_void_p)]),
    ("maclab_set_stream", c_int, [c_void_p, c_void_p]),
    ("maclab_step", c_int, [c_void_p, c_int64]),
    ("maclab_set_graph_steps", c_int, [c_void_p, c_int]),
    ("maclab_get_state", c_int, [c_void_p, P(c_double), P(c_double), P(c_double)]),
    ("maclab_set_state", c_int, [c_void_p, P(c_double), P(c_double), P(c_double)]),
    ("maclab_residual", c_int, [c_void_p, P(c_double)]),
    ("maclab_mark", c_int, [c_void_p]),
    ("maclab_residual_since_mark", c_int, [c_void_p, P(c_double)]),
    ("maclab_residual_noalloc", c_int, [c_int, c_int, c_int, c_int] + [c_void_p] * 7 +
     [P(ctypes.c_uint8), c_double, c_void_p, P(c_double)]),
    ("maclab_run_to_steady", c_int, [c_void_p, c_double, c_int64, c_int, P(c_int64),
                                     P(c_double)]),
    ("maclab_time", c_int, [c_void_p, P(c_double), P(c_int64)]),
    ("maclab_set_tile_rows", c_int, [c_void_p, c_int]),
    ("maclab_set_launch", c_int, [c_void_p, c_int, c_int]),
    ("maclab_autotune", c_int, [c_void_p, c_int, P(c_int)]),
    ("maclab_set_step_kernel", c_int, [c_void_p, c_int]),
    ("maclab_set_temporal_block", c_int, [c_void_p, c_int]),
    ("maclab_set_relaxation", c_int, [c_void_p, c_double]),
    ("maclab_set_hbar_level", c_int, [c_void_p, c_int]),
    ("maclab_set_profiling", c_int, [c_void_p, c_int]),
    ("maclab_get_profile", c_int, [c_void_p, P(c_double), P(c_int64)]),
    ("maclab_get_info", c_int, [c_void_p, P(Info)]),
    ("maclab_measure_fp64", c_int, [P(c_double)]),
    ("maclab_device_state", c_int, [c_void_p, P(c_void_p), P(c_void_p), P(c_void_p)]),
    ("maclab_last_error", ctypes.c_char_p, [c_void_p]),
    ("maclab_batch_create", c_int, [c_int, P(Grid), P(Params), P(BC), P(P(c_double)),
                                    P(P(ctypes.c_uint8)), P(P(c_double)), P(P(c_double)),
                                    P(P(c_double)), P(Allocator), c_void_p, P(c_void_p)]),
    ("maclab_batch_step", c_int, [c_void_p, c_int64]),
    ("maclab_batch_set_graph_steps", c_int, [c_void_p, c_int]),
    ("maclab_batch_set_persistent", c_int, [c_void_p, c_int]),
    ("maclab_batch_set_barrier_test", c_int, [c_void_p, c_int, ctypes.c_uint]),
    ("maclab_batch_residual", c_int, [c_void_p, P(c_double)]),
    ("maclab_batch_mark", c_int, [c_void_p]),
    ("maclab_batch_residual_since_mark", c_int, [c_void_p, P(c_double)]),
    ("maclab_batch_set_active", c_int, [c_void_p, P(ctypes.c_uint8)]),
    ("maclab_batch_run_to_steady", c_int, [c_void_p, c_double, c_int64, c_int, P(c_int64),
                                           P(c_double), P(c_double)]),
    ("maclab_batch_get_state", c_int, [c_void_p, c_int, P(c_double), P(c_double), P(c_double)]),
    ("maclab_batch_set_state", c_int, [c_void_p, c_int, P(c_double), P(c_double), P(c_double)]),
    ("maclab_batch_info", c_int, [c_void_p, P(c_int), P(c_int64), P(c_int64), P(c_int64)]),
    ("maclab_batch_device_state", c_int, [c_void_p, c_int, P(c_void_p), P(c_void_p), P(c_void_p), P(c_int)]),
    ("maclab_batch_last_error", ctypes.c_char_p, [c_void_p]),
    ("maclab_batch_destroy", None, [c_void_p]),
    ("maclab_destroy", None, [c_void_p]),
    # learned warm start (maclab_ws.h)
    ("maclab_ws_create", c_int, [P(WSConfig), c_void_p, P(c_void_p)]),
    ("maclab_ws_destroy", None, [c_void_p]),
    ("maclab_ws_param_count", c_int, [c_void_p, P(c_int64)]),
    ("maclab_ws_get_params", c_int, [c_void_p, P(c_float), c_int64]),
    ("maclab_ws_set_params", c_int, [c_void_p, P(c_float), c_int64]),
    ("maclab_ws_forward", c_int, [c_void_p, c_int, c_void_p, c_void_p]),
    ("maclab_ws_gradients", c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p, c_void_p, P(c_float), c_int64,
                                    P(c_double)]),
    ("maclab_ws_train_step", c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p, c_void_p, c_float,
                                     P(c_double)]),
    ("maclab_ws_keep_gradients", c_int, [c_void_p, c_int]),
    ("maclab_ws_inspect", c_int, [c_void_p, c_int, c_int, c_int, c_void_p, c_int64]),
    ("maclab_ws_encode", c_int, [c_void_p, c_int, c_void_p, c_void_p, c_double, c_double, c_double, c_double,
                                 c_void_p,
                                 c_void_p, c_void_p, c_int, P(c_double), c_void_p, c_void_p, c_void_p]),
    ("maclab_ws_decode", c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p, P(c_double), c_double, c_void_p,
                                 c_void_p, c_void_p]),
]

_lock = threading.Lock()
_lib = None


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load the in-tree CUDA library.  Raises if it is missing and cannot be
    built: there is no fallback implementation."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if os.environ.get("MACLAB_LIB"):
                # an alternative build of the same sources (tuning experiments)
                path = os.environ["MACLAB_LIB"]
            elif build_if_missing:
                path = _build.build()
            if not os.path.exists(path):
                raise RuntimeError("maclab CUDA library not built: %s (run build())" % path)
            lib = ctypes.CDLL(path)
            for name, res, args in PROTOTYPES:
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib
