"""ctypes loader for libpfem.so: argument marshalling only.

Every function here has the name and argument order of the C entry point it wraps
(include/pfem.h), takes torch tensors for device buffers, and raises PfemError on a
non-zero status.  There is no fallback: if the library is missing, loading fails loudly.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpfem.so")

PFEM_F64, PFEM_F32, PFEM_BF16 = 0, 1, 2
PFEM_SHAPE_LINEAR, PFEM_SHAPE_QUADRATIC = 0, 1
PFEM_SOLVE_F64, PFEM_SOLVE_F32, PFEM_SOLVE_F32_REFINED, PFEM_SOLVE_F32_REFINED_FF = 0, 1, 2, 3
PFEM_BACKWARD_RECOMPUTE, PFEM_BACKWARD_CHECKPOINT = 0, 1
PFEM_KMAX = 16
PFEM_KW_MAX = 64

STATUS = {0: "PFEM_OK", 1: "PFEM_ERR_INVALID_ARG", 2: "PFEM_ERR_CUDA", 3: "PFEM_ERR_WORKSPACE",
          4: "PFEM_ERR_CAPACITY", 5: "PFEM_ERR_DEGENERATE", 6: "PFEM_ERR_TIMEOUT"}

# exported symbols and their C signatures (restype, argtypes)
_i32, _i64, _sz, _p = ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t, ctypes.c_void_p
SIGNATURES = {
    "pfem_abi_version": (ctypes.c_int, []),
    "pfem_launch_count": (ctypes.c_uint64, []),
    "pfem_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "pfem_options_default": (None, [_p]),
    "pfem_create": (ctypes.c_int, [ctypes.POINTER(_p), _p]),
    "pfem_destroy": (None, [_p]),
    "pfem_get_options": (ctypes.c_int, [_p, _p]),
    "pfem_last_error": (ctypes.c_char_p, [_p]),
    "pfem_set_stage_events": (ctypes.c_int, [_p, _p, _i32]),
    "pfem_set_values_event": (ctypes.c_int, [_p, _p]),
    "pfem_default_bins": (_i32, [_i32, _i64]),
    "pfem_workspace_size": (_sz, [_i32, _i32, _i64, _i32]),
    "pfem_read_status": (ctypes.c_int, [_p, ctypes.POINTER(_i32), ctypes.POINTER(_i64), _p]),
    "pfem_get_device_status": (ctypes.c_int, [_p, _p, ctypes.POINTER(_i32), ctypes.POINTER(_i64), _p]),
    "pfem_reset_status": (ctypes.c_int, [_p, _p]),
    "pfem_build_cells": (ctypes.c_int, [_p, _i32, _i64, _p, ctypes.c_int, _p, _p, _p, _p, _p, _sz, _p]),
    "pfem_build_cells_noalloc": (ctypes.c_int, [_i32, _i64, _p, ctypes.c_int, _p, _p, _p, _p, _p]),
    "pfem_delaunay_stars": (ctypes.c_int, [_p, _i32, _i64, _p, _p, _p, _p, _p, _sz, _p]),
    "pfem_shape_quadratic": (ctypes.c_int, [_p, _i32, _i32, _i64, _p, ctypes.c_int, _p, _p,
                                            ctypes.c_int, ctypes.c_int, _i32, _p, _p, ctypes.c_int,
                                            _p, _sz, _p]),
    "pfem_project_p2m": (ctypes.c_int, [_p, _i32, _i32, _i64, _p, ctypes.c_int, _p, _p, _p, _i32, _p,
                                        ctypes.c_int, ctypes.c_int, ctypes.c_int, _p, _p, _i32,
                                        ctypes.c_int, _p, _p, _sz, _p]),
    "pfem_interp_m2p": (ctypes.c_int, [_p, _i32, _i64, _p, ctypes.c_int, _i32, _p, _p, ctypes.c_int, _p]),
    "pfem_backward_workspace_size": (_sz, [_i32, _i64, _i32]),
    "pfem_interp_m2p_quadratic": (ctypes.c_int, [_p, _i32, _i64, _p, ctypes.c_int, _i32, _p, _p,
                                                 ctypes.c_int, _p]),
    "pfem_project_backward": (ctypes.c_int, [_p, _i32, _i32, _i64, _p, ctypes.c_int, _p, _p, _p, _i32,
                                             _p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int, _p, _p, _i32, ctypes.c_int, _p, _p, _p,
                                             _p, _sz, _p]),
    "pfem_interp_m2p_backward": (ctypes.c_int, [_p, _i32, _i32, _i64, _p, ctypes.c_int, _p, _p, _i32,
                                                _p, _p, ctypes.c_int, _p, _p, _p]),
    "pfem_advect_midpoint": (ctypes.c_int, [_p, _i32, _i64, _p, ctypes.c_int, _p, ctypes.c_double,
                                            _p, _p]),
    "pfem_update_workspace_size": (_sz, [_i32, _i64]),
    "pfem_update_cells": (ctypes.c_int, [_p, _i32, _i64, _p, ctypes.c_int, _p, _p, _p, _p, _p, _p,
                                         _p, _p, _sz, _p]),
    "pfem_batch_plan_size": (_sz, [_i32]),
    "pfem_batch_plan_init": (ctypes.c_int, [_p, _i32, _p, _p, ctypes.POINTER(_i64)]),
    "pfem_batch_workspace_size": (_sz, [_i64, _i64, _i64]),
    "pfem_batch_build_cells": (ctypes.c_int, [_p, _p, _i64, _i64, _p, ctypes.c_int, _p, _p, _p, _p,
                                              _p, _sz, _p]),
    "pfem_batch_project_p2m": (ctypes.c_int, [_p, _p, _i64, _i64, _p, ctypes.c_int, _p, _p, _p, _i32,
                                              _p, ctypes.c_int, ctypes.c_int, ctypes.c_int, _p, _i32,
                                              _i32, _p, _sz, _p]),
    "pfem_batch_interp_m2p": (ctypes.c_int, [_p, _p, _p, ctypes.c_int, _i32, _p, _p, ctypes.c_int,
                                             _i32, _p]),
}


class Options(ctypes.Structure):
    """pfem_options (include/pfem.h); zero fields take their defaults."""
    _fields_ = [("walk_max_steps", ctypes.c_int32), ("star_capacity", ctypes.c_int32),
                ("node_capacity", ctypes.c_int32), ("search_radius_max", ctypes.c_int32),
                ("batch_tile_rows", ctypes.c_int32), ("batch_p2m_blocks", ctypes.c_int32),
                ("batch_m2p_blocks", ctypes.c_int32), ("reserved", ctypes.c_int32 * 9)]


class BatchProblem(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nb", ctypes.c_int32), ("N", ctypes.c_int64)]


class PfemError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {STATUS.get(code, code)}")
        self.code = code


class LibraryMissing(ImportError):
    pass


_lib = None


def load(path: Optional[str] = None):
    """Load libpfem.so (built by build.py; PFEM_LIB selects another build of it); raises
    LibraryMissing if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or os.environ.get("PFEM_LIB") or LIB_PATH
    if not os.path.exists(p):
        raise LibraryMissing(f"{p} is missing: build it with paper_1610_05266_gb300.build.build()")
    L = ctypes.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def dtype_code(t: torch.dtype) -> int:
    if t == torch.float64:
        return PFEM_F64
    if t == torch.float32:
        return PFEM_F32
    if t == torch.bfloat16:
        return PFEM_BF16
    raise TypeError(f"unsupported dtype {t}")


def ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("device buffers must be CUDA tensors")
    if not t.is_contiguous():
        raise ValueError("buffers must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def stream_ptr(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def check(code: int, what: str, ctx=None):
    """Raise PfemError for a non-zero status, with the library's last-error text."""
    if code != 0:
        text = load().pfem_last_error(ctx_ptr(ctx))
        detail = text.decode() if text else ""
        raise PfemError(code, f"{what} ({detail})" if detail else what)


def ctx_ptr(ctx):
    """The pfem_ctx* of a Context (or None for the defaults)."""
    return None if ctx is None else ctx.handle
