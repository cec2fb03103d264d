"""ctypes declarations of the C ABI in include/rips.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

STATUS = {0: "ok", -1: "bad argument", -2: "bad modulus", -3: "overflow", -4: "out of memory",
          -5: "CUDA error", -6: "device timeout", -7: "internal error"}


class RipsError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {STATUS.get(status, status)} ({status})")
        self.status = status


class Bar(C.Structure):
    _fields_ = [("dim", C.c_int32), ("birth", C.c_float), ("death", C.c_float), ("cloud", C.c_int32),
                ("birth_simplex", C.c_uint64), ("death_simplex", C.c_uint64)]


class Stats(C.Structure):
    _fields_ = [("simplices", C.c_int64), ("apparent_cofacet", C.c_int64), ("apparent_facet", C.c_int64),
                ("cleared", C.c_int64), ("columns", C.c_int64), ("emergent", C.c_int64),
                ("pairs", C.c_int64), ("zero_pairs", C.c_int64), ("essential", C.c_int64),
                ("reduction_steps", C.c_int64), ("rounds", C.c_int64), ("longest_chain", C.c_int64),
                ("compacted_entries", C.c_int64), ("added_entries", C.c_int64)]


class Limits(C.Structure):
    _fields_ = [("barrier_wait_ns", C.c_uint64), ("chain_ns", C.c_uint64), ("arena_entries", C.c_uint64),
                ("table_slots", C.c_uint64)]


class Tuning(C.Structure):
    _fields_ = [("warp_chain_limit", C.c_int32), ("warp_merge_max", C.c_int32),
                ("reduce_blocks_per_sm", C.c_int32), ("scan_blocks_per_sm", C.c_int32)]


# every symbol declared in include/rips.h
EXPORTS = [
    "rips_barcodes", "rips_barcodes_device", "rips_distance_matrix_device", "rips_barcodes_batched",
    "rips_barcodes_backward", "rips_barcodes_packed", "rips_barcodes_sparse", "rips_barcodes_sparse_points", "rips_barcodes_batched_dists", "rips_barcodes_backward_dist", "rips_result_num_bars", "rips_result_bars", "rips_result_num_clouds",
    "rips_result_dim_max", "rips_result_threshold", "rips_result_stats", "rips_result_phase_ms",
    "rips_result_free", "rips_status_string", "rips_kernel_launch_count", "rips_set_kernel_timing",
    "rips_result_kernel_ms", "rips_h0_barcode_noalloc", "rips_set_tuning", "rips_get_tuning", "rips_clear_tuning",
    "rips_set_limits", "rips_get_limits", "rips_set_options", "rips_get_options", "rips_batch_plan_create", "rips_batch_plan_run", "rips_batch_plan_result",
    "rips_batch_plan_free",
]

KERNEL_CLASSES = ["prologue", "edge_sort", "h0", "enumerate", "apparent", "col_sort", "pivot_init", "reduce",
                  "readout"]

_lib = None


def load(build_if_missing: bool = True):
    """Load librips.so.  Raises if it is missing and cannot be built: there is no
    CPU fallback."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.library_path()
    if not os.path.exists(path) or not _build.up_to_date():
        if not build_if_missing:
            raise RuntimeError(f"librips.so is not built ({path}); run paper_1908_02518_gb300.build.build()")
        path = _build.build()
    lib = C.CDLL(path)
    vp, fp, i64, i32, u32 = C.c_void_p, C.POINTER(C.c_float), C.c_int64, C.c_int32, C.c_uint32
    pres = C.POINTER(C.c_void_p)
    lib.rips_barcodes.argtypes = [fp, i64, i32, C.c_float, u32, pres]
    lib.rips_barcodes.restype = C.c_int
    lib.rips_barcodes_device.argtypes = [vp, i64, i32, C.c_float, u32, vp, pres]
    lib.rips_barcodes_device.restype = C.c_int
    lib.rips_distance_matrix_device.argtypes = [vp, i64, i32, vp, vp]
    lib.rips_distance_matrix_device.restype = C.c_int
    lib.rips_barcodes_batched.argtypes = [vp, C.POINTER(C.c_int64), i32, i32, i32, C.c_float, u32, vp, pres]
    lib.rips_barcodes_batched.restype = C.c_int
    lib.rips_barcodes_backward.argtypes = [vp, vp, i32, vp, vp, vp, vp, vp]
    lib.rips_barcodes_backward.restype = C.c_int
    lib.rips_barcodes_sparse.argtypes = [vp, vp, vp, i64, i64, i32, C.c_float, u32, vp, pres]
    lib.rips_barcodes_sparse.restype = C.c_int
    lib.rips_barcodes_sparse_points.argtypes = [vp, i64, i32, i32, C.c_float, u32, vp, pres]
    lib.rips_barcodes_sparse_points.restype = C.c_int
    lib.rips_barcodes_packed.argtypes = [vp, i64, i32, i32, C.c_float, u32, vp, pres]
    lib.rips_barcodes_packed.restype = C.c_int
    lib.rips_barcodes_batched_dists.argtypes = [C.POINTER(vp), C.POINTER(C.c_int64), i32, i32, C.c_float, u32, vp,
                                                pres]
    lib.rips_barcodes_batched_dists.restype = C.c_int
    lib.rips_barcodes_backward_dist.argtypes = [vp, C.POINTER(vp), vp, vp, C.POINTER(vp), vp]
    lib.rips_barcodes_backward_dist.restype = C.c_int
    lib.rips_result_num_bars.argtypes = [vp, i32, i32]
    lib.rips_result_num_bars.restype = i64
    lib.rips_result_bars.argtypes = [vp, i32, i32]
    lib.rips_result_bars.restype = C.POINTER(Bar)
    lib.rips_result_num_clouds.argtypes = [vp]
    lib.rips_result_num_clouds.restype = i32
    lib.rips_result_dim_max.argtypes = [vp]
    lib.rips_result_dim_max.restype = i32
    lib.rips_result_threshold.argtypes = [vp, i32]
    lib.rips_result_threshold.restype = C.c_float
    lib.rips_result_stats.argtypes = [vp, i32, i32, C.POINTER(Stats)]
    lib.rips_result_stats.restype = C.c_int
    lib.rips_result_phase_ms.argtypes = [vp, fp, i32]
    lib.rips_result_phase_ms.restype = i32
    lib.rips_result_free.argtypes = [vp]
    lib.rips_result_free.restype = None
    lib.rips_status_string.argtypes = [C.c_int]
    lib.rips_status_string.restype = C.c_char_p
    lib.rips_kernel_launch_count.argtypes = [C.c_int]
    lib.rips_kernel_launch_count.restype = i64
    lib.rips_set_kernel_timing.argtypes = [C.c_int]
    lib.rips_set_kernel_timing.restype = C.c_int
    lib.rips_result_kernel_ms.argtypes = [vp, i32, fp, C.POINTER(C.c_int64)]
    lib.rips_result_kernel_ms.restype = C.c_int
    lib.rips_h0_barcode_noalloc.argtypes = [vp, i64, C.c_float, vp, vp, vp]
    lib.rips_h0_barcode_noalloc.restype = C.c_int
    lib.rips_set_tuning.argtypes = [i32, i64, i64, C.POINTER(Tuning)]
    lib.rips_set_tuning.restype = C.c_int
    lib.rips_get_tuning.argtypes = [i32, i64, C.POINTER(Tuning)]
    lib.rips_get_tuning.restype = C.c_int
    lib.rips_clear_tuning.argtypes = []
    lib.rips_clear_tuning.restype = None
    lib.rips_set_limits.argtypes = [C.POINTER(Limits)]
    lib.rips_set_limits.restype = C.c_int
    lib.rips_set_options.argtypes = [u32]
    lib.rips_set_options.restype = C.c_int
    lib.rips_get_options.argtypes = []
    lib.rips_get_options.restype = u32
    lib.rips_get_limits.argtypes = [C.POINTER(Limits)]
    lib.rips_get_limits.restype = C.c_int
    lib.rips_batch_plan_create.argtypes = [C.POINTER(C.c_int64), i32, i32, C.c_float, u32, i64, pres]
    lib.rips_batch_plan_create.restype = C.c_int
    lib.rips_batch_plan_run.argtypes = [vp, vp, vp]
    lib.rips_batch_plan_run.restype = C.c_int
    lib.rips_batch_plan_result.argtypes = [vp, vp, pres]
    lib.rips_batch_plan_result.restype = C.c_int
    lib.rips_batch_plan_free.argtypes = [vp]
    lib.rips_batch_plan_free.restype = None
    _lib = lib
    return lib


def check(status: int, what: str):
    if status != 0:
        raise RipsError(status, what)
