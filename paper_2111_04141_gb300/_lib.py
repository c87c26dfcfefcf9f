"""ctypes declarations of the libgw C ABI (include/gw.h).

Loading fails loudly when the compiled library is missing: there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
# GW_DEBUG_BOUNDS=1 selects the build with device-side bounds checks
# (build(debug=True)); the default is the release library
LIB_PATH = os.path.join(_HERE, "libgw_debug.so" if os.environ.get("GW_DEBUG_BOUNDS") == "1"
                        else "libgw.so")

GW_C64, GW_BF16X2, GW_F16X2 = 0, 1, 2
GW_FLAG_VALID, GW_FLAG_CONJ = 1, 2

c_i32, c_i64, c_f64, c_vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p


class GwError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: status {status}: {message}")
        self.status = status


class PlanDesc(ctypes.Structure):
    _fields_ = [("grid_n", c_i32), ("cell_rad", c_f64), ("support_min", c_i32),
                ("support_max", c_i32), ("oversample", c_i32), ("n_wplanes", c_i32),
                ("w_max_lambda", c_f64), ("npol", c_i32), ("vis_dtype", c_i32),
                ("table_dtype", c_i32), ("max_vis_per_call", c_i64)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("grid_n", c_i32), ("npol", c_i32), ("oversample", c_i32), ("n_wplanes", c_i32),
                ("grid_tile_u", c_i32), ("grid_tile_v", c_i32), ("degrid_tile", c_i32),
                ("device", c_i32), ("table_elems", c_i64), ("chunk_vis", c_i64),
                ("field", c_f64), ("taper_c", c_f64), ("table_scale", c_f64),
                ("vis_dtype", c_i32), ("table_dtype", c_i32), ("table_exp2", c_i32),
                ("plane_groups", c_i32), ("table_bytes", c_i64), ("scratch_bytes", c_i64)]


class Tuning(ctypes.Structure):
    _fields_ = [("item_max", c_i32), ("degrid_kernel", c_i32), ("grid_kernel", c_i32),
                ("compress_min_gain", c_i32), ("plane_groups", c_i32)]


class Timing(ctypes.Structure):
    _fields_ = [("index_ms", c_f64), ("bin_ms", c_f64), ("grid_ms", c_f64), ("degrid_ms", c_f64),
                ("index_calls", c_i64), ("bin_calls", c_i64), ("grid_calls", c_i64),
                ("degrid_calls", c_i64), ("valid_vis", c_i64), ("taps", c_i64)]


_SIGS = {
    "gw_api_version": (c_i32, []),
    "gw_launch_count": (ctypes.c_uint64, []),
    "gw_strerror": (ctypes.c_char_p, [c_i32]),
    "gw_last_error": (ctypes.c_char_p, []),
    "gw_plan_create": (c_i32, [ctypes.POINTER(PlanDesc), c_vp, ctypes.POINTER(c_vp)]),
    "gw_plan_destroy": (c_i32, [c_vp]),
    "gw_plan_info_get": (c_i32, [c_vp, ctypes.POINTER(PlanInfo)]),
    "gw_plan_clone": (c_i32, [c_vp, c_i64, c_vp, ctypes.POINTER(c_vp)]),
    "gw_plan_set_tuning": (c_i32, [c_vp, ctypes.POINTER(Tuning)]),
    "gw_plan_get_tuning": (c_i32, [c_vp, ctypes.POINTER(Tuning)]),
    "gw_grid_vis": (c_i32, [c_vp, c_vp, c_vp, c_i64, c_i32, c_vp, c_vp, c_vp,
                            ctypes.POINTER(c_i64), c_vp]),
    "gw_grid_vis_compensated": (c_i32, [c_vp, c_vp, c_vp, c_i64, c_i32, c_vp, c_vp, c_vp, c_vp,
                                        ctypes.POINTER(c_i64), c_vp]),
    "gw_grid_fold": (c_i32, [c_vp, c_vp, c_vp, c_vp]),
    "gw_grid_vis_host": (c_i32, [c_vp, c_vp, c_vp, c_i64, c_i32, c_vp, c_vp, c_vp,
                                 ctypes.POINTER(c_i64), c_vp]),
    "gw_hybrid_grid": (c_i32, [c_vp, c_vp, c_vp, c_i64, c_i32, c_vp, c_vp, c_i32, c_vp,
                               ctypes.POINTER(c_i64), c_vp]),
    "gw_hybrid_prune": (c_i32, [c_vp, c_i32, c_vp, c_vp, c_vp]),
    "gw_hybrid_shift": (c_i32, [c_vp, c_vp, c_vp]),
    "gw_hybrid_image": (c_i32, [c_vp, c_i32, c_vp, c_vp, c_vp]),
    "gw_grid_vis_wstack": (c_i32, [c_vp, c_vp, c_vp, c_i64, c_i32, c_vp, c_vp, c_i32, c_f64, c_f64,
                                   c_vp, ctypes.POINTER(c_i64), c_vp]),
    "gw_wstack_combine": (c_i32, [c_vp, c_vp, c_i32, c_f64, c_f64, c_vp, c_vp]),
    "gw_grid_vis_compressed": (c_i32, [c_vp, c_vp, c_vp, c_i64, c_i32, c_vp, c_vp, c_vp,
                                       ctypes.POINTER(c_i64), ctypes.POINTER(c_i64), c_vp]),
    "gw_grid_vis_devcount": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_i64, c_i32, c_vp, c_vp, c_vp]),
    "gw_grid_vis_devcount_readback": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_i64, c_i32, c_vp, c_vp,
                                              c_vp, c_i32, c_vp]),
    "gw_degrid_vis_devcount": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_i64, c_i32, c_vp, c_vp, c_vp]),
    "gw_degrid_vis": (c_i32, [c_vp, c_vp, c_vp, c_i64, c_i32, c_vp, c_vp,
                              ctypes.POINTER(c_i64), c_vp]),
    "gw_degrid_vis_static": (c_i32, [c_vp, c_vp, c_vp, c_i64, c_i32, c_vp, c_vp,
                                     ctypes.POINTER(c_i64), c_vp]),
    "gw_grid_correct": (c_i32, [c_vp, c_vp, c_i32, c_vp]),
    "gw_grid_shift": (c_i32, [c_vp, c_vp, c_vp]),
    "gw_index_vis": (c_i32, [c_vp, c_vp, c_vp, c_i64, c_i32, c_vp, ctypes.POINTER(c_i64), c_vp]),
    "gw_plan_copy_tables": (c_i32, [c_vp, c_vp, c_vp, c_vp]),
    "gw_plan_copy_stored_tables": (c_i32, [c_vp, c_vp]),
    "gw_plan_copy_corrector": (c_i32, [c_vp, c_vp]),
    "gw_ffma_peak": (c_i32, [c_i32, ctypes.POINTER(c_f64), c_vp]),
    "gw_plan_timing_enable": (c_i32, [c_vp, c_i32]),
    "gw_plan_timing_get": (c_i32, [c_vp, ctypes.POINTER(Timing)]),
    "gw_debug_bins": (c_i32, [c_vp, c_vp, c_vp, c_i64, c_i32, c_i32, c_vp, c_vp, c_i64, c_vp]),
    "gw_debug_fail_alloc": (c_i32, [c_i64]),
    "gw_debug_live_plans": (c_i64, []),
    "gw_debug_live_bytes": (c_i64, []),
    "gw_plan_device_status": (c_i32, [c_vp, c_vp]),
}

EXPORTED = tuple(_SIGS)

_lib = None


def load(path: str = LIB_PATH):
    """Load libgw.so (building nothing).  Raises if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libgw.so not found at {path}; build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(status: int, where: str):
    if status != 0:
        lib = load()
        msg = lib.gw_last_error().decode(errors="replace")
        name = lib.gw_strerror(status).decode()
        raise GwError(status, where, f"{name}: {msg}")
