"""ctypes loader for libtc.so (the C ABI of include/tc.h).

The library must have been built (``__graft_entry__.build()``); there is no
fallback: importing a function from a missing library raises.
"""
import ctypes
import os

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libtc.so")

# names and signatures of every entry point declared in include/tc.h
_c = ctypes
_vp = _c.c_void_p
_i32, _i64, _dbl = _c.c_int32, _c.c_int64, _c.c_double
SIGNATURES = {
    "tc_create": (_i32, [_c.POINTER(_vp), _vp]),
    "tc_destroy": (_i32, [_vp]),
    "tc_last_error": (_c.c_char_p, [_vp]),
    "tc_sync": (_i32, [_vp]),
    "tc_build": (_i32, [_vp, _vp, _i64, _i32]),
    "tc_moments": (_i32, [_vp, _vp, _vp, _vp, _i32]),
    "tc_eval": (_i32, [_vp, _vp, _i64, _dbl, _i32, _vp]),
    "tc_velocity_host": (_i32, [_vp, _vp, _vp, _vp, _vp, _i64, _i32, _dbl, _i32, _vp]),
    "tc_adjoint": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "tc_update_positions": (_i32, [_vp, _vp]),
    "tc_eval_frozen": (_i32, [_vp, _vp]),
    "tc_direct": (_i32, [_vp, _vp, _vp, _vp, _i64, _vp, _i64, _i32, _vp, _vp]),
    "tc_direct_noalloc": (_i32, [_vp, _vp, _vp, _vp, _i64, _vp, _i64, _i32, _vp, _vp]),
    "tc_direct_reg": (_i32, [_vp, _vp, _vp, _vp, _i64, _vp, _i64, _dbl, _i32, _vp, _vp]),
    "tc_stats": (_i32, [_vp, _vp, _vp, _vp]),
    "tc_eval_counts": (_i32, [_vp, _vp, _vp]),
    "tc_list_stats": (_i32, [_vp, _vp, _vp, _vp]),
    "tc_tune": (_i32, [_vp, _vp, _vp, _vp, _vp, _i64, _vp, _i32, _vp, _i32, _vp, _i32, _vp, _i64, _dbl, _vp, _vp, _vp]),
    "tc_tree_info": (_i32, [_vp, _vp, _vp, _vp, _vp]),
    "tc_tree_export": (_i32, [_vp] + [_vp] * 9),
    "tc_tree_order": (_i32, [_vp, _vp]),
    "tc_moments_export": (_i32, [_vp, _i64, _vp, _vp]),
    "tc_batch_create": (_i32, [_c.POINTER(_vp), _vp]),
    "tc_batch_destroy": (_i32, [_vp]),
    "tc_batch_last_error": (_c.c_char_p, [_vp]),
    "tc_batch_set": (_i32, [_vp, _i32, _i32]),
    "tc_batch_build": (_i32, [_vp, _vp, _i32, _vp, _i32]),
    "tc_batch_moments": (_i32, [_vp, _vp, _vp, _vp, _i32]),
    "tc_batch_eval": (_i32, [_vp, _dbl, _i32, _vp]),
    "tc_batch_eval_separate": (_i32, [_vp, _dbl, _i32, _vp]),
    "tc_batch_info": (_i32, [_vp, _vp, _vp]),
    "tc_batch_system": (_vp, [_vp, _i32]),
    "tc_profile": (_i32, [_vp, _i32]),
    "tc_phase_times": (_i32, [_vp, _vp]),
    "tc_kernel_launches": (_i64, []),
    "tc_fma_peak": (_i32, [_i32, _vp, _vp]),
    "tc_fail_allocations": (None, [_i64]),
}
PHASES = ("build", "moments", "tables", "targets", "lists", "far", "near", "final", "adj_far_target",
          "adj_far_source", "adj_near_target", "adj_near_source", "adj_rest")


class TCConfig(ctypes.Structure):
    _fields_ = [("precision", _i32), ("shrink", _i32), ("stream", _vp), ("rec64", _i32), ("reserved1", _i32),
                ("reg_eps", _dbl)]


_lib = None


def lib():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libtc.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
    h = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(h, name)
        fn.restype = res
        fn.argtypes = args
    _lib = h
    return h
