"""ctypes declarations of the C ABI in include/lob.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# LOB_CHECKED=1 selects the variant built with invariant checks
LIB_PATH = os.path.join(HERE, "liblob_checked.so" if os.environ.get("LOB_CHECKED") == "1"
                        else "liblob.so")

vp = ctypes.c_void_p
i32 = ctypes.c_int32
i64 = ctypes.c_int64


class LobConfig(ctypes.Structure):
    _fields_ = [("n_books", i32), ("capacity", i32), ("trade_capacity", i32),
                ("overflow_rule", i32), ("flags", i32)]


class LobEnvConfig(ctypes.Structure):
    _fields_ = [("n_steps", i32), ("parent_qty", i32), ("agent_tid", i32), ("depth", i32),
                ("p_init_fallback", i32), ("msgs_per_step", i32), ("lam", ctypes.c_double),
                ("passive_ticks", i32), ("tick_size", i32)]


class LobServeDesc(ctypes.Structure):
    """lob_serve_desc: the generator's functions travel as plain addresses."""
    _fields_ = [(name, vp) for name in (
        "engine", "gen_params", "gen_init", "gen_advance", "d_geo_px", "d_geo_q",
        "d_gen_states", "d_gen_pools", "d_win0", "d_win1", "d_bid_px", "d_bid_qty",
        "d_ask_px", "d_ask_qty", "d_trade_counts", "proc_stream", "gen_stream")] + \
        [("slots", i32), ("max_msgs", i32), ("depth", i32), ("ring", i32)]


# name -> (restype, argtypes); every symbol of include/lob.h
SIGNATURES = {
    "lob_create": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.POINTER(LobConfig), vp]),
    "lob_destroy": (ctypes.c_int, [vp]),
    "lob_reset": (ctypes.c_int, [vp, vp]),
    "lob_reset_books": (ctypes.c_int, [vp, vp, i32, vp]),
    "lob_process_batch": (ctypes.c_int, [vp, vp, vp, vp, i32, vp]),
    "lob_inject_orders": (ctypes.c_int, [vp, vp, vp, vp, i32, vp]),
    "lob_process_segments": (ctypes.c_int, [vp, vp, vp, vp, vp, i32, vp]),
    "lob_process_batch_l1": (ctypes.c_int, [vp, vp, vp, vp, i32, vp, vp]),
    "lob_clear_trades": (ctypes.c_int, [vp, vp]),
    "lob_get_levels": (ctypes.c_int, [vp, i32, vp, vp, vp, vp, vp]),
    "lob_get_levels_books": (ctypes.c_int, [vp, vp, i32, i32, vp, vp, vp, vp, vp]),
    "lob_get_trades": (ctypes.c_int, [vp, vp, vp, vp]),
    "lob_get_book": (ctypes.c_int, [vp, vp, vp, vp, vp, vp, vp, vp]),
    "lob_set_book": (ctypes.c_int, [vp, vp, vp, vp, vp, vp, vp, vp]),
    "lob_init_from_levels": (ctypes.c_int, [vp, vp, vp, vp, vp, i32, i64, vp]),
    "lob_get_stats": (ctypes.c_int, [vp, vp, vp, vp]),
    "lob_set_launch": (ctypes.c_int, [vp, i32, i32, i32]),
    "lob_launch_count": (i64, [vp]),
    "lob_process_streams_static": (ctypes.c_int, [vp, vp, i32, i32, i32, i32] + [vp] * 10 + [vp]),
    "lob_env_create": (ctypes.c_int, [ctypes.POINTER(vp), vp, ctypes.POINTER(LobEnvConfig), vp]),
    "lob_env_destroy": (ctypes.c_int, [vp]),
    "lob_env_reset": (ctypes.c_int, [vp, vp]),
    "lob_env_run": (ctypes.c_int, [vp, vp, i64, i32, i32] + [vp] * 9 + [vp]),
    "lob_env_observe": (ctypes.c_int, [vp, vp, i64, vp, vp, vp]),
    "lob_process_host": (ctypes.c_int, [vp, vp, i64, i32, vp]),
    "lob_selftest_wait": (ctypes.c_int, [i64, vp, vp, vp]),
    "lob_literal_process": (ctypes.c_int, [vp, vp, i32, i32, i32, i32, i32] + [vp] * 8 + [vp]),
    "lob_env_get_state": (ctypes.c_int, [vp, vp, vp, vp]),
    "lob_env_segments": (ctypes.c_int32, [vp]),
    "lob_serve_create": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.POINTER(LobServeDesc)]),
    "lob_serve_admit": (ctypes.c_int, [vp, ctypes.c_uint64, i64, i32, ctypes.POINTER(i32)]),
    "lob_serve_tick": (ctypes.c_int, [vp, i32, i32, vp, vp, vp, vp, vp]),
    "lob_serve_timings": (ctypes.c_int, [vp, vp, vp, vp, i32, ctypes.POINTER(i32)]),
    "lob_serve_ready": (ctypes.c_int, [vp]),
    "lob_serve_destroy": (ctypes.c_int, [vp]),
    "lob_last_error": (ctypes.c_char_p, []),
    "lob_abi_version": (ctypes.c_int, []),
}

_lib = None


def load():
    """Load liblob.so; raises (never falls back) when it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("%s is not built; run paper_2308_13289_b300.build.build() "
                              "(the engine has no CPU fallback)" % os.path.basename(LIB_PATH))
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class LobError(RuntimeError):
    def __init__(self, code, where):
        msg = load().lob_last_error()
        super().__init__("%s failed (%d): %s" % (where, code, msg.decode() if msg else ""))
        self.code = code


def check(code, where):
    if code != 0:
        raise LobError(code, where)
