"""ctypes declarations of the C ABI in include/ci_prng.h.

Loads the in-tree libci_prng.so; raises loudly when it is missing (there is no
CPU fallback).  Names match the C entry points one to one.
"""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
# CI_PRNG_CHECKED=1 selects the bounds-checked debugging build (build.py
# build(checked=True)); it must exist then, like the ordinary one.
CHECKED = os.environ.get("CI_PRNG_CHECKED") == "1"
LIB_PATH = os.path.join(PKG, "libci_prng_checked.so" if CHECKED else "libci_prng.so")

CI_OK, CI_PENDING = 0, 1
CI_E_INVAL, CI_E_NOMEM, CI_E_CUDA, CI_E_BUSY, CI_E_TIMEOUT, CI_E_STATE, CI_E_CANCELED = -1, -2, -3, -4, -5, -6, -7
CI_VAR_XOR, CI_VAR_BBS, CI_VAR_BBS16 = 0, 1, 2
CI_SINK_WRITTEN, CI_SINK_QC, CI_SINK_DIGEST = 0, 1, 2
CI_NOALLOC_MAX_ITEMS = 1024
CI_XL_XOR128, CI_XL_XORSHIFT32, CI_XL_XOR64 = 0, 1, 2

STATUS_NAMES = {0: "CI_OK", 1: "CI_PENDING", -1: "CI_E_INVAL", -2: "CI_E_NOMEM", -3: "CI_E_CUDA",
                -4: "CI_E_BUSY", -5: "CI_E_TIMEOUT", -6: "CI_E_STATE",
                -7: "CI_E_CANCELED"}


class ci_params(ctypes.Structure):
    _fields_ = [
        ("variant", ctypes.c_int32),
        ("xl", ctypes.c_int32),
        ("comb_size", ctypes.c_uint32),
        ("flags", ctypes.c_uint32),
        ("seed", ctypes.c_uint64),
        ("comb_seed", ctypes.c_uint64),
        ("first_stream", ctypes.c_uint64),
        ("comb", ctypes.c_void_p),
    ]


class ci_states_desc(ctypes.Structure):
    _fields_ = [
        ("variant", ctypes.c_int32),
        ("xl", ctypes.c_int32),
        ("comb_size", ctypes.c_uint32),
        ("reserved", ctypes.c_uint32),
        ("n_streams", ctypes.c_uint64),
        ("n_lanes", ctypes.c_uint64),
        ("state_bytes", ctypes.c_uint64),
        ("state_dev", ctypes.c_void_p),
        ("comb", ctypes.c_uint8 * 512),
    ]


class ci_batch_item(ctypes.Structure):
    _fields_ = [
        ("states", ctypes.c_void_p),
        ("n_per_stream", ctypes.c_uint64),
        ("sink", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("out_dev", ctypes.c_void_p),
        ("out_capacity_u32", ctypes.c_uint64),
        ("aux_dev", ctypes.c_void_p),
    ]


class ci_server_config(ctypes.Structure):
    _fields_ = [
        ("max_slots", ctypes.c_uint32),
        ("max_inflight", ctypes.c_uint32),
        ("slice_xor", ctypes.c_uint64),
        ("slice_bbs", ctypes.c_uint64),
        ("split_min_slices", ctypes.c_uint64),
    ]


class ci_request(ctypes.Structure):
    _fields_ = [
        ("params", ci_params),
        ("n_streams", ctypes.c_uint64),
        ("n_per_stream", ctypes.c_uint64),
        ("continue_ticket", ctypes.c_uint64),
    ]


class ci_result(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("out_dev", ctypes.c_void_p),
        ("n_streams", ctypes.c_uint64),
        ("n_per_stream", ctypes.c_uint64),
        ("states", ctypes.c_void_p),
        ("submit_ns", ctypes.c_uint64),
        ("admit_ns", ctypes.c_uint64),
        ("done_ns", ctypes.c_uint64),
    ]


class ci_server_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("submitted", "admitted", "completed", "released", "waves", "units",
                                                "arena_bytes", "arena_used", "arena_peak", "pending", "active", "gpu_ns",
                                                "max_wave_units", "host_admit_ns", "host_launch_ns",
                                                "split_jobs")]


class ci_tune_choice(ctypes.Structure):
    _fields_ = [
        ("warps_per_block", ctypes.c_uint32),
        ("tile_depth", ctypes.c_uint32),
        ("cache_policy", ctypes.c_uint32),
        ("ms", ctypes.c_float),
    ]


class ci_tune_table(ctypes.Structure):
    _fields_ = [
        ("choice", (ci_tune_choice * 4) * 5),
        ("batch_warps_per_block", ctypes.c_uint32),
        ("batch_ms", ctypes.c_float),
    ]


class CIError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        self.status = status
        super().__init__("%s failed with %s: %s" % (where, STATUS_NAMES.get(status, status), message))


_lib = None

_VP, _U32, _U64, _I32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32
_SIGNATURES = {
    "ci_state_bytes": [_VP, _U64, _VP],
    "ci_init_states": [_VP, _U64, _VP, _VP],
    "ci_init_states_at": [_VP, _U64, _VP, _U64, _VP, _VP],
    "ci_init_states_many": [_VP, _VP, _U32, _VP, _VP],
    "ci_free_states": [_VP],
    "ci_states_query": [_VP, _VP],
    "ci_generate": [_VP, _U64, _VP, _U64, _VP],
    "ci_generate_bbs": [_VP, _U64, _VP, _U64, _VP],
    "ci_generate_fused_qc": [_VP, _U64, _VP, _VP],
    "ci_generate_digest": [_VP, _U64, _VP, _VP],
    "ci_batch_create": [_U32, _VP],
    "ci_batch_run": [_VP, _VP, _U32, _VP],
    "ci_batch_destroy": [_VP],
    "ci_batch_run_noalloc": [_VP, _U32, _VP],
    "ci_generate_split": [_VP, _U64, _I32, _VP, _U64, _U32, _VP],
    "ci_naive_state_bytes": [_U64, _VP],
    "ci_naive_init": [_U64, _U64, _U64, _VP, _U64, _VP],
    "ci_naive_generate": [_VP, _U64, _U64, _VP, _U64, _VP],
    "ci_bg_encrypt": [_U64, _U64, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP],
    "ci_bg_decrypt": [_U64, _U64, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP],
    "ci_server_create": [_VP, _U64, _VP, _VP],
    "ci_submit": [_VP, _VP, _VP],
    "ci_poll": [_VP, _U64, _VP],
    "ci_wait": [_VP, _U64, _U32, _VP],
    "ci_release": [_VP, _U64],
    "ci_release_states": [_VP, _U64],
    "ci_cancel": [_VP, _U64],
    "ci_server_get_stats": [_VP, _VP],
    "ci_server_drive": [_VP, _VP, _VP, _VP, _VP, _U32, _VP, _VP],
    "ci_server_destroy": [_VP],
    "ci_autotune": [_U32, _VP, _VP],
    "ci_tune_get": [_VP],
    "ci_tune_set": [_VP],
    "ci_export_state": [_VP, _VP, _U64, _VP],
    "ci_import_state": [_VP, _VP, _U64, _VP],
    "ci_check_status": [_VP, _VP],
    "ci_check_probe": [_VP],
}


def lib() -> ctypes.CDLL:
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("%s is not built (run `python -c 'import __graft_entry__ as g; g.build()'` or "
                              "`python paper_1112_5239_gb300/build.py%s`); there is no CPU fallback"
                              % (os.path.basename(LIB_PATH), " --checked" if CHECKED else ""))
        L = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = _I32
        L.ci_last_error.argtypes = []
        L.ci_last_error.restype = ctypes.c_char_p
        L.ci_version.argtypes = []
        L.ci_version.restype = _U32
        _lib = L
    return _lib


def check(status: int, where: str) -> int:
    if status < 0:
        msg = lib().ci_last_error()
        raise CIError(status, where, msg.decode() if msg else "")
    return status


def call(name: str, *args) -> int:
    """Calls C entry point `name` and raises CIError on a negative status."""
    return check(getattr(lib(), name)(*args), name)
