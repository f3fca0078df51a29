"""Python binding of libtcks (include/tcks.h): RNS-CKKS encrypted-vector arithmetic on one GB300.

Argument marshalling only: every step of every operation runs in the CUDA library. Each C function
is reachable under its own name through `lib()` (e.g. `lib().tcks_add`), and the classes below wrap
the handles (Params, Context, Ciphertext, Plaintext, Matrix) with the same operation names. There is
no CPU fallback: if the compiled library is missing, importing the classes works but any call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# TCKS_DEBUG_CHECKS=1 in the environment selects the debug build (descriptor and range checks).
DEBUG_BUILD = os.environ.get("TCKS_DEBUG_CHECKS", "") == "1"
LIB_PATH = os.path.join(HERE, "_build_debug" if DEBUG_BUILD else "_build", "libtcks.so")

TCKS_AUTO_RELIN = 1
TCKS_AUTO_RESCALE = 2
TCKS_DOUBLE_HOIST = 4
TCKS_RECT_DIAG = 8
TCKS_CONV_HOIST = 16
TCKS_CONV_SHARED = 32
TCKS_CONV_PACK = 64
TCKS_MERGED_RESCALE = 128
TCKS_CONV_FOLD = 256
TCKS_CTA_ADD, TCKS_CTA_SUB, TCKS_CTA_MUL = 0, 1, 2  # ciphertext-array operations
KEY_SECRET, KEY_PUBLIC, KEY_RELIN, KEY_GALOIS = 0, 1, 2, 3

_u64p = ctypes.POINTER(ctypes.c_uint64)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_i32p = ctypes.POINTER(ctypes.c_int32)
_dblp = ctypes.POINTER(ctypes.c_double)
_vp = ctypes.c_void_p
_vpp = ctypes.POINTER(ctypes.c_void_p)


class TcksError(RuntimeError):
    def __init__(self, status: int, name: str, detail: str):
        super().__init__(f"{name} ({status}): {detail}")
        self.status = status
        self.name = name
        self.detail = detail


class _Allocator(ctypes.Structure):
    _fields_ = [("alloc", ctypes.CFUNCTYPE(_vp, ctypes.c_size_t, _vp, _vp)),
                ("free", ctypes.CFUNCTYPE(None, _vp, _vp, _vp)),
                ("user", _vp)]


# name -> (restype, argtypes); status-returning functions use c_int32
_SIGS = {
    "tcks_status_string": (ctypes.c_char_p, [ctypes.c_int32]),
    "tcks_last_error_detail": (ctypes.c_char_p, []),
    "tcks_params_create": (ctypes.c_int32, [ctypes.c_uint32, _u32p, ctypes.c_uint32, ctypes.c_double, _vpp]),
    "tcks_params_create_primes": (ctypes.c_int32, [ctypes.c_uint32, _u64p, ctypes.c_uint32, ctypes.c_double, _vpp]),
    "tcks_params_create_hybrid": (ctypes.c_int32, [ctypes.c_uint32, _u64p, ctypes.c_uint32, ctypes.c_uint32,
                                                   ctypes.c_uint32, ctypes.c_double, _vpp]),
    "tcks_params_free": (None, [_vp]),
    "tcks_params_primes": (ctypes.c_int32, [_vp, _u64p, ctypes.c_uint32]),
    "tcks_context_create": (ctypes.c_int32, [_vp, ctypes.c_uint64, ctypes.c_uint32, _vp, _vp, _vpp]),
    "tcks_ctx_free": (None, [_vp]),
    "tcks_ctx_info": (ctypes.c_int32, [_vp, _u32p, _u32p, _dblp]),
    "tcks_ctx_key_bytes": (ctypes.c_int32, [_vp, _u64p]),
    "tcks_ctx_synchronize": (ctypes.c_int32, [_vp]),
    "tcks_gen_galois_keys": (ctypes.c_int32, [_vp, _i32p, ctypes.c_uint32, ctypes.c_uint32]),
    "tcks_has_galois_key": (ctypes.c_int32, [_vp, ctypes.c_int32, _u32p]),
    "tcks_export_key": (ctypes.c_int32, [_vp, ctypes.c_uint32, ctypes.c_int32, _u64p, ctypes.c_size_t]),
    "tcks_import_key": (ctypes.c_int32, [_vp, ctypes.c_uint32, ctypes.c_int32, ctypes.c_uint32, _u64p,
                                          ctypes.c_size_t]),
    "tcks_encode": (ctypes.c_int32, [_vp, _dblp, ctypes.c_size_t, ctypes.c_double, ctypes.c_uint32, _vpp]),
    "tcks_encode_device": (ctypes.c_int32, [_vp, _vp, ctypes.c_size_t, ctypes.c_double, ctypes.c_uint32, _vpp]),
    "tcks_decode": (ctypes.c_int32, [_vp, _vp, _dblp, ctypes.c_size_t]),
    "tcks_encrypt": (ctypes.c_int32, [_vp, _vp, ctypes.c_uint64, _vpp]),
    "tcks_decrypt": (ctypes.c_int32, [_vp, _vp, _vpp]),
    "tcks_ct_import": (ctypes.c_int32, [_vp, _u64p, ctypes.c_uint32, ctypes.c_double, _vpp]),
    "tcks_ct_export": (ctypes.c_int32, [_vp, _u64p, ctypes.c_size_t]),
    "tcks_ct_import_sized": (ctypes.c_int32, [_vp, _u64p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_double, _vpp]),
    "tcks_ct_size": (ctypes.c_int32, [_vp, _u32p]),
    "tcks_relinearize": (ctypes.c_int32, [_vp]),
    "tcks_pt_import": (ctypes.c_int32, [_vp, _u64p, ctypes.c_uint32, ctypes.c_double, _vpp]),
    "tcks_pt_export": (ctypes.c_int32, [_vp, _u64p, ctypes.c_size_t]),
    "tcks_ct_info": (ctypes.c_int32, [_vp, _u32p, _dblp]),
    "tcks_pt_info": (ctypes.c_int32, [_vp, _u32p, _dblp]),
    "tcks_ct_device_ptr": (ctypes.c_int32, [_vp, ctypes.POINTER(_u64p)]),
    "tcks_ct_free": (None, [_vp]),
    "tcks_pt_free": (None, [_vp]),
    "tcks_add": (ctypes.c_int32, [_vp, _vp, _vpp]),
    "tcks_sub": (ctypes.c_int32, [_vp, _vp, _vpp]),
    "tcks_negate": (ctypes.c_int32, [_vp, _vpp]),
    "tcks_add_plain": (ctypes.c_int32, [_vp, _vp, _vpp]),
    "tcks_sub_plain": (ctypes.c_int32, [_vp, _vp, _vpp]),
    "tcks_mul_plain": (ctypes.c_int32, [_vp, _vp, _vpp]),
    "tcks_mul": (ctypes.c_int32, [_vp, _vp, _vpp]),
    "tcks_square": (ctypes.c_int32, [_vp, _vpp]),
    "tcks_cta_free": (None, [_vp]),
    "tcks_cta_info": (ctypes.c_int32, [_vp, _u32p, _u32p, _dblp]),
    "tcks_cta_import": (ctypes.c_int32, [_vp, _u64p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_double, _vpp]),
    "tcks_cta_export": (ctypes.c_int32, [_vp, _u64p, ctypes.c_size_t]),
    "tcks_cta_from_cts": (ctypes.c_int32, [_vpp, ctypes.c_uint32, _vpp]),
    "tcks_cta_get": (ctypes.c_int32, [_vp, ctypes.c_uint32, _vpp]),
    "tcks_cta_encrypt": (ctypes.c_int32, [_vp, _dblp, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                          ctypes.c_uint64, _vpp]),
    "tcks_cta_decrypt": (ctypes.c_int32, [_vp, _dblp, ctypes.c_uint32]),
    "tcks_cta_binary": (ctypes.c_int32, [ctypes.c_uint32, _vp, _vp, _vpp]),
    "tcks_cta_negate": (ctypes.c_int32, [_vp, _vpp]),
    "tcks_cta_plain": (ctypes.c_int32, [ctypes.c_uint32, _vp, _dblp, ctypes.c_uint32, _vpp]),
    "tcks_cta_combine": (ctypes.c_int32, [_vp, _u32p, _dblp, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int32,
                                          _vpp]),
    "tcks_cta_sum_slots": (ctypes.c_int32, [_vp, ctypes.c_uint32, _vpp]),
    "tcks_cta_power": (ctypes.c_int32, [_vp, ctypes.c_uint32, _vpp]),
    "tcks_cta_polyval": (ctypes.c_int32, [_vp, _dblp, ctypes.c_uint32, _vpp]),
    "tcks_cta_rescale": (ctypes.c_int32, [_vp]),
    "tcks_cta_mod_switch": (ctypes.c_int32, [_vp, ctypes.c_uint32]),
    "tcks_power": (ctypes.c_int32, [_vp, ctypes.c_uint32, _vpp]),
    "tcks_power_batch": (ctypes.c_int32, [_vpp, ctypes.c_uint32, ctypes.c_uint32, _vpp]),
    "tcks_polyval": (ctypes.c_int32, [_vp, _dblp, ctypes.c_uint32, _vpp]),
    "tcks_polyval_batch": (ctypes.c_int32, [_vpp, ctypes.c_uint32, _dblp, ctypes.c_uint32, _vpp]),
    "tcks_rescale": (ctypes.c_int32, [_vp]),
    "tcks_mod_switch": (ctypes.c_int32, [_vp, ctypes.c_uint32]),
    "tcks_rescale_noalloc": (ctypes.c_int32, [_vp, _vp, ctypes.c_uint32, _vp]),
    "tcks_rotate": (ctypes.c_int32, [_vp, ctypes.c_int32, _vpp]),
    "tcks_rotate_hoisted": (ctypes.c_int32, [_vp, _i32p, ctypes.c_uint32, _vpp]),
    "tcks_ntt_inplace": (ctypes.c_int32, [_vp, _vp, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int32]),
    "tcks_sum": (ctypes.c_int32, [_vp, ctypes.c_uint32, _vpp]),
    "tcks_dot": (ctypes.c_int32, [_vp, _vp, ctypes.c_uint32, _vpp]),
    "tcks_dot_plain": (ctypes.c_int32, [_vp, _dblp, ctypes.c_uint32, _vpp]),
    "tcks_matrix_encode": (ctypes.c_int32, [_vp, _dblp, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, _vpp]),
    "tcks_matrix_encode_rect": (ctypes.c_int32, [_vp, _dblp, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                                  _vpp]),
    "tcks_matrix_import_rect": (ctypes.c_int32, [_vp, _u64p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                                  ctypes.c_double, _vpp]),
    "tcks_matrix_import_ext": (ctypes.c_int32, [_vp, _u64p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                                 ctypes.c_double, _vpp]),
    "tcks_ctx_set_flags": (ctypes.c_int32, [_vp, ctypes.c_uint32]),
    "tcks_matrix_import": (ctypes.c_int32, [_vp, _u64p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                             ctypes.c_double, _vpp]),
    "tcks_matrix_free": (None, [_vp]),
    "tcks_vecmat_plain": (ctypes.c_int32, [_vp, _vp, _vpp]),
    "tcks_im2col_encode": (ctypes.c_int32, [_dblp, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                             ctypes.c_uint32, ctypes.c_uint32, _dblp, ctypes.c_size_t, _u32p]),
    "tcks_conv2d_im2col": (ctypes.c_int32, [_vp, _dblp, ctypes.c_uint32, ctypes.c_uint32, _vpp]),
    "tcks_conv2d_im2col_pt": (ctypes.c_int32, [_vp, _vp, ctypes.c_uint32, ctypes.c_uint32, _vpp]),
    "tcks_autotune": (ctypes.c_int32, [_vp, ctypes.c_char_p, _u32p]),
    "tcks_cnn_autotune": (ctypes.c_int32, [_vp, ctypes.c_uint32, ctypes.c_char_p, _u32p, _u32p, _u32p]),
    "tcks_launch_count": (ctypes.c_uint64, []),
    "tcks_debug_checks": (ctypes.c_int32, []),
    "tcks_ctx_set_launch_shape": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32]),
    "tcks_ctx_get_launch_shape": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint32),
                                                   ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint32)]),
    "tcks_debug_selftest": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32,
                                             ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32)]),
    "tcks_profile_start": (ctypes.c_int32, []),
    "tcks_profile_stop": (ctypes.c_int32, []),
    "tcks_profile_count": (ctypes.c_uint32, []),
    "tcks_profile_read_ops": (ctypes.c_int32, [ctypes.c_uint32, _dblp]),
    "tcks_calibrate_butterflies": (ctypes.c_int32, [ctypes.c_uint32, _dblp]),
    "tcks_calibrate_macs": (ctypes.c_int32, [ctypes.c_uint32, _dblp]),
    "tcks_calibrate_dh_macs": (ctypes.c_int32, [ctypes.c_uint32, _dblp]),
    "tcks_profile_records": (ctypes.c_int32, [ctypes.c_uint32, ctypes.c_uint32, _u32p, _dblp, _dblp, _u32p]),
    "tcks_profile_read": (ctypes.c_int32, [ctypes.c_uint32, ctypes.POINTER(ctypes.c_char_p),
                                            ctypes.POINTER(ctypes.c_uint64), _dblp, _dblp]),
    "tcks_server_create": (ctypes.c_int32, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, _vpp]),
    "tcks_server_free": (None, [_vp]),
    "tcks_server_add_cnn": (ctypes.c_int32, [_vp, _vp, _u32p]),
    "tcks_server_add_vecmat": (ctypes.c_int32, [_vp, _vp, _u32p]),
    "tcks_server_submit": (ctypes.c_int32, [_vp, ctypes.c_uint32, _vp, _u64p]),
    "tcks_server_step": (ctypes.c_int32, [_vp, _u32p]),
    "tcks_server_poll": (ctypes.c_int32, [_vp, _u64p, ctypes.c_uint32, _u32p]),
    "tcks_server_take": (ctypes.c_int32, [_vp, ctypes.c_uint64, _vpp]),
    "tcks_server_stats": (ctypes.c_int32, [_vp, _u64p, _u64p, _u64p, _u64p, _u64p]),
    "tcks_cnn_create": (ctypes.c_int32, [_vp, _dblp, _dblp, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                          _dblp, _dblp, ctypes.c_uint32, _dblp, _dblp, ctypes.c_uint32, _vpp]),
    "tcks_cnn_free": (None, [_vp]),
    "tcks_cnn_galois_steps": (ctypes.c_int32, [_vp, _i32p, _u32p, ctypes.c_uint32, _u32p]),
    "tcks_cnn_forward": (ctypes.c_int32, [_vp, _vp, _vpp]),
    "tcks_cnn_forward_batch": (ctypes.c_int32, [_vp, _vpp, ctypes.c_uint32, _vpp]),
    "tcks_cnn_forward_host": (ctypes.c_int32, [_vp, _u64p, ctypes.c_uint32, _u64p]),
    "tcks_cnn_forward_device": (ctypes.c_int32, [_vp, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p]),
    "tcks_cnn_wire_sizes": (ctypes.c_int32, [_vp, _u64p, _u64p, _u64p]),
    "tcks_cnn_pipe_create": (ctypes.c_int32, [_vp, ctypes.c_uint32, ctypes.c_uint64, _vpp]),
    "tcks_cnn_pipe_submit": (ctypes.c_int32, [_vp, ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64)]),
    "tcks_cnn_pipe_wait": (ctypes.c_int32, [_vp, ctypes.c_uint64]),
    "tcks_cnn_pipe_free": (None, [_vp]),
    "tcks_cnn_forward_wire": (ctypes.c_int32, [_vp, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32,
                                               ctypes.c_void_p, ctypes.c_uint64]),
    "tcks_vecmat_plain_batch": (ctypes.c_int32, [_vpp, ctypes.c_uint32, _vp, _vpp]),
    "tcks_ct_import_batch": (ctypes.c_int32, [_vp, _u64p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_double, _vpp]),
    "tcks_ct_export_batch": (ctypes.c_int32, [_vpp, ctypes.c_uint32, _u64p, ctypes.c_size_t]),
    "tcks_ct_serialized_size": (ctypes.c_int32, [_vp, _u64p]),
    "tcks_ct_serialize": (ctypes.c_int32, [_vp, ctypes.c_void_p, ctypes.c_uint64, _u64p]),
    "tcks_ct_deserialize": (ctypes.c_int32, [_vp, ctypes.c_void_p, ctypes.c_uint64, _vpp]),
    "tcks_encrypt_symmetric": (ctypes.c_int32, [_vp, _vp, ctypes.c_uint64, ctypes.c_uint64, _vpp]),
    "tcks_ct_serialized_size_seeded": (ctypes.c_int32, [_vp, _u64p]),
    "tcks_ct_serialize_seeded": (ctypes.c_int32, [_vp, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_uint64, _u64p]),
    "tcks_rotate_sum_hoisted": (ctypes.c_int32, [_vp, _i32p, ctypes.c_uint32, _vpp]),
    "tcks_batch_run": (ctypes.c_int32, [_vp, ctypes.c_uint32]),
    "tcks_executor_start": (ctypes.c_int32, [_vp, ctypes.c_uint32, ctypes.c_int64, _vpp]),
    "tcks_executor_post": (ctypes.c_int32, [_vp, ctypes.c_uint32, _vp, _vp, ctypes.c_uint32, ctypes.c_uint32, _u64p]),
    "tcks_executor_wait": (ctypes.c_int32, [_vp, ctypes.c_uint64, ctypes.c_int64]),
    "tcks_executor_close": (ctypes.c_int32, [_vp, ctypes.POINTER(ctypes.c_int32)]),
    "tcks_executor_free": (None, [_vp]),
    "tcks_batch_submit": (ctypes.c_int32, [_vp, ctypes.c_uint32, _vpp]),
    "tcks_batch_wait": (ctypes.c_int32, [_vp, ctypes.c_int64]),
    "tcks_batch_free": (None, [_vp]),
    "tcks_batch_graph_create": (ctypes.c_int32, [_vp, ctypes.c_uint32, _vpp]),
    "tcks_batch_graph_run": (ctypes.c_int32, [_vp]),
    "tcks_batch_graph_launches": (ctypes.c_int32, [_vp, _u64p]),
    "tcks_batch_graph_free": (None, [_vp]),
    "tcks_cnn_graph_create": (ctypes.c_int32, [_vp, ctypes.c_uint32, _vpp]),
    "tcks_cnn_graph_run": (ctypes.c_int32, [_vp, _vpp, _vpp]),
    "tcks_cnn_graph_free": (None, [_vp]),
    "tcks_cnn_export_plaintext": (ctypes.c_int32, [_vp, ctypes.c_uint32, ctypes.c_uint32, _u64p, ctypes.c_size_t,
                                                    _u32p, _dblp]),
}

_lib = None


def lib(build_if_missing: bool = False):
    """The loaded CUDA library. Raises if it has not been built (no fallback path exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        if build_if_missing:
            from .build import build
            build(debug=DEBUG_BUILD)
        else:
            raise RuntimeError(f"libtcks.so is not built ({LIB_PATH}); run paper_2104_03152_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in _SIGS.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def check(status: int):
    if status != 0:
        L = lib()
        raise TcksError(status, L.tcks_status_string(status).decode(), L.tcks_last_error_detail().decode())


def launch_count() -> int:
    return int(lib().tcks_launch_count())


def debug_checks() -> bool:
    """True when the loaded library is the debug build (descriptor and device range checks)."""
    return bool(lib().tcks_debug_checks())


def debug_selftest(ctx: "Context", d_ptr: int, polys: int, level: int, understate: int) -> int:
    """Forward NTT in place through the multi-context descriptor launch with the descriptor declaring
    `understate` limbs fewer than the grid covers; returns the error word the range checks set."""
    w = ctypes.c_uint32()
    check(lib().tcks_debug_selftest(ctx.h, _vp(d_ptr), polys, level, understate, ctypes.byref(w)))
    return w.value


def profile_start():
    check(lib().tcks_profile_start())


def profile_stop():
    check(lib().tcks_profile_stop())


def profile_read(with_ops: bool = False) -> dict:
    """{kernel family: (launches, device ms, algorithmic bytes[, algorithmic integer ops])} of the
    records since profile_start; ops are modular butterflies plus modular multiply(-accumulate)s."""
    L = lib()
    out = {}
    for i in range(L.tcks_profile_count()):
        name, n, ms, by = ctypes.c_char_p(), ctypes.c_uint64(), ctypes.c_double(), ctypes.c_double()
        check(L.tcks_profile_read(i, ctypes.byref(name), ctypes.byref(n), ctypes.byref(ms), ctypes.byref(by)))
        if n.value:
            rec = (n.value, ms.value, by.value)
            if with_ops:
                ops = ctypes.c_double()
                check(L.tcks_profile_read_ops(i, ctypes.byref(ops)))
                rec += (ops.value,)
            out[name.value.decode()] = rec
    return out


def profile_records(family: str) -> list:
    """[(shape tag, device ms, algorithmic ops)] of the profiled launches of one kernel family, in order."""
    L = lib()
    for i in range(L.tcks_profile_count()):
        name = ctypes.c_char_p()
        check(L.tcks_profile_read(i, ctypes.byref(name), None, None, None))
        if name.value.decode() != family:
            continue
        n = ctypes.c_uint32()
        check(L.tcks_profile_records(i, 0, None, None, None, ctypes.byref(n)))
        tags = np.zeros(n.value, dtype=np.uint32)
        ms = np.zeros(n.value, dtype=np.float64)
        ops = np.zeros(n.value, dtype=np.float64)
        check(L.tcks_profile_records(i, n.value, _p(tags), _p(ms), _p(ops), ctypes.byref(n)))
        return [(int(t), float(m), float(o)) for t, m, o in zip(tags, ms, ops)]
    return []


def calibrate_butterflies(word_bits: int = 64) -> float:
    """Modular butterflies per second of the integer pipe on the current device (registers only)."""
    v = ctypes.c_double()
    check(lib().tcks_calibrate_butterflies(word_bits, ctypes.byref(v)))
    return v.value


def calibrate_macs(word_bits: int) -> float:
    """Measured modular multiply-accumulates per second (32- or 64-bit words), registers only."""
    v = ctypes.c_double()
    check(lib().tcks_calibrate_macs(word_bits, ctypes.byref(v)))
    return v.value


def calibrate_dh_macs(ell: int) -> float:
    """Product-accumulates per second of the double-hoisted accumulation's own form at level ell."""
    v = ctypes.c_double()
    check(lib().tcks_calibrate_dh_macs(ell, ctypes.byref(v)))
    return v.value


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as({np.dtype(np.uint64): _u64p, np.dtype(np.float64): _dblp,
                             np.dtype(np.uint32): _u32p, np.dtype(np.int32): _i32p}[a.dtype])


class Params:
    """CKKS parameters: N = 2^log_n and the prime chain (data primes, then P), chosen from bit sizes
    (`bits`) or given explicitly (`primes`). n_special > 1 or alpha > 1: hybrid key switching with the
    last n_special primes special and digits of alpha data primes (tcks_params_create_hybrid)."""

    def __init__(self, log_n: int, bits=None, scale: float = 2.0 ** 40, primes=None, n_special: int = 1,
                 alpha: int = 1):
        h = _vp()
        self.n_special, self.alpha = int(n_special), int(alpha)
        if self.n_special > 1 or self.alpha > 1:
            if primes is None:  # the chain from bit sizes, then its primes
                tmp = Params(log_n, bits, scale)
                primes = tmp.primes
            q_in = np.ascontiguousarray([int(x) for x in primes], dtype=np.uint64)
            check(lib().tcks_params_create_hybrid(log_n, _p(q_in), len(q_in), self.n_special, self.alpha,
                                                  float(scale), ctypes.byref(h)))
            bits = [int(x).bit_length() for x in primes]
        elif primes is not None:
            q_in = np.ascontiguousarray([int(x) for x in primes], dtype=np.uint64)
            check(lib().tcks_params_create_primes(log_n, _p(q_in), len(q_in), float(scale), ctypes.byref(h)))
            bits = [int(x).bit_length() for x in primes]
        else:
            b = np.ascontiguousarray(bits, dtype=np.uint32)
            check(lib().tcks_params_create(log_n, _p(b), len(b), float(scale), ctypes.byref(h)))
        self.h = h
        self.log_n = log_n
        self.N = 1 << log_n
        self.bits = list(bits)
        self.scale = float(scale)
        q = np.zeros(len(self.bits), dtype=np.uint64)
        check(lib().tcks_params_primes(h, _p(q), len(q)))
        self.primes = [int(x) for x in q]

    def __del__(self):
        if getattr(self, "h", None):
            lib().tcks_params_free(self.h)
            self.h = None


# Allocator callbacks handed to the library stay referenced for the life of the process: a context
# outlives its Python wrapper while ciphertexts still hold it, and frees through these callbacks last.
_CALLBACKS_IN_USE = []


def _torch_allocator():
    """tcks_allocator backed by PyTorch's caching allocator (stream-ordered)."""
    import torch

    @ctypes.CFUNCTYPE(_vp, ctypes.c_size_t, _vp, _vp)
    def _alloc(nbytes, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), stream=stream or 0)
        except Exception:  # out of memory -> NULL, reported by the library as OUT_OF_MEMORY
            return None

    @ctypes.CFUNCTYPE(None, _vp, _vp, _vp)
    def _free(ptr, stream, user):
        torch.cuda.caching_allocator_delete(ptr)

    a = _Allocator(_alloc, _free, None)
    _CALLBACKS_IN_USE.append((a, _alloc, _free))
    return a, (_alloc, _free)


class Context:
    """TenSEAL context (§2.1): keys on the device, auto relinearize / rescale flags."""

    def __init__(self, params: Params, seed: int = 0x7E5EA1, flags: int = TCKS_AUTO_RELIN | TCKS_AUTO_RESCALE,
                 stream: int | None = None, allocator: str = "pool"):
        self.params = params
        self.N = params.N
        self.slots = params.N // 2
        self.primes = params.primes
        self.L = len(params.primes) - params.n_special
        self.stream = stream  # the cudaStream_t handle given by the caller (None: the context's own)
        self._alloc_keep = None
        aptr = None
        if allocator == "torch":
            a, keep = _torch_allocator()
            self._alloc_keep = (a, keep)
            aptr = ctypes.cast(ctypes.pointer(a), _vp)
        h = _vp()
        self.flags = flags
        check(lib().tcks_context_create(params.h, seed, flags, aptr, _vp(stream) if stream else None,
                                        ctypes.byref(h)))
        self.h = h

    def __del__(self):
        if getattr(self, "h", None):
            lib().tcks_ctx_free(self.h)
            self.h = None

    def synchronize(self):
        check(lib().tcks_ctx_synchronize(self.h))

    def set_launch_shape(self, limb_threads: int = 0, accum_rpt: int = 0, accum_form: int = 0):
        """Launch shape of the context's kernels (bit-identical results for every shape); accum_form 0 (the
        default) loads the accumulation's operands thread by thread, 1..4 stage them with bulk copies."""
        check(lib().tcks_ctx_set_launch_shape(self.h, limb_threads, accum_rpt, accum_form))

    def launch_shape(self) -> tuple:
        a, b, c = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
        check(lib().tcks_ctx_get_launch_shape(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return a.value, b.value, c.value

    def autotune(self, cache_path: str | None = None) -> int:
        t = ctypes.c_uint32()
        check(lib().tcks_autotune(self.h, cache_path.encode() if cache_path else None, ctypes.byref(t)))
        return t.value

    def key_bytes(self) -> int:
        v = ctypes.c_uint64()
        check(lib().tcks_ctx_key_bytes(self.h, ctypes.byref(v)))
        return v.value

    def gen_galois_keys(self, steps, max_level: int = 0):
        s = np.ascontiguousarray(list(steps), dtype=np.int32)
        check(lib().tcks_gen_galois_keys(self.h, _p(s), len(s), max_level))

    def galois_key_level(self, step: int) -> int | None:
        v = ctypes.c_uint32()
        st = lib().tcks_has_galois_key(self.h, step, ctypes.byref(v))
        return v.value if st == 0 else None

    def _switch_key_shape(self, K: int):
        """[digits][2][K + special primes][N] for a switching key of level K."""
        a, sp = self.params.alpha, self.params.n_special
        return (-(-K // a), 2, K + sp, self.N)

    def _key_shape(self, kind: int, step: int):
        N, L = self.N, self.L
        if kind == KEY_SECRET:
            return (L + self.params.n_special, N)
        if kind == KEY_PUBLIC:
            return (2, L, N)
        if kind == KEY_RELIN:
            return self._switch_key_shape(L)
        K = self.galois_key_level(step)
        if K is None:
            raise KeyError(step)
        return self._switch_key_shape(K)

    def export_key(self, kind: int, step: int = 0) -> np.ndarray:
        a = np.zeros(self._key_shape(kind, step), dtype=np.uint64)
        check(lib().tcks_export_key(self.h, kind, step, _p(a), a.size))
        return a

    def import_key(self, kind: int, data: np.ndarray, step: int = 0, key_level: int = 0):
        a = np.ascontiguousarray(data, dtype=np.uint64)
        check(lib().tcks_import_key(self.h, kind, step, key_level, _p(a), a.size))

    # encode / encrypt
    def encode(self, v, scale: float = 0.0, level: int = 0) -> "Plaintext":
        a = np.ascontiguousarray(v, dtype=np.float64)
        h = _vp()
        check(lib().tcks_encode(self.h, _p(a), len(a), float(scale), level, ctypes.byref(h)))
        return Plaintext(self, h)

    def decode(self, pt: "Plaintext", n: int | None = None) -> np.ndarray:
        n = self.slots if n is None else n
        out = np.zeros(n, dtype=np.float64)
        check(lib().tcks_decode(self.h, pt.h, _p(out), n))
        return out

    def encrypt(self, pt: "Plaintext", seed: int) -> "Ciphertext":
        h = _vp()
        check(lib().tcks_encrypt(self.h, pt.h, seed, ctypes.byref(h)))
        return Ciphertext(self, h)

    def encrypt_symmetric(self, pt: "Plaintext", seed_a: int, seed_e: int) -> "Ciphertext":
        """Secret-key encryption: c1 from the public seed seed_a, the error from the private seed seed_e."""
        h = _vp()
        check(lib().tcks_encrypt_symmetric(self.h, pt.h, seed_a, seed_e, ctypes.byref(h)))
        return Ciphertext(self, h)

    def decrypt(self, ct: "Ciphertext") -> "Plaintext":
        h = _vp()
        check(lib().tcks_decrypt(self.h, ct.h, ctypes.byref(h)))
        return Plaintext(self, h)

    def encrypt_values(self, v, seed: int, level: int = 0) -> "Ciphertext":
        return self.encrypt(self.encode(v, level=level), seed)

    def decrypt_values(self, ct: "Ciphertext", n: int | None = None) -> np.ndarray:
        return self.decode(self.decrypt(ct), n)

    def ct_import(self, limbs: np.ndarray, scale: float) -> "Ciphertext":
        """A ciphertext from host limbs [size][level][N] (size 2, or 3 for an unrelinearized product)."""
        a = np.ascontiguousarray(limbs, dtype=np.uint64)
        size, level = a.shape[0], a.shape[1]
        h = _vp()
        if size == 2:
            check(lib().tcks_ct_import(self.h, _p(a), level, float(scale), ctypes.byref(h)))
        else:
            check(lib().tcks_ct_import_sized(self.h, _p(a), size, level, float(scale), ctypes.byref(h)))
        return Ciphertext(self, h)

    def ct_import_batch(self, limbs: np.ndarray, scale: float) -> list:
        """Ciphertexts from host limbs [count][2][level][N] (one wait for all the copies)."""
        a = np.ascontiguousarray(limbs, dtype=np.uint64)
        outs = (_vp * a.shape[0])()
        check(lib().tcks_ct_import_batch(self.h, _p(a), a.shape[0], a.shape[2], float(scale), outs))
        return [Ciphertext(self, _vp(outs[i])) for i in range(a.shape[0])]

    def ct_deserialize(self, data: bytes) -> "Ciphertext":
        """A ciphertext from the bit-packed wire format (see tcks_ct_serialize)."""
        buf = ctypes.create_string_buffer(bytes(data), len(data))
        h = _vp()
        check(lib().tcks_ct_deserialize(self.h, buf, len(data), ctypes.byref(h)))
        return Ciphertext(self, h)

    def pt_import(self, limbs: np.ndarray, scale: float) -> "Plaintext":
        a = np.ascontiguousarray(limbs, dtype=np.uint64)
        h = _vp()
        check(lib().tcks_pt_import(self.h, _p(a), a.shape[0], float(scale), ctypes.byref(h)))
        return Plaintext(self, h)

    def rescale_noalloc(self, d_in: int, level: int, d_out: int):
        """Allocation-free rescale of device limbs [2][level][N] into [2][level-1][N] (see tcks.h)."""
        check(lib().tcks_rescale_noalloc(self.h, _vp(d_in), level, _vp(d_out)))

    def ntt_inplace(self, d_ptr: int, polys: int, level: int, inverse: bool):
        check(lib().tcks_ntt_inplace(self.h, _vp(d_ptr), polys, level, 1 if inverse else 0))

    def matrix_encode(self, M: np.ndarray, level: int = 0) -> "Matrix":
        a = np.ascontiguousarray(M, dtype=np.float64)
        h = _vp()
        check(lib().tcks_matrix_encode(self.h, _p(a), a.shape[0], a.shape[1], level, ctypes.byref(h)))
        return Matrix(self, h, a.shape[0], a.shape[1])

    def matrix_import(self, diag_limbs: np.ndarray, rows: int, cols: int, scale: float) -> "Matrix":
        a = np.ascontiguousarray(diag_limbs, dtype=np.uint64)
        h = _vp()
        check(lib().tcks_matrix_import(self.h, _p(a), rows, cols, a.shape[1], float(scale), ctypes.byref(h)))
        return Matrix(self, h, rows, cols)

    def matrix_encode_rect(self, M: np.ndarray, level: int = 0) -> "Matrix":
        """Rectangular (hybrid) diagonals: fewer rotations; slots >= cols of the product hold partial sums."""
        a = np.ascontiguousarray(M, dtype=np.float64)
        h = _vp()
        check(lib().tcks_matrix_encode_rect(self.h, _p(a), a.shape[0], a.shape[1], level, ctypes.byref(h)))
        return Matrix(self, h, a.shape[0], a.shape[1])

    def matrix_import_rect(self, diag_limbs: np.ndarray, rows: int, cols: int, scale: float) -> "Matrix":
        """Rectangular-form diagonals over the extended basis [m'][level+1][N]."""
        a = np.ascontiguousarray(diag_limbs, dtype=np.uint64)
        h = _vp()
        check(lib().tcks_matrix_import_rect(self.h, _p(a), rows, cols, a.shape[1] - 1, float(scale), ctypes.byref(h)))
        return Matrix(self, h, rows, cols)

    def matrix_import_ext(self, diag_limbs: np.ndarray, rows: int, cols: int, scale: float) -> "Matrix":
        """Diagonals over the extended basis [rows][level+1][N] (limb `level` modulo P)."""
        a = np.ascontiguousarray(diag_limbs, dtype=np.uint64)
        h = _vp()
        check(lib().tcks_matrix_import_ext(self.h, _p(a), rows, cols, a.shape[1] - 1, float(scale), ctypes.byref(h)))
        return Matrix(self, h, rows, cols)

    def set_flags(self, flags: int):
        check(lib().tcks_ctx_set_flags(self.h, flags))
        self.flags = flags


def im2col_encode(img: np.ndarray, kh: int, kw: int, stride: int, cap: int):
    """Client-side im2col (§3.2): (slot vector of length cap, number of windows)."""
    a = np.ascontiguousarray(img, dtype=np.float64)
    out = np.zeros(cap, dtype=np.float64)
    w = ctypes.c_uint32()
    check(lib().tcks_im2col_encode(_p(a), a.shape[0], a.shape[1], kh, kw, stride, _p(out), cap, ctypes.byref(w)))
    return out, w.value


class Plaintext:
    def __init__(self, ctx: Context, h):
        self.ctx = ctx
        self.h = h

    def __del__(self):
        if getattr(self, "h", None):
            lib().tcks_pt_free(self.h)
            self.h = None

    def info(self):
        lv, sc = ctypes.c_uint32(), ctypes.c_double()
        check(lib().tcks_pt_info(self.h, ctypes.byref(lv), ctypes.byref(sc)))
        return lv.value, sc.value

    @property
    def level(self) -> int:
        return self.info()[0]

    @property
    def scale(self) -> float:
        return self.info()[1]

    def export(self) -> np.ndarray:
        a = np.zeros((self.level, self.ctx.N), dtype=np.uint64)
        check(lib().tcks_pt_export(self.h, _p(a), a.size))
        return a


class Matrix:
    def __init__(self, ctx: Context, h, rows: int, cols: int):
        self.ctx = ctx
        self.h = h
        self.rows = rows
        self.cols = cols

    def __del__(self):
        if getattr(self, "h", None):
            lib().tcks_matrix_free(self.h)
            self.h = None

    def vecmat_batch(self, cts) -> list:
        """cts[i] x this matrix for a batch of one level and scale (one batched pass)."""
        ins = (_vp * len(cts))(*[c.h.value if isinstance(c.h, _vp) else c.h for c in cts])
        outs = (_vp * len(cts))()
        check(lib().tcks_vecmat_plain_batch(ins, len(cts), self.h, outs))
        return [Ciphertext(self.ctx, _vp(outs[i])) for i in range(len(cts))]


class Ciphertext:
    """A CKKSVector: up to N/2 encrypted real slots in one ciphertext (§2.3)."""

    def __init__(self, ctx: Context, h):
        self.ctx = ctx
        self.h = h

    def __del__(self):
        if getattr(self, "h", None):
            lib().tcks_ct_free(self.h)
            self.h = None

    def info(self):
        lv, sc = ctypes.c_uint32(), ctypes.c_double()
        check(lib().tcks_ct_info(self.h, ctypes.byref(lv), ctypes.byref(sc)))
        return lv.value, sc.value

    @property
    def level(self) -> int:
        return self.info()[0]

    @property
    def scale(self) -> float:
        return self.info()[1]

    def serialize(self) -> bytes:
        """The bit-packed wire format (bit_length(q_i) bits per residue, 16-byte header)."""
        size = np.zeros(1, dtype=np.uint64)
        check(lib().tcks_ct_serialized_size(self.h, _p(size)))
        buf = ctypes.create_string_buffer(int(size[0]))
        written = np.zeros(1, dtype=np.uint64)
        check(lib().tcks_ct_serialize(self.h, buf, int(size[0]), _p(written)))
        return buf.raw[: int(written[0])]

    def serialize_seeded(self, seed_a: int) -> bytes:
        """Wire kind 1 (c0 and the seed of c1) of a fresh secret-key ciphertext."""
        size = np.zeros(1, dtype=np.uint64)
        check(lib().tcks_ct_serialized_size_seeded(self.h, _p(size)))
        buf = ctypes.create_string_buffer(int(size[0]))
        written = np.zeros(1, dtype=np.uint64)
        check(lib().tcks_ct_serialize_seeded(self.h, seed_a, buf, int(size[0]), _p(written)))
        return buf.raw[: int(written[0])]

    @property
    def size(self) -> int:
        """Components: 2, or 3 for an enc x enc product taken without automatic relinearization."""
        v = ctypes.c_uint32()
        check(lib().tcks_ct_size(self.h, ctypes.byref(v)))
        return v.value

    def export(self) -> np.ndarray:
        a = np.zeros((self.size, self.level, self.ctx.N), dtype=np.uint64)
        check(lib().tcks_ct_export(self.h, _p(a), a.size))
        return a

    def device_ptr(self) -> int:
        p = _u64p()
        check(lib().tcks_ct_device_ptr(self.h, ctypes.byref(p)))
        return ctypes.cast(p, _vp).value

    def _unary(self, fn, *args) -> "Ciphertext":
        h = _vp()
        check(fn(self.h, *args, ctypes.byref(h)))
        return Ciphertext(self.ctx, h)

    def add(self, o: "Ciphertext"):
        return self._unary(lib().tcks_add, o.h)

    def sub(self, o: "Ciphertext"):
        return self._unary(lib().tcks_sub, o.h)

    def negate(self):
        return self._unary(lib().tcks_negate)

    def add_plain(self, p: Plaintext):
        return self._unary(lib().tcks_add_plain, p.h)

    def sub_plain(self, p: Plaintext):
        return self._unary(lib().tcks_sub_plain, p.h)

    def mul_plain(self, p: Plaintext):
        return self._unary(lib().tcks_mul_plain, p.h)

    def mul(self, o: "Ciphertext"):
        return self._unary(lib().tcks_mul, o.h)

    def square(self):
        return self._unary(lib().tcks_square)

    def power(self, k: int):
        """x^k element-wise with the minimum depth ceil(log2 k)."""
        return self._unary(lib().tcks_power, k)

    def polyval(self, coeffs):
        """sum_i coeffs[i] x^i element-wise (lowest degree first); result at the context scale."""
        a = np.ascontiguousarray(coeffs, dtype=np.float64)
        return self._unary(lib().tcks_polyval, _p(a), len(a))

    def relinearize_(self):
        """Relinearize in place (three components -> two); a two-component ciphertext is unchanged."""
        check(lib().tcks_relinearize(self.h))
        return self

    def rescale_(self):
        check(lib().tcks_rescale(self.h))
        return self

    def mod_switch_(self, level: int):
        check(lib().tcks_mod_switch(self.h, level))
        return self

    def rotate(self, step: int):
        return self._unary(lib().tcks_rotate, step)

    def rotate_sum_hoisted(self, steps):
        """self + sum of rot(self, s) over steps, one ModUp and one ModDown for all of them."""
        st = np.ascontiguousarray(list(steps), dtype=np.int32)
        return self._unary(lib().tcks_rotate_sum_hoisted, _p(st), len(st))

    def rotate_hoisted(self, steps) -> list:
        s = np.ascontiguousarray(list(steps), dtype=np.int32)
        outs = (_vp * len(s))()
        check(lib().tcks_rotate_hoisted(self.h, _p(s), len(s), outs))
        return [Ciphertext(self.ctx, _vp(outs[i])) for i in range(len(s))]

    def sum(self, n: int):
        return self._unary(lib().tcks_sum, n)

    def dot(self, o: "Ciphertext", n: int):
        return self._unary(lib().tcks_dot, o.h, n)

    def dot_plain(self, w, n: int | None = None):
        a = np.ascontiguousarray(w, dtype=np.float64)
        return self._unary(lib().tcks_dot_plain, _p(a), len(a) if n is None else n)

    def vecmat_plain(self, M: Matrix):
        return self._unary(lib().tcks_vecmat_plain, M.h)

    def conv2d_im2col(self, kernel, windows: int):
        k = np.ascontiguousarray(kernel, dtype=np.float64).reshape(-1)
        return self._unary(lib().tcks_conv2d_im2col, _p(k), len(k), windows)

    def conv2d_im2col_pt(self, kernel: Plaintext, taps: int, windows: int):
        return self._unary(lib().tcks_conv2d_im2col_pt, kernel.h, taps, windows)


def _handles(cts):
    return (_vp * len(cts))(*[c.h.value if isinstance(c.h, _vp) else c.h for c in cts])


def power_batch(cts, k: int) -> list:
    """x^k for ciphertexts of one level and scale in batched launches."""
    if not cts:
        return []
    outs = (_vp * len(cts))()
    check(lib().tcks_power_batch(_handles(cts), len(cts), k, outs))
    return [Ciphertext(cts[0].ctx, _vp(outs[i])) for i in range(len(cts))]


def polyval_batch(cts, coeffs) -> list:
    """sum_i coeffs[i] x^i for ciphertexts of one level and scale in batched launches."""
    if not cts:
        return []
    a = np.ascontiguousarray(coeffs, dtype=np.float64)
    outs = (_vp * len(cts))()
    check(lib().tcks_polyval_batch(_handles(cts), len(cts), _p(a), len(a), outs))
    return [Ciphertext(cts[0].ctx, _vp(outs[i])) for i in range(len(cts))]


class CNN:
    """The encrypted MNIST-shaped network of §5 (conv -> square -> FC -> square -> FC)."""

    def __init__(self, ctx: Context, conv_w, conv_b, fc1_w, fc1_b, fc2_w, fc2_b, windows: int = 64):
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (conv_w, conv_b, fc1_w, fc1_b, fc2_w, fc2_b)]
        self._keep = arrs
        cw, cb, w1, b1, w2, b2 = arrs
        h = _vp()
        check(lib().tcks_cnn_create(ctx.h, _p(cw), _p(cb), cw.shape[0], cw.shape[1], windows, _p(w1), _p(b1),
                                    w1.shape[0], _p(w2), _p(b2), w2.shape[0], ctypes.byref(h)))
        self.ctx = ctx
        self.h = h
        self.classes = w2.shape[0]

    def __del__(self):
        if getattr(self, "h", None):
            lib().tcks_cnn_free(self.h)
            self.h = None

    def galois_steps(self) -> dict:
        n = ctypes.c_uint32()
        check(lib().tcks_cnn_galois_steps(self.h, None, None, 0, ctypes.byref(n)))
        st = np.zeros(n.value, dtype=np.int32)
        lv = np.zeros(n.value, dtype=np.uint32)
        check(lib().tcks_cnn_galois_steps(self.h, _p(st), _p(lv), n.value, ctypes.byref(n)))
        return {int(s): int(l) for s, l in zip(st, lv)}

    def gen_keys(self):
        """Galois keys for every step, each trimmed to the level it is used at."""
        by_level = {}
        for s, l in self.galois_steps().items():
            by_level.setdefault(l, []).append(s)
        for l, steps in sorted(by_level.items()):
            self.ctx.gen_galois_keys(steps, l)

    def forward(self, ct: Ciphertext) -> Ciphertext:
        h = _vp()
        check(lib().tcks_cnn_forward(self.h, ct.h, ctypes.byref(h)))
        return Ciphertext(self.ctx, h)

    def forward_batch(self, cts) -> list:
        ins = (_vp * len(cts))(*[c.h.value if isinstance(c.h, _vp) else c.h for c in cts])
        outs = (_vp * len(cts))()
        check(lib().tcks_cnn_forward_batch(self.h, ins, len(cts), outs))
        return [Ciphertext(self.ctx, _vp(outs[i])) for i in range(len(cts))]

    def forward_device(self, d_in: int, count: int, d_out: int):
        """The batched forward pass on device buffers (pointers to [count][2][L][N] and
        [count][2][L-6][N] words), enqueued on the context's stream."""
        check(lib().tcks_cnn_forward_device(self.h, d_in, count, d_out))

    def forward_host(self, host_in: np.ndarray, host_out: np.ndarray):
        """The batched forward pass from host limbs [count][2][L][N] into host_out [count][2][L-6][N]."""
        assert host_in.dtype == np.uint64 and host_out.dtype == np.uint64
        check(lib().tcks_cnn_forward_host(self.h, _p(host_in), host_in.shape[0], _p(host_out)))
        return host_out

    def autotune(self, batch: int, cache_path: str | None = None) -> tuple[int, int, int]:
        """Times the batched forward pass at `batch` requests over the launch shapes and keeps the fastest
        (CTA size of the limb kernels, requests per thread of the accumulation, its form: 0 per-thread
        loads, 1..4 staged by bulk copies); returns that triple."""
        t, r, f = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
        check(lib().tcks_cnn_autotune(self.h, batch, cache_path.encode() if cache_path else None, ctypes.byref(t),
                                      ctypes.byref(r), ctypes.byref(f)))
        return t.value, r.value, f.value

    def wire_sizes(self) -> tuple[int, int, int]:
        """Bytes of one serialized input (both components), one seeded input, one serialized output."""
        v = np.zeros(3, dtype=np.uint64)
        check(lib().tcks_cnn_wire_sizes(self.h, _p(v[0:]), _p(v[1:]), _p(v[2:])))
        return int(v[0]), int(v[1]), int(v[2])

    def forward_wire(self, host_in: np.ndarray, count: int, host_out: np.ndarray) -> np.ndarray:
        """The batched forward pass on serialized ciphertexts: host_in = count inputs of one size (uint8,
        [count][in_size]), host_out [count][out_size] uint8 receives the serialized outputs."""
        assert host_in.dtype == np.uint8 and host_out.dtype == np.uint8
        assert host_in.flags.c_contiguous and host_out.flags.c_contiguous
        in_size, out_size = host_in.size // max(count, 1), host_out.size // max(count, 1)
        check(lib().tcks_cnn_forward_wire(self.h, host_in.ctypes.data, in_size, count, host_out.ctypes.data,
                                          out_size))
        return host_out

    def graph(self, count: int) -> "CNNGraph":
        return CNNGraph(self, count)

    def pipe(self, count: int, in_size: int) -> "CNNPipe":
        return CNNPipe(self, count, in_size)

    def export_plaintext(self, kind: int, index: int):
        lv = {0: self.ctx.L, 1: self.ctx.L - 1, 2: self.ctx.L - 2 - 2 * index, 3: self.ctx.L - 3,
              4: self.ctx.L - 5, 5: self.ctx.L - 2, 6: self.ctx.L - 4, 7: self.ctx.L + 1, 8: self.ctx.L + 1}[kind]
        a = np.zeros((lv, self.ctx.N), dtype=np.uint64)
        l, sc = ctypes.c_uint32(), ctypes.c_double()
        check(lib().tcks_cnn_export_plaintext(self.h, kind, index, _p(a), a.size, ctypes.byref(l), ctypes.byref(sc)))
        return a, sc.value


JOB_NTT, JOB_INTT, JOB_RELIN, JOB_ROTATE = 0, 1, 2, 3


class _BatchJob(ctypes.Structure):
    _fields_ = [("ctx", _vp), ("op", ctypes.c_uint32), ("step", ctypes.c_int32), ("count", ctypes.c_uint32),
                ("level", ctypes.c_uint32), ("d_in", _vp), ("d_out", _vp)]


def _job_array(jobs):
    """jobs: (context, op, step, count, level, d_in, d_out) tuples with device pointers as ints."""
    arr = (_BatchJob * len(jobs))()
    for i, (ctx, op, step, count, level, d_in, d_out) in enumerate(jobs):
        arr[i] = _BatchJob(ctx.h, op, step, count, level, _vp(d_in), _vp(d_out))
    return arr


def batch_run(jobs):
    """Runs a descriptor table of NTT / INTT / relinearize / rotate jobs over raw device buffers,
    possibly of several contexts and levels, as one batched unit (asynchronous on the first job's
    context stream)."""
    arr = _job_array(jobs)
    check(lib().tcks_batch_run(arr, len(jobs)))


EXEC_NTT, EXEC_INTT = 0, 1


class Executor:
    """A persistent kernel taking NTT / INTT jobs from a queue (tcks_executor_*); every wait inside it is
    bounded by idle_timeout_ns."""

    def __init__(self, ctx: "Context", capacity: int = 4096, idle_timeout_ns: int = 1_000_000_000):
        self.ctx = ctx
        h = _vp()
        check(lib().tcks_executor_start(ctx.h, capacity, int(idle_timeout_ns), ctypes.byref(h)))
        self.h = h

    def post(self, op: int, d_in: int, d_out: int, polys: int, level: int) -> int:
        t = np.zeros(1, dtype=np.uint64)
        check(lib().tcks_executor_post(self.h, op, _vp(d_in), _vp(d_out), polys, level, _p(t)))
        return int(t[0])

    def wait(self, ticket: int, timeout_ns: int = -1):
        check(lib().tcks_executor_wait(self.h, ticket, int(timeout_ns)))

    def close(self) -> int:
        """Stops the kernel; returns its status word (0, or the TIMEOUT code)."""
        st = ctypes.c_int32()
        check(lib().tcks_executor_close(self.h, ctypes.byref(st)))
        return st.value

    def __del__(self):
        if getattr(self, "h", None):
            lib().tcks_executor_free(self.h)
            self.h = None


class Batch:
    """A submitted job table with a completion handle (tcks_batch_submit / tcks_batch_wait)."""

    def __init__(self, jobs):
        self._ctxs = [j[0] for j in jobs]
        arr = _job_array(jobs)
        h = _vp()
        check(lib().tcks_batch_submit(arr, len(jobs), ctypes.byref(h)))
        self.h = h

    def wait(self, timeout_ns: int = -1):
        """Waits up to timeout_ns (negative: without limit); raises TcksError TIMEOUT if not done."""
        check(lib().tcks_batch_wait(self.h, int(timeout_ns)))

    def __del__(self):
        if getattr(self, "h", None):
            lib().tcks_batch_free(self.h)
            self.h = None


class BatchGraph:
    """A job table captured once as a CUDA graph and replayed over the same buffers."""

    def __init__(self, jobs):
        self._ctxs = [j[0] for j in jobs]  # the contexts outlive the graph
        arr = _job_array(jobs)
        h = _vp()
        check(lib().tcks_batch_graph_create(arr, len(jobs), ctypes.byref(h)))
        self.h = h
        n = np.zeros(1, dtype=np.uint64)
        check(lib().tcks_batch_graph_launches(h, _p(n)))
        self.launches = int(n[0])

    def run(self):
        check(lib().tcks_batch_graph_run(self.h))

    def __del__(self):
        if getattr(self, "h", None):
            lib().tcks_batch_graph_free(self.h)
            self.h = None


class CNNPipe:
    """Pipelined serialized batches (tcks_cnn_pipe_*): submit queues a batch of `count` inputs of
    in_size bytes and returns a ticket; wait(ticket) returns once its outputs are in its host_out. The
    arrays must stay alive and unchanged until their batch completes (pinned memory lets the copies
    run asynchronously)."""

    def __init__(self, model: "CNN", count: int, in_size: int):
        h = _vp()
        check(lib().tcks_cnn_pipe_create(model.h, count, in_size, ctypes.byref(h)))
        self.model, self.count, self.in_size, self.h = model, count, in_size, h
        self._held = {}

    def submit(self, host_in: np.ndarray, host_out: np.ndarray) -> int:
        assert host_in.dtype == np.uint8 and host_out.dtype == np.uint8
        assert host_in.flags.c_contiguous and host_out.flags.c_contiguous
        assert host_in.size == self.count * self.in_size
        t = ctypes.c_uint64()
        check(lib().tcks_cnn_pipe_submit(self.h, host_in.ctypes.data, host_out.ctypes.data, ctypes.byref(t)))
        self._held[t.value] = (host_in, host_out)
        for k in [k for k in self._held if k + 2 <= t.value]:  # completed by this submit
            del self._held[k]
        return t.value

    def wait(self, ticket: int):
        check(lib().tcks_cnn_pipe_wait(self.h, ticket))
        self._held.pop(ticket, None)

    def __del__(self):
        if getattr(self, "h", None):
            lib().tcks_cnn_pipe_free(self.h)
            self.h = None


class CNNGraph:
    """The batched forward captured as a CUDA graph for `count` requests per replay."""

    def __init__(self, model: CNN, count: int):
        h = _vp()
        check(lib().tcks_cnn_graph_create(model.h, count, ctypes.byref(h)))
        self.model = model
        self.count = count
        self.h = h

    def __del__(self):
        if getattr(self, "h", None):
            lib().tcks_cnn_graph_free(self.h)
            self.h = None

    def run(self, cts) -> list:
        assert len(cts) == self.count
        ins = (_vp * len(cts))(*[c.h.value if isinstance(c.h, _vp) else c.h for c in cts])
        outs = (_vp * len(cts))()
        check(lib().tcks_cnn_graph_run(self.h, ins, outs))
        return [Ciphertext(self.model.ctx, _vp(outs[i])) for i in range(len(cts))]


class Server:
    """Continuous-batching serving loop with HBM-budget admission (see tcks_server_* in tcks.h)."""

    def __init__(self, hbm_budget_bytes: int, max_in_flight: int = 1024, max_batch: int = 64):
        h = _vp()
        check(lib().tcks_server_create(int(hbm_budget_bytes), max_in_flight, max_batch, ctypes.byref(h)))
        self.h = h
        self._keep = []

    def __del__(self):
        if getattr(self, "h", None):
            lib().tcks_server_free(self.h)
            self.h = None

    def add_cnn(self, model: CNN) -> int:
        lane = ctypes.c_uint32()
        check(lib().tcks_server_add_cnn(self.h, model.h, ctypes.byref(lane)))
        self._keep.append(model)
        return lane.value

    def add_vecmat(self, M: Matrix) -> int:
        lane = ctypes.c_uint32()
        check(lib().tcks_server_add_vecmat(self.h, M.h, ctypes.byref(lane)))
        self._keep.append(M)
        return lane.value

    def submit(self, lane: int, ct: Ciphertext) -> int:
        rid = ctypes.c_uint64()
        check(lib().tcks_server_submit(self.h, lane, ct.h, ctypes.byref(rid)))
        return rid.value

    def step(self) -> int:
        n = ctypes.c_uint32()
        check(lib().tcks_server_step(self.h, ctypes.byref(n)))
        return n.value

    def poll(self, cap: int = 4096) -> list:
        ids = np.zeros(cap, dtype=np.uint64)
        n = ctypes.c_uint32()
        check(lib().tcks_server_poll(self.h, _p(ids), cap, ctypes.byref(n)))
        return [int(x) for x in ids[: n.value]]

    def take(self, rid: int, ctx: Context) -> Ciphertext:
        h = _vp()
        check(lib().tcks_server_take(self.h, rid, ctypes.byref(h)))
        return Ciphertext(ctx, h)

    def stats(self) -> dict:
        v = [ctypes.c_uint64() for _ in range(5)]
        check(lib().tcks_server_stats(self.h, *[ctypes.byref(x) for x in v]))
        return dict(zip(["queued", "in_flight", "finished", "bytes_in_use", "bytes_resident"], [x.value for x in v]))

from .tensor import CKKSTensor  # noqa: E402,F401
