"""Thin ctypes binding of libicm (include/icm.h), with the C entry points under the same names.

Argument marshalling only: every step of the matching path runs in the library's CUDA kernels.
PyTorch provides device memory (uint8 tensors sized by the *_bytes queries) and streams.  If the
compiled library is missing, importing the binding raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libicm.so")

ICM_OK, ICM_EINVAL, ICM_ENOMEM, ICM_ECUDA, ICM_ETIMEOUT, ICM_EBOUND, ICM_EUNSUPPORTED = range(7)
ICM_FORM_U64, ICM_FORM_I8_DIGITS, ICM_FORM_I8_CRT, ICM_FORM_F16_CRT, ICM_FORM_I8_P2 = range(5)
FORMS = {"u64": ICM_FORM_U64, "i8_digits": ICM_FORM_I8_DIGITS, "i8_crt": ICM_FORM_I8_CRT, "f16_crt": ICM_FORM_F16_CRT,
         "i8_p2": ICM_FORM_I8_P2}


class IcmError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        self.status = status
        super().__init__(f"{where}: status {status} ({detail})")


class icm_server_cfg(ctypes.Structure):
    _fields_ = [("max_eyes", ctypes.c_uint32), ("window_us", ctypes.c_uint32), ("form", ctypes.c_int),
                ("max_pending", ctypes.c_uint32), ("max_batches", ctypes.c_uint32)]


class icm_params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in (
        "log_n_db", "log_n_q", "n_limbs", "n_limbs_q", "prime_bits", "code_bits", "d2", "rho", "fold_k",
        "hamming_weight", "log2_delta", "noise_eta")] + [("seed", ctypes.c_uint64)]


class icm_fold_mc_args(ctypes.Structure):
    _fields_ = [("coef", ctypes.c_void_p), ("degree", ctypes.c_uint32), ("k", ctypes.c_uint32),
                ("mu", ctypes.c_double), ("sigma", ctypes.c_double), ("nf_lo", ctypes.c_double),
                ("nf_hi", ctypes.c_double), ("pf_lo", ctypes.c_double), ("pf_hi", ctypes.c_double),
                ("pos_lo", ctypes.c_double), ("pos_hi", ctypes.c_double), ("hist_lo", ctypes.c_double),
                ("hist_hi", ctypes.c_double), ("n_bins", ctypes.c_uint32), ("accumulate", ctypes.c_uint32),
                ("seed", ctypes.c_uint64), ("trial0", ctypes.c_uint64), ("n_trials", ctypes.c_uint64)]


_lib = None
_vp, _sz, _u32, _u64, _i32 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int

_SIGS = {
    "icm_status_str": (ctypes.c_char_p, [_i32]),
    "icm_last_error": (ctypes.c_char_p, []),
    "icm_ctx_create": (_i32, [ctypes.POINTER(icm_params), ctypes.POINTER(_vp)]),
    "icm_ctx_destroy": (None, [_vp]),
    "icm_ctx_primes": (_i32, [_vp, _vp, _sz]),
    "icm_ctx_crt_moduli": (_i32, [_vp, _vp, _sz, ctypes.POINTER(_sz)]),
    "icm_keygen": (_i32, [_vp]),
    "icm_db_bytes": (_i32, [_vp, _sz, ctypes.POINTER(_sz), ctypes.POINTER(_sz)]),
    "icm_db_encrypt": (_i32, [_vp, _vp, _vp, _sz, _u64, _vp, _sz, _vp, ctypes.POINTER(_vp)]),
    "icm_match_launches": (_i32, [_vp, _vp, _sz, ctypes.c_int, ctypes.POINTER(_sz)]),
    "icm_db_bytes_slots": (_i32, [_vp, _sz, ctypes.POINTER(_sz), ctypes.POINTER(_sz)]),
    "icm_db_encrypt_slots": (_i32, [_vp, _vp, _vp, _sz, _u32, _u64, _vp, _sz, _vp, ctypes.POINTER(_vp)]),
    "icm_normalize_bytes": (_i32, [_vp, ctypes.POINTER(_sz), ctypes.POINTER(_sz)]),
    "icm_normalize": (_i32, [_vp, _vp, _vp, _vp, _u32, _vp, _sz, _vp, _sz, _vp]),
    "icm_decrypt_slots": (_i32, [_vp, _vp, _vp, _sz, _u32, _vp, _sz, _vp]),
    "icm_db_destroy": (None, [_vp]),
    "icm_query_ct_bytes": (_i32, [_vp, _sz, ctypes.POINTER(_sz)]),
    "icm_query_encrypt": (_i32, [_vp, _vp, _vp, _vp, _sz, _vp, _sz, _vp]),
    "icm_query_op_bytes": (_i32, [_vp, _sz, _i32, ctypes.POINTER(_sz)]),
    "icm_query_prepare": (_i32, [_vp, _vp, _sz, _i32, _vp, _sz, _vp, ctypes.POINTER(_vp)]),
    "icm_query_destroy": (None, [_vp]),
    "icm_scores_bytes": (_i32, [_vp, _vp, _sz, _i32, ctypes.POINTER(_sz)]),
    "icm_match_workspace_bytes": (_i32, [_vp, _vp, _sz, _i32, ctypes.POINTER(_sz)]),
    "icm_match": (_i32, [_vp, _vp, _vp, _vp, _sz, _vp, _sz, _vp, ctypes.POINTER(_vp)]),
    "icm_fold": (_i32, [_vp, _vp, _vp, _sz, _vp, ctypes.POINTER(_vp)]),
    "icm_scores_destroy": (None, [_vp]),
    "icm_scores_shape": (_i32, [_vp, ctypes.POINTER(_sz), ctypes.POINTER(_sz), ctypes.POINTER(_sz)]),
    "icm_decrypt_scores": (_i32, [_vp, _vp, _vp, _sz, _vp]),
    "icm_decrypt_scores_max_error": (_i32, [_vp, _vp, _vp, _sz, _vp, _vp]),
    "icm_rescale_bytes": (_i32, [_vp, ctypes.POINTER(_sz)]),
    "icm_rescale": (_i32, [_vp, _vp, _vp, _sz, _vp, ctypes.POINTER(_vp)]),
    "icm_ppmm_workspace_bytes": (_i32, [_i32, _u32, _sz, _sz, _sz, ctypes.POINTER(_sz)]),
    "icm_ppmm": (_i32, [_i32, _vp, _u32, _vp, _vp, _vp, _sz, _sz, _sz, _vp, _sz, _vp]),
    "icm_sync": (_i32, [_vp, _u32]),
    "icm_ppmm_noalloc": (_i32, [_i32, _vp, _u32, _vp, _vp, _vp, _sz, _sz, _sz, _vp]),
    "icm_ctx_set_variant": (_i32, [_vp, _i32]),
    "icm_ctx_set_device_wait": (_i32, [_vp, ctypes.c_uint64, _i32]),
    "icm_device_status": (_i32, [_i32]),
    "icm_match_host_workspace_bytes": (_i32, [_vp, _vp, _sz, _i32, ctypes.POINTER(_sz)]),
    "icm_match_host": (_i32, [_vp, _vp, _vp, _sz, _i32, _vp, _vp, _sz, _vp]),
    "icm_probe_peak": (_i32, [_i32, ctypes.POINTER(ctypes.c_double), _vp]),
    "icm_match_batch_workspace_bytes": (_i32, [_vp, _vp, _sz, _sz, _i32, ctypes.POINTER(_sz)]),
    "icm_match_batch": (_i32, [_vp, _vp, _sz, _vp, _vp, _vp, _vp, _sz, _vp, _vp]),
    "icm_plan_create": (_i32, [_vp, _vp, _sz, _sz, _i32, _vp, _vp, _sz, _vp, _vp, _vp, _vp, _vp, _sz, _vp,
                               ctypes.POINTER(_vp)]),
    "icm_plan_launch": (_i32, [_vp, _vp]),
    "icm_plan_destroy": (None, [_vp]),
    "icm_server_device_bytes": (_i32, [_vp, _vp, _sz, _vp, ctypes.POINTER(_sz)]),
    "icm_server_create": (_i32, [_vp, _vp, _sz, _vp, _vp, _sz, ctypes.POINTER(_vp)]),
    "icm_server_eye_words": (_i32, [_vp, ctypes.POINTER(_sz), ctypes.POINTER(_sz)]),
    "icm_server_submit": (_i32, [_vp, _vp, _vp, ctypes.POINTER(_u64)]),
    "icm_server_wait": (_i32, [_vp, _u64, _u32, ctypes.POINTER(ctypes.c_double)]),
    "icm_server_stats": (_i32, [_vp, ctypes.POINTER(_u64), ctypes.POINTER(_u64), ctypes.POINTER(ctypes.c_double)]),
    "icm_server_destroy": (_i32, [_vp, _u32]),
    "icm_server_memory": (_i32, [_vp, ctypes.POINTER(_sz), ctypes.POINTER(_sz), ctypes.POINTER(_sz),
                                 ctypes.POINTER(_u32)]),
    "icm_fold_mc": (_i32, [ctypes.POINTER(icm_fold_mc_args), _vp, _vp, _vp, _vp]),
    "icm_fold_poly_range": (_i32, [_vp, _u32, ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_double)]),
    "icm_autotune": (_i32, [_vp, _vp, _sz, _vp, _vp, _vp, _vp, _sz, _vp, ctypes.POINTER(_i32),
                            ctypes.POINTER(ctypes.c_float), _sz]),
}


def lib() -> ctypes.CDLL:
    """Load libicm.so (built by paper_2601_17561_gb300.build); raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libicm.so not built at {LIB_PATH}: run paper_2601_17561_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status: int, where: str):
    if status != ICM_OK:
        detail = lib().icm_last_error().decode()
        raise IcmError(status, where, detail or lib().icm_status_str(status).decode())


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(stream)


def _ptr(x):
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return ctypes.c_void_p(x.data_ptr())
    if hasattr(x, "ctypes"):
        return x.ctypes.data_as(ctypes.c_void_p)
    return ctypes.c_void_p(x)


# ------------------------------------------------------------------ same-name wrappers

def icm_status_str(s: int) -> str:
    return lib().icm_status_str(s).decode()


def icm_ctx_create(p: icm_params):
    h = ctypes.c_void_p()
    _check(lib().icm_ctx_create(ctypes.byref(p), ctypes.byref(h)), "icm_ctx_create")
    return h


def icm_ctx_destroy(ctx):
    lib().icm_ctx_destroy(ctx)


def icm_ctx_primes(ctx, n: int = 8):
    arr = (ctypes.c_uint64 * n)()
    _check(lib().icm_ctx_primes(ctx, arr, n), "icm_ctx_primes")
    return list(arr)


def icm_ctx_crt_moduli(ctx):
    """The CRT forms' small moduli (list of ints)."""
    n = _sz()
    _check(lib().icm_ctx_crt_moduli(ctx, None, 0, ctypes.byref(n)), "icm_ctx_crt_moduli")
    arr = (ctypes.c_int32 * n.value)()
    _check(lib().icm_ctx_crt_moduli(ctx, arr, n.value, ctypes.byref(n)), "icm_ctx_crt_moduli")
    return list(arr)


def icm_keygen(ctx):
    _check(lib().icm_keygen(ctx), "icm_keygen")


def icm_db_bytes(ctx, n_db: int):
    b, m = ctypes.c_size_t(), ctypes.c_size_t()
    _check(lib().icm_db_bytes(ctx, n_db, ctypes.byref(b), ctypes.byref(m)), "icm_db_bytes")
    return b.value, m.value


def icm_db_encrypt(ctx, codes, masks, n_db, chunk_id, dev_buf, nbytes, stream=None):
    h = ctypes.c_void_p()
    _check(lib().icm_db_encrypt(ctx, _ptr(codes), _ptr(masks), n_db, chunk_id, _ptr(dev_buf), nbytes,
                                _stream(stream), ctypes.byref(h)), "icm_db_encrypt")
    return h


def icm_match_launches(ctx, db, n_eyes: int, form) -> int:
    n = _sz()
    _check(lib().icm_match_launches(ctx, db, n_eyes, form, ctypes.byref(n)), "icm_match_launches")
    return n.value


def icm_db_bytes_slots(ctx, n_db: int):
    b, m = ctypes.c_size_t(), ctypes.c_size_t()
    _check(lib().icm_db_bytes_slots(ctx, n_db, ctypes.byref(b), ctypes.byref(m)), "icm_db_bytes_slots")
    return b.value, m.value


def icm_db_encrypt_slots(ctx, codes, masks, n_db, log2_scale, chunk_id, dev_buf, nbytes, stream=None):
    h = ctypes.c_void_p()
    _check(lib().icm_db_encrypt_slots(ctx, _ptr(codes), _ptr(masks), n_db, log2_scale, chunk_id, _ptr(dev_buf),
                                      nbytes, _stream(stream), ctypes.byref(h)), "icm_db_encrypt_slots")
    return h


def icm_normalize_bytes(scores):
    a, b = ctypes.c_size_t(), ctypes.c_size_t()
    _check(lib().icm_normalize_bytes(scores, ctypes.byref(a), ctypes.byref(b)), "icm_normalize_bytes")
    return a.value, b.value


def icm_normalize(ctx, scores, dev_q_masks, dev_db_masks, log2_scale_mu, dev_out, nbytes, dev_ws, ws_bytes,
                  stream=None):
    _check(lib().icm_normalize(ctx, scores, _ptr(dev_q_masks), _ptr(dev_db_masks), log2_scale_mu, _ptr(dev_out),
                               nbytes, _ptr(dev_ws), ws_bytes, _stream(stream)), "icm_normalize")


def icm_decrypt_slots(ctx, scores, dev_norm, norm_bytes, log2_scale_mu, dev_hd, n, stream=None):
    _check(lib().icm_decrypt_slots(ctx, scores, _ptr(dev_norm), norm_bytes, log2_scale_mu, _ptr(dev_hd), n,
                                   _stream(stream)), "icm_decrypt_slots")


def icm_db_destroy(h):
    lib().icm_db_destroy(h)


def icm_query_ct_bytes(ctx, n_eyes):
    b = ctypes.c_size_t()
    _check(lib().icm_query_ct_bytes(ctx, n_eyes, ctypes.byref(b)), "icm_query_ct_bytes")
    return b.value


def icm_query_encrypt(ctx, codes, masks, eye_ids, n_eyes, dev_ct, nbytes, stream=None):
    _check(lib().icm_query_encrypt(ctx, _ptr(codes), _ptr(masks), _ptr(eye_ids), n_eyes, _ptr(dev_ct), nbytes,
                                   _stream(stream)), "icm_query_encrypt")


def icm_query_op_bytes(ctx, n_eyes, form):
    b = ctypes.c_size_t()
    _check(lib().icm_query_op_bytes(ctx, n_eyes, form, ctypes.byref(b)), "icm_query_op_bytes")
    return b.value


def icm_query_prepare(ctx, dev_ct, n_eyes, form, dev_op, nbytes, stream=None):
    h = ctypes.c_void_p()
    _check(lib().icm_query_prepare(ctx, _ptr(dev_ct), n_eyes, form, _ptr(dev_op), nbytes, _stream(stream),
                                   ctypes.byref(h)), "icm_query_prepare")
    return h


def icm_query_destroy(h):
    lib().icm_query_destroy(h)


def icm_scores_bytes(ctx, db, n_eyes, folded):
    b = ctypes.c_size_t()
    _check(lib().icm_scores_bytes(ctx, db, n_eyes, int(folded), ctypes.byref(b)), "icm_scores_bytes")
    return b.value


def icm_match_workspace_bytes(ctx, db, n_eyes, form):
    b = ctypes.c_size_t()
    _check(lib().icm_match_workspace_bytes(ctx, db, n_eyes, form, ctypes.byref(b)), "icm_match_workspace_bytes")
    return b.value


def icm_match(ctx, db, q, dev_out, nbytes, dev_ws=None, ws_bytes=0, stream=None):
    h = ctypes.c_void_p()
    _check(lib().icm_match(ctx, db, q, _ptr(dev_out), nbytes, _ptr(dev_ws), ws_bytes, _stream(stream), ctypes.byref(h)),
           "icm_match")
    return h


def icm_fold(ctx, scores, dev_out, nbytes, stream=None):
    h = ctypes.c_void_p()
    _check(lib().icm_fold(ctx, scores, _ptr(dev_out), nbytes, _stream(stream), ctypes.byref(h)), "icm_fold")
    return h


def icm_rescale_bytes(scores):
    n = _sz()
    _check(lib().icm_rescale_bytes(scores, ctypes.byref(n)), "icm_rescale_bytes")
    return n.value


def icm_rescale(ctx, scores, dev_out, nbytes, stream=None):
    h = _vp()
    _check(lib().icm_rescale(ctx, scores, _ptr(dev_out), nbytes, _stream(stream), ctypes.byref(h)), "icm_rescale")
    return h


def icm_scores_destroy(h):
    lib().icm_scores_destroy(h)


def icm_scores_shape(h):
    a, b, c = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_size_t()
    _check(lib().icm_scores_shape(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "icm_scores_shape")
    return a.value, b.value, c.value


def icm_decrypt_scores(ctx, scores, dev_num, n, stream=None):
    _check(lib().icm_decrypt_scores(ctx, scores, _ptr(dev_num), n, _stream(stream)), "icm_decrypt_scores")


def icm_decrypt_scores_max_error(ctx, scores, dev_num, n, dev_max_err, stream=None):
    _check(lib().icm_decrypt_scores_max_error(ctx, scores, _ptr(dev_num), n, _ptr(dev_max_err), _stream(stream)),
           "icm_decrypt_scores_max_error")


def icm_ppmm_workspace_bytes(form, n_limbs, M, N, K):
    b = ctypes.c_size_t()
    _check(lib().icm_ppmm_workspace_bytes(form, n_limbs, M, N, K, ctypes.byref(b)), "icm_ppmm_workspace_bytes")
    return b.value


def icm_ppmm(form, q, n_limbs, dev_A, dev_B, dev_C, M, N, K, dev_ws=None, ws_bytes=0, stream=None):
    qa = (ctypes.c_uint64 * n_limbs)(*[int(x) for x in q[:n_limbs]])
    _check(lib().icm_ppmm(form, qa, n_limbs, _ptr(dev_A), _ptr(dev_B), _ptr(dev_C), M, N, K, _ptr(dev_ws),
                          ws_bytes, _stream(stream)), "icm_ppmm")


def icm_match_host_workspace_bytes(ctx, db, n_eyes, form):
    b = ctypes.c_size_t()
    _check(lib().icm_match_host_workspace_bytes(ctx, db, n_eyes, form, ctypes.byref(b)), "icm_match_host_workspace_bytes")
    return b.value


def icm_match_host(ctx, db, host_ct, n_eyes, form, host_folded, dev_ws, ws_bytes, stream=None):
    _check(lib().icm_match_host(ctx, db, _ptr(host_ct), n_eyes, form, _ptr(host_folded), _ptr(dev_ws), ws_bytes,
                                _stream(stream)), "icm_match_host")


def icm_probe_peak(kind: int, stream=None) -> float:
    v = ctypes.c_double()
    _check(lib().icm_probe_peak(kind, ctypes.byref(v), _stream(stream)), "icm_probe_peak")
    return v.value


def _ptr_array(xs):
    return (ctypes.c_void_p * len(xs))(*[(_ptr(x).value if x is not None else None) for x in xs])


def _handle_array(hs):
    return (ctypes.c_void_p * len(hs))(*[h.value for h in hs])


def _size_array(ns):
    return (ctypes.c_size_t * len(ns))(*ns)


def icm_match_batch_workspace_bytes(ctx, dbs, n_eyes, form):
    b = ctypes.c_size_t()
    _check(lib().icm_match_batch_workspace_bytes(ctx, _handle_array(dbs), len(dbs), n_eyes, form, ctypes.byref(b)),
           "icm_match_batch_workspace_bytes")
    return b.value


def icm_match_batch(ctx, dbs, q, dev_outs, out_bytes, dev_ws, ws_bytes, stream=None):
    outs = (ctypes.c_void_p * len(dbs))()
    _check(lib().icm_match_batch(ctx, _handle_array(dbs), len(dbs), q, _ptr_array(dev_outs), _size_array(out_bytes),
                                 _ptr(dev_ws), ws_bytes, _stream(stream), outs), "icm_match_batch")
    return [ctypes.c_void_p(h) for h in outs]


def icm_plan_create(ctx, dbs, n_eyes, form, dev_ct, dev_op, op_bytes, dev_scores, scores_bytes, dev_folded,
                    folded_bytes, dev_ws, ws_bytes, stream):
    h = ctypes.c_void_p()
    _check(lib().icm_plan_create(ctx, _handle_array(dbs), len(dbs), n_eyes, form, _ptr(dev_ct), _ptr(dev_op), op_bytes,
                                 _ptr_array(dev_scores), _size_array(scores_bytes), _ptr_array(dev_folded),
                                 _size_array(folded_bytes), _ptr(dev_ws), ws_bytes, _stream(stream), ctypes.byref(h)),
           "icm_plan_create")
    return h


def icm_plan_launch(plan, stream=None):
    _check(lib().icm_plan_launch(plan, _stream(stream)), "icm_plan_launch")


def icm_plan_destroy(plan):
    lib().icm_plan_destroy(plan)


def icm_autotune(ctx, dbs, q, dev_outs, out_bytes, dev_ws, ws_bytes, stream=None):
    best = ctypes.c_int()
    ms = (ctypes.c_float * len(VARIANTS))()
    _check(lib().icm_autotune(ctx, _handle_array(dbs), len(dbs), q, _ptr_array(dev_outs), _size_array(out_bytes),
                              _ptr(dev_ws), ws_bytes, _stream(stream), ctypes.byref(best), ms, len(VARIANTS)),
           "icm_autotune")
    return best.value, list(ms)


# CRT product kernel variants in the autotuner's order (icm_autotune's ms_per_choice)
VARIANTS = {128: "mma.sync-128", 256: "mma.sync-256", 1: "tcgen05-r8s4", 2: "tcgen05-r8s4-wave", 3: "tcgen05-r4s8"}


def icm_ctx_set_variant(ctx, variant: int):
    _check(lib().icm_ctx_set_variant(ctx, variant), "icm_ctx_set_variant")


def icm_ctx_set_device_wait(ctx, wait_ns: int = 0, inject_stall: bool = False):
    _check(lib().icm_ctx_set_device_wait(ctx, wait_ns, 1 if inject_stall else 0), "icm_ctx_set_device_wait")


def icm_device_status(clear: bool = True):
    _check(lib().icm_device_status(1 if clear else 0), "icm_device_status")


def icm_server_device_bytes(ctx, dbs, cfg):
    b = ctypes.c_size_t()
    _check(lib().icm_server_device_bytes(ctx, _handle_array(dbs), len(dbs), ctypes.byref(cfg), ctypes.byref(b)),
           "icm_server_device_bytes")
    return b.value


def icm_server_create(ctx, dbs, cfg, dev_ws, ws_bytes):
    h = ctypes.c_void_p()
    _check(lib().icm_server_create(ctx, _handle_array(dbs), len(dbs), ctypes.byref(cfg), _ptr(dev_ws), ws_bytes,
                                   ctypes.byref(h)), "icm_server_create")
    return h


def icm_server_eye_words(srv):
    a, b = ctypes.c_size_t(), ctypes.c_size_t()
    _check(lib().icm_server_eye_words(srv, ctypes.byref(a), ctypes.byref(b)), "icm_server_eye_words")
    return a.value, b.value


def icm_server_submit(srv, host_ct, host_out):
    t = ctypes.c_uint64()
    _check(lib().icm_server_submit(srv, _ptr(host_ct), _ptr(host_out), ctypes.byref(t)), "icm_server_submit")
    return t.value


def icm_server_wait(srv, ticket, timeout_ms=600000):
    lat = ctypes.c_double()
    _check(lib().icm_server_wait(srv, ticket, timeout_ms, ctypes.byref(lat)), "icm_server_wait")
    return lat.value


def icm_server_stats(srv):
    a, b, m = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_double()
    _check(lib().icm_server_stats(srv, ctypes.byref(a), ctypes.byref(b), ctypes.byref(m)), "icm_server_stats")
    return a.value, b.value, m.value


def icm_server_memory(srv):
    """(pool bytes, bytes of one full batch, peak reserved bytes, peak batches in flight)"""
    a, b, c, d = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_uint32()
    _check(lib().icm_server_memory(srv, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d)),
           "icm_server_memory")
    return a.value, b.value, c.value, d.value


def icm_server_destroy(srv, timeout_ms=600000):
    _check(lib().icm_server_destroy(srv, timeout_ms), "icm_server_destroy")


def icm_ppmm_noalloc(form, q, n_limbs, dev_A, dev_B, dev_C, M, N, K, stream=None):
    qa = (ctypes.c_uint64 * n_limbs)(*[int(x) for x in q[:n_limbs]])
    _check(lib().icm_ppmm_noalloc(form, qa, n_limbs, _ptr(dev_A), _ptr(dev_B), _ptr(dev_C), M, N, K, _stream(stream)),
           "icm_ppmm_noalloc")


def icm_sync(stream=None, timeout_ms: int = 600000):
    _check(lib().icm_sync(_stream(stream), timeout_ms), "icm_sync")


def icm_fold_mc(args: icm_fold_mc_args, dev_counts, dev_hist=None, dev_sums=None, stream=None):
    _check(lib().icm_fold_mc(ctypes.byref(args), _ptr(dev_counts), _ptr(dev_hist), _ptr(dev_sums), _stream(stream)),
           "icm_fold_mc")


def icm_fold_poly_range(coef, lo: float, hi: float):
    c = (ctypes.c_double * len(coef))(*coef)
    mn, mx = ctypes.c_double(), ctypes.c_double()
    _check(lib().icm_fold_poly_range(c, len(coef) - 1, lo, hi, ctypes.byref(mn), ctypes.byref(mx)),
           "icm_fold_poly_range")
    return mn.value, mx.value
