"""ctypes binding of libsemiring.so (include/semiring.h), argument marshalling only.

Every function has the C name and argument order.  Pointer arguments accept
an int (a device address) or any object with ``data_ptr()`` (a torch tensor);
``stream`` accepts None (torch's current stream), an int handle, or an object
with ``cuda_stream``.  A non-OK status raises SemiringError carrying the
library's message.  No computation happens here: a missing library raises at
import, and there is no fallback.
"""

from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libsemiring.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build it with `python -c \"import __graft_entry__ as g; g.build()\"` "
        "(paper_1705_08743_gb300.build.build()); there is no fallback implementation")

lib = ctypes.CDLL(LIB_PATH)

# status codes / enums (include/semiring.h)
SR_OK, SR_EINVAL, SR_ENOMEM, SR_ECUDA, SR_ETIMEOUT, SR_EAGAIN, SR_EBUSY, SR_ENOTFOUND, SR_ECANCELED = range(9)
SR_BOOL_W32, SR_BOOL_W64, SR_U8, SR_U16, SR_U32 = range(5)
SR_CLOSURE_WARSHALL, SR_CLOSURE_SQUARING = 0, 1
SR_OP_ANTIDIST_MUL, SR_OP_BOOL_MUL, SR_OP_ANTIDIST_CLOSURE, SR_OP_BOOL_CLOSURE = range(4)
SR_PEAK_DPX_S16X2, SR_PEAK_U16_PAIR, SR_PEAK_LOP3, SR_PEAK_IADD, SR_PEAK_U32_PAIR, SR_PEAK_TC_F8 = range(6)
SR_OPT_BOOL_TENSOR = 1
SR_OPT_BOOL_FOUR_RUSSIANS = 2
SR_OPT_SPIN_LIMIT = 3
SR_OPT_CLOSURE_BLOCK = 4
SR_OPT_CLOSURE_PERSISTENT = 5
SR_OPT_CLOSURE_PANEL_SHARE = 6
SR_OPT_BOOL_SIDE_SMS = 7
SR_OPT_PRODUCT_SPLIT = 8
SR_OPT_CLOSURE_FUSED = 9
SR_TUNE_BOOL_WORDS, SR_TUNE_BOOL_TABLES, SR_TUNE_BOOL_TENSOR, SR_TUNE_PERSISTENT, SR_TUNE_FUSED = 0, 1, 2, 1, 2
SR_OP_DIST_MUL = 4
SR_EW_AND, SR_EW_OR, SR_EW_XOR, SR_EW_NOT = range(4)

STATUS_NAMES = {0: "SR_OK", 1: "SR_EINVAL", 2: "SR_ENOMEM", 3: "SR_ECUDA", 4: "SR_ETIMEOUT",
                5: "SR_EAGAIN", 6: "SR_EBUSY", 7: "SR_ENOTFOUND", 8: "SR_ECANCELED"}


class SemiringError(RuntimeError):
    def __init__(self, status: int, fn: str, msg: str):
        super().__init__(f"{fn}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class sr_config(ctypes.Structure):
    _fields_ = [("workspace_bytes", ctypes.c_size_t), ("spin_limit", ctypes.c_int),
                ("tune_cache", ctypes.c_char_p), ("reserved", ctypes.c_int * 4)]


_vp, _i64, _int, _st = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int


class sr_desc(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int), ("dtype", ctypes.c_int), ("A", ctypes.c_void_p), ("B", ctypes.c_void_p),
                ("C", ctypes.c_void_p), ("lda", ctypes.c_int64), ("ldb", ctypes.c_int64), ("ldc", ctypes.c_int64),
                ("R", ctypes.c_int64), ("K", ctypes.c_int64), ("N", ctypes.c_int64), ("accumulate", ctypes.c_int),
                ("method", ctypes.c_int)]

class sr_request(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int), ("dtype", ctypes.c_int), ("R", ctypes.c_int64), ("K", ctypes.c_int64),
                ("N", ctypes.c_int64), ("A", ctypes.c_void_p), ("B", ctypes.c_void_p), ("rA", ctypes.c_uint64),
                ("rB", ctypes.c_uint64), ("out", ctypes.c_void_p), ("keep", ctypes.c_int), ("method", ctypes.c_int)]


class sr_serve_config(ctypes.Structure):
    _fields_ = [("arena_bytes", ctypes.c_size_t), ("slots", ctypes.c_int), ("max_pending", ctypes.c_int),
                ("batch_max_d", ctypes.c_int), ("batch_max_graphs", ctypes.c_int), ("backfill_ms", ctypes.c_int)]


class sr_result_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("latency_ms", ctypes.c_double), ("queue_ms", ctypes.c_double),
                ("resident", ctypes.c_uint64)]


class sr_serve_stats_t(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("failed", ctypes.c_uint64),
                ("batches", ctypes.c_uint64), ("batched_requests", ctypes.c_uint64), ("cancelled", ctypes.c_uint64),
                ("arena_bytes", ctypes.c_size_t), ("arena_in_use", ctypes.c_size_t),
                ("arena_peak_bytes", ctypes.c_size_t), ("pending", ctypes.c_int), ("inflight", ctypes.c_int),
                ("residents", ctypes.c_int)]


_SIGS = {
    "sr_create": (_st, [ctypes.POINTER(_vp), ctypes.POINTER(sr_config)]),
    "sr_destroy": (None, [_vp]),
    "sr_last_error": (ctypes.c_char_p, []),
    "sr_version": (ctypes.c_char_p, []),
    "sr_workspace_query": (_st, [_int, _int, _i64, _int, ctypes.POINTER(ctypes.c_size_t)]),
    "sr_stream_status": (_st, [_vp, _vp]),
    "sr_kernel_launches": (ctypes.c_uint64, []),
    "sr_set_option": (_st, [_vp, _int, _int]),
    "sr_peak_probe": (_st, [_int, _int, _int, _vp, ctypes.POINTER(ctypes.c_double),
                            ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "antidist_encode": (_st, [_vp, _vp, _i64, _vp, _i64, _i64, _i64, _int, _vp]),
    "bool_pack": (_st, [_vp, _vp, _i64, _vp, _i64, _i64, _i64, _int, _vp]),
    "bool_unpack": (_st, [_vp, _vp, _i64, _vp, _i64, _i64, _i64, _int, _vp]),
    "antidist_mul": (_st, [_vp, _vp, _i64, _vp, _i64, _vp, _i64, _i64, _i64, _i64, _int, _int, _vp]),
    "bool_mul": (_st, [_vp, _vp, _i64, _vp, _i64, _vp, _i64, _i64, _i64, _i64, _int, _int, _vp]),
    "antidist_closure": (_st, [_vp, _vp, _i64, _i64, _int, _vp]),
    "bool_closure": (_st, [_vp, _vp, _i64, _i64, _int, _int, _vp]),
    "bool_closure_squaring_noalloc": (_st, [_vp, _i64, _i64, _int, _vp]),
    "sr_closure_order": (ctypes.c_longlong, [_i64, _int, _vp, ctypes.c_longlong]),
    "sr_shard_rows": (_st, [_i64, _int, _int, _i64, ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
    "sr_host_mapped": (_st, [_vp, ctypes.POINTER(_int)]),
    "sr_autotune_closure": (_st, [_vp, _int, _i64, _vp, _int, _int, ctypes.POINTER(_int),
                                  ctypes.POINTER(ctypes.c_double)]),
    "sr_autotune_mul": (_st, [_vp, _int, _int, _i64, _vp, _int, _int, ctypes.POINTER(_int),
                              ctypes.POINTER(ctypes.c_double)]),
    "sr_tune_get": (_st, [_vp, _int, _int, _i64, ctypes.POINTER(_int), ctypes.POINTER(ctypes.c_double)]),
    "sr_tune_set": (_st, [_vp, _int, _int, _i64, _int]),
    "sr_tune_save": (_st, [_vp, ctypes.c_char_p]),
    "sr_tune_load": (_st, [_vp, ctypes.c_char_p]),
    "sr_batch_create": (_st, [_vp, ctypes.POINTER(sr_desc), _int, ctypes.POINTER(_vp)]),
    "sr_batch_launch": (_st, [_vp, _int, _vp]),
    "sr_batch_set_tuning": (_st, [_vp, _int, _int, _int]),
    "sr_batch_get_tuning": (_st, [_vp, ctypes.POINTER(_int), ctypes.POINTER(_int), ctypes.POINTER(_int)]),
    "sr_batch_autotune": (_st, [_vp, _vp, _vp, _int, ctypes.POINTER(ctypes.c_double)]),
    "sr_batch_info": (_st, [_vp, ctypes.POINTER(_int), ctypes.POINTER(_int), ctypes.POINTER(ctypes.c_double)]),
    "sr_batch_set_timing": (_st, [_vp, _int]),
    "sr_batch_completion_ms": (_st, [_vp, ctypes.POINTER(ctypes.c_double)]),
    "sr_batch_destroy": (None, [_vp]),
    "sr_batched": (_st, [_vp, ctypes.POINTER(sr_desc), _int, _vp]),
    "dist_mul": (_st, [_vp, _vp, _i64, _vp, _i64, _vp, _i64, _i64, _i64, _i64, _int, _int, _vp]),
    "dist_closure": (_st, [_vp, _vp, _i64, _i64, _int, _vp]),
    "sr_entrywise": (_st, [_vp, _int, _vp, _i64, _vp, _i64, _vp, _i64, _i64, _i64, _int, _vp]),
    "sr_reflexive": (_st, [_vp, _vp, _i64, _i64, _int, _vp]),
    "sr_serve_start": (_st, [_vp, ctypes.POINTER(sr_serve_config)]),
    "sr_serve_stop": (_st, [_vp]),
    "sr_submit": (_st, [_vp, ctypes.POINTER(sr_request), ctypes.POINTER(ctypes.c_uint64)]),
    "sr_poll": (_st, [_vp, ctypes.c_uint64, ctypes.POINTER(_int)]),
    "sr_wait": (_st, [_vp, ctypes.c_uint64, _int]),
    "sr_result": (_st, [_vp, ctypes.c_uint64, ctypes.POINTER(sr_result_info)]),
    "sr_release": (_st, [_vp, ctypes.c_uint64]),
    "sr_cancel": (_st, [_vp, ctypes.c_uint64]),
    "sr_resident_put": (_st, [_vp, _vp, _i64, _i64, _int, ctypes.POINTER(ctypes.c_uint64)]),
    "sr_resident_get": (_st, [_vp, ctypes.c_uint64, _vp]),
    "sr_resident_free": (_st, [_vp, ctypes.c_uint64]),
    "sr_serve_stats": (_st, [_vp, ctypes.POINTER(sr_serve_stats_t)]),
}

for _name, (_res, _args) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def exported_symbols():
    return list(_SIGS)


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "value"):
        return x.value
    raise TypeError(f"cannot take a device pointer from {type(x)}")


def _stream(s):
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(st: int, fn: str):
    if st != SR_OK:
        raise SemiringError(st, fn, last_error())


def last_error() -> str:
    return (lib.sr_last_error() or b"").decode()


def version() -> str:
    return lib.sr_version().decode()


def sr_create(workspace_bytes: int = 0, spin_limit: int = 0, tune_cache: str | None = None):
    cfg = sr_config(workspace_bytes=workspace_bytes, spin_limit=spin_limit,
                    tune_cache=tune_cache.encode() if tune_cache else None)
    h = _vp()
    _check(lib.sr_create(ctypes.byref(h), ctypes.byref(cfg)), "sr_create")
    return h.value


def sr_destroy(ctx):
    lib.sr_destroy(ctx)


def sr_workspace_query(op: int, dtype: int, D: int, method: int = 0) -> int:
    n = ctypes.c_size_t()
    _check(lib.sr_workspace_query(op, dtype, D, method, ctypes.byref(n)), "sr_workspace_query")
    return n.value


def sr_closure_order(D: int, share: int = 128):
    """The persistent closure's work order: a list of (type, pivot block, tile row, tile
    column, second tile column or -1); type 0 phase-3 tiles, 1 row-panel tile, 2
    column-panel tile, 3 diagonal block."""
    n = lib.sr_closure_order(D, share, None, 0)
    if n < 0:
        raise SemiringError(SR_EINVAL, "sr_closure_order", f"D = {D} is outside the persistent schedule's range")
    buf = (ctypes.c_int * (5 * n))()
    lib.sr_closure_order(D, share, ctypes.cast(buf, _vp), n)
    return [tuple(buf[5 * q:5 * q + 5]) for q in range(n)]


def sr_autotune_closure(ctx, dtype: int, D: int, stream=None, reps: int = 2, force: bool = False):
    """-> (choice, ms): block width 128/256/512, SR_TUNE_PERSISTENT or SR_TUNE_FUSED, and its time."""
    ch, ms = _int(), ctypes.c_double()
    _check(lib.sr_autotune_closure(ctx, dtype, D, _stream(stream), reps, 1 if force else 0, ctypes.byref(ch),
                                   ctypes.byref(ms)), "sr_autotune_closure")
    return ch.value, ms.value


def sr_autotune_mul(ctx, op: int, dtype: int, D: int, stream=None, reps: int = 2, force: bool = False):
    ch, ms = _int(), ctypes.c_double()
    _check(lib.sr_autotune_mul(ctx, op, dtype, D, _stream(stream), reps, 1 if force else 0, ctypes.byref(ch),
                               ctypes.byref(ms)), "sr_autotune_mul")
    return ch.value, ms.value


def sr_tune_get(ctx, op: int, dtype: int, D: int):
    """-> (choice, ms), or None if nothing is recorded for that bucket."""
    ch, ms = _int(), ctypes.c_double()
    st = lib.sr_tune_get(ctx, op, dtype, D, ctypes.byref(ch), ctypes.byref(ms))
    if st == SR_ENOTFOUND:
        return None
    _check(st, "sr_tune_get")
    return ch.value, ms.value


def sr_tune_set(ctx, op: int, dtype: int, D: int, choice: int):
    _check(lib.sr_tune_set(ctx, op, dtype, D, choice), "sr_tune_set")


def sr_tune_save(ctx, path: str):
    _check(lib.sr_tune_save(ctx, path.encode()), "sr_tune_save")


def sr_tune_load(ctx, path: str):
    _check(lib.sr_tune_load(ctx, path.encode()), "sr_tune_load")


def sr_host_mapped(p) -> bool:
    """Whether p (a pointer, or a tensor's data_ptr()) is pinned host memory the current
    device addresses at the same pointer."""
    m = _int()
    ptr = p.data_ptr() if hasattr(p, "data_ptr") else p
    _check(lib.sr_host_mapped(ptr, ctypes.byref(m)), "sr_host_mapped")
    return bool(m.value)


def sr_shard_rows(R: int, world: int, rank: int, align: int = 128):
    """-> (r0, r1): this rank's rows of a row-sharded product."""
    r0, r1 = _i64(), _i64()
    _check(lib.sr_shard_rows(R, world, rank, align, ctypes.byref(r0), ctypes.byref(r1)), "sr_shard_rows")
    return r0.value, r1.value


def sr_stream_status(ctx, stream=None):
    _check(lib.sr_stream_status(ctx, _stream(stream)), "sr_stream_status")


def sr_set_option(ctx, option: int, value: int):
    _check(lib.sr_set_option(ctx, option, value), "sr_set_option")


def sr_kernel_launches() -> int:
    return int(lib.sr_kernel_launches())


def sr_peak_probe(op: int, iters: int = 4096, blocks_per_sm: int = 8, stream=None):
    """-> (ms, instructions/s, semiring ops/s) of one inner operation on all SMs."""
    ms, ips, ops = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib.sr_peak_probe(op, iters, blocks_per_sm, _stream(stream), ctypes.byref(ms), ctypes.byref(ips),
                             ctypes.byref(ops)), "sr_peak_probe")
    return ms.value, ips.value, ops.value


def antidist_encode(ctx, W, ldw, T, ldt, R, C, dtype, stream=None):
    _check(lib.antidist_encode(ctx, _ptr(W), ldw, _ptr(T), ldt, R, C, dtype, _stream(stream)), "antidist_encode")


def bool_pack(ctx, dense, ldd, M, ldm, R, C, dtype, stream=None):
    _check(lib.bool_pack(ctx, _ptr(dense), ldd, _ptr(M), ldm, R, C, dtype, _stream(stream)), "bool_pack")


def bool_unpack(ctx, M, ldm, dense, ldd, R, C, dtype, stream=None):
    _check(lib.bool_unpack(ctx, _ptr(M), ldm, _ptr(dense), ldd, R, C, dtype, _stream(stream)), "bool_unpack")


def antidist_mul(ctx, A, lda, B, ldb, C, ldc, R, K, N, dtype, accumulate=0, stream=None):
    _check(lib.antidist_mul(ctx, _ptr(A), lda, _ptr(B), ldb, _ptr(C), ldc, R, K, N, dtype, int(accumulate),
                            _stream(stream)), "antidist_mul")


def bool_mul(ctx, A, lda, B, ldb, C, ldc, R, K, N, dtype, accumulate=0, stream=None):
    _check(lib.bool_mul(ctx, _ptr(A), lda, _ptr(B), ldb, _ptr(C), ldc, R, K, N, dtype, int(accumulate),
                        _stream(stream)), "bool_mul")


def antidist_closure(ctx, T, ldt, D, dtype, stream=None):
    _check(lib.antidist_closure(ctx, _ptr(T), ldt, D, dtype, _stream(stream)), "antidist_closure")


def bool_closure(ctx, T, ldt, D, dtype, method=SR_CLOSURE_WARSHALL, stream=None):
    _check(lib.bool_closure(ctx, _ptr(T), ldt, D, dtype, method, _stream(stream)), "bool_closure")


NOALLOC_SCRATCH_BYTES = 16 << 20


def bool_closure_squaring_noalloc(T, ldt, D, dtype, stream=None):
    """Allocation-free Boolean closure by squaring (library-owned 16 MiB scratch)."""
    _check(lib.bool_closure_squaring_noalloc(_ptr(T), ldt, D, dtype, _stream(stream)),
           "bool_closure_squaring_noalloc")


def closure_desc(T, ldt, D, dtype):
    """sr_desc of an in-place anti-distance closure."""
    return sr_desc(op=SR_OP_ANTIDIST_CLOSURE, dtype=dtype, A=None, B=None, C=_ptr(T), lda=0, ldb=0, ldc=ldt,
                   R=D, K=D, N=D, accumulate=0, method=0)


def _desc_array(descs):
    arr = (sr_desc * len(descs))(*descs)
    return arr


def sr_batch_create(ctx, descs):
    arr = _desc_array(descs)
    h = _vp()
    _check(lib.sr_batch_create(ctx, arr, len(descs), ctypes.byref(h)), "sr_batch_create")
    return h.value


def sr_batch_launch(batch, use_graph=0, stream=None):
    _check(lib.sr_batch_launch(batch, int(use_graph), _stream(stream)), "sr_batch_launch")


def sr_batch_set_tuning(batch, cluster, coop_threshold, ctas_per_sm):
    _check(lib.sr_batch_set_tuning(batch, cluster, coop_threshold, ctas_per_sm), "sr_batch_set_tuning")


def sr_batch_get_tuning(batch):
    a, b, c = _int(), _int(), _int()
    _check(lib.sr_batch_get_tuning(batch, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "sr_batch_get_tuning")
    return a.value, b.value, c.value


def sr_batch_autotune(ctx, batch, stream=None, reps=2):
    ms = ctypes.c_double()
    _check(lib.sr_batch_autotune(ctx, batch, _stream(stream), reps, ctypes.byref(ms)), "sr_batch_autotune")
    return ms.value


def sr_batch_info(batch):
    n, it, ops = _int(), _int(), ctypes.c_double()
    _check(lib.sr_batch_info(batch, ctypes.byref(n), ctypes.byref(it), ctypes.byref(ops)), "sr_batch_info")
    return n.value, it.value, ops.value


def sr_batch_set_timing(batch, enable: bool = True):
    _check(lib.sr_batch_set_timing(batch, 1 if enable else 0), "sr_batch_set_timing")


def sr_batch_completion_ms(batch):
    """Per-graph completion times (ms since the last timed launch's start), descriptor order."""
    n, _, _ = sr_batch_info(batch)
    out = (ctypes.c_double * n)()
    _check(lib.sr_batch_completion_ms(batch, out), "sr_batch_completion_ms")
    return list(out)


def sr_batch_destroy(batch):
    lib.sr_batch_destroy(batch)


def sr_batched(ctx, descs, stream=None):
    arr = _desc_array(descs)
    _check(lib.sr_batched(ctx, arr, len(descs), _stream(stream)), "sr_batched")


def _hptr(x):
    """Host pointer of a numpy array or a (pinned) CPU torch tensor."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return x.ctypes.data


def sr_serve_start(ctx, arena_bytes=1 << 30, slots=4, max_pending=4096, batch_max_d=512, batch_max_graphs=64,
                   backfill_ms=0):
    cfg = sr_serve_config(arena_bytes=arena_bytes, slots=slots, max_pending=max_pending, batch_max_d=batch_max_d,
                          batch_max_graphs=batch_max_graphs, backfill_ms=backfill_ms)
    _check(lib.sr_serve_start(ctx, ctypes.byref(cfg)), "sr_serve_start")


def sr_serve_stop(ctx):
    _check(lib.sr_serve_stop(ctx), "sr_serve_stop")


def make_request(op, dtype, R, K=0, N=0, A=None, B=None, rA=0, rB=0, out=None, keep=0, method=0):
    return sr_request(op=op, dtype=dtype, R=R, K=K or R, N=N or R, A=_hptr(A), B=_hptr(B), rA=rA, rB=rB,
                      out=_hptr(out), keep=keep, method=method)


def sr_submit(ctx, req):
    t = ctypes.c_uint64()
    _check(lib.sr_submit(ctx, ctypes.byref(req), ctypes.byref(t)), "sr_submit")
    return t.value


def sr_poll(ctx, ticket):
    d = _int()
    _check(lib.sr_poll(ctx, ticket, ctypes.byref(d)), "sr_poll")
    return bool(d.value)


def sr_wait(ctx, ticket, timeout_ms=60000):
    _check(lib.sr_wait(ctx, ticket, timeout_ms), "sr_wait")


def sr_result(ctx, ticket):
    info = sr_result_info()
    _check(lib.sr_result(ctx, ticket, ctypes.byref(info)), "sr_result")
    return info


def sr_release(ctx, ticket):
    _check(lib.sr_release(ctx, ticket), "sr_release")


def sr_cancel(ctx, ticket):
    _check(lib.sr_cancel(ctx, ticket), "sr_cancel")


def sr_resident_put(ctx, host, rows, cols, dtype):
    h = ctypes.c_uint64()
    _check(lib.sr_resident_put(ctx, _hptr(host), rows, cols, dtype, ctypes.byref(h)), "sr_resident_put")
    return h.value


def sr_resident_get(ctx, handle, host):
    _check(lib.sr_resident_get(ctx, handle, _hptr(host)), "sr_resident_get")


def sr_resident_free(ctx, handle):
    _check(lib.sr_resident_free(ctx, handle), "sr_resident_free")


def sr_serve_stats(ctx):
    st = sr_serve_stats_t()
    _check(lib.sr_serve_stats(ctx, ctypes.byref(st)), "sr_serve_stats")
    return {f: getattr(st, f) for f, _ in sr_serve_stats_t._fields_}


def dist_mul(ctx, A, lda, B, ldb, C, ldc, R, K, N, dtype, accumulate=0, stream=None):
    _check(lib.dist_mul(ctx, _ptr(A), lda, _ptr(B), ldb, _ptr(C), ldc, R, K, N, dtype, int(accumulate),
                        _stream(stream)), "dist_mul")


def dist_closure(ctx, T, ldt, D, dtype, stream=None):
    _check(lib.dist_closure(ctx, _ptr(T), ldt, D, dtype, _stream(stream)), "dist_closure")


def sr_entrywise(ctx, op, A, lda, B, ldb, C, ldc, R, N, dtype, stream=None):
    _check(lib.sr_entrywise(ctx, op, _ptr(A), lda, _ptr(B), ldb, _ptr(C), ldc, R, N, dtype, _stream(stream)),
           "sr_entrywise")


def sr_reflexive(ctx, T, ldt, D, dtype, stream=None):
    _check(lib.sr_reflexive(ctx, _ptr(T), ldt, D, dtype, _stream(stream)), "sr_reflexive")
