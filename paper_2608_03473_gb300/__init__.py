"""GB300-native certified-split lexer -- Python binding of ``include/lexgpu.h``.

Argument marshalling only: every step of the lexing path runs in
``liblexgpu.so`` (CUDA kernels for sm_103a).  PyTorch supplies device memory
and streams.  The functions keep the C names:

    ts  = lx_compile_tokenset(dfa, discarded)        # host-only analysis
    ex, mo = lx_certificates(ts)                       # 256-bit masks as bytes
    ctx = lx_ctx_create()
    rc, n_tokens, consumed = lx_lex(ctx, ts, d_in, mode, d_kinds, d_lens)

and the other entry points: ``lx_lex_host`` (host buffers), ``lx_lex_batch``
(many documents, one graph launch; ``BatchDocs`` prebuilds its arrays),
``lx_lex_noalloc`` (no allocation), ``lx_lex_enumerative`` and
``lx_lex_speculative`` (token sets that certify no byte; ``Model`` and
``train_context_model`` for the entry-context predictor),
``lx_ctx_set_config`` / ``lx_autotune`` (launch configuration).

``dfa`` is any object with ``n_states, q0, n_kinds`` and numpy arrays
``byte_class[256]``, ``next[n_classes, n_states]`` (-1 = undefined) and
``accept[n_states]`` (-1 = not accepting).

If the shared library is missing the import still succeeds, but every call
raises ``RuntimeError``: there is no CPU fallback.
"""

from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblexgpu.so")

LX_OK = 0
LX_E_INVAL = -1
LX_E_NOMEM = -2
LX_E_CAPACITY = -3
LX_E_CUDA = -4
LX_E_TIMEOUT = -5
LX_E_MODE = -6
LX_E_TOOBIG = -7
LX_NONE = 0xFFFFFFFF
LX_NO_KIND = 0xFFFF

LX_FULL_EXACT = 0
LX_FILTERED_EXACT = 1
LX_FILTERED_MODULO = 2

# every function declared in include/lexgpu.h
EXPORTED = (
    "lx_compile_tokenset", "lx_compile_tokenset_framed", "lx_certificates", "lx_tokenset_info", "lx_tokenset_table", "lx_tokenset_class_table",
    "lx_tokenset_walk_table", "lx_window_certificates", "lx_tokenset_scan_table", "lx_tokenset_liveness",
    "lx_liveness",
    "lx_tokenset_free",
    "lx_ctx_create", "lx_ctx_free", "lx_ctx_set_timeout_ms", "lx_ctx_enable_timing", "lx_ctx_last_kernel_ms",
    "lx_ctx_set_config", "lx_ctx_get_config", "lx_autotune", "lx_ctx_debug_withhold", "lx_ctx_set_kernel",
    "lx_ctx_set_warps", "lx_ctx_set_warp_geometry", "lx_lex_async",
    "lx_lex", "lx_lex_host", "lx_lex_noalloc", "lx_lex_batch", "lx_lex_enumerative", "lx_chunk_contexts",
    "lx_lex_speculative", "lx_model_create", "lx_model_free", "lx_model_info", "lx_model_get_params",
    "lx_model_set_params", "lx_model_windows", "lx_model_forward", "lx_model_gradient", "lx_model_train_step",
    "lx_strerror",
)


class LexError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {lx_strerror(code)} ({code})" if what else f"{lx_strerror(code)} ({code})")


class _Dfa(ctypes.Structure):
    _fields_ = [
        ("n_states", ctypes.c_uint32), ("n_classes", ctypes.c_uint32), ("q0", ctypes.c_uint32),
        ("n_kinds", ctypes.c_uint32), ("byte_class", ctypes.c_void_p), ("next", ctypes.c_void_p),
        ("accept_kind", ctypes.c_void_p),
    ]


class _Doc(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("n", ctypes.c_uint64), ("set", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]


class _DocResult(ctypes.Structure):
    _fields_ = [("out_off", ctypes.c_uint64), ("n_tokens", ctypes.c_uint64), ("consumed", ctypes.c_uint64)]


_lib = None
_lock = threading.Lock()


def load_library(path: Optional[str] = None):
    """Load liblexgpu.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"{p} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(p)
        vp, u32, u64, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
        sig = {
            "lx_compile_tokenset": (i32, [vp, vp, u32, vp]),
            "lx_compile_tokenset_framed": (i32, [vp, vp, u32, u32, i32, vp]),
            "lx_certificates": (i32, [vp, vp, vp]),
            "lx_tokenset_info": (i32, [vp, i32, vp, vp, vp, vp, vp]),
            "lx_tokenset_table": (i32, [vp, i32, vp, u32, vp, u32]),
            "lx_tokenset_class_table": (i32, [vp, i32, vp, u32, vp, u32]),
            "lx_tokenset_walk_table": (i32, [vp, i32, vp, u32, vp, u32]),
            "lx_window_certificates": (i32, [vp, vp]),
            "lx_tokenset_scan_table": (i32, [vp, vp, u32, vp, u32]),
            "lx_tokenset_liveness": (i32, [vp, vp, u32, vp, u32]),
            "lx_liveness": (i32, [vp, vp, vp, u64, vp, vp]),
            "lx_tokenset_free": (None, [vp]),
            "lx_ctx_create": (i32, [vp]),
            "lx_ctx_free": (None, [vp]),
            "lx_ctx_set_timeout_ms": (i32, [vp, u32]),
            "lx_ctx_enable_timing": (i32, [vp, i32]),
            "lx_ctx_last_kernel_ms": (i32, [vp, vp]),
            "lx_ctx_set_config": (i32, [vp, vp, i32, u32, u32, u32]),
            "lx_ctx_debug_withhold": (i32, [vp, u32]),
            "lx_ctx_set_kernel": (i32, [vp, i32]),
            "lx_ctx_set_warps": (i32, [vp, u32]),
            "lx_ctx_set_warp_geometry": (i32, [vp, i32]),
            "lx_lex_async": (i32, [vp, vp, vp, u64, i32, vp, vp, u64, vp, vp]),
            "lx_ctx_get_config": (i32, [vp, vp, i32, vp, vp, vp, vp]),
            "lx_autotune": (i32, [vp, vp, i32, vp, u64, vp, vp, u64, vp]),
            "lx_lex": (i32, [vp, vp, vp, u64, i32, vp, vp, u64, vp, vp, vp]),
            "lx_lex_host": (i32, [vp, vp, vp, u64, i32, vp, vp, u64, vp, vp, vp]),
            "lx_lex_noalloc": (i32, [vp, vp, u64, i32, vp, vp, u64, vp, vp, vp]),
            "lx_lex_batch": (i32, [vp, vp, u32, vp, u32, i32, vp, vp, u64, vp, vp, vp]),
            "lx_lex_enumerative": (i32, [vp, vp, vp, u64, i32, vp, vp, u64, vp, vp, vp]),
            "lx_chunk_contexts": (i32, [vp, vp, vp, u64, vp, vp, u64, vp, vp]),
            "lx_lex_speculative": (i32, [vp, vp, vp, vp, u64, i32, vp, vp, u64, vp, vp, vp, vp]),
            "lx_model_create": (i32, [u32, u32, u64, vp]),
            "lx_model_free": (None, [vp]),
            "lx_model_info": (i32, [vp, vp, vp, vp, vp, vp]),
            "lx_model_get_params": (i32, [vp, vp, u64]),
            "lx_model_set_params": (i32, [vp, vp, u64]),
            "lx_model_windows": (i32, [vp, u64, vp, u32, vp, vp]),
            "lx_model_forward": (i32, [vp, vp, u32, vp, vp]),
            "lx_model_gradient": (i32, [vp, vp, vp, u32, vp, u64, vp, vp]),
            "lx_model_train_step": (i32, [vp, vp, vp, u32, ctypes.c_float, vp, vp]),
            "lx_strerror": (ctypes.c_char_p, [i32]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        if path is None:
            _lib = lib
        return lib


def lx_strerror(code: int) -> str:
    try:
        return load_library().lx_strerror(int(code)).decode()
    except RuntimeError:
        return f"status {code}"


class Tokenset:
    """Owning handle of an ``lx_tokenset``."""

    def __init__(self, handle: int, n_kinds: int):
        self.handle = handle
        self.n_kinds = n_kinds

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.lx_tokenset_free(self.handle)
            self.handle = None


class Ctx:
    """Owning handle of an ``lx_ctx``."""

    def __init__(self, handle: int):
        self.handle = handle

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.lx_ctx_free(self.handle)
            self.handle = None


def lx_compile_tokenset(dfa, discarded: Sequence[int] = ()) -> Tokenset:
    lib = load_library()
    nxt = np.ascontiguousarray(dfa.next, dtype=np.int64)
    n_classes, n_states = nxt.shape
    nxt32 = np.where(nxt < 0, LX_NONE, nxt).astype(np.uint32)
    acc = np.ascontiguousarray(dfa.accept, dtype=np.int64)
    acc16 = np.where(acc < 0, LX_NO_KIND, acc).astype(np.uint16)
    cls = np.ascontiguousarray(dfa.byte_class, dtype=np.uint8)
    n_kinds = int(getattr(dfa, "n_kinds", 0) or (int(acc.max()) + 1))
    d = _Dfa(n_states, n_classes, int(dfa.q0), n_kinds, cls.ctypes.data, nxt32.ctypes.data, acc16.ctypes.data)
    disc = np.ascontiguousarray(list(discarded), dtype=np.uint16)
    out = ctypes.c_void_p()
    rc = lib.lx_compile_tokenset(ctypes.byref(d), disc.ctypes.data if disc.size else None, int(disc.size),
                                 ctypes.byref(out))
    if rc != LX_OK:
        raise LexError(rc, "lx_compile_tokenset")
    return Tokenset(out.value, n_kinds)


def lx_compile_tokenset_framed(dfa, discarded: Sequence[int] = (), frame_byte: int = 0x1E,
                               frame_discarded: bool = False) -> Tokenset:
    """The token set of ``dfa`` with ``frame_byte`` reserved for framing at the
    producer: a kind of its own (numbered dfa.n_kinds), rejected inside every
    other token."""
    lib = load_library()
    nxt = np.ascontiguousarray(dfa.next, dtype=np.int64)
    n_classes, n_states = nxt.shape
    nxt32 = np.where(nxt < 0, LX_NONE, nxt).astype(np.uint32)
    acc = np.ascontiguousarray(dfa.accept, dtype=np.int64)
    acc16 = np.where(acc < 0, LX_NO_KIND, acc).astype(np.uint16)
    cls = np.ascontiguousarray(dfa.byte_class, dtype=np.uint8)
    n_kinds = int(getattr(dfa, "n_kinds", 0) or (int(acc.max()) + 1))
    d = _Dfa(n_states, n_classes, int(dfa.q0), n_kinds, cls.ctypes.data, nxt32.ctypes.data, acc16.ctypes.data)
    disc = np.ascontiguousarray(list(discarded), dtype=np.uint16)
    out = ctypes.c_void_p()
    rc = lib.lx_compile_tokenset_framed(ctypes.byref(d), disc.ctypes.data if disc.size else None, int(disc.size),
                                        int(frame_byte), 1 if frame_discarded else 0, ctypes.byref(out))
    if rc != LX_OK:
        raise LexError(rc, "lx_compile_tokenset_framed")
    return Tokenset(out.value, n_kinds + 1)


def _mask_to_bytes(words) -> np.ndarray:
    w = np.array(words, dtype=np.uint32)
    return np.array([(w[b >> 5] >> (b & 31)) & 1 for b in range(256)], dtype=bool)


def lx_certificates(ts: Tokenset) -> Tuple[np.ndarray, np.ndarray]:
    """Useful exact and modulo-I certificate masks, as bool[256]."""
    lib = load_library()
    ex = (ctypes.c_uint32 * 8)()
    mo = (ctypes.c_uint32 * 8)()
    rc = lib.lx_certificates(ts.handle, ex, mo)
    if rc != LX_OK:
        raise LexError(rc, "lx_certificates")
    return _mask_to_bytes(list(ex)), _mask_to_bytes(list(mo))


def lx_tokenset_info(ts: Tokenset, mode: int = LX_FULL_EXACT) -> dict:
    lib = load_library()
    ns, nl, tr = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
    re_, tf = ctypes.c_int(), ctypes.c_int()
    rc = lib.lx_tokenset_info(ts.handle, int(mode), ctypes.byref(ns), ctypes.byref(nl), ctypes.byref(re_),
                              ctypes.byref(tf), ctypes.byref(tr))
    return {"status": rc, "n_states": ns.value, "n_live": nl.value, "reentrant": bool(re_.value),
            "table_form": tf.value, "table_rows": tr.value}


def lx_tokenset_table(ts: Tokenset, mode: int, class_table: bool = False) -> Tuple[int, np.ndarray, dict]:
    """(status, blob bytes, layout) of the packed walk table for ``mode`` (the
    class-indexed one with ``class_table``)."""
    lib = load_library()
    fn = lib.lx_tokenset_class_table if class_table else lib.lx_tokenset_table
    meta = (ctypes.c_uint32 * 11)()
    rc = fn(ts.handle, int(mode), None, 0, meta, 11)
    blob = np.zeros(max(meta[0], 1), dtype=np.uint8)
    fn(ts.handle, int(mode), blob.ctypes.data, int(meta[0]), None, 0)
    keys = ("blob_bytes", "form", "n_rows", "ncols", "row_bytes", "table_bytes", "p_start", "p_flag", "p_slow")
    info = {k: int(meta[i]) for i, k in enumerate(keys)}
    info["kind_off"] = int(meta[9]) & 0xFFFF
    info["cmap_off"] = int(meta[9]) >> 16
    info["cert_off"] = int(meta[10])
    return rc, blob[:meta[0]], info


def lx_tokenset_walk_table(ts: Tokenset, mode: int) -> Tuple[int, np.ndarray, dict]:
    """The event-code walk table of ``mode`` (status, blob, layout)."""
    lib = load_library()
    meta = (ctypes.c_uint32 * 12)()
    lib.lx_tokenset_walk_table(ts.handle, int(mode), None, 0, meta, 12)
    blob = np.zeros(max(int(meta[0]), 1), np.uint8)
    rc = lib.lx_tokenset_walk_table(ts.handle, int(mode), blob.ctypes.data, int(blob.size), meta, 12)
    keys = ("bytes", "form", "n_rows", "row_shift", "p_start", "p_pre", "acc_off", "kmap_off", "cmap_off", "cut_off",
            "n_ctx", "ctx_off")
    return rc, blob[:int(meta[0])], dict(zip(keys, [int(x) for x in meta]))


def lx_window_certificates(ts: Tokenset) -> Tuple[int, np.ndarray]:
    """(status, bool[256, 256]): [a, b] when a cut before b is certified after a."""
    lib = load_library()
    words = np.zeros(256 * 8, np.uint32)
    rc = lib.lx_window_certificates(ts.handle, words.ctypes.data)
    bits = np.unpackbits(words.view(np.uint8).reshape(256, 32), axis=1, bitorder="little")
    return rc, bits.astype(bool)


def lx_ctx_create() -> Ctx:
    lib = load_library()
    out = ctypes.c_void_p()
    rc = lib.lx_ctx_create(ctypes.byref(out))
    if rc != LX_OK:
        raise LexError(rc, "lx_ctx_create")
    return Ctx(out.value)


def lx_ctx_set_timeout_ms(ctx: Ctx, ms: int) -> int:
    return load_library().lx_ctx_set_timeout_ms(ctx.handle, int(ms))


LX_KERNEL_AUTO, LX_KERNEL_TILE, LX_KERNEL_WARP = 0, 1, 2


def lx_ctx_set_kernel(ctx: Ctx, kernel: int) -> int:
    """Which kernel lx_lex uses: LX_KERNEL_AUTO (warp-tile kernel where it
    applies), LX_KERNEL_TILE or LX_KERNEL_WARP."""
    return load_library().lx_ctx_set_kernel(ctx.handle, int(kernel))


def lx_ctx_set_warps(ctx: Ctx, warps: int) -> int:
    """Warps per CTA of the warp-tile kernel (0: as many as fit)."""
    return load_library().lx_ctx_set_warps(ctx.handle, int(warps))


LX_WARP_GEOMETRY_AUTO, LX_WARP_GEOMETRY_SPARSE, LX_WARP_GEOMETRY_DENSE = 0, 1, 2


def lx_ctx_set_warp_geometry(ctx: Ctx, geometry: int) -> int:
    """The warp-tile kernel's geometry: LX_WARP_GEOMETRY_AUTO (chosen from the
    previous call on the same token set and mode), _SPARSE (512-byte halo,
    1536 staged tokens) or _DENSE (2048 and 768, the rest staged in global
    memory)."""
    return load_library().lx_ctx_set_warp_geometry(ctx.handle, int(geometry))


class AsyncResult(ctypes.Structure):
    """lx_async_result: the record lx_lex_async writes to device memory."""
    _fields_ = [("status", ctypes.c_int32), ("reserved", ctypes.c_uint32), ("n_tokens", ctypes.c_uint64),
                ("consumed", ctypes.c_uint64)]


def lx_lex_async(ctx: Ctx, ts: Tokenset, d_in, mode: int, d_kinds, d_lens, d_result, n: Optional[int] = None,
                 capacity: Optional[int] = None, stream=None) -> int:
    """Launch lx_lex without a host round trip; the result record (24 bytes:
    status, reserved, n_tokens, consumed) lands in the device buffer
    ``d_result`` in stream order.  Returns the launch status."""
    lib = load_library()
    n = d_in.numel() if n is None else int(n)
    cap = min(d_kinds.numel(), d_lens.numel()) if capacity is None else int(capacity)
    if d_result.numel() * d_result.element_size() < ctypes.sizeof(AsyncResult):
        raise ValueError("d_result needs 24 bytes")
    return lib.lx_lex_async(ctx.handle, ts.handle, d_in.data_ptr(), n, int(mode), d_kinds.data_ptr(),
                            d_lens.data_ptr(), cap, d_result.data_ptr(), _stream_handle(stream))


def async_result(buf) -> Tuple[int, int, int]:
    """(status, n_tokens, consumed) from the bytes of an lx_async_result."""
    a = np.asarray(buf).view(np.uint8)
    st = int(a[:4].view(np.int32)[0])
    nt, con = a[8:24].view(np.uint64).tolist()
    return st, int(nt), int(con)


def lx_ctx_enable_timing(ctx: Ctx, on: bool = True) -> int:
    return load_library().lx_ctx_enable_timing(ctx.handle, 1 if on else 0)


def lx_ctx_last_kernel_ms(ctx: Ctx) -> float:
    ms = ctypes.c_float()
    rc = load_library().lx_ctx_last_kernel_ms(ctx.handle, ctypes.byref(ms))
    if rc != LX_OK:
        raise LexError(rc, "lx_ctx_last_kernel_ms")
    return ms.value


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return int(getattr(stream, "cuda_stream", stream))


def lx_lex(ctx: Ctx, ts: Tokenset, d_in, mode: int, d_kinds, d_lens, n: Optional[int] = None,
           capacity: Optional[int] = None, stream=None) -> Tuple[int, int, int]:
    """Lex the device tensor ``d_in`` (uint8).  Returns (status, n_tokens, consumed)."""
    lib = load_library()
    n = d_in.numel() if n is None else int(n)
    cap = min(d_kinds.numel(), d_lens.numel()) if capacity is None else int(capacity)
    nt, con = ctypes.c_uint64(), ctypes.c_uint64()
    rc = lib.lx_lex(ctx.handle, ts.handle, d_in.data_ptr(), n, int(mode), d_kinds.data_ptr(), d_lens.data_ptr(),
                    cap, ctypes.byref(nt), ctypes.byref(con), _stream_handle(stream))
    return rc, nt.value, con.value


def lx_lex_host(ctx: Ctx, ts: Tokenset, h_in, mode: int, h_kinds, h_lens, n: Optional[int] = None,
                capacity: Optional[int] = None, stream=None) -> Tuple[int, int, int]:
    """Lex a host buffer (numpy array or CPU tensor, ideally pinned)."""
    lib = load_library()

    def ptr(x):
        return x.data_ptr() if hasattr(x, "data_ptr") else x.ctypes.data

    def size(x):
        return x.numel() if hasattr(x, "numel") else x.size

    n = size(h_in) if n is None else int(n)
    cap = min(size(h_kinds), size(h_lens)) if capacity is None else int(capacity)
    nt, con = ctypes.c_uint64(), ctypes.c_uint64()
    rc = lib.lx_lex_host(ctx.handle, ts.handle, ptr(h_in), n, int(mode), ptr(h_kinds), ptr(h_lens), cap,
                         ctypes.byref(nt), ctypes.byref(con), _stream_handle(stream))
    return rc, nt.value, con.value


LX_NOALLOC_SCRATCH_BYTES = 512 * 1024
LX_NOALLOC_MAX_INPUT = 57336 * 17408


def lx_lex_noalloc(ts: Tokenset, d_in, mode: int, d_kinds, d_lens, n: Optional[int] = None,
                   capacity: Optional[int] = None, stream=None) -> Tuple[int, int, int]:
    """``lx_lex`` without any allocation: for callers that may not allocate
    device or pinned memory while lexing (fixed-budget allocators,
    latency-sensitive code).  Uses one fixed device scratch array shared by
    every call, so overlapping calls race.  Returns (status, n_tokens, consumed)."""
    lib = load_library()
    n = d_in.numel() if n is None else int(n)
    cap = min(d_kinds.numel(), d_lens.numel()) if capacity is None else int(capacity)
    nt, con = ctypes.c_uint64(), ctypes.c_uint64()
    rc = lib.lx_lex_noalloc(ts.handle, d_in.data_ptr(), n, int(mode), d_kinds.data_ptr(), d_lens.data_ptr(), cap,
                            ctypes.byref(nt), ctypes.byref(con), _stream_handle(stream))
    return rc, nt.value, con.value


class BatchDocs:
    """The C arrays of one batch (token sets, document descriptors, result
    records), built once so that repeated lx_lex_batch calls on the same
    batch do no per-document Python work.  ``docs`` is a sequence of (device
    uint8 tensor or (pointer, n), set index)."""

    def __init__(self, sets, docs):
        self.sets = list(sets)
        self.n_sets, self.n_docs = len(self.sets), len(docs)
        self.set_arr = (ctypes.c_void_p * max(self.n_sets, 1))(*[ts.handle for ts in self.sets])
        self.doc_arr = (_Doc * max(self.n_docs, 1))()
        for i, (buf, set_idx) in enumerate(docs):
            if isinstance(buf, tuple):
                ptr, n = buf
            else:
                ptr, n = buf.data_ptr(), buf.numel()
            self.doc_arr[i] = _Doc(ptr if n else None, int(n), int(set_idx), 0)
        self.res_arr = (_DocResult * max(self.n_docs, 1))()

    def results(self):
        r = self.res_arr
        return [(r[i].out_off, r[i].n_tokens, r[i].consumed) for i in range(self.n_docs)]


def lx_lex_batch(ctx: Ctx, sets, docs, mode: int, d_kinds, d_lens, capacity: Optional[int] = None,
                 stream=None, want_results: bool = True):
    """Lex many documents in one graph launch.  ``sets`` is a sequence of
    Tokenset (ignored when ``docs`` is a BatchDocs); ``docs`` a BatchDocs or
    a sequence of (device uint8 tensor or (pointer, n), set index).  Returns
    (status, n_total, results) with results a list of (out_off, n_tokens,
    consumed) per document, in the order given (None if not wanted)."""
    lib = load_library()
    b = docs if isinstance(docs, BatchDocs) else BatchDocs(sets, docs)
    cap = min(d_kinds.numel(), d_lens.numel()) if capacity is None else int(capacity)
    total = ctypes.c_uint64()
    rc = lib.lx_lex_batch(ctx.handle, b.set_arr, b.n_sets, b.doc_arr, b.n_docs, int(mode), d_kinds.data_ptr(),
                          d_lens.data_ptr(), cap, b.res_arr, ctypes.byref(total), _stream_handle(stream))
    return rc, total.value, (b.results() if want_results else None)


def lx_lex_enumerative(ctx: Ctx, ts: Tokenset, d_in, mode: int, d_kinds, d_lens, n: Optional[int] = None,
                       capacity: Optional[int] = None, stream=None) -> Tuple[int, int, int]:
    """Lex a device buffer whose token set certifies no byte by enumerating
    chunk entry contexts.  Returns (status, n_tokens, consumed) as lx_lex."""
    lib = load_library()
    n = d_in.numel() if n is None else int(n)
    cap = min(d_kinds.numel(), d_lens.numel()) if capacity is None else int(capacity)
    nt, con = ctypes.c_uint64(), ctypes.c_uint64()
    rc = lib.lx_lex_enumerative(ctx.handle, ts.handle, d_in.data_ptr(), n, int(mode), d_kinds.data_ptr(),
                                d_lens.data_ptr(), cap, ctypes.byref(nt), ctypes.byref(con), _stream_handle(stream))
    return rc, nt.value, con.value


def lx_tokenset_scan_table(ts: Tokenset):
    """(status, blob uint8 array, meta dict) of the plain DFA scan table."""
    lib = load_library()
    meta = (ctypes.c_uint32 * 9)()
    lib.lx_tokenset_scan_table(ts.handle, None, 0, meta, 9)
    blob = np.zeros(max(meta[0], 1), np.uint8)
    rc = lib.lx_tokenset_scan_table(ts.handle, blob.ctypes.data, meta[0], meta, 9)
    keys = ("bytes", "S", "C", "q0", "next_off", "acc_off", "cbeg_off", "cand_off", "max_cand")
    return rc, blob[:meta[0]], dict(zip(keys, list(meta)))


def lx_tokenset_liveness(ts: Tokenset):
    """(status, blob uint8 array, meta dict) of the liveness automaton of the
    failed-lookahead guard."""
    lib = load_library()
    meta = (ctypes.c_uint32 * 8)()
    lib.lx_tokenset_liveness(ts.handle, None, 0, meta, 8)
    blob = np.zeros(max(meta[0], 1), np.uint8)
    rc = lib.lx_tokenset_liveness(ts.handle, blob.ctypes.data, meta[0], meta, 8)
    keys = ("bytes", "R", "C", "S", "W", "next_off", "reset_off", "member_off")
    return rc, blob[:meta[0]], dict(zip(keys, list(meta)))


def lx_liveness(ctx: Ctx, ts: Tokenset, d_in, d_live, n: Optional[int] = None, stream=None) -> int:
    """The liveness automaton's state at every offset 0..n of the device
    buffer d_in into the device buffer d_live (n + 1 bytes)."""
    lib = load_library()
    n = d_in.numel() if n is None else int(n)
    if d_live.numel() < n + 1:
        raise ValueError("d_live needs n + 1 bytes")
    return lib.lx_liveness(ctx.handle, ts.handle, d_in.data_ptr(), n, d_live.data_ptr(), _stream_handle(stream))


LX_KS_MIN, LX_KS_MAX = 16, 96


def lx_ctx_set_config(ctx: Ctx, ts: Tokenset, mode: int, ks: int, ctas_per_sm: int = 0,
                      class_table: int = 0) -> int:
    return load_library().lx_ctx_set_config(ctx.handle, ts.handle, int(mode), int(ks), int(ctas_per_sm),
                                            int(class_table))


def lx_ctx_get_config(ctx: Ctx, ts: Tokenset, mode: int):
    """(ks, ctas_per_sm, class_table, ms) in force for (ts, mode)."""
    ks, ctas, cls, ms = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_float()
    load_library().lx_ctx_get_config(ctx.handle, ts.handle, int(mode), ctypes.byref(ks), ctypes.byref(ctas),
                                     ctypes.byref(cls), ctypes.byref(ms))
    return ks.value, ctas.value, cls.value, ms.value


def lx_autotune(ctx: Ctx, ts: Tokenset, mode: int, d_sample, d_kinds, d_lens, n: Optional[int] = None,
                capacity: Optional[int] = None, stream=None) -> int:
    """Time the launch configurations on a device sample and keep the fastest."""
    n = d_sample.numel() if n is None else int(n)
    cap = min(d_kinds.numel(), d_lens.numel()) if capacity is None else int(capacity)
    return load_library().lx_autotune(ctx.handle, ts.handle, int(mode), d_sample.data_ptr(), n,
                                      d_kinds.data_ptr(), d_lens.data_ptr(), cap, _stream_handle(stream))


CTX_BOUNDARY = 0xFFFE
CTX_NONE = 0xFFFF


def lx_chunk_contexts(ctx: Ctx, ts: Tokenset, d_in, n: Optional[int] = None, stream=None):
    """(status, starts uint64 device tensor, contexts uint16 device tensor) per
    4096-byte chunk target: the true entry context at every chunk start."""
    import torch
    lib = load_library()
    n = d_in.numel() if n is None else int(n)
    count = ctypes.c_uint64()
    lib.lx_chunk_contexts(ctx.handle, ts.handle, d_in.data_ptr(), n, None, None, 0, ctypes.byref(count),
                          _stream_handle(stream))
    m = max(count.value, 1)
    starts = torch.empty(m, dtype=torch.int64, device=d_in.device)
    cx = torch.empty(m, dtype=torch.int16, device=d_in.device)
    rc = lib.lx_chunk_contexts(ctx.handle, ts.handle, d_in.data_ptr(), n, starts.data_ptr(), cx.data_ptr(), m,
                               ctypes.byref(count), _stream_handle(stream))
    return rc, starts[:count.value], cx[:count.value]


class _SpecStats(ctypes.Structure):
    _fields_ = [("chunks", ctypes.c_uint64), ("rounds", ctypes.c_uint32), ("rescanned", ctypes.c_uint32),
                ("judged", ctypes.c_uint64)]


class Model:
    """Owning handle of an ``lx_model`` (the entry-context predictor)."""

    def __init__(self, n_contexts: int, hidden: int = 64, seed: int = 1):
        lib = load_library()
        h = ctypes.c_void_p()
        rc = lib.lx_model_create(int(n_contexts), int(hidden), int(seed), ctypes.byref(h))
        if rc != 0:
            raise LexError(rc, "lx_model_create")
        self.handle = h.value
        c, hd, w, e, n = (ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32(),
                          ctypes.c_uint64())
        lib.lx_model_info(self.handle, ctypes.byref(c), ctypes.byref(hd), ctypes.byref(w), ctypes.byref(e),
                          ctypes.byref(n))
        self.n_contexts, self.hidden, self.window, self.embed, self.n_params = c.value, hd.value, w.value, \
            e.value, n.value

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.lx_model_free(self.handle)
            self.handle = None

    def get_params(self) -> np.ndarray:
        out = np.empty(self.n_params, np.float32)
        rc = load_library().lx_model_get_params(self.handle, out.ctypes.data, self.n_params)
        if rc != 0:
            raise LexError(rc, "lx_model_get_params")
        return out

    def set_params(self, p: np.ndarray):
        p = np.ascontiguousarray(p, np.float32)
        rc = load_library().lx_model_set_params(self.handle, p.ctypes.data, p.size)
        if rc != 0:
            raise LexError(rc, "lx_model_set_params")

    def windows(self, d_in, d_pos, stream=None):
        import torch
        cnt = d_pos.numel()
        win = torch.empty((max(cnt, 1), self.window), dtype=torch.int16, device=d_in.device)
        rc = load_library().lx_model_windows(d_in.data_ptr(), d_in.numel(), d_pos.data_ptr(), cnt,
                                             win.data_ptr(), _stream_handle(stream))
        if rc != 0:
            raise LexError(rc, "lx_model_windows")
        return win[:cnt]

    def forward(self, d_windows, stream=None):
        import torch
        b = d_windows.shape[0]
        logits = torch.empty((b, self.n_contexts), dtype=torch.float32, device=d_windows.device)
        rc = load_library().lx_model_forward(self.handle, d_windows.data_ptr(), b, logits.data_ptr(),
                                             _stream_handle(stream))
        if rc != 0:
            raise LexError(rc, "lx_model_forward")
        return logits

    def gradient(self, d_windows, d_labels, stream=None):
        g = np.empty(self.n_params, np.float32)
        loss = ctypes.c_float()
        rc = load_library().lx_model_gradient(self.handle, d_windows.data_ptr(), d_labels.data_ptr(),
                                              d_windows.shape[0], g.ctypes.data, self.n_params,
                                              ctypes.byref(loss), _stream_handle(stream))
        if rc != 0:
            raise LexError(rc, "lx_model_gradient")
        return g, loss.value

    def train_step(self, d_windows, d_labels, lr: float, stream=None) -> float:
        loss = ctypes.c_float()
        rc = load_library().lx_model_train_step(self.handle, d_windows.data_ptr(), d_labels.data_ptr(),
                                                d_windows.shape[0], ctypes.c_float(lr), ctypes.byref(loss),
                                                _stream_handle(stream))
        if rc != 0:
            raise LexError(rc, "lx_model_train_step")
        return loss.value


def lx_lex_speculative(ctx: Ctx, ts: Tokenset, model: Optional[Model], d_in, mode: int, d_kinds, d_lens,
                       n: Optional[int] = None, capacity: Optional[int] = None, stream=None):
    """Speculative lexing of a token set with no certified byte.  Returns
    (status, n_tokens, consumed, stats dict)."""
    lib = load_library()
    n = d_in.numel() if n is None else int(n)
    cap = min(d_kinds.numel(), d_lens.numel()) if capacity is None else int(capacity)
    nt, con = ctypes.c_uint64(), ctypes.c_uint64()
    st = _SpecStats()
    rc = lib.lx_lex_speculative(ctx.handle, ts.handle, model.handle if model is not None else None,
                                d_in.data_ptr(), n, int(mode), d_kinds.data_ptr(), d_lens.data_ptr(), cap,
                                ctypes.byref(nt), ctypes.byref(con), ctypes.byref(st), _stream_handle(stream))
    return rc, nt.value, con.value, {"chunks": st.chunks, "rounds": st.rounds, "rescanned": st.rescanned,
                                   "judged": bool(st.judged)}


def context_training_set(ctx: Ctx, ts: Tokenset, model: Model, d_in, stream=None):
    """(windows, labels) on the device for every chunk start of d_in, the
    labels being the entry contexts resolved by lx_chunk_contexts (class
    index: a DFA state, or n_contexts - 1 for BOUNDARY)."""
    import torch
    rc, starts, cx = lx_chunk_contexts(ctx, ts, d_in, stream=stream)
    if rc != 0:
        raise LexError(rc, "lx_chunk_contexts")
    keep = (starts >= 0) & (starts > 0)   # targets with a start, chunk 0 excluded (always BOUNDARY)
    starts, cx = starts[keep].contiguous(), cx[keep].contiguous()
    lab = cx.to(torch.int32) & 0xFFFF
    lab = torch.where(lab == CTX_BOUNDARY, torch.full_like(lab, model.n_contexts - 1), lab)
    return model.windows(d_in, starts, stream=stream), lab.to(torch.int16).contiguous()


def train_context_model(ctx: Ctx, ts: Tokenset, samples, hidden: int = 64, epochs: int = 4, batch: int = 512,
                        lr: float = 2e-3, seed: int = 1, stream=None) -> Model:
    """Train an entry-context model for ``ts`` on device buffers ``samples``
    (labels from enumeration, every step in this library's kernels)."""
    import torch
    info = lx_tokenset_scan_table(ts)[2]
    model = Model(info["S"] + 1, hidden=hidden, seed=seed)
    wins, labs = [], []
    for d in samples:
        w, y = context_training_set(ctx, ts, model, d, stream=stream)
        wins.append(w)
        labs.append(y)
    W = torch.cat(wins)
    Y = torch.cat(labs)
    g = torch.Generator(device="cpu").manual_seed(seed)
    for _ in range(epochs):
        perm = torch.randperm(W.shape[0], generator=g).to(W.device)
        for i in range(0, W.shape[0] - batch + 1, batch):
            idx = perm[i:i + batch]
            model.train_step(W[idx].contiguous(), Y[idx].contiguous(), lr, stream=stream)
    return model


def lx_ctx_debug_withhold(ctx: Ctx, tile: int) -> int:
    """Failure-detection test hook: tile ``tile`` never publishes its
    look-back aggregate (0xFFFFFFFF: off)."""
    return load_library().lx_ctx_debug_withhold(ctx.handle, int(tile) & 0xFFFFFFFF)
