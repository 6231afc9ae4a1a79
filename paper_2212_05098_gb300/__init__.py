"""Python binding of libgbutf (validating UTF-8 <-> UTF-16LE transcoding on GB300).

Argument marshalling only: every function here forwards to the C ABI of
``include/gbutf.h`` with the same name, passing raw device pointers, sizes
and the CUDA stream handle. All transcoding work runs in the library's CUDA
kernels. There is no fallback: if the library cannot be built or loaded, the
import of the function raises.

Convenience wrappers (``Context.utf8_to_utf16le`` ...) take torch CUDA tensors
and allocate worst-case outputs; torch provides device memory and streams only.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

from . import build as _build

GBU_OK = 0
GBU_HEADER_BITS = 1
GBU_TOO_SHORT = 2
GBU_TOO_LONG = 3
GBU_OVERLONG = 4
GBU_TOO_LARGE = 5
GBU_SURROGATE = 6
GBU_LONE_HIGH_SURROGATE = 7
GBU_LONE_LOW_SURROGATE = 8
GBU_OUTPUT_TOO_SMALL = 16
GBU_INVALID_ARG = 17
GBU_DEVICE_ERROR = 18
GBU_DEVICE_TIMEOUT = 19
GBU_SMALL_MAX_CHUNKS = 8    # largest input (in 12 KiB chunks) of the one-launch path


class gbu_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("reserved", ctypes.c_uint32),
                ("in_offset", ctypes.c_uint64), ("out_len", ctypes.c_uint64)]


@dataclass(frozen=True)
class Result:
    status: int
    in_offset: int
    out_len: int

    @property
    def ok(self) -> bool:
        return self.status == GBU_OK

    @property
    def name(self) -> str:
        return status_name(self.status)


GBU_OP_UTF8_TO_UTF16LE = 0
GBU_OP_UTF16LE_TO_UTF8 = 1
GBU_OP_UTF16_LENGTH_FROM_UTF8 = 2
GBU_OP_UTF8_LENGTH_FROM_UTF16LE = 3
GBU_OP_UTF8_TO_UTF16BE = 4
GBU_OP_UTF16BE_TO_UTF8 = 5
GBU_OP_UTF8_LENGTH_FROM_UTF16BE = 6


class gbu_batch_item(ctypes.Structure):
    _fields_ = [("in_", ctypes.c_void_p), ("n", ctypes.c_uint64), ("out", ctypes.c_void_p),
                ("cap", ctypes.c_uint64), ("op", ctypes.c_int32), ("reserved", ctypes.c_uint32)]


class gbu_tune(ctypes.Structure):
    _fields_ = [("look_width", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("small_chunks", ctypes.c_int32), ("chunk_bytes", ctypes.c_int32),
                ("compute_threads", ctypes.c_int32)]


class gbu_request(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("reserved", ctypes.c_uint32), ("in_", ctypes.c_void_p),
                ("n", ctypes.c_uint64), ("out_copy", ctypes.c_void_p),
                ("out_copy_cap_bytes", ctypes.c_uint64), ("tag", ctypes.c_uint64)]


class gbu_completion(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_uint64), ("result", gbu_result), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_launch", ctypes.c_double),
                ("t_done", ctypes.c_double), ("batch", ctypes.c_uint32),
                ("batch_items", ctypes.c_uint32)]


class gbu_server_stats_t(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("batches", ctypes.c_uint64), ("pool_bytes", ctypes.c_uint64),
                ("pool_high_water", ctypes.c_uint64)]


# name -> (restype, argtypes)
_VP, _U64, _I32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int32
_RP = ctypes.POINTER(gbu_result)
SIGNATURES = {
    "gbu_create": (_VP, [ctypes.c_int]),
    "gbu_destroy": (None, [_VP]),
    "gbu_reserve": (_I32, [_VP, _U64]),
    "gbu_utf8_to_utf16le": (gbu_result, [_VP, _VP, _U64, _VP, _U64, _VP]),
    "gbu_utf16le_to_utf8": (gbu_result, [_VP, _VP, _U64, _VP, _U64, _VP]),
    "gbu_utf16_length_from_utf8": (gbu_result, [_VP, _VP, _U64, _VP]),
    "gbu_utf8_length_from_utf16le": (gbu_result, [_VP, _VP, _U64, _VP]),
    "gbu_utf8_to_utf16be": (gbu_result, [_VP, _VP, _U64, _VP, _U64, _VP]),
    "gbu_utf16be_to_utf8": (gbu_result, [_VP, _VP, _U64, _VP, _U64, _VP]),
    "gbu_utf8_length_from_utf16be": (gbu_result, [_VP, _VP, _U64, _VP]),
    "gbu_validate_utf16be": (gbu_result, [_VP, _VP, _U64, _VP]),
    "gbu_utf8_to_utf32le": (gbu_result, [_VP, _VP, _U64, _VP, _U64, _VP]),
    "gbu_utf32le_to_utf8": (gbu_result, [_VP, _VP, _U64, _VP, _U64, _VP]),
    "gbu_utf32_length_from_utf8": (gbu_result, [_VP, _VP, _U64, _VP]),
    "gbu_utf8_length_from_utf32le": (gbu_result, [_VP, _VP, _U64, _VP]),
    "gbu_validate_utf32le": (gbu_result, [_VP, _VP, _U64, _VP]),
    "gbu_utf8_to_utf16be_async": (_I32, [_VP, _VP, _U64, _VP, _U64, _VP, _VP]),
    "gbu_utf16be_to_utf8_async": (_I32, [_VP, _VP, _U64, _VP, _U64, _VP, _VP]),
    "gbu_validate_utf8": (gbu_result, [_VP, _VP, _U64, _VP]),
    "gbu_validate_utf16le": (gbu_result, [_VP, _VP, _U64, _VP]),
    "gbu_validate_utf8_async": (_I32, [_VP, _VP, _U64, _VP, _VP]),
    "gbu_validate_utf16le_async": (_I32, [_VP, _VP, _U64, _VP, _VP]),
    "gbu_utf8_to_utf16le_async": (_I32, [_VP, _VP, _U64, _VP, _U64, _VP, _VP]),
    "gbu_utf16le_to_utf8_async": (_I32, [_VP, _VP, _U64, _VP, _U64, _VP, _VP]),
    "gbu_utf16_length_from_utf8_async": (_I32, [_VP, _VP, _U64, _VP, _VP]),
    "gbu_utf8_length_from_utf16le_async": (_I32, [_VP, _VP, _U64, _VP, _VP]),
    "gbu_utf8_to_utf16le_host": (gbu_result, [_VP, _VP, _U64, _VP, _U64, _VP]),
    "gbu_utf16le_to_utf8_host": (gbu_result, [_VP, _VP, _U64, _VP, _U64, _VP]),
    "gbu_batch_plan": (_I32, [_VP, ctypes.POINTER(gbu_batch_item), ctypes.c_uint32, _VP, _VP]),
    "gbu_batch_launch": (_I32, [_VP, _VP]),
    "gbu_batch_launch_graph": (_I32, [_VP, _VP]),
    "gbu_get_tune": (_I32, [_VP, ctypes.POINTER(gbu_tune)]),
    "gbu_set_tune": (_I32, [_VP, ctypes.POINTER(gbu_tune)]),
    "gbu_tune_shapes": (_I32, [ctypes.POINTER(gbu_tune), ctypes.c_int32]),
    "gbu_call_shape": (_I32, [_VP, _U64, ctypes.POINTER(gbu_tune)]),
    "gbu_set_wait_limit": (_I32, [_VP, _U64]),
    "gbu_test_skip_chunks": (_I32, [_VP, ctypes.c_uint32]),
    "gbu_batch_autotune": (_I32, [_VP, _VP, ctypes.c_char_p, ctypes.POINTER(gbu_tune)]),
    "gbu_server_create": (_VP, [ctypes.c_int, _U64, ctypes.c_uint32, ctypes.c_uint32]),
    "gbu_server_destroy": (None, [_VP]),
    "gbu_server_submit": (_I32, [_VP, ctypes.POINTER(gbu_request)]),
    "gbu_server_poll": (ctypes.c_uint32, [_VP, ctypes.POINTER(gbu_completion), ctypes.c_uint32]),
    "gbu_server_wait_idle": (_I32, [_VP, ctypes.c_double]),
    "gbu_server_replay": (_I32, [_VP, ctypes.POINTER(gbu_request), ctypes.POINTER(ctypes.c_double),
                                 ctypes.c_uint32, ctypes.POINTER(gbu_completion), ctypes.c_double]),
    "gbu_server_stats": (_I32, [_VP, ctypes.POINTER(gbu_server_stats_t)]),
    "gbu_utf8_to_utf16le_noalloc": (gbu_result, [_VP, _U64, _VP, _U64, _VP]),
    "gbu_status_name": (ctypes.c_char_p, [_I32]),
    "gbu_kernel_launch_count": (_U64, []),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libgbutf.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is None:
        path = _build.build() if build_if_missing else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libgbutf.so not found at {path}; run build()")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def _res(r: gbu_result) -> Result:
    return Result(int(r.status), int(r.in_offset), int(r.out_len))


# ---- raw C-ABI mirrors (same names, integer pointers) -----------------------

def gbu_create(device: int = 0) -> int:
    h = load().gbu_create(device)
    if not h:
        raise RuntimeError(f"gbu_create({device}) failed")
    return h


def gbu_destroy(ctx: int) -> None:
    load().gbu_destroy(ctx)


def gbu_reserve(ctx: int, max_input_bytes: int) -> int:
    return load().gbu_reserve(ctx, max_input_bytes)


def gbu_utf8_to_utf16le(ctx, d_in, n_bytes, d_out, cap_units, stream=0) -> Result:
    return _res(load().gbu_utf8_to_utf16le(ctx, d_in, n_bytes, d_out, cap_units, stream))


def gbu_utf16le_to_utf8(ctx, d_in, n_units, d_out, cap_bytes, stream=0) -> Result:
    return _res(load().gbu_utf16le_to_utf8(ctx, d_in, n_units, d_out, cap_bytes, stream))


def gbu_utf16_length_from_utf8(ctx, d_in, n_bytes, stream=0) -> Result:
    return _res(load().gbu_utf16_length_from_utf8(ctx, d_in, n_bytes, stream))


def gbu_utf8_length_from_utf16le(ctx, d_in, n_units, stream=0) -> Result:
    return _res(load().gbu_utf8_length_from_utf16le(ctx, d_in, n_units, stream))


def gbu_utf8_to_utf16be(ctx, d_in, n_bytes, d_out, cap_units, stream=0) -> Result:
    return _res(load().gbu_utf8_to_utf16be(ctx, d_in, n_bytes, d_out, cap_units, stream))


def gbu_utf16be_to_utf8(ctx, d_in, n_units, d_out, cap_bytes, stream=0) -> Result:
    return _res(load().gbu_utf16be_to_utf8(ctx, d_in, n_units, d_out, cap_bytes, stream))


def gbu_utf8_length_from_utf16be(ctx, d_in, n_units, stream=0) -> Result:
    return _res(load().gbu_utf8_length_from_utf16be(ctx, d_in, n_units, stream))


def gbu_validate_utf16be(ctx, d_in, n_units, stream=0) -> Result:
    return _res(load().gbu_validate_utf16be(ctx, d_in, n_units, stream))


def gbu_utf8_to_utf32le(ctx, d_in, n_bytes, d_out, cap_units, stream=0) -> Result:
    return _res(load().gbu_utf8_to_utf32le(ctx, d_in, n_bytes, d_out, cap_units, stream))


def gbu_utf32le_to_utf8(ctx, d_in, n_units, d_out, cap_bytes, stream=0) -> Result:
    return _res(load().gbu_utf32le_to_utf8(ctx, d_in, n_units, d_out, cap_bytes, stream))


def gbu_utf32_length_from_utf8(ctx, d_in, n_bytes, stream=0) -> Result:
    return _res(load().gbu_utf32_length_from_utf8(ctx, d_in, n_bytes, stream))


def gbu_utf8_length_from_utf32le(ctx, d_in, n_units, stream=0) -> Result:
    return _res(load().gbu_utf8_length_from_utf32le(ctx, d_in, n_units, stream))


def gbu_validate_utf32le(ctx, d_in, n_units, stream=0) -> Result:
    return _res(load().gbu_validate_utf32le(ctx, d_in, n_units, stream))


def gbu_utf8_to_utf16be_async(ctx, d_in, n_bytes, d_out, cap_units, d_result, stream=0) -> int:
    return load().gbu_utf8_to_utf16be_async(ctx, d_in, n_bytes, d_out, cap_units, d_result, stream)


def gbu_utf16be_to_utf8_async(ctx, d_in, n_units, d_out, cap_bytes, d_result, stream=0) -> int:
    return load().gbu_utf16be_to_utf8_async(ctx, d_in, n_units, d_out, cap_bytes, d_result, stream)


def gbu_validate_utf8(ctx, d_in, n_bytes, stream=0) -> Result:
    return _res(load().gbu_validate_utf8(ctx, d_in, n_bytes, stream))


def gbu_validate_utf16le(ctx, d_in, n_units, stream=0) -> Result:
    return _res(load().gbu_validate_utf16le(ctx, d_in, n_units, stream))


def gbu_validate_utf8_async(ctx, d_in, n_bytes, d_result, stream=0) -> int:
    return load().gbu_validate_utf8_async(ctx, d_in, n_bytes, d_result, stream)


def gbu_validate_utf16le_async(ctx, d_in, n_units, d_result, stream=0) -> int:
    return load().gbu_validate_utf16le_async(ctx, d_in, n_units, d_result, stream)


def gbu_utf8_to_utf16le_async(ctx, d_in, n_bytes, d_out, cap_units, d_result, stream=0) -> int:
    return load().gbu_utf8_to_utf16le_async(ctx, d_in, n_bytes, d_out, cap_units, d_result, stream)


def gbu_utf16le_to_utf8_async(ctx, d_in, n_units, d_out, cap_bytes, d_result, stream=0) -> int:
    return load().gbu_utf16le_to_utf8_async(ctx, d_in, n_units, d_out, cap_bytes, d_result, stream)


def gbu_utf16_length_from_utf8_async(ctx, d_in, n_bytes, d_result, stream=0) -> int:
    return load().gbu_utf16_length_from_utf8_async(ctx, d_in, n_bytes, d_result, stream)


def gbu_utf8_length_from_utf16le_async(ctx, d_in, n_units, d_result, stream=0) -> int:
    return load().gbu_utf8_length_from_utf16le_async(ctx, d_in, n_units, d_result, stream)


def gbu_utf8_to_utf16le_host(ctx, h_in, n_bytes, h_out, cap_units, stream=0) -> Result:
    return _res(load().gbu_utf8_to_utf16le_host(ctx, h_in, n_bytes, h_out, cap_units, stream))


def gbu_utf16le_to_utf8_host(ctx, h_in, n_units, h_out, cap_bytes, stream=0) -> Result:
    return _res(load().gbu_utf16le_to_utf8_host(ctx, h_in, n_units, h_out, cap_bytes, stream))


def gbu_batch_plan(ctx, items, results_ptr, stream=0) -> int:
    """items: sequence of (in_ptr, n, out_ptr, cap, op) tuples or gbu_batch_item."""
    arr = (gbu_batch_item * max(1, len(items)))()
    for i, it in enumerate(items):
        arr[i] = it if isinstance(it, gbu_batch_item) else gbu_batch_item(*it, 0)
    return load().gbu_batch_plan(ctx, arr, len(items), results_ptr, stream)


def gbu_batch_launch(ctx, stream=0) -> int:
    return load().gbu_batch_launch(ctx, stream)


def gbu_batch_launch_graph(ctx, stream=0) -> int:
    return load().gbu_batch_launch_graph(ctx, stream)


def gbu_get_tune(ctx) -> gbu_tune:
    t = gbu_tune()
    st = load().gbu_get_tune(ctx, ctypes.byref(t))
    if st != GBU_OK:
        raise RuntimeError(status_name(st))
    return t


def gbu_set_wait_limit(ctx, ns: int) -> int:
    return load().gbu_set_wait_limit(ctx, ns)


def gbu_test_skip_chunks(ctx, first_chunk: int) -> int:
    return load().gbu_test_skip_chunks(ctx, first_chunk)


def gbu_set_tune(ctx, look_width: int, ctas_per_sm: int,
                 small_chunks: int = GBU_SMALL_MAX_CHUNKS, chunk_bytes: int = 0,
                 compute_threads: int = 0) -> int:
    t = gbu_tune(look_width, ctas_per_sm, small_chunks, chunk_bytes, compute_threads)
    return load().gbu_set_tune(ctx, ctypes.byref(t))


def gbu_call_shape(ctx, input_bytes: int) -> gbu_tune:
    """Launch parameters of a single-buffer call with this many input bytes."""
    t = gbu_tune()
    st = load().gbu_call_shape(ctx, input_bytes, ctypes.byref(t))
    if st != GBU_OK:
        raise RuntimeError(status_name(st))
    return t


def gbu_tune_shapes() -> list[tuple[int, int]]:
    """The compiled kernel shapes as (chunk_bytes, compute_threads); the first
    is the default."""
    n = load().gbu_tune_shapes(None, 0)
    arr = (gbu_tune * max(1, n))()
    load().gbu_tune_shapes(arr, n)
    return [(arr[i].chunk_bytes, arr[i].compute_threads) for i in range(n)]


def gbu_batch_autotune(ctx, stream=0, cache_path: str | None = None):
    """Returns (status, gbu_tune chosen)."""
    t = gbu_tune()
    path = cache_path.encode() if cache_path else None
    st = load().gbu_batch_autotune(ctx, stream, path, ctypes.byref(t))
    return st, t


def gbu_server_create(device: int, pool_bytes: int, slots: int, max_batch_items: int) -> int:
    return load().gbu_server_create(device, pool_bytes, slots, max_batch_items)


def gbu_server_destroy(srv) -> None:
    load().gbu_server_destroy(srv)


def gbu_server_submit(srv, op: int, in_ptr: int, n: int, out_copy: int = 0,
                      out_copy_cap_bytes: int = 0, tag: int = 0) -> int:
    r = gbu_request(op, 0, in_ptr or None, n, out_copy or None, out_copy_cap_bytes, tag)
    return load().gbu_server_submit(srv, ctypes.byref(r))


def gbu_server_poll(srv, max_items: int = 1024) -> list:
    buf = (gbu_completion * max_items)()
    k = load().gbu_server_poll(srv, buf, max_items)
    return [buf[i] for i in range(k)]


def gbu_server_wait_idle(srv, timeout_s: float = 60.0) -> int:
    return load().gbu_server_wait_idle(srv, timeout_s)


def gbu_server_replay(srv, requests, t_arrival, timeout_s: float = 120.0):
    """requests: sequence of (op, in_ptr, n, out_copy, out_copy_cap_bytes, tag);
    t_arrival: seconds after the call. Returns (status, completion array)."""
    k = len(requests)
    reqs = (gbu_request * max(1, k))()
    for i, (op, inp, n, oc, occ, tag) in enumerate(requests):
        reqs[i] = gbu_request(op, 0, inp or None, n, oc or None, occ, tag)
    times = (ctypes.c_double * max(1, k))(*t_arrival)
    out = (gbu_completion * max(1, k))()
    st = load().gbu_server_replay(srv, reqs, times, k, out, timeout_s)
    return st, out


def gbu_server_stats(srv) -> gbu_server_stats_t:
    st = gbu_server_stats_t()
    load().gbu_server_stats(srv, ctypes.byref(st))
    return st


def gbu_utf8_to_utf16le_noalloc(d_in, n_bytes, d_out, cap_units, stream=0) -> Result:
    return _res(load().gbu_utf8_to_utf16le_noalloc(d_in, n_bytes, d_out, cap_units, stream))


GBU_NOALLOC_MAX_BYTES = 64 << 20


def gbu_kernel_launch_count() -> int:
    return int(load().gbu_kernel_launch_count())


def status_name(status: int) -> str:
    return load().gbu_status_name(status).decode()


# ---- torch convenience layer (device memory + streams only) -------------------

def _stream_handle(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


class Context:
    """Owns one gbu_ctx (scratch for one in-flight call) on one device."""

    def __init__(self, device: int = 0):
        self.device = device
        self.handle = gbu_create(device)

    def close(self):
        if self.handle:
            gbu_destroy(self.handle)
            self.handle = None

    def __del__(self):  # pragma: no cover - interpreter shutdown order
        try:
            self.close()
        except Exception:
            pass

    def reserve(self, max_input_bytes: int) -> None:
        st = gbu_reserve(self.handle, max_input_bytes)
        if st != GBU_OK:
            raise RuntimeError(f"gbu_reserve failed: {status_name(st)}")

    def utf8_to_utf16le(self, src, out=None, stream=None):
        """src: uint8 CUDA tensor. Returns (Result, int16 tensor holding the words)."""
        import torch
        n = src.numel()
        if out is None:
            out = torch.empty(max(n, 1), dtype=torch.int16, device=src.device)
        r = gbu_utf8_to_utf16le(self.handle, src.data_ptr(), n, out.data_ptr(), out.numel(),
                                _stream_handle(stream))
        return r, out

    def utf16le_to_utf8(self, src, out=None, stream=None):
        """src: int16/uint16-sized CUDA tensor of words. Returns (Result, uint8 tensor)."""
        import torch
        n = src.numel()
        if out is None:
            out = torch.empty(max(3 * n, 1), dtype=torch.uint8, device=src.device)
        r = gbu_utf16le_to_utf8(self.handle, src.data_ptr(), n, out.data_ptr(), out.numel(),
                                _stream_handle(stream))
        return r, out

    def utf16_length_from_utf8(self, src, stream=None) -> Result:
        return gbu_utf16_length_from_utf8(self.handle, src.data_ptr(), src.numel(),
                                          _stream_handle(stream))

    def utf8_length_from_utf16le(self, src, stream=None) -> Result:
        return gbu_utf8_length_from_utf16le(self.handle, src.data_ptr(), src.numel(),
                                            _stream_handle(stream))
