"""Oracle: scalar CPU UTF-8 <-> UTF-16LE (and UTF-8 <-> UTF-32LE) transcoder
(test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package. The product
library never loads it, and it shares no code with the CUDA path.

Each function follows the paper's statement of the encodings (Clausecker &
Lemire, arXiv 2212.05098): Fig. 1(a) and Table 1 (byte layouts), Sec. 2.1
(UTF-16 surrogates), Sec. 6.4 (UTF-8 validation rules 1-6), Sec. 7.4
(surrogate sequencing) and the valid-prefix-then-stop behaviour of Sec. 6.4 and
Sec. 7.5. The C source (``oracle.c``) states the readings taken where the
paper is silent (error kinds and their precedence, capacity handling).

Arrays are numpy ``uint8`` buffers; UTF-16LE data is passed as bytes
(``2 * n_units``), low byte first, UTF-32LE data likewise (``4 * n_units``).
UTF-32 units above U+10FFFF are TOO_LARGE and units in D800-DFFF SURROGATE
(the library's convention; Sec. 2 defines UTF-32 as the code point itself).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

OK = 0
HEADER_BITS = 1
TOO_SHORT = 2
TOO_LONG = 3
OVERLONG = 4
TOO_LARGE = 5
SURROGATE = 6
LONE_HIGH_SURROGATE = 7
LONE_LOW_SURROGATE = 8
OUTPUT_TOO_SMALL = 16

STATUS_NAMES = {
    OK: "OK", HEADER_BITS: "HEADER_BITS", TOO_SHORT: "TOO_SHORT",
    TOO_LONG: "TOO_LONG", OVERLONG: "OVERLONG", TOO_LARGE: "TOO_LARGE",
    SURROGATE: "SURROGATE", LONE_HIGH_SURROGATE: "LONE_HIGH_SURROGATE",
    LONE_LOW_SURROGATE: "LONE_LOW_SURROGATE", OUTPUT_TOO_SMALL: "OUTPUT_TOO_SMALL",
}


class _CResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32),
                ("in_offset", ctypes.c_uint64),
                ("out_len", ctypes.c_uint64)]


@dataclass(frozen=True)
class Result:
    status: int
    in_offset: int
    out_len: int

    @property
    def ok(self) -> bool:
        return self.status == OK


_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        rp = ctypes.POINTER(_CResult)
        for name in ("oracle_utf8_to_utf16le", "oracle_utf16le_to_utf8",
                     "oracle_utf8_to_utf32le", "oracle_utf32le_to_utf8"):
            f = getattr(lib, name)
            f.argtypes = [u8p, ctypes.c_uint64, u8p, ctypes.c_uint64, rp]
            f.restype = None
        for name in ("oracle_utf16_length_from_utf8", "oracle_utf8_length_from_utf16le",
                     "oracle_utf32_length_from_utf8", "oracle_utf8_length_from_utf32le"):
            f = getattr(lib, name)
            f.argtypes = [u8p, ctypes.c_uint64, rp]
            f.restype = None
        _lib = lib
    return _lib


def _as_u8(buf) -> np.ndarray:
    if isinstance(buf, (bytes, bytearray, memoryview)):
        return np.frombuffer(bytes(buf), dtype=np.uint8)
    a = np.ascontiguousarray(buf)
    return a.view(np.uint8).reshape(-1)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def utf8_to_utf16le(data, cap_units: int | None = None):
    """Transcode UTF-8 bytes; returns (Result, uint16 array of length min(out_len, cap))."""
    lib = _load()
    src = _as_u8(data)
    n = src.size
    if cap_units is None:
        cap_units = n  # worst case: one unit per input byte
    out = np.zeros(max(cap_units, 1) * 2, dtype=np.uint8)
    r = _CResult()
    lib.oracle_utf8_to_utf16le(_ptr(src), n, _ptr(out), cap_units, ctypes.byref(r))
    res = Result(r.status, r.in_offset, r.out_len)
    keep = min(res.out_len, cap_units)
    return res, out[: 2 * keep].view("<u2").copy()


def utf16le_to_utf8(data, cap_bytes: int | None = None):
    """Transcode UTF-16LE (uint16 array or LE bytes); returns (Result, uint8 array)."""
    lib = _load()
    src = _as_u8(data)
    if src.size % 2:
        raise ValueError("UTF-16LE input must have an even number of bytes")
    n = src.size // 2
    if cap_bytes is None:
        cap_bytes = 3 * n  # worst case: three bytes per input unit
    out = np.zeros(max(cap_bytes, 1), dtype=np.uint8)
    r = _CResult()
    lib.oracle_utf16le_to_utf8(_ptr(src), n, _ptr(out), cap_bytes, ctypes.byref(r))
    res = Result(r.status, r.in_offset, r.out_len)
    keep = min(res.out_len, cap_bytes)
    return res, out[:keep].copy()


def utf16_length_from_utf8(data) -> Result:
    lib = _load()
    src = _as_u8(data)
    r = _CResult()
    lib.oracle_utf16_length_from_utf8(_ptr(src), src.size, ctypes.byref(r))
    return Result(r.status, r.in_offset, r.out_len)


def utf8_length_from_utf16le(data) -> Result:
    lib = _load()
    src = _as_u8(data)
    if src.size % 2:
        raise ValueError("UTF-16LE input must have an even number of bytes")
    r = _CResult()
    lib.oracle_utf8_length_from_utf16le(_ptr(src), src.size // 2, ctypes.byref(r))
    return Result(r.status, r.in_offset, r.out_len)


# UTF-16BE (Sec. 2.1: the same words with the high byte first): the UTF-16LE
# oracle applied to byte-swapped words, which is the definition of the order.
def _swap_words(data) -> np.ndarray:
    src = _as_u8(data)
    if src.size % 2:
        raise ValueError("UTF-16 input must have an even number of bytes")
    return src.reshape(-1, 2)[:, ::-1].reshape(-1).copy()


def utf8_to_utf16be(data, cap_units: int | None = None):
    """Transcode UTF-8 bytes to UTF-16BE; returns (Result, big-endian bytes)."""
    res, out = utf8_to_utf16le(data, cap_units)
    return res, _swap_words(out.view(np.uint8))


def utf16be_to_utf8(data, cap_bytes: int | None = None):
    """Transcode UTF-16BE bytes; returns (Result, uint8 array)."""
    return utf16le_to_utf8(_swap_words(data), cap_bytes)


def utf8_length_from_utf16be(data) -> Result:
    return utf8_length_from_utf16le(_swap_words(data))


def library_path() -> str:
    return os.path.abspath(_build.build())


# ---- UTF-32LE (Sec. 2: one 32-bit unit per code point) ---------------------

def utf8_to_utf32le(data, cap_units: int | None = None):
    """Transcode UTF-8 bytes; returns (Result, uint32 array of length min(out_len, cap))."""
    lib = _load()
    src = _as_u8(data)
    n = src.size
    if cap_units is None:
        cap_units = n  # worst case: one unit per input byte
    out = np.zeros(max(cap_units, 1) * 4, dtype=np.uint8)
    r = _CResult()
    lib.oracle_utf8_to_utf32le(_ptr(src), n, _ptr(out), cap_units, ctypes.byref(r))
    res = Result(r.status, r.in_offset, r.out_len)
    keep = min(res.out_len, cap_units)
    return res, out[: 4 * keep].view("<u4").copy()


def utf32le_to_utf8(data, cap_bytes: int | None = None):
    """Transcode UTF-32LE (uint32 array or LE bytes); returns (Result, uint8 array)."""
    lib = _load()
    src = _as_u8(data)
    if src.size % 4:
        raise ValueError("UTF-32LE input must have a multiple of 4 bytes")
    n = src.size // 4
    if cap_bytes is None:
        cap_bytes = 4 * n  # worst case: four bytes per input unit
    out = np.zeros(max(cap_bytes, 1), dtype=np.uint8)
    r = _CResult()
    lib.oracle_utf32le_to_utf8(_ptr(src), n, _ptr(out), cap_bytes, ctypes.byref(r))
    res = Result(r.status, r.in_offset, r.out_len)
    keep = min(res.out_len, cap_bytes)
    return res, out[:keep].copy()


def utf32_length_from_utf8(data) -> Result:
    lib = _load()
    src = _as_u8(data)
    r = _CResult()
    lib.oracle_utf32_length_from_utf8(_ptr(src), src.size, ctypes.byref(r))
    return Result(r.status, r.in_offset, r.out_len)


def utf8_length_from_utf32le(data) -> Result:
    lib = _load()
    src = _as_u8(data)
    if src.size % 4:
        raise ValueError("UTF-32LE input must have a multiple of 4 bytes")
    r = _CResult()
    lib.oracle_utf8_length_from_utf32le(_ptr(src), src.size // 4, ctypes.byref(r))
    return Result(r.status, r.in_offset, r.out_len)
