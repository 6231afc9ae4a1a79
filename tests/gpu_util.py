"""Helpers for the GPU parity tests: guarded device buffers and calls through
the C ABI (via the thin Python binding), compared with the oracle."""
from __future__ import annotations

import numpy as np

import oracle
import paper_2212_05098_gb300 as gbu

GUARD = 64          # canary bytes on each side of every output buffer
CANARY = 0xA5


def torch():
    import torch as _t
    return _t


class DevIn:
    """Input bytes copied to the device at byte offset `off` of a larger buffer."""

    def __init__(self, data: np.ndarray, off: int = 0):
        t = torch()
        data = np.ascontiguousarray(data, dtype=np.uint8)
        self.buf = t.zeros(data.size + off + 32, dtype=t.uint8, device="cuda")
        if data.size:
            self.buf[off:off + data.size] = t.from_numpy(np.array(data, copy=True)).cuda()
        self.ptr = self.buf.data_ptr() + off
        self.nbytes = data.size


class DevOut:
    """Output buffer of `cap_bytes` at byte offset `off`, surrounded by canaries."""

    def __init__(self, cap_bytes: int, off: int = 0):
        t = torch()
        self.off = GUARD + off
        self.cap_bytes = cap_bytes
        self.buf = t.full((cap_bytes + self.off + GUARD,), CANARY, dtype=t.uint8, device="cuda")
        self.ptr = self.buf.data_ptr() + self.off

    def host(self) -> np.ndarray:
        return self.buf.cpu().numpy()

    def data(self, nbytes: int) -> np.ndarray:
        return self.host()[self.off:self.off + nbytes]

    def guards_intact(self) -> bool:
        h = self.host()
        return bool((h[:self.off] == CANARY).all() and (h[self.off + self.cap_bytes:] == CANARY).all())


def gpu_u8_to_u16(ctx, data: np.ndarray, cap_units=None, in_off=0, out_off=0, stream=0):
    din = DevIn(data, in_off)
    if cap_units is None:
        cap_units = max(data.size, 0)
    dout = DevOut(2 * cap_units, out_off)
    r = gbu.gbu_utf8_to_utf16le(ctx, din.ptr, data.size, dout.ptr, cap_units, stream)
    return r, dout


def gpu_u16_to_u8(ctx, data: np.ndarray, cap_bytes=None, in_off=0, out_off=0, stream=0):
    assert data.size % 2 == 0 and in_off % 2 == 0
    din = DevIn(data, in_off)
    n = data.size // 2
    if cap_bytes is None:
        cap_bytes = 3 * n
    dout = DevOut(cap_bytes, out_off)
    r = gbu.gbu_utf16le_to_utf8(ctx, din.ptr, n, dout.ptr, cap_bytes, stream)
    return r, dout


def triple(r) -> tuple:
    return (r.status, r.in_offset, r.out_len)


def check_u8(ctx, data: np.ndarray, cap_units=None, in_off=0, out_off=0):
    """UTF-8 -> UTF-16 on the GPU vs the oracle: result, output bytes, canaries."""
    data = np.ascontiguousarray(data, dtype=np.uint8)
    ref, ref_out = oracle.utf8_to_utf16le(data, cap_units)
    r, dout = gpu_u8_to_u16(ctx, data, cap_units, in_off, out_off)
    assert triple(r) == triple(ref), (triple(r), triple(ref))
    cap = data.size if cap_units is None else cap_units
    keep = min(ref.out_len, cap)
    got = dout.data(2 * keep)
    want = ref_out[:keep].view(np.uint8)
    if not np.array_equal(got, want):
        bad = int(np.nonzero(got != want)[0][0])
        raise AssertionError(f"output differs at byte {bad} of {2 * keep}")
    assert dout.guards_intact(), "write outside [0, cap)"
    din = DevIn(data, in_off)
    lr = gbu.gbu_utf16_length_from_utf8(ctx, din.ptr, data.size, 0)
    lref = oracle.utf16_length_from_utf8(data)
    assert triple(lr) == triple(lref), (triple(lr), triple(lref))
    vr = gbu.gbu_validate_utf8(ctx, din.ptr, data.size, 0)
    assert triple(vr) == (lref.status, lref.in_offset, 0), (triple(vr), triple(lref))
    return r


def check_u16(ctx, data: np.ndarray, cap_bytes=None, in_off=0, out_off=0):
    """UTF-16 -> UTF-8 on the GPU vs the oracle: result, output bytes, canaries."""
    data = np.ascontiguousarray(data, dtype=np.uint8)
    ref, ref_out = oracle.utf16le_to_utf8(data, cap_bytes)
    r, dout = gpu_u16_to_u8(ctx, data, cap_bytes, in_off, out_off)
    assert triple(r) == triple(ref), (triple(r), triple(ref))
    cap = 3 * (data.size // 2) if cap_bytes is None else cap_bytes
    keep = min(ref.out_len, cap)
    got = dout.data(keep)
    if not np.array_equal(got, ref_out[:keep]):
        bad = int(np.nonzero(got != ref_out[:keep])[0][0])
        raise AssertionError(f"output differs at byte {bad} of {keep}")
    assert dout.guards_intact(), "write outside [0, cap)"
    din = DevIn(data, in_off)
    lr = gbu.gbu_utf8_length_from_utf16le(ctx, din.ptr, data.size // 2, 0)
    lref = oracle.utf8_length_from_utf16le(data)
    assert triple(lr) == triple(lref), (triple(lr), triple(lref))
    vr = gbu.gbu_validate_utf16le(ctx, din.ptr, data.size // 2, 0)
    assert triple(vr) == (lref.status, lref.in_offset, 0), (triple(vr), triple(lref))
    return r


def check_u8_be(ctx, data: np.ndarray, cap_units=None, in_off=0, out_off=0):
    """UTF-8 -> UTF-16BE on the GPU vs the oracle."""
    data = np.ascontiguousarray(data, dtype=np.uint8)
    ref, ref_out = oracle.utf8_to_utf16be(data, cap_units)
    din = DevIn(data, in_off)
    cap = data.size if cap_units is None else cap_units
    dout = DevOut(2 * cap, out_off)
    r = gbu.gbu_utf8_to_utf16be(ctx, din.ptr, data.size, dout.ptr, cap, 0)
    assert triple(r) == triple(ref), (triple(r), triple(ref))
    keep = min(ref.out_len, cap)
    assert np.array_equal(dout.data(2 * keep), ref_out[: 2 * keep])
    assert dout.guards_intact(), "write outside [0, cap)"
    return r


def check_u16_be(ctx, data: np.ndarray, cap_bytes=None, in_off=0, out_off=0):
    """UTF-16BE (bytes, high byte first) -> UTF-8 on the GPU vs the oracle,
    plus the BE length and validation calls."""
    data = np.ascontiguousarray(data, dtype=np.uint8)
    ref, ref_out = oracle.utf16be_to_utf8(data, cap_bytes)
    din = DevIn(data, in_off)
    n = data.size // 2
    cap = 3 * n if cap_bytes is None else cap_bytes
    dout = DevOut(cap, out_off)
    r = gbu.gbu_utf16be_to_utf8(ctx, din.ptr, n, dout.ptr, cap, 0)
    assert triple(r) == triple(ref), (triple(r), triple(ref))
    keep = min(ref.out_len, cap)
    assert np.array_equal(dout.data(keep), ref_out[:keep])
    assert dout.guards_intact(), "write outside [0, cap)"
    lr = gbu.gbu_utf8_length_from_utf16be(ctx, din.ptr, n, 0)
    lref = oracle.utf8_length_from_utf16be(data)
    assert triple(lr) == triple(lref)
    vr = gbu.gbu_validate_utf16be(ctx, din.ptr, n, 0)
    assert triple(vr) == (lref.status, lref.in_offset, 0)
    return r
