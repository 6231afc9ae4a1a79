"""GPU parity of the UTF-32LE calls against the oracle: results, output
bytes and canaries, for every text profile at ragged sizes, invalid UTF-32
units and invalid UTF-8 at tile edges, small capacities, lengths and
validation, empty input and misaligned pointers."""
import numpy as np
import pytest

import oracle
import paper_2212_05098_gb300 as gbu
import textgen

from gpu_util import DevIn, DevOut, triple

pytestmark = pytest.mark.gpu

TILE32 = 2048     # UTF-32 units per tile of the UTF-32 kernels
TILE8 = 8192      # UTF-8 bytes per tile


@pytest.fixture(scope="module")
def ctx():
    import torch
    torch.cuda.init()
    h = gbu.gbu_create(0)
    yield h
    gbu.gbu_destroy(h)


def check_u32_to_u8(ctx, units: np.ndarray, cap_bytes=None, out_off=0):
    units = np.ascontiguousarray(units, dtype="<u4")
    data = units.view(np.uint8)
    n = units.size
    if cap_bytes is None:
        cap_bytes = 4 * n
    ref, ref_out = oracle.utf32le_to_utf8(data, cap_bytes)
    din = DevIn(data, 0)
    dout = DevOut(cap_bytes, out_off)
    r = gbu.gbu_utf32le_to_utf8(ctx, din.ptr, n, dout.ptr, cap_bytes, 0)
    assert triple(r) == triple(ref), (triple(r), triple(ref))
    keep = min(ref.out_len, cap_bytes)
    assert np.array_equal(dout.data(keep), ref_out[:keep])
    assert dout.guards_intact(), "write outside [0, cap)"
    lr = gbu.gbu_utf8_length_from_utf32le(ctx, din.ptr, n, 0)
    lref = oracle.utf8_length_from_utf32le(data)
    assert triple(lr) == triple(lref), (triple(lr), triple(lref))
    vr = gbu.gbu_validate_utf32le(ctx, din.ptr, n, 0)
    assert triple(vr) == (lref.status, lref.in_offset, 0)
    return r


def check_u8_to_u32(ctx, data: np.ndarray, cap_units=None, in_off=0):
    data = np.ascontiguousarray(data, dtype=np.uint8)
    if cap_units is None:
        cap_units = data.size
    ref, ref_out = oracle.utf8_to_utf32le(data, cap_units)
    din = DevIn(data, in_off)
    dout = DevOut(4 * cap_units, 0)
    r = gbu.gbu_utf8_to_utf32le(ctx, din.ptr, data.size, dout.ptr, cap_units, 0)
    assert triple(r) == triple(ref), (triple(r), triple(ref))
    keep = min(ref.out_len, cap_units)
    assert np.array_equal(dout.data(4 * keep), ref_out[:keep].view(np.uint8))
    assert dout.guards_intact(), "write outside [0, cap)"
    lr = gbu.gbu_utf32_length_from_utf8(ctx, din.ptr, data.size, 0)
    lref = oracle.utf32_length_from_utf8(data)
    assert triple(lr) == triple(lref), (triple(lr), triple(lref))
    return r


@pytest.mark.parametrize("profile", list(textgen.PROFILES))
def test_profiles_both_directions(ctx, profile):
    for k, nbytes in enumerate([1, 3, 257, TILE8 - 1, TILE8 + 5, 3 * TILE8 + 1001, 200_003]):
        t = textgen.generate(profile, nbytes, textgen.UTF8, seed=300 + k)
        r = check_u8_to_u32(ctx, t.data, in_off=k % 5)
        assert r.status == gbu.GBU_OK
        units = t.cps.astype("<u4") if t.cps is not None else oracle.utf8_to_utf32le(t.data)[1]
        r = check_u32_to_u8(ctx, units, out_off=k % 3)
        assert r.status == gbu.GBU_OK


def test_invalid_utf32_units_at_tile_edges(ctx):
    base = textgen.generate("emoji", 3 * 4 * TILE32, textgen.UTF8, seed=31)
    units = oracle.utf8_to_utf32le(base.data)[1]
    assert units.size > 3 * TILE32
    for pos in [0, 1, TILE32 - 1, TILE32, TILE32 + 1, 2 * TILE32 - 1, units.size - 1, 777]:
        for bad in (0xD800, 0xDFFF, 0x110000, 0xFFFFFFFF):
            u = units.copy()
            u[pos] = bad
            r = check_u32_to_u8(ctx, u)
            assert r.in_offset == pos
    # two errors: the first one counts
    u = units.copy()
    u[TILE32 + 3] = 0x110000
    u[5] = 0xDC00
    assert check_u32_to_u8(ctx, u).in_offset == 5


def test_invalid_utf8_and_tile_edges(ctx):
    base = textgen.generate("mix", 3 * TILE8 + 100, textgen.UTF8, seed=32).data
    for i, pos in enumerate([0, 5, TILE8 - 1, TILE8, TILE8 + 1, 2 * TILE8 - 2, base.size - 1]):
        d = base.copy()
        d[pos] = [0xFF, 0x80, 0xC0, 0xED][i % 4]
        check_u8_to_u32(ctx, d)
    for i in range(8):
        check_u8_to_u32(ctx, textgen.mutate(base, 1 + i % 3, seed=900 + i)[: base.size - 11 * i])


def test_small_capacities(ctx):
    t = textgen.generate("emoji", 5 * TILE8, textgen.UTF8, seed=33)
    units = oracle.utf8_to_utf32le(t.data)[1]
    for cap in [0, 1, 7, TILE32, units.size - 1]:
        r = check_u8_to_u32(ctx, t.data, cap_units=cap)
        assert r.status == gbu.GBU_OUTPUT_TOO_SMALL
    need = oracle.utf8_length_from_utf32le(units).out_len
    for cap in [0, 1, 4, 4 * TILE32 + 3, need - 1]:
        r = check_u32_to_u8(ctx, units, cap_bytes=cap)
        assert r.status == gbu.GBU_OUTPUT_TOO_SMALL and r.out_len == need


def test_empty_and_misaligned(ctx):
    import torch
    buf = torch.zeros(64, dtype=torch.uint8, device="cuda")
    p = buf.data_ptr()
    r = gbu.gbu_utf32le_to_utf8(ctx, p, 0, p, 0, 0)
    assert triple(r) == (gbu.GBU_OK, 0, 0)
    r = gbu.gbu_utf8_to_utf32le(ctx, p, 0, p, 0, 0)
    assert triple(r) == (gbu.GBU_OK, 0, 0)
    assert gbu.gbu_utf32le_to_utf8(ctx, p + 2, 4, p, 64, 0).status == gbu.GBU_INVALID_ARG
    assert gbu.gbu_utf8_to_utf32le(ctx, p, 4, p + 2, 4, 0).status == gbu.GBU_INVALID_ARG
    assert gbu.gbu_validate_utf32le(ctx, p + 1, 4, 0).status == gbu.GBU_INVALID_ARG
