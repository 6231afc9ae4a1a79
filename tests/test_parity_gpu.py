"""GPU parity: the CUDA path, called through the C ABI, against the oracle.

Bit-exact on output bytes, status, first-error offset and output length, on
seeded synthetic text of every profile, at sizes that span several chunks
with ragged tails, at every input/output alignment, with random corruption,
with too-small outputs (canary-guarded), and on the paper's worked examples.
"""
import os

import numpy as np
import pytest

import oracle
import paper_2212_05098_gb300 as gbu
import textgen
from textgen import inject

from gpu_util import (DevIn, DevOut, check_u16, check_u8, gpu_u8_to_u16, triple)

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def ctx():
    import torch
    torch.cuda.init()
    h = gbu.gbu_create(0)
    yield h
    gbu.gbu_destroy(h)


def _golden(name):
    with open(os.path.join(HERE, "golden", name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                yield [c.strip() for c in line.split("|")]


def test_paper_examples(ctx):
    for row in _golden("fig1b_examples.txt"):
        words = np.array([int(w, 2) for w in row[1].split()], dtype="<u2")
        utf8 = np.array([int(b, 2) for b in row[2].split()], dtype=np.uint8)
        r = check_u8(ctx, utf8)
        assert r.status == gbu.GBU_OK and r.out_len == words.size
        r = check_u16(ctx, words.view(np.uint8))
        assert r.status == gbu.GBU_OK and r.out_len == utf8.size
    for row in _golden("worked_examples.txt"):
        data = np.frombuffer(bytes.fromhex(row[1]), dtype=np.uint8)
        check_u8(ctx, data)
        _, out = oracle.utf8_to_utf16le(data)
        check_u16(ctx, out.view(np.uint8))


def test_mix_1mib_seed0(ctx):
    """1 MiB of the 60/25/10/5 mix, seed 0, both directions."""
    t8 = textgen.generate("mix", 1 << 20, textgen.UTF8, seed=0)
    r = check_u8(ctx, t8.data)
    assert r.status == gbu.GBU_OK
    t16 = textgen.generate("mix", 1 << 20, textgen.UTF16, seed=0)
    r = check_u16(ctx, t16.data)
    assert r.status == gbu.GBU_OK


SIZES = [1, 2, 3, 4, 15, 16, 17, 31, 32, 33, 255, 4095, 4096, 4097, 8191, 8192, 8193,
         3 * 8192 + 123, 100_003, (1 << 20) + 5]


@pytest.mark.parametrize("profile", list(textgen.PROFILES))
def test_profiles_ragged_sizes(ctx, profile):
    big8 = textgen.generate(profile, SIZES[-1] + 16, textgen.UTF8, seed=21)
    big16 = textgen.generate(profile, 2 * (SIZES[-1] + 16), textgen.UTF16, seed=22)
    for n in SIZES:
        check_u8(ctx, big8.data[:n])            # may cut a character: TOO_SHORT at its lead
        check_u16(ctx, big16.data[:2 * n])      # may cut a pair: LONE_HIGH at the end


def test_every_alignment(ctx):
    t8 = textgen.generate("emoji", 70_001, textgen.UTF8, seed=31)
    t16 = textgen.generate("emoji", 2 * 40_001, textgen.UTF16, seed=32)
    for off in range(16):
        check_u8(ctx, t8.data, in_off=off, out_off=2 * (off % 8))
        check_u16(ctx, t16.data, in_off=2 * (off % 8), out_off=off)


@pytest.mark.parametrize("profile", ["mix", "cjk", "emoji"])
def test_fuzz_corrupted(ctx, profile):
    base8 = textgen.generate(profile, 40_000, textgen.UTF8, seed=41)
    base16 = textgen.generate(profile, 80_000, textgen.UTF16, seed=42)
    for i in range(40):
        d = textgen.mutate(base8.data, 1 + i % 3, seed=500 + i)
        check_u8(ctx, d[: 40_000 - 37 * i])
        words = base16.data.copy().view("<u2")
        rng = np.random.Generator(np.random.Philox(key=600 + i))
        words[rng.integers(0, words.size, size=1 + i % 3)] = rng.integers(0xD800, 0xE000, size=1 + i % 3)
        check_u16(ctx, words.view(np.uint8)[: 80_000 - 46 * i])


def test_random_bytes(ctx):
    for i in range(30):
        d = textgen.random_bytes(1 + 997 * i, seed=700 + i)
        check_u8(ctx, d)
        check_u16(ctx, d[: d.size - (d.size % 2)])


def test_all_scalars(ctx):
    cps = np.concatenate([np.arange(0, 0xD800), np.arange(0xE000, 0x110000)]).astype(np.uint32)
    s = cps.astype("<u4").tobytes().decode("utf-32-le")
    check_u8(ctx, np.frombuffer(s.encode("utf-8"), np.uint8))
    check_u16(ctx, np.frombuffer(s.encode("utf-16-le"), np.uint8))


def test_output_too_small_and_canaries(ctx):
    t8 = textgen.generate("cjk", 50_000, textgen.UTF8, seed=51)
    full, _ = oracle.utf8_to_utf16le(t8.data)
    for cap in [0, 1, 7, 8, 9, full.out_len // 2, full.out_len - 1, full.out_len]:
        r = check_u8(ctx, t8.data, cap_units=cap, out_off=2 * (cap % 8))
        assert r.status == (gbu.GBU_OK if cap >= full.out_len else gbu.GBU_OUTPUT_TOO_SMALL)
    t16 = textgen.generate("emoji", 60_000, textgen.UTF16, seed=52)
    full, _ = oracle.utf16le_to_utf8(t16.data)
    for cap in [0, 1, 3, 15, 16, 17, full.out_len // 3, full.out_len - 1, full.out_len]:
        r = check_u16(ctx, t16.data, cap_bytes=cap, out_off=cap % 16)
        assert r.status == (gbu.GBU_OK if cap >= full.out_len else gbu.GBU_OUTPUT_TOO_SMALL)


def test_error_beats_small_output(ctx):
    d = np.frombuffer(bytes.fromhex("41 42 43 80 44"), np.uint8)
    r = check_u8(ctx, d, cap_units=1)
    assert triple(r) == (gbu.GBU_TOO_LONG, 3, 3)


def test_empty_input(ctx):
    r, _ = gpu_u8_to_u16(ctx, np.zeros(0, np.uint8))
    assert triple(r) == (gbu.GBU_OK, 0, 0)
    d = DevOut(16)
    r = gbu.gbu_utf16le_to_utf8(ctx, d.ptr, 0, d.ptr, 16, 0)
    assert triple(r) == (gbu.GBU_OK, 0, 0)


def test_invalid_arguments(ctx):
    d = DevOut(64)
    assert gbu.gbu_utf16le_to_utf8(ctx, d.ptr + 1, 4, d.ptr, 16, 0).status == gbu.GBU_INVALID_ARG
    assert gbu.gbu_utf8_to_utf16le(ctx, d.ptr, 4, d.ptr + 1, 16, 0).status == gbu.GBU_INVALID_ARG
    assert gbu.gbu_utf8_to_utf16le(ctx, d.ptr, 1 << 40, d.ptr, 16, 0).status == gbu.GBU_INVALID_ARG


def test_async_result_in_device_memory(ctx):
    import torch
    t8 = textgen.generate("latin", 300_000, textgen.UTF8, seed=61)
    din = DevIn(t8.data)
    dout = DevOut(2 * t8.data.size)
    res = torch.zeros(4, dtype=torch.int64, device="cuda")     # 32 bytes >= sizeof(gbu_result)
    stream = torch.cuda.Stream()
    st = gbu.gbu_utf8_to_utf16le_async(ctx, din.ptr, t8.data.size, dout.ptr, t8.data.size,
                                       res.data_ptr(), stream.cuda_stream)
    assert st == gbu.GBU_OK
    stream.synchronize()
    h = res.cpu().numpy()
    status = int(h[0] & 0xFFFFFFFF)
    ref, ref_out = oracle.utf8_to_utf16le(t8.data)
    assert (status, int(h[1]), int(h[2])) == triple(ref)
    assert np.array_equal(dout.data(2 * ref.out_len), ref_out.view(np.uint8))
    # length-only, async, other direction
    t16 = textgen.generate("cyrillic", 200_000, textgen.UTF16, seed=62)
    din16 = DevIn(t16.data)
    st = gbu.gbu_utf8_length_from_utf16le_async(ctx, din16.ptr, t16.data.size // 2,
                                                res.data_ptr(), stream.cuda_stream)
    assert st == gbu.GBU_OK
    stream.synchronize()
    h = res.cpu().numpy()
    assert (int(h[0] & 0xFFFFFFFF), int(h[1]), int(h[2])) == triple(oracle.utf8_length_from_utf16le(t16.data))


def test_host_buffer_api(ctx):
    import ctypes
    t8 = textgen.generate("mix", 123_457, textgen.UTF8, seed=71)
    out = np.zeros(t8.data.size, dtype="<u2")
    r = gbu.gbu_utf8_to_utf16le_host(ctx, t8.data.ctypes.data, t8.data.size,
                                     out.ctypes.data, out.size, 0)
    ref, ref_out = oracle.utf8_to_utf16le(t8.data)
    assert triple(r) == triple(ref)
    assert np.array_equal(out[: ref.out_len], ref_out)
    t16 = textgen.generate("emoji", 2 * 77_777, textgen.UTF16, seed=72)
    out8 = np.zeros(3 * t16.data.size // 2, dtype=np.uint8)
    r = gbu.gbu_utf16le_to_utf8_host(ctx, t16.data.ctypes.data, t16.data.size // 2,
                                     out8.ctypes.data, out8.size, 0)
    ref, ref_out = oracle.utf16le_to_utf8(t16.data)
    assert triple(r) == triple(ref)
    assert np.array_equal(out8[: ref.out_len], ref_out)


@pytest.mark.parametrize("enc", [textgen.UTF8, textgen.UTF16])
def test_injected_errors_at_chunk_edges(ctx, enc):
    """Every error kind, including sequences cut exactly at 4..64 KiB edges."""
    text = textgen.generate("cjk", 1 << 22, enc, seed=81)
    starts, outs = text.char_starts(), text.out_starts()
    ncases = len(inject.UTF8_CASES if enc == textgen.UTF8 else inject.UTF16_CASES)
    for i in range(5 * ncases):
        p = inject.make_patch(text, i, seed=81, starts=starts, out_starts=outs)
        data = p.apply(text.data)
        r = check_u8(ctx, data) if enc == textgen.UTF8 else check_u16(ctx, data)
        assert triple(r) == (p.kind, p.err_unit, p.prefix_out), p.case


@pytest.mark.parametrize("profile", list(textgen.PROFILES))
def test_utf16be_both_directions(ctx, profile):
    """UTF-16BE forms: ragged sizes, both directions, corrupted copies."""
    from gpu_util import check_u16_be, check_u8_be
    big8 = textgen.generate(profile, 3 * 8192 + 200, textgen.UTF8, seed=61)
    t16 = textgen.generate(profile, 2 * (3 * 8192 + 200), textgen.UTF16, seed=62)
    be16 = t16.data.reshape(-1, 2)[:, ::-1].reshape(-1).copy()
    for n in (1, 2, 17, 4095, 4096, 4097, 8193, 3 * 8192 + 101):
        check_u8_be(ctx, big8.data[:n])
        check_u16_be(ctx, be16[: 2 * n])
    check_u8_be(ctx, big8.data, in_off=3, out_off=6)
    check_u16_be(ctx, be16, in_off=2, out_off=5)
    for k in range(4):
        check_u8_be(ctx, textgen.mutate(big8.data, 2, seed=63 + k))
        bad = be16.copy().view(">u2")
        bad[1000 + 3000 * k] = 0xDC00 + k      # lone low surrogate
        check_u16_be(ctx, bad.view(np.uint8))
    check_u8_be(ctx, big8.data, cap_units=100)
    check_u16_be(ctx, be16, cap_bytes=333)


def _patchwork(seed: int, n_runs: int = 300):
    """Code points in runs of a few hundred bytes, each run from one text
    class (ASCII only, or one profile), so that neighbouring warps of a chunk
    see different classes of text and pick different paths."""
    rng = np.random.Generator(np.random.Philox(key=seed))
    profiles = ["latin", "cyrillic", "cjk", "emoji", "mix"]
    parts = []
    for i in range(n_runs):
        nbytes = int(rng.integers(40, 2600))
        k = int(rng.integers(len(profiles) + 1))
        if k == len(profiles):
            parts.append(rng.integers(0x20, 0x7F, size=nbytes).astype(np.uint32))
        else:
            parts.append(textgen.generate(profiles[k], nbytes, textgen.UTF8,
                                          seed=seed * 1000 + i).cps)
    return np.concatenate(parts)


@pytest.mark.parametrize("seed", [71, 72, 73])
def test_mixed_classes_per_warp(ctx, seed):
    """Text whose class changes every few hundred bytes, valid and with one
    injected error, in both directions: the per-warp paths (ASCII / 2-byte /
    3-byte / 4-byte leads, 1-2-byte / BMP / surrogate UTF-16) meet at
    arbitrary positions inside chunks and threads."""
    cps = _patchwork(seed)
    d8 = textgen.encode(cps, textgen.UTF8).copy()
    d16 = textgen.encode(cps, textgen.UTF16).copy()
    check_u8(ctx, d8)
    check_u16(ctx, d16)
    rng = np.random.Generator(np.random.Philox(key=seed + 100))
    for i in range(6):
        bad8 = d8.copy()
        bad8[int(rng.integers(bad8.size))] = [0xFF, 0x80, 0xC0, 0xED][i % 4]
        check_u8(ctx, bad8[: bad8.size - 13 * i])
        words = d16.copy().view("<u2")
        words[int(rng.integers(words.size))] = [0xD800, 0xDC00, 0xDBFF][i % 3]
        check_u16(ctx, words.view(np.uint8)[: d16.size - 26 * i])
