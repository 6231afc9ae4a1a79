"""The one-launch path for inputs of a few chunks, against the oracle.

An input that spans at most `small_chunks` chunks (12 KiB each, counted from
the 16-byte boundary at or before it) runs as one thread-block cluster with
one CTA per chunk; longer inputs, and every input when small_chunks is 0, run
on the persistent grid. Both settings must give the oracle's result, output
bytes, lengths and validation results: ragged sizes around every chunk count
up to the path's limit and one past it, every input alignment at the largest
size, injected errors of every kind, too-small outputs, UTF-16BE.
"""
import numpy as np
import pytest

import oracle
import paper_2212_05098_gb300 as gbu
import textgen
from textgen import inject

from gpu_util import check_u16, check_u16_be, check_u8, check_u8_be, triple

pytestmark = pytest.mark.gpu

CHUNK = 12288                      # input bytes of a chunk
LIMIT = gbu.GBU_SMALL_MAX_CHUNKS * CHUNK
SIZES = [1, 2, 3, 15, 16, 17, 100, 4095, 4096, 4097, CHUNK - 1, CHUNK, CHUNK + 1,
         2 * CHUNK + 7, 3 * CHUNK - 3, 5 * CHUNK + 1001, LIMIT - 17, LIMIT - 16, LIMIT,
         LIMIT + 1, LIMIT + 4 * CHUNK]


@pytest.fixture(scope="module", params=["small", "persistent"])
def ctx(request):
    import torch
    torch.cuda.init()
    h = gbu.gbu_create(0)
    small = gbu.GBU_SMALL_MAX_CHUNKS if request.param == "small" else 0
    # the default shape pinned (12 KiB chunks; by size, inputs up to 1 MiB
    # would take the 8 KiB shape)
    assert gbu.gbu_set_tune(h, 1, 0, small, CHUNK, 256) == gbu.GBU_OK
    assert gbu.gbu_get_tune(h).small_chunks == small
    yield h
    gbu.gbu_destroy(h)


def test_tune_limits():
    import torch
    torch.cuda.init()
    h = gbu.gbu_create(0)
    try:
        assert gbu.gbu_get_tune(h).small_chunks == gbu.GBU_SMALL_MAX_CHUNKS   # the default
        assert gbu.gbu_set_tune(h, 1, 0, gbu.GBU_SMALL_MAX_CHUNKS + 1) == gbu.GBU_INVALID_ARG
        assert gbu.gbu_set_tune(h, 1, 0, -1) == gbu.GBU_INVALID_ARG
        assert gbu.gbu_set_tune(h, 1, 0, 3) == gbu.GBU_OK
        assert gbu.gbu_get_tune(h).small_chunks == 3
    finally:
        gbu.gbu_destroy(h)


@pytest.mark.parametrize("profile", ["mix", "latin", "cjk", "emoji"])
def test_ragged_sizes(ctx, profile):
    t8 = textgen.generate(profile, SIZES[-1], textgen.UTF8, seed=140)
    t16 = textgen.generate(profile, 2 * SIZES[-1], textgen.UTF16, seed=141)
    for n in SIZES:
        check_u8(ctx, t8.data[:n])             # may cut a character: TOO_SHORT at its lead
        check_u16(ctx, t16.data[:2 * n])       # may cut a pair: LONE_HIGH at the end


def test_every_alignment_at_the_limit(ctx):
    t8 = textgen.generate("emoji", LIMIT, textgen.UTF8, seed=142)
    t16 = textgen.generate("emoji", LIMIT, textgen.UTF16, seed=143)
    for off in range(16):
        # the largest input of the path at this offset, and one byte more
        for n in (LIMIT - off, LIMIT - off + 1):
            check_u8(ctx, t8.data[:min(n, LIMIT)], in_off=off, out_off=2 * (off % 8))
        if off % 2 == 0:
            n16 = (LIMIT - off) // 2
            check_u16(ctx, t16.data[:2 * n16], in_off=off, out_off=off)


@pytest.mark.parametrize("enc", [textgen.UTF8, textgen.UTF16])
def test_injected_errors(ctx, enc):
    """Every error kind, at chunk edges (4..64 KiB) inside an input of 7.5
    chunks."""
    text = textgen.generate("cjk", 15 * CHUNK // 2, enc, seed=144)
    starts, outs = text.char_starts(), text.out_starts()
    ncases = len(inject.UTF8_CASES if enc == textgen.UTF8 else inject.UTF16_CASES)
    for i in range(3 * ncases):
        p = inject.make_patch(text, i, seed=144, starts=starts, out_starts=outs)
        data = p.apply(text.data)
        r = check_u8(ctx, data) if enc == textgen.UTF8 else check_u16(ctx, data)
        assert triple(r) == (p.kind, p.err_unit, p.prefix_out), p.case


def test_random_corruption(ctx):
    base8 = textgen.generate("mix", 6 * CHUNK + 555, textgen.UTF8, seed=145).data
    base16 = textgen.generate("mix", 6 * CHUNK + 556, textgen.UTF16, seed=146).data
    for i in range(24):
        check_u8(ctx, textgen.mutate(base8, 1 + i % 4, seed=900 + i)[: base8.size - 301 * i])
        words = base16.copy().view("<u2")
        rng = np.random.Generator(np.random.Philox(key=950 + i))
        words[rng.integers(0, words.size, size=1 + i % 3)] = rng.integers(0xD800, 0xE000, size=1 + i % 3)
        check_u16(ctx, words.view(np.uint8)[: base16.size - 2 * 151 * i])


def test_output_too_small(ctx):
    t8 = textgen.generate("cyrillic", 4 * CHUNK + 9, textgen.UTF8, seed=147).data
    t16 = textgen.generate("cyrillic", 4 * CHUNK + 10, textgen.UTF16, seed=148).data
    need8 = oracle.utf8_to_utf16le(t8)[0].out_len
    need16 = oracle.utf16le_to_utf8(t16)[0].out_len
    for cap in (0, 1, 7, CHUNK // 2 + 3, need8 - 1):
        check_u8(ctx, t8, cap_units=cap)
    for cap in (1, 5, CHUNK + 1, need16 - 1):
        check_u16(ctx, t16, cap_bytes=cap)
    # an error inside the part that fits wins over the small output
    bad = t8.copy()
    bad[CHUNK + 5] = 0xFF
    check_u8(ctx, bad, cap_units=need8 // 2)


@pytest.mark.parametrize("profile", ["mix", "emoji"])
def test_utf16be(ctx, profile):
    t8 = textgen.generate(profile, 3 * CHUNK + 77, textgen.UTF8, seed=149).data
    t16 = textgen.generate(profile, 3 * CHUNK + 78, textgen.UTF16, seed=150).data
    be = t16.reshape(-1, 2)[:, ::-1].reshape(-1).copy()
    for n in (1, 17, CHUNK + 1, t8.size):
        check_u8_be(ctx, t8[:n])
    for n in (2, 18, CHUNK + 2, be.size):
        check_u16_be(ctx, be[:n])


SHAPES = [(12288, 256), (8192, 256), (16384, 512), (6144, 128), (24576, 512)]


@pytest.mark.parametrize("shape", SHAPES[1:])
def test_other_shapes(shape):
    """The one-launch path and the persistent grid of every other kernel
    shape, around its own chunk and path limits."""
    import torch
    torch.cuda.init()
    chunk, threads = shape
    limit = gbu.GBU_SMALL_MAX_CHUNKS * chunk
    h = gbu.gbu_create(0)
    try:
        t8 = textgen.generate("emoji", limit + 3 * chunk, textgen.UTF8, seed=152).data
        t16 = textgen.generate("cjk", limit + 3 * chunk, textgen.UTF16, seed=153).data
        bad8 = textgen.mutate(t8, 2, seed=154)
        for small in (gbu.GBU_SMALL_MAX_CHUNKS, 0):
            assert gbu.gbu_set_tune(h, 1, 0, small, chunk, threads) == gbu.GBU_OK
            for n in (1, 17, chunk - 1, chunk, chunk + 1, 3 * chunk + 5, limit - 1, limit,
                      limit + 1, limit + 3 * chunk):
                check_u8(h, t8[:n])
                check_u8(h, bad8[:n])
                check_u16(h, t16[:2 * (n // 2)])
            check_u8(h, t8[:limit - 7], in_off=7)
            check_u16(h, t16[:limit - 6], in_off=6)
    finally:
        gbu.gbu_destroy(h)


def test_call_shape_by_size():
    import torch
    torch.cuda.init()
    h = gbu.gbu_create(0)
    try:
        for n, want in ((1, (8192, 256)), (4096, (8192, 256)), (1 << 20, (8192, 256)),
                        ((1 << 20) + 1, (12288, 256)), (1 << 30, (12288, 256))):
            t = gbu.gbu_call_shape(h, n)
            assert (t.chunk_bytes, t.compute_threads) == want, n
            assert t.small_chunks == gbu.GBU_SMALL_MAX_CHUNKS
        assert gbu.gbu_set_tune(h, 4, 0, 2, 24576, 512) == gbu.GBU_OK
        t = gbu.gbu_call_shape(h, 100)
        assert (t.look_width, t.small_chunks, t.chunk_bytes, t.compute_threads) == (4, 2, 24576, 512)
    finally:
        gbu.gbu_destroy(h)


def test_one_launch_per_call(ctx):
    t8 = textgen.generate("latin", 2 * CHUNK, textgen.UTF8, seed=151).data
    before = gbu.gbu_kernel_launch_count()
    check_u8(ctx, t8)       # transcode, length, validation
    # one launch each on the one-launch path; beyond it a validation is the
    # streaming kernel plus the result kernel
    small = gbu.gbu_get_tune(ctx).small_chunks > 0
    assert gbu.gbu_kernel_launch_count() == before + (3 if small else 4)


def test_concurrent_streams():
    """One-launch calls on several streams at once (they share no scratch):
    every result and output equals the oracle's."""
    import torch
    torch.cuda.init()
    h = gbu.gbu_create(0)
    try:
        streams = [torch.cuda.Stream() for _ in range(4)]
        cases = []
        for i in range(32):
            n = 100 + 2000 * i      # all within the one-launch path (8 chunks of 8 KiB)
            d = textgen.generate(["mix", "emoji", "cjk", "cyrillic"][i % 4], n, textgen.UTF8,
                                 seed=210 + i).data
            if i % 5 == 4:
                d = textgen.mutate(d, 1, seed=260 + i)
            din = torch.from_numpy(np.array(d, copy=True)).cuda()
            dout = torch.zeros(2 * n + 16, dtype=torch.uint8, device="cuda")
            res = torch.zeros(4, dtype=torch.int64, device="cuda")
            cases.append((d, din, dout, res))
        torch.cuda.synchronize()
        for i, (d, din, dout, res) in enumerate(cases):
            s = streams[i % len(streams)]
            assert gbu.gbu_utf8_to_utf16le_async(h, din.data_ptr(), d.size, dout.data_ptr(), d.size,
                                                 res.data_ptr(), s.cuda_stream) == gbu.GBU_OK
        torch.cuda.synchronize()
        for d, din, dout, res in cases:
            ref, ref_out = oracle.utf8_to_utf16le(d)
            r = res.cpu().numpy()
            assert (int(r[0]) & 0xFFFFFFFF, int(r[1]), int(r[2])) == triple(ref)
            n = min(ref.out_len, d.size)
            assert np.array_equal(dout.cpu().numpy()[: 2 * n].view("<u2"), ref_out[:n])
    finally:
        gbu.gbu_destroy(h)
