"""The validation-only calls on the streaming kernel (inputs longer than the
one-launch path) against the oracle: errors planted at the edges of a
thread's 32 bytes, of a warp's 1 KiB and of a CTA's 8 KiB, at the first and
last positions, at every input alignment, for UTF-8, UTF-16LE and UTF-16BE."""
import numpy as np
import pytest

import oracle
import paper_2212_05098_gb300 as gbu
import textgen

from gpu_util import DevIn, triple

pytestmark = pytest.mark.gpu

N = 300_000   # bytes: beyond the one-launch path of every size class


@pytest.fixture(scope="module")
def ctx():
    import torch
    torch.cuda.init()
    h = gbu.gbu_create(0)
    yield h
    gbu.gbu_destroy(h)


def _check8(ctx, data, off):
    want = oracle.utf16_length_from_utf8(data)
    d = DevIn(data, off)
    got = gbu.gbu_validate_utf8(ctx, d.ptr, data.size, 0)
    assert triple(got) == (want.status, want.in_offset, 0), (off, triple(got), triple(want))


def _check16(ctx, data, off, be=False):
    want = oracle.utf8_length_from_utf16le(data)
    src = data.reshape(-1, 2)[:, ::-1].reshape(-1).copy() if be else data
    d = DevIn(src, off)
    f = gbu.gbu_validate_utf16be if be else gbu.gbu_validate_utf16le
    got = f(ctx, d.ptr, data.size // 2, 0)
    assert triple(got) == (want.status, want.in_offset, 0), (off, be, triple(got), triple(want))


EDGES = [0, 1, 2, 3, 29, 30, 31, 32, 33, 1021, 1022, 1023, 1024, 1025, 8190, 8191, 8192, 8193]
PATTERNS8 = [b"\x80", b"\xc1\xbf", b"\xe0\x9f\x80", b"\xed\xa0\x80", b"\xf0\x8f\x80\x80",
             b"\xf4\x90\x80\x80", b"\xf5", b"\xe4\xb8", b"\xf0\x9f\x98"]


def test_valid_inputs_every_alignment(ctx):
    for prof in ("mix", "cjk", "emoji"):
        t8 = textgen.generate(prof, N, textgen.UTF8, seed=160).data
        t16 = textgen.generate(prof, N, textgen.UTF16, seed=161).data
        for off in range(16):
            _check8(ctx, t8, off)
            if off % 2 == 0:
                _check16(ctx, t16, off)
                _check16(ctx, t16, off, be=True)


def test_utf8_errors_at_block_edges(ctx):
    base = textgen.generate("cjk", N, textgen.UTF8, seed=162).data
    rng = np.random.default_rng(163)
    for k, pat in enumerate(PATTERNS8):
        for e in EDGES + [N - 1, N - 2, N - 3, N - 4]:
            for shift in (0, -1, -2):
                p = e + shift
                if p < 0 or p >= N:
                    continue
                data = base.copy()
                q = min(p, N - len(pat))
                data[q:q + len(pat)] = np.frombuffer(pat, np.uint8)
                _check8(ctx, data, int(rng.integers(0, 16)))


def test_utf16_errors_at_block_edges(ctx):
    base = textgen.generate("emoji", N, textgen.UTF16, seed=164).data
    units = N // 2
    rng = np.random.default_rng(165)
    for e in [0, 1, 14, 15, 16, 17, 511, 512, 513, 4095, 4096, 4097, units - 2, units - 1]:
        for bad in (0xD83D, 0xDE00):           # a lone high or low surrogate
            data = base.copy()
            w = data.view("<u2")
            w[e] = bad
            if e + 1 < units and bad == 0xD83D:
                w[e + 1] = 0x0041
            if e > 0 and bad == 0xDE00:
                w[e - 1] = 0x0041
            off = 2 * int(rng.integers(0, 8))
            _check16(ctx, data, off)
            _check16(ctx, data, off, be=True)


def test_utf16_surrogates_in_bmp_text(ctx):
    """Surrogates alone in text without them (threads holding no surrogate
    skip the pairing check): lone halves and valid pairs at the edges of a
    thread's 16 units, a warp's 512 and a CTA's 4096, with their neighbours
    surrogate-free."""
    base = textgen.generate("cjk", N, textgen.UTF16, seed=166).data
    units = N // 2
    rng = np.random.default_rng(167)
    edges = [0, 1, 14, 15, 16, 17, 31, 32, 511, 512, 4095, 4096, units - 2, units - 1]
    for e in edges:
        for case in ("high", "low", "pair", "pair+lone"):
            data = base.copy()
            w = data.view("<u2")
            if case == "high":
                w[e] = 0xDBFF
            elif case == "low":
                w[e] = 0xDC00
            elif e + 1 < units:
                w[e], w[e + 1] = 0xD83D, 0xDE00     # valid: no error
                if case == "pair+lone" and e + 3 < units:
                    w[e + 3] = 0xDFFF                # a lone low two units on
            off = 2 * int(rng.integers(0, 8))
            _check16(ctx, data, off)
            _check16(ctx, data, off, be=True)


def test_random_and_corrupted(ctx):
    for i in range(12):
        d = textgen.random_bytes(N + 977 * i, seed=170 + i)
        _check8(ctx, d, i % 16)
        _check16(ctx, d[: d.size - (d.size % 2)], 2 * (i % 8))
        t = textgen.generate("emoji", N, textgen.UTF8, seed=180 + i).data
        _check8(ctx, textgen.mutate(t, 1 + i % 3, seed=190 + i), (3 * i) % 16)


def test_two_launches_and_reuse(ctx):
    t = textgen.generate("mix", N, textgen.UTF8, seed=200).data
    bad = t.copy()
    bad[N // 2] = 0xFF
    before = gbu.gbu_kernel_launch_count()
    for data in (bad, t, bad, t):           # the error word is reset by every call
        _check8(ctx, data, 0)
    assert gbu.gbu_kernel_launch_count() == before + 8


def test_async_results_in_device_memory(ctx):
    """The asynchronous validation calls on the streaming kernel, results in
    device memory, one call after another on a stream."""
    import torch
    s = torch.cuda.Stream()
    res = torch.zeros((6, 4), dtype=torch.int64, device="cuda")
    datas, wants = [], []
    for i in range(6):
        t = textgen.generate(["mix", "cjk", "emoji"][i % 3], N + 1000 * i,
                             textgen.UTF8 if i % 2 == 0 else textgen.UTF16, seed=220 + i).data
        if i >= 3:
            t = textgen.mutate(t, 1, seed=230 + i)
        datas.append(DevIn(t, 2 * i))
        wants.append(oracle.utf16_length_from_utf8(t) if i % 2 == 0
                     else oracle.utf8_length_from_utf16le(t))
    torch.cuda.synchronize()
    for i, d in enumerate(datas):
        if i % 2 == 0:
            st = gbu.gbu_validate_utf8_async(ctx, d.ptr, d.nbytes, res[i].data_ptr(), s.cuda_stream)
        else:
            st = gbu.gbu_validate_utf16le_async(ctx, d.ptr, d.nbytes // 2, res[i].data_ptr(),
                                                s.cuda_stream)
        assert st == gbu.GBU_OK
    s.synchronize()
    h = res.cpu().numpy()
    for i, w in enumerate(wants):
        assert (int(h[i, 0]) & 0xFFFFFFFF, int(h[i, 1]), int(h[i, 2])) == (w.status, w.in_offset, 0)
