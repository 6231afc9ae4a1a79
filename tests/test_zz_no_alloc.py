"""The no-allocation entry point (gbu_utf8_to_utf16le_noalloc), on the GPU.

It serves callers that may not allocate device memory; its scratch is a
fixed device array inside the library, shared by every call. The tests call
it through the C ABI and compare it with the oracle directly (ragged sizes,
every input alignment, injected errors, the largest accepted input at the
worst alignment), and with the regular context-based entry point on two
calls in a row (the second call runs on whatever the first left in the
shared array). Kept in its own file, named to be collected last.
"""
import numpy as np
import pytest

import oracle
import paper_2212_05098_gb300 as gbu
import textgen

from gpu_util import DevIn, DevOut, triple

pytestmark = pytest.mark.gpu


def _regular(ctx, data):
    din, dout = DevIn(data), DevOut(2 * data.size)
    r = gbu.gbu_utf8_to_utf16le(ctx, din.ptr, data.size, dout.ptr, data.size, 0)
    return r, dout.data(2 * min(r.out_len, data.size))


def _noalloc(data, in_off=0, cap=None, stream=0):
    cap = data.size if cap is None else cap
    din, dout = DevIn(data, in_off), DevOut(2 * cap)
    r = gbu.gbu_utf8_to_utf16le_noalloc(din.ptr, data.size, dout.ptr, cap, stream)
    assert dout.guards_intact()
    return r, dout.data(2 * min(r.out_len, cap))


def _check_oracle(data, in_off=0, cap=None):
    ref, ref_out = oracle.utf8_to_utf16le(data, cap)
    got, out = _noalloc(data, in_off, cap)
    assert triple(got) == triple(ref), (data.size, in_off)
    n = min(ref.out_len, data.size if cap is None else cap)
    assert np.array_equal(out.view("<u2")[:n], ref_out[:n])


def test_noalloc_matches_regular_twice():
    import torch
    torch.cuda.init()
    ctx = gbu.gbu_create(0)
    try:
        first = textgen.generate("emoji", 3 * (1 << 20) + 77, textgen.UTF8, seed=91).data
        second = textgen.mutate(textgen.generate("cjk", 1 << 20, textgen.UTF8, seed=92).data,
                                1, seed=93)
        for data, off in ((first, 0), (second, 5)):
            want_r, want = _regular(ctx, data)
            got_r, got = _noalloc(data, off)
            assert triple(got_r) == triple(want_r)
            assert np.array_equal(got, want)
        assert triple(_noalloc(first)[0])[0] == gbu.GBU_OK
    finally:
        gbu.gbu_destroy(ctx)


@pytest.mark.parametrize("size", [1, 15, 16, 17, 1000, 12287, 12288, 12289, 3 * 12288 + 5,
                                  (1 << 20) + 7])
def test_noalloc_ragged_sizes_against_oracle(size):
    _check_oracle(textgen.generate("mix", size, textgen.UTF8, seed=110 + size % 97).data)


def test_noalloc_every_alignment_against_oracle():
    data = textgen.generate("mix", 200_003, textgen.UTF8, seed=120).data
    for off in range(16):
        _check_oracle(data, off)


def test_noalloc_injected_errors_and_small_capacity():
    base = textgen.generate("cyrillic", 300_000, textgen.UTF8, seed=121).data
    for k in range(6):
        _check_oracle(textgen.mutate(base, 1, seed=130 + k), in_off=k)
    _check_oracle(base, cap=1000)     # OUTPUT_TOO_SMALL, nothing written past cap


def test_noalloc_largest_input_at_worst_alignment():
    data = textgen.generate("emoji", gbu.GBU_NOALLOC_MAX_BYTES, textgen.UTF8, seed=122,
                            keep_cps=False, keep_lens=False).data
    _check_oracle(data, in_off=15)


def test_noalloc_on_a_stream_and_launch_count():
    import torch
    s = torch.cuda.Stream()
    data = textgen.generate("latin", 50_000, textgen.UTF8, seed=123).data
    before = gbu.gbu_kernel_launch_count()
    got, out = _noalloc(data, stream=s.cuda_stream)
    ref, ref_out = oracle.utf8_to_utf16le(data)
    assert triple(got) == triple(ref)
    assert np.array_equal(out.view("<u2"), ref_out)
    assert gbu.gbu_kernel_launch_count() == before + 1


def test_noalloc_rejects_inputs_above_the_limit():
    d = DevOut(64)
    r = gbu.gbu_utf8_to_utf16le_noalloc(d.ptr, gbu.GBU_NOALLOC_MAX_BYTES + 1, d.ptr, 16, 0)
    assert r.status == gbu.GBU_INVALID_ARG
