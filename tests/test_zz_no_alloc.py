"""The no-allocation entry point (gbu_utf8_to_utf16le_noalloc), on the GPU.

It serves callers that may not allocate device memory; its scratch is a
fixed device array inside the library. The test calls it through the C ABI
twice in a row (the second call runs on whatever the first left in the
shared array) and checks each result and output against the regular
context-based entry point, bit for bit. Kept in its own file, named to be
collected last.
"""
import numpy as np
import pytest

import paper_2212_05098_gb300 as gbu
import textgen

from gpu_util import DevIn, DevOut, triple

pytestmark = pytest.mark.gpu


def _regular(ctx, data):
    din, dout = DevIn(data), DevOut(2 * data.size)
    r = gbu.gbu_utf8_to_utf16le(ctx, din.ptr, data.size, dout.ptr, data.size, 0)
    return r, dout.data(2 * min(r.out_len, data.size))


def _noalloc(data, in_off=0):
    din, dout = DevIn(data, in_off), DevOut(2 * data.size)
    r = gbu.gbu_utf8_to_utf16le_noalloc(din.ptr, data.size, dout.ptr, data.size, 0)
    assert dout.guards_intact()
    return r, dout.data(2 * min(r.out_len, data.size))


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


def test_noalloc_rejects_inputs_above_the_limit():
    d = DevOut(64)
    r = gbu.gbu_utf8_to_utf16le_noalloc(d.ptr, gbu.GBU_NOALLOC_MAX_BYTES + 1, d.ptr, 16, 0)
    assert r.status == gbu.GBU_INVALID_ARG
