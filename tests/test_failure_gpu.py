"""Failure detection of the single-pass scan, on the GPU, without faulting it.

Every wait inside the kernels is bounded by a limit of GPU global time. The
tests shorten the limit to a few milliseconds and make a launch skip its
first chunks from the host (gbu_test_skip_chunks): the look-back of the chunk
after them then waits for a prefix that nobody publishes. Nothing faults, no
wait is unbounded, and the launch must report GBU_DEVICE_TIMEOUT; a launch
that processes no chunk at all must report GBU_DEVICE_ERROR (its chunk count
does not add up). The next call on the same context must again match the
oracle exactly.
"""
import time

import numpy as np
import pytest

import paper_2212_05098_gb300 as gbu
import textgen

from gpu_util import check_u16, check_u8, gpu_u16_to_u8, gpu_u8_to_u16, triple

pytestmark = pytest.mark.gpu

SHORT_NS = 2_000_000   # 2 ms


@pytest.fixture()
def ctx():
    import torch
    torch.cuda.init()
    c = gbu.gbu_create(0)
    assert c
    yield c
    gbu.gbu_destroy(c)


def test_wait_limit_arguments(ctx):
    assert gbu.gbu_set_wait_limit(ctx, 61 * 10**9) == gbu.GBU_INVALID_ARG
    assert gbu.gbu_set_wait_limit(ctx, SHORT_NS) == gbu.GBU_OK
    assert gbu.gbu_set_wait_limit(ctx, 0) == gbu.GBU_OK
    assert gbu.gbu_set_wait_limit(0, SHORT_NS) == gbu.GBU_INVALID_ARG
    assert gbu.gbu_test_skip_chunks(0, 1) == gbu.GBU_INVALID_ARG


def test_short_limit_does_not_fire_on_normal_calls(ctx):
    assert gbu.gbu_set_wait_limit(ctx, SHORT_NS) == gbu.GBU_OK
    t8 = textgen.generate("emoji", 3 << 20, textgen.UTF8, seed=96).data
    t16 = textgen.generate("cjk", 2 << 20, textgen.UTF16, seed=97).data
    for _ in range(3):
        check_u8(ctx, t8)
        check_u16(ctx, t16)


@pytest.mark.parametrize("direction", ["utf8", "utf16"])
def test_skipped_chunks_time_out_and_context_recovers(ctx, direction):
    assert gbu.gbu_set_wait_limit(ctx, SHORT_NS) == gbu.GBU_OK
    if direction == "utf8":
        data = textgen.generate("cjk", 1 << 20, textgen.UTF8, seed=98).data   # dozens of chunks
        run, check = gpu_u8_to_u16, check_u8
    else:
        data = textgen.generate("emoji", 1 << 20, textgen.UTF16, seed=99).data
        run, check = gpu_u16_to_u8, check_u16
    check(ctx, data)
    assert gbu.gbu_test_skip_chunks(ctx, 5) == gbu.GBU_OK
    t0 = time.time()
    r, _ = run(ctx, data)
    elapsed = time.time() - t0
    assert r.status == gbu.GBU_DEVICE_TIMEOUT, triple(r)
    assert (r.in_offset, r.out_len) == (0, 0)
    assert elapsed < 5.0      # every bounded wait gave up after a few ms
    # clean scan state again: exact results, several times
    for _ in range(2):
        check(ctx, data)


def test_launch_without_chunks_reports_device_error(ctx):
    assert gbu.gbu_set_wait_limit(ctx, SHORT_NS) == gbu.GBU_OK
    data = textgen.generate("latin", 4000, textgen.UTF8, seed=100).data   # one chunk
    assert gbu.gbu_test_skip_chunks(ctx, 1) == gbu.GBU_OK
    r, _ = gpu_u8_to_u16(ctx, data)
    assert r.status == gbu.GBU_DEVICE_ERROR, triple(r)
    check_u8(ctx, data)
    # the length-only call after a failed launch
    rl = gbu.gbu_utf16_length_from_utf8
    import torch
    d = torch.from_numpy(np.array(data, copy=True)).cuda()
    got = rl(ctx, d.data_ptr(), data.size, 0)
    import oracle
    assert triple(got) == triple(oracle.utf16_length_from_utf8(data))
