"""Inputs beyond 4 GiB: byte offsets, output lengths, chunk numbers and error
positions above 2^32 end to end, against the oracle.

- UTF-8 -> UTF-16LE of 4.6 GB of mix-profile text: the whole output compared
  with the oracle's; then one invalid byte planted 4.4 GB in: the transcoding,
  length and validation calls report the oracle's kind, offset and prefix.
- UTF-16LE -> UTF-8 of 2.25 G units of CJK-like text (4.5 GB in, 6.3 GB
  out): result triple against the oracle's length call, and the output's
  tail against the oracle run on the last 4 MiB of the input (cut at a unit
  that is not a low surrogate).
"""
import numpy as np
import pytest

import oracle
import paper_2212_05098_gb300 as gbu
import textgen

from gpu_util import triple

pytestmark = pytest.mark.gpu

N8 = (4 << 30) + (300 << 20) + 12345        # UTF-8 bytes
N16 = (2 << 30) + (100 << 20) + 777         # UTF-16 units


@pytest.fixture(scope="module")
def env():
    import torch
    torch.cuda.init()
    pool = textgen.process_pool()
    ctx = gbu.gbu_create(0)
    yield torch, pool, ctx
    gbu.gbu_destroy(ctx)
    pool.shutdown()


def test_utf8_beyond_4gib(env):
    torch, pool, ctx = env
    t = textgen.generate("mix", N8, textgen.UTF8, seed=300, executor=pool,
                         keep_cps=False, keep_lens=False).data
    d_in = torch.from_numpy(t).cuda()
    d_out = torch.empty(2 * N8, dtype=torch.uint8, device="cuda")
    r = gbu.gbu_utf8_to_utf16le(ctx, d_in.data_ptr(), N8, d_out.data_ptr(), N8, 0)
    ref, ref_out = oracle.utf8_to_utf16le(t)
    assert triple(r) == triple(ref)
    assert ref.out_len > (1 << 32) // 2        # more than 4 GiB of output bytes
    got = d_out[: 2 * ref.out_len].cpu().numpy().view("<u2")
    assert np.array_equal(got, ref_out)
    del got, ref_out
    # one invalid byte 4.4 GB in
    p = 4_400_000_000
    t[p] = 0xFF
    d_in[p] = 0xFF
    want = oracle.utf16_length_from_utf8(t)
    assert want.status != gbu.GBU_OK and want.in_offset > (1 << 32)
    r = gbu.gbu_utf8_to_utf16le(ctx, d_in.data_ptr(), N8, d_out.data_ptr(), N8, 0)
    assert triple(r) == triple(want)
    assert triple(gbu.gbu_utf16_length_from_utf8(ctx, d_in.data_ptr(), N8, 0)) == triple(want)
    v = gbu.gbu_validate_utf8(ctx, d_in.data_ptr(), N8, 0)
    assert triple(v) == (want.status, want.in_offset, 0)


def test_utf16_beyond_4gib(env):
    torch, pool, ctx = env
    t = textgen.generate("cjk", 2 * N16, textgen.UTF16, seed=301, executor=pool,
                         keep_cps=False, keep_lens=False).data
    want = oracle.utf8_length_from_utf16le(t)
    assert want.status == gbu.GBU_OK and want.out_len > (1 << 32)
    d_in = torch.from_numpy(t).cuda()
    d_out = torch.empty(3 * N16, dtype=torch.uint8, device="cuda")
    r = gbu.gbu_utf16le_to_utf8(ctx, d_in.data_ptr(), N16, d_out.data_ptr(), 3 * N16, 0)
    assert triple(r) == triple(want)
    assert triple(gbu.gbu_utf8_length_from_utf16le(ctx, d_in.data_ptr(), N16, 0)) == triple(want)
    v = gbu.gbu_validate_utf16le(ctx, d_in.data_ptr(), N16, 0)
    assert triple(v) == (gbu.GBU_OK, N16, 0)
    # the output's tail: the oracle on the input's last 4 MiB (from a unit
    # that starts a character)
    w = t.view("<u2")
    s = N16 - (2 << 20)
    while 0xDC00 <= int(w[s]) <= 0xDFFF:
        s += 1
    tail_ref, tail_out = oracle.utf16le_to_utf8(t[2 * s:])
    assert tail_ref.status == gbu.GBU_OK
    got = d_out[want.out_len - tail_ref.out_len: want.out_len].cpu().numpy()
    assert np.array_equal(got, tail_out)
