"""Full-size GPU parity, in the launch configuration the benchmark times.

- Every profile x direction at 1 GiB: whole outputs, lengths and status
  compared with the oracle byte for byte.
- Validation stress on 256 MiB of CJK-like text per direction: 1000 seeded
  injected errors each (every UTF-8 / UTF-16 error kind, sequences cut at
  4-64 KiB edges and at the end of the buffer). Each case is patched into the
  resident device buffer; kind, first-error offset and prefix length must match
  the injector's expectation, the valid prefix must match the oracle's output
  of the unpatched text, and every 100th case is rerun through the oracle.
"""
import numpy as np
import pytest

import oracle
import paper_2212_05098_gb300 as gbu
import textgen
from textgen import inject

pytestmark = pytest.mark.gpu

GIB = 1 << 30


@pytest.fixture(scope="module")
def env():
    import torch
    torch.cuda.init()
    pool = textgen.process_pool()
    ctx = gbu.gbu_create(0)
    gbu.gbu_reserve(ctx, GIB)
    yield torch, pool, ctx
    gbu.gbu_destroy(ctx)
    pool.shutdown()


def _run(torch, ctx, enc, d_in, n_units, d_out, cap):
    if enc == textgen.UTF8:
        return gbu.gbu_utf8_to_utf16le(ctx, d_in.data_ptr(), n_units, d_out.data_ptr(), cap, 0)
    return gbu.gbu_utf16le_to_utf8(ctx, d_in.data_ptr(), n_units, d_out.data_ptr(), cap, 0)


@pytest.mark.parametrize("profile", textgen.BENCH_PROFILES)
@pytest.mark.parametrize("enc", [textgen.UTF8, textgen.UTF16])
def test_one_gib_matches_oracle(env, profile, enc):
    torch, pool, ctx = env
    t = textgen.generate(profile, GIB, enc, executor=pool, keep_cps=False, keep_lens=False)
    if enc == textgen.UTF8:
        ref, ref_out = oracle.utf8_to_utf16le(t.data)
        n, cap, ub = t.data.size, t.data.size, 2
    else:
        ref, ref_out = oracle.utf16le_to_utf8(t.data)
        n, cap, ub = t.data.size // 2, 3 * (t.data.size // 2), 1
    d_in = torch.from_numpy(t.data).cuda()
    del t
    d_out = torch.empty(cap * ub, dtype=torch.uint8, device="cuda")
    r = _run(torch, ctx, enc, d_in, n, d_out, cap)
    assert (r.status, r.in_offset, r.out_len) == (ref.status, ref.in_offset, ref.out_len)
    want = torch.from_numpy(ref_out.view(np.uint8)).cuda()
    assert torch.equal(d_out[: ref.out_len * ub], want)


@pytest.mark.parametrize("enc", [textgen.UTF8, textgen.UTF16])
def test_validation_stress_1000_cases(env, enc):
    torch, pool, ctx = env
    size = 256 << 20
    t = textgen.generate("cjk", size, enc, seed=3, executor=pool, keep_cps=False)
    starts, outs = t.char_starts(), t.out_starts()
    ub_in = 1 if enc == textgen.UTF8 else 2
    ub_out = 2 if enc == textgen.UTF8 else 1
    n = t.data.size // ub_in
    cap = n if enc == textgen.UTF8 else 3 * n
    if enc == textgen.UTF8:
        base_ref, base_out = oracle.utf8_to_utf16le(t.data)
    else:
        base_ref, base_out = oracle.utf16le_to_utf8(t.data)
    assert base_ref.status == oracle.OK
    base_dev = torch.from_numpy(base_out.view(np.uint8)).cuda()
    d_in = torch.from_numpy(t.data).cuda()
    d_out = torch.empty(cap * ub_out, dtype=torch.uint8, device="cuda")
    ncases = 1000
    for i in range(ncases):
        p = inject.make_patch(t, i, seed=3, starts=starts, out_starts=outs)
        lo, hi = p.offset, p.offset + p.data.size
        d_in[lo:hi] = torch.from_numpy(p.data).cuda()
        r = _run(torch, ctx, enc, d_in, n, d_out, cap)
        assert (r.status, r.in_offset, r.out_len) == (p.kind, p.err_unit, p.prefix_out), (i, p.case)
        # valid prefix: the unpatched text's output up to the window, then spaces
        w_out = int(outs[np.searchsorted(starts, lo // ub_in)]) * ub_out
        assert torch.equal(d_out[:w_out], base_dev[:w_out]), (i, p.case)
        tail = d_out[w_out: r.out_len * ub_out].cpu().numpy()
        spaces = np.full(r.out_len - w_out // ub_out, 0x20, "<u2" if ub_out == 2 else np.uint8)
        assert np.array_equal(tail, spaces.view(np.uint8)), (i, p.case)
        if i % 100 == 0:
            patched = p.apply(t.data)
            if enc == textgen.UTF8:
                ref = oracle.utf16_length_from_utf8(patched)
            else:
                ref = oracle.utf8_length_from_utf16le(patched)
            assert (r.status, r.in_offset, r.out_len) == (ref.status, ref.in_offset, ref.out_len)
        d_in[lo:hi] = torch.from_numpy(t.data[lo:hi]).cuda()   # undo the patch
