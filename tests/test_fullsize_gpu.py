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
    v = (gbu.gbu_validate_utf8(ctx, d_in.data_ptr(), n, 0) if enc == textgen.UTF8
         else gbu.gbu_validate_utf16le(ctx, d_in.data_ptr(), n, 0))
    assert (v.status, v.in_offset, v.out_len) == (ref.status, ref.in_offset, 0)


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
        if i % 10 == 0:   # validation-only call: same first error
            v = (gbu.gbu_validate_utf8(ctx, d_in.data_ptr(), n, 0) if enc == textgen.UTF8
                 else gbu.gbu_validate_utf16le(ctx, d_in.data_ptr(), n, 0))
            assert (v.status, v.in_offset, v.out_len) == (p.kind, p.err_unit, 0), (i, p.case)
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


def test_batched_200k_strings(env):
    """The batched workload at full size: 200,000 strings, lengths log-uniform
    16 B - 1 MiB (about 18 GiB), windows of 256 MiB corpora of the four
    profiles in both encodings, one autotuned graph. Every result is checked
    against properties of valid text (status OK, whole input consumed, output
    length from the characters' encoded sizes), and every string's result and
    output against the oracle byte for byte (the oracle on 16 host threads,
    the outputs copied back 8192 strings at a time)."""
    torch, pool, ctx = env
    from textgen import batch as tbatch
    corpora, d_corp = [], []
    for p in textgen.BENCH_PROFILES:
        for enc in (textgen.UTF8, textgen.UTF16):
            t = textgen.generate(p, 256 << 20, enc, executor=pool, keep_cps=False, keep_lens=False)
            corpora.append((p, enc, t.data))
            d_corp.append(torch.from_numpy(t.data).cuda())
    lay = tbatch.layout(corpora, 200_000, 16, 1 << 20, seed=4)
    n = lay.nbytes.size
    is16 = np.array([corpora[k][1] == textgen.UTF16 for k in lay.corpus])
    cap_b = np.where(is16, 3 * (lay.nbytes // 2), 2 * lay.nbytes)
    off = np.zeros(n + 1, np.int64)
    np.cumsum((cap_b + 15) // 16 * 16, out=off[1:])
    d_out = torch.empty(int(off[-1]) + 16, dtype=torch.uint8, device="cuda")
    d_res = torch.zeros(n * 24, dtype=torch.uint8, device="cuda")
    items = []
    for i in range(n):
        k = int(lay.corpus[i])
        inp = d_corp[k].data_ptr() + int(lay.start[i])
        u = int(lay.nbytes[i]) // (2 if is16[i] else 1)
        items.append((inp if u else 0, u, d_out.data_ptr() + int(off[i]),
                      3 * u if is16[i] else u,
                      gbu.GBU_OP_UTF16LE_TO_UTF8 if is16[i] else gbu.GBU_OP_UTF8_TO_UTF16LE))
    assert gbu.gbu_batch_plan(ctx, items, d_res.data_ptr(), 0) == gbu.GBU_OK
    st, _ = gbu.gbu_batch_autotune(ctx, 0, None)
    try:
        assert st == gbu.GBU_OK
        d_out.fill_(0xA5)
        assert gbu.gbu_batch_launch_graph(ctx, 0) == gbu.GBU_OK
        torch.cuda.synchronize()
        res = np.frombuffer(d_res.cpu().numpy().tobytes(),
                            dtype=[("status", "<i4"), ("r", "<u4"), ("off", "<u8"), ("len", "<u8")])
        assert (res["status"] == 0).all()
        assert (res["off"] == lay.nbytes // np.where(is16, 2, 1)).all()
        # output length of valid text: UTF-8 -> UTF-16 units = non-continuation
        # bytes + 4-byte leads; UTF-16 -> UTF-8 bytes = per-unit sizes, 2 per
        # surrogate (4 per pair)
        for k, (p, enc, data) in enumerate(corpora):
            sel = np.nonzero(lay.corpus == k)[0]
            if enc == textgen.UTF8:
                w = (((data & 0xC0) != 0x80).astype(np.int64) + (data >= 0xF0))
            else:
                u = data.view("<u2")
                w = np.where(u < 0x80, 1, np.where(u < 0x800, 2, np.where((u & 0xF800) == 0xD800, 2, 3)))
                w = w.astype(np.int64)
            cum = np.zeros(w.size + 1, np.int64)
            np.cumsum(w, out=cum[1:])
            ub = 2 if enc == textgen.UTF16 else 1
            s0, s1 = lay.start[sel] // ub, (lay.start[sel] + lay.nbytes[sel]) // ub
            assert (res["len"][sel] == cum[s1] - cum[s0]).all(), (p, enc)
        from concurrent.futures import ThreadPoolExecutor

        def ref_of(i):
            k = int(lay.corpus[i])
            src = corpora[k][2][int(lay.start[i]):int(lay.start[i] + lay.nbytes[i])]
            if is16[i]:
                ref, ref_out = oracle.utf16le_to_utf8(src)
                return ref, ref_out
            ref, ref_out = oracle.utf8_to_utf16le(src)
            return ref, ref_out.view(np.uint8)

        with ThreadPoolExecutor(16) as ex:   # the oracle's C calls release the GIL
            for g0 in range(0, n, 8192):
                g1 = min(n, g0 + 8192)
                host = d_out[int(off[g0]):int(off[g1])].cpu().numpy()
                for i, (ref, want) in zip(range(g0, g1), ex.map(ref_of, range(g0, g1))):
                    assert (int(res["status"][i]), int(res["off"][i]), int(res["len"][i])) == \
                        (ref.status, ref.in_offset, ref.out_len), i
                    o = int(off[i] - off[g0])
                    assert np.array_equal(host[o:o + want.size], want), i
    finally:
        assert gbu.gbu_set_tune(ctx, 1, 0) == gbu.GBU_OK


@pytest.mark.parametrize("enc", [textgen.UTF8, textgen.UTF16])
def test_host_buffer_pipeline(env, enc):
    """The host-buffer calls on 256 MiB inputs (cut into slices that are copied
    in, transcoded and copied out in a pipeline): valid text, an error in a
    middle slice, an error right after a slice cut, and a too-small output,
    each against the oracle."""
    torch, pool, ctx = env
    size = 256 << 20
    t = textgen.generate("emoji", size, enc, seed=71, executor=pool, keep_cps=False, keep_lens=False)
    n = t.data.size if enc == textgen.UTF8 else t.data.size // 2
    cap = n if enc == textgen.UTF8 else 3 * n
    ub = 2 if enc == textgen.UTF8 else 1
    h_in = torch.from_numpy(t.data).pin_memory()
    h_out = torch.empty(cap * ub, dtype=torch.uint8).pin_memory()
    call = gbu.gbu_utf8_to_utf16le_host if enc == textgen.UTF8 else gbu.gbu_utf16le_to_utf8_host
    ref_fn = oracle.utf8_to_utf16le if enc == textgen.UTF8 else oracle.utf16le_to_utf8

    def check(data, capacity):
        h_in.copy_(torch.from_numpy(data))
        h_out.fill_(0xA5)
        r = call(ctx, h_in.data_ptr(), n, h_out.data_ptr(), capacity, 0)
        ref, out = ref_fn(data, capacity)
        assert (r.status, r.in_offset, r.out_len) == (ref.status, ref.in_offset, ref.out_len)
        keep = min(ref.out_len, capacity) * ub
        assert np.array_equal(h_out[:keep].numpy(), out.view(np.uint8)[:keep])
        assert (h_out[capacity * ub:].numpy() == 0xA5).all()

    check(t.data, cap)
    bad = t.data.copy()
    if enc == textgen.UTF8:
        bad[size // 2 + 12345] = 0xFF
        bad2 = t.data.copy()
        bad2[(size // 8) + 1] = 0x80         # near a slice cut (32 MiB slices)
    else:
        bad.view("<u2")[n // 2 + 999] = 0xDC00
        bad2 = t.data.copy()
        bad2.view("<u2")[(n // 8) + 1] = 0xD800
    check(bad, cap)
    check(bad2, cap)
    check(t.data, cap // 3)                    # OUTPUT_TOO_SMALL with the required length
