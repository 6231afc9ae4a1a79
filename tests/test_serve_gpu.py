"""GPU tests of the serving loop: every request's result and output are the
same alone (the single-buffer call) and in the mix (continuous batching),
and agree with the oracle; admission by bytes against a small pool."""
import numpy as np
import pytest

import oracle
import paper_2212_05098_gb300 as gbu
import textgen
from textgen import batch as tbatch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    torch.cuda.init()
    corpora = [(p, e, textgen.generate(p, 8 << 20, e, keep_cps=False, keep_lens=False).data)
               for p in textgen.BENCH_PROFILES for e in (textgen.UTF8, textgen.UTF16)]
    d_corp = [torch.from_numpy(c[2]).cuda() for c in corpora]
    ctx = gbu.gbu_create(0)
    yield torch, corpora, d_corp, ctx
    gbu.gbu_destroy(ctx)


def _requests(torch, corpora, d_corp, trace, ops_length_every=7):
    """Device inputs (windows, or patched copies for the error requests),
    output destinations and the request tuples."""
    lay = trace.layout
    keep, reqs, meta = [], [], []
    for i in range(lay.nbytes.size):
        k = int(lay.corpus[i])
        enc = corpora[k][1]
        s, nb = int(lay.start[i]), int(lay.nbytes[i])
        host = corpora[k][2][s:s + nb]
        if trace.error_at[i] >= 0:
            host = tbatch.inject_error(host, int(trace.error_at[i]), enc)
            dev = torch.from_numpy(host.copy()).cuda() if nb else None
            keep.append(dev)
            ptr = dev.data_ptr() if nb else 0
        else:
            ptr = d_corp[k].data_ptr() + s if nb else 0
        u16 = enc == textgen.UTF16
        n = nb // 2 if u16 else nb
        length_only = i % ops_length_every == 3
        if u16:
            op = gbu.GBU_OP_UTF8_LENGTH_FROM_UTF16LE if length_only else gbu.GBU_OP_UTF16LE_TO_UTF8
        else:
            op = gbu.GBU_OP_UTF16_LENGTH_FROM_UTF8 if length_only else gbu.GBU_OP_UTF8_TO_UTF16LE
        cap_b = 0 if length_only else (3 * n if u16 else 2 * n)
        out = torch.full((cap_b + 64,), 0xA5, dtype=torch.uint8, device="cuda")
        keep.append(out)
        reqs.append((op, ptr, n, out.data_ptr() if cap_b else 0, cap_b, 1000 + i))
        meta.append((host, u16, length_only, out, cap_b))
    return keep, reqs, meta


def _alone(ctx, req, meta):
    """The same request through the single-buffer call."""
    op, ptr, n, _, cap_b, _ = req
    host, u16, length_only, _, _ = meta
    import torch
    if length_only:
        f = gbu.gbu_utf8_length_from_utf16le if u16 else gbu.gbu_utf16_length_from_utf8
        return f(ctx, ptr, n, 0), None
    out = torch.empty(cap_b + 16, dtype=torch.uint8, device="cuda")
    if u16:
        r = gbu.gbu_utf16le_to_utf8(ctx, ptr, n, out.data_ptr(), 3 * n, 0)
        return r, out[: min(r.out_len, 3 * n)].cpu().numpy()
    r = gbu.gbu_utf8_to_utf16le(ctx, ptr, n, out.data_ptr(), n, 0)
    return r, out[: 2 * min(r.out_len, n)].cpu().numpy()


def _check_trace(env, trace, pool_bytes, slots, max_items, oracle_every=10):
    torch, corpora, d_corp, ctx = env
    keep, reqs, meta = _requests(torch, corpora, d_corp, trace)
    srv = gbu.gbu_server_create(0, pool_bytes, slots, max_items)
    assert srv
    try:
        st, comp = gbu.gbu_server_replay(srv, reqs, list(trace.t_arrival), 120.0)
        assert st == gbu.GBU_OK
        stats = gbu.gbu_server_stats(srv)
        assert stats.submitted == stats.completed == len(reqs)
        assert stats.pool_high_water <= pool_bytes
    finally:
        gbu.gbu_server_destroy(srv)
    torch.cuda.synchronize()
    n_batched = 0
    for i, (req, m) in enumerate(zip(reqs, meta)):
        c = comp[i]
        assert c.tag == req[5]
        assert c.t_submit <= c.t_admit <= c.t_launch <= c.t_done
        n_batched += c.batch_items > 1
        got = (c.result.status, c.result.in_offset, c.result.out_len)
        r1, out1 = _alone(ctx, req, m)
        assert got == (r1.status, r1.in_offset, r1.out_len), (i, got)
        host, u16, length_only, out, cap_b = m
        if not length_only:
            ub = 1 if u16 else 2
            got_out = out[: ub * min(c.result.out_len, cap_b // ub)].cpu().numpy()
            assert np.array_equal(got_out, out1), i
        if i % oracle_every == 0:
            if u16:
                ref = oracle.utf8_length_from_utf16le(host) if length_only else oracle.utf16le_to_utf8(host)[0]
            else:
                ref = oracle.utf16_length_from_utf8(host) if length_only else oracle.utf8_to_utf16le(host)[0]
            assert got == (ref.status, ref.in_offset, ref.out_len), i
    return comp, n_batched


def test_mix_equals_alone(env):
    """400 requests arriving within a few ms: they run in shared batches, two
    slots in flight, and each equals its single-buffer result."""
    torch, corpora, _, _ = env
    trace = tbatch.serving_trace(corpora, 400, 1e5, seed=51, lo=64, hi=1 << 20, error_frac=0.05)
    comp, n_batched = _check_trace(env, trace, 1 << 30, 2, 256)
    assert n_batched > 100            # the mix really shared launches
    assert len({c.batch for c in comp}) > 1


def test_slow_arrivals_run_alone(env):
    """Requests far apart in time: each runs as its own batch."""
    torch, corpora, _, _ = env
    trace = tbatch.serving_trace(corpora, 30, 200.0, seed=52, lo=64, hi=256 << 10, error_frac=0.1)
    comp, _ = _check_trace(env, trace, 64 << 20, 2, 64, oracle_every=1)
    assert sum(c.batch_items == 1 for c in comp) >= 20


def test_small_pool_admission(env):
    """A pool that holds only a few requests at a time: admission waits for
    space, everything completes, results unchanged."""
    torch, corpora, _, _ = env
    trace = tbatch.serving_trace(corpora, 120, 1e6, seed=53, lo=64 << 10, hi=512 << 10,
                                 error_frac=0.05)
    comp, _ = _check_trace(env, trace, 4 << 20, 3, 64)
    # every batch's inputs and worst-case outputs fit into the pool together
    lay = trace.layout
    per_batch = {}
    for i, c in enumerate(comp):
        u16 = corpora[int(lay.corpus[i])][1] == textgen.UTF16
        nb = int(lay.nbytes[i])
        out_b = 0 if i % 7 == 3 else (3 * (nb // 2) if u16 else 2 * nb)   # length-only: no output
        per_batch[c.batch] = per_batch.get(c.batch, 0) + nb + out_b
    assert max(per_batch.values()) <= 4 << 20
    assert len(per_batch) >= 10


def test_submit_rejects(env):
    torch, _, d_corp, _ = env
    srv = gbu.gbu_server_create(0, 2 << 20, 1, 16)
    assert srv
    try:
        p = d_corp[0].data_ptr()
        assert gbu.gbu_server_submit(srv, 9, p, 16) == gbu.GBU_INVALID_ARG            # bad op
        assert gbu.gbu_server_submit(srv, 0, 0, 16) == gbu.GBU_INVALID_ARG            # null input
        assert gbu.gbu_server_submit(srv, 1, p + 1, 16) == gbu.GBU_INVALID_ARG        # odd UTF-16
        assert gbu.gbu_server_submit(srv, 0, p, 4 << 20) == gbu.GBU_INVALID_ARG       # never fits
        assert gbu.gbu_server_submit(srv, 0, p, 1000, tag=7) == gbu.GBU_OK
        assert gbu.gbu_server_wait_idle(srv, 30.0) == gbu.GBU_OK
        got = gbu.gbu_server_poll(srv)
        assert len(got) == 1 and got[0].tag == 7
        assert gbu.gbu_server_create(0, 1 << 20, 0, 16) is None
    finally:
        gbu.gbu_server_destroy(srv)


def test_big_endian_requests(env):
    """UTF-16BE requests through the server equal the single-buffer calls."""
    torch, corpora, d_corp, ctx = env
    srv = gbu.gbu_server_create(0, 64 << 20, 2, 64)
    assert srv
    try:
        reqs, keep = [], []
        for i, (prof, enc, data) in enumerate(corpora):
            src = data[: 200_000 + 1000 * i]
            if enc == textgen.UTF16:
                src = src.reshape(-1, 2)[:, ::-1].reshape(-1).copy()       # as UTF-16BE
                op, n = gbu.GBU_OP_UTF16BE_TO_UTF8, src.size // 2
                cap_b = 3 * n
            else:
                op, n = gbu.GBU_OP_UTF8_TO_UTF16BE, src.size
                cap_b = 2 * n
            d_in = torch.from_numpy(src).cuda()
            d_out = torch.full((cap_b + 64,), 0xA5, dtype=torch.uint8, device="cuda")
            keep.append((d_in, d_out, op, n, cap_b, src))
            reqs.append((op, d_in.data_ptr(), n, d_out.data_ptr(), cap_b, i))
        st, comp = gbu.gbu_server_replay(srv, reqs, [0.0] * len(reqs), 60.0)
        assert st == gbu.GBU_OK
    finally:
        gbu.gbu_server_destroy(srv)
    torch.cuda.synchronize()
    for i, (d_in, d_out, op, n, cap_b, src) in enumerate(keep):
        c = comp[i]
        if op == gbu.GBU_OP_UTF16BE_TO_UTF8:
            ref, out = oracle.utf16be_to_utf8(src)
        else:
            ref, out = oracle.utf8_to_utf16be(src)
        assert (c.result.status, c.result.in_offset, c.result.out_len) == \
            (ref.status, ref.in_offset, ref.out_len), i
        assert np.array_equal(d_out[: out.size].cpu().numpy(), out), i
