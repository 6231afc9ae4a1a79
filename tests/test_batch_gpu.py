"""GPU parity of the batch API: many inputs, any mix of the four calls, in one
launch of the persistent kernel, each result and output compared with the
oracle's single-buffer answer on the same input."""
import numpy as np
import pytest

import oracle
import paper_2212_05098_gb300 as gbu
import textgen
from textgen import inject

from gpu_util import GUARD, CANARY

pytestmark = pytest.mark.gpu

RESULT_DTYPE = np.dtype([("status", "<i4"), ("reserved", "<u4"), ("in_offset", "<u8"),
                         ("out_len", "<u8")])


@pytest.fixture(scope="module")
def ctx():
    import torch
    torch.cuda.init()
    h = gbu.gbu_create(0)
    yield h
    gbu.gbu_destroy(h)


def _case(rng, i):
    """One batch item: (op, input bytes, cap units or None)."""
    op = int(rng.integers(0, 4))
    utf16 = op in (gbu.GBU_OP_UTF16LE_TO_UTF8, gbu.GBU_OP_UTF8_LENGTH_FROM_UTF16LE)
    profile = list(textgen.PROFILES)[int(rng.integers(0, len(textgen.PROFILES)))]
    kind = rng.random()
    if kind < 0.05:
        n = 0
    elif kind < 0.35:
        n = int(rng.integers(1, 64))
    else:
        n = int(np.exp(rng.uniform(np.log(64), np.log(300_000))))
    enc = textgen.UTF16 if utf16 else textgen.UTF8
    t = textgen.generate(profile, (n + 9) & ~1, enc, seed=1000 + i)
    data = t.data[: (n // 2) * 2 if utf16 else n].copy()
    if data.size and rng.random() < 0.25:
        data = textgen.mutate(data, int(rng.integers(1, 4)), seed=2000 + i)
    cap = None
    if op <= 1 and rng.random() < 0.2:
        cap = int(rng.integers(0, max(1, data.size)))
    return op, data, cap


def _expected(op, data, cap):
    if op == gbu.GBU_OP_UTF8_TO_UTF16LE:
        r, out = oracle.utf8_to_utf16le(data, cap)
        c = data.size if cap is None else cap
        return r, out[: min(r.out_len, c)].view(np.uint8), 2 * c
    if op == gbu.GBU_OP_UTF16LE_TO_UTF8:
        r, out = oracle.utf16le_to_utf8(data, cap)
        c = 3 * (data.size // 2) if cap is None else cap
        return r, out[: min(r.out_len, c)], c
    if op == gbu.GBU_OP_UTF16_LENGTH_FROM_UTF8:
        return oracle.utf16_length_from_utf8(data), None, 0
    return oracle.utf8_length_from_utf16le(data), None, 0


class Batch:
    """Inputs at random alignments in one device arena, outputs in another,
    every output surrounded by canaries."""

    def __init__(self, cases, rng):
        import torch
        self.cases = cases
        self.want = [_expected(*c) for c in cases]
        in_offs, out_offs = [], []
        pos = 0
        for op, data, _ in cases:
            pos = (pos + 15) & ~15
            a = int(rng.integers(0, 16))
            if op in (1, 3):
                a &= ~1
            in_offs.append(pos + a)
            pos += a + data.size + 32
        self.din = torch.zeros(pos + 16, dtype=torch.uint8, device="cuda")
        hin = np.zeros(pos + 16, dtype=np.uint8)
        for (op, data, _), o in zip(cases, in_offs):
            hin[o:o + data.size] = data
        self.din.copy_(torch.from_numpy(hin))
        pos = 0
        for (op, data, cap), w in zip(cases, self.want):
            pos = (pos + 15) & ~15
            a = int(rng.integers(0, 16))
            if op == 0:
                a &= ~1
            pos += GUARD
            out_offs.append(pos + a)
            pos += a + w[2] + GUARD
        self.out_size = pos + 16
        self.dout = torch.empty(self.out_size, dtype=torch.uint8, device="cuda")
        self.res = torch.empty(len(cases) * RESULT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        self.in_offs, self.out_offs = in_offs, out_offs
        base_in, base_out = self.din.data_ptr(), self.dout.data_ptr()
        self.items = []
        for (op, data, cap), w, io, oo in zip(cases, self.want, in_offs, out_offs):
            unit = 2 if op in (1, 3) else 1
            n = data.size // unit
            if op <= 1:
                c = w[2] // (2 if op == 0 else 1)
                self.items.append((base_in + io if n else 0, n, base_out + oo, c, op))
            else:
                self.items.append((base_in + io if n else 0, n, 0, 0, op))

    def reset(self):
        self.dout.fill_(CANARY)
        self.res.fill_(0xEE)

    def check(self):
        res = np.frombuffer(self.res.cpu().numpy().tobytes(), dtype=RESULT_DTYPE)
        out = self.dout.cpu().numpy()
        prev_end = 0
        for i, ((op, data, cap), (r, want, outb), oo) in enumerate(
                zip(self.cases, self.want, self.out_offs)):
            got = (int(res[i]["status"]), int(res[i]["in_offset"]), int(res[i]["out_len"]))
            assert got == (r.status, r.in_offset, r.out_len), (i, op, data.size, cap, got,
                                                                (r.status, r.in_offset, r.out_len))
            if want is not None:
                assert np.array_equal(out[oo:oo + want.size], want), (i, op, data.size)
                # canaries between the previous item's output and past this one's capacity
                assert (out[prev_end:oo] == CANARY).all(), (i, "write before output")
                prev_end = oo + outb
        assert (out[prev_end:] == CANARY).all(), "write past the last output"


def _run(ctx, batch, launch, times=2):
    import torch
    s = torch.cuda.Stream()
    for _ in range(times):
        batch.reset()
        torch.cuda.synchronize()
        assert launch(ctx, s.cuda_stream) == gbu.GBU_OK
        s.synchronize()
        batch.check()


def test_mixed_batch_launch_and_graph(ctx):
    rng = np.random.default_rng(77)
    cases = [_case(rng, i) for i in range(80)]
    b = Batch(cases, rng)
    assert gbu.gbu_batch_plan(ctx, b.items, b.res.data_ptr(), 0) == gbu.GBU_OK
    _run(ctx, b, gbu.gbu_batch_launch)
    _run(ctx, b, gbu.gbu_batch_launch_graph)
    _run(ctx, b, gbu.gbu_batch_launch)


def test_batch_replan_and_single_items(ctx):
    """Re-planning with another batch, a one-item batch, and a batch of empty inputs."""
    rng = np.random.default_rng(78)
    for count in (1, 3, 17):
        cases = [_case(rng, 100 * count + i) for i in range(count)]
        b = Batch(cases, rng)
        assert gbu.gbu_batch_plan(ctx, b.items, b.res.data_ptr(), 0) == gbu.GBU_OK
        _run(ctx, b, gbu.gbu_batch_launch_graph)
        _run(ctx, b, gbu.gbu_batch_launch, times=1)
    empty = [(op, np.zeros(0, np.uint8), None) for op in range(4)]
    b = Batch(empty, rng)
    assert gbu.gbu_batch_plan(ctx, b.items, b.res.data_ptr(), 0) == gbu.GBU_OK
    _run(ctx, b, gbu.gbu_batch_launch)


def test_batch_injected_errors_at_chunk_edges(ctx):
    """Errors planted around chunk edges of several items in one batch."""
    rng = np.random.default_rng(79)
    cases = []
    for i in range(24):
        utf16 = i % 2 == 1
        enc = textgen.UTF16 if utf16 else textgen.UTF8
        t = textgen.generate(["cjk", "emoji", "mix", "cyrillic"][i % 4], 200_000, enc, seed=300 + i)
        ncases = len(inject.UTF16_CASES if utf16 else inject.UTF8_CASES)
        p = inject.make_patch(t, i % ncases, seed=400 + i)
        data = p.apply(t.data)
        cases.append((1 if utf16 else 0, data, None))
        cases.append((3 if utf16 else 2, data, None))
    b = Batch(cases, rng)
    assert gbu.gbu_batch_plan(ctx, b.items, b.res.data_ptr(), 0) == gbu.GBU_OK
    _run(ctx, b, gbu.gbu_batch_launch)
    _run(ctx, b, gbu.gbu_batch_launch_graph)


def test_batch_results_in_mapped_host_memory(ctx):
    """Results may go to pinned host memory mapped into the device."""
    import torch
    rng = np.random.default_rng(80)
    cases = [_case(rng, 500 + i) for i in range(12)]
    b = Batch(cases, rng)
    host = torch.empty(b.res.numel(), dtype=torch.uint8, pin_memory=True)
    assert gbu.gbu_batch_plan(ctx, b.items, host.data_ptr(), 0) == gbu.GBU_OK
    b.dout.fill_(CANARY)
    host.fill_(0xEE)
    torch.cuda.synchronize()
    assert gbu.gbu_batch_launch(ctx, 0) == gbu.GBU_OK
    torch.cuda.synchronize()
    b.res.copy_(host)
    b.check()


def test_batch_invalid_items(ctx):
    import torch
    buf = torch.zeros(64, dtype=torch.uint8, device="cuda")
    res = torch.zeros(64, dtype=torch.uint8, device="cuda")
    p = buf.data_ptr()
    bad = [
        (p, 4, p, 4, 7),          # unknown op
        (0, 4, p, 4, 0),          # null input with n > 0
        (p + 1, 4, p, 4, 1),      # odd UTF-16 input
        (p, 4, p + 1, 4, 0),      # odd UTF-16 output
        (p, 4, 0, 4, 1),          # null output with cap > 0
    ]
    for it in bad:
        assert gbu.gbu_batch_plan(ctx, [it], res.data_ptr(), 0) == gbu.GBU_INVALID_ARG, it
    assert gbu.gbu_batch_plan(ctx, [(p, 4, p, 4, 0)], 0, 0) == gbu.GBU_INVALID_ARG


SHAPES = [(12288, 256), (8192, 256), (16384, 512), (6144, 128), (24576, 512)]


def test_compiled_shapes():
    assert gbu.gbu_tune_shapes() == SHAPES


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("look", [1, 2, 4, 8, 16])
def test_results_do_not_depend_on_tuning(ctx, look, shape):
    """Every kernel shape, look-back width and CTAs per SM gives the oracle's
    results, for a batch and for single-buffer calls."""
    import torch
    from gpu_util import check_u16, check_u8
    rng = np.random.default_rng(81)
    cases = [_case(rng, 700 + i) for i in range(24)]
    b = Batch(cases, rng)
    t8 = textgen.generate("emoji", 300_001, textgen.UTF8, seed=82)
    t16 = textgen.generate("cjk", 300_000, textgen.UTF16, seed=83)
    bad8 = textgen.mutate(t8.data, 2, seed=84)
    try:
        for ctas in (1, 2, 3):
            st = gbu.gbu_set_tune(ctx, look, ctas, gbu.GBU_SMALL_MAX_CHUNKS, *shape)
            if ctas > 1 and st == gbu.GBU_INVALID_ARG:
                break   # more CTAs per SM than fit on this device
            assert st == gbu.GBU_OK
            t = gbu.gbu_get_tune(ctx)
            assert (t.look_width, t.ctas_per_sm, t.chunk_bytes, t.compute_threads) == (look, ctas, *shape)
            assert gbu.gbu_batch_plan(ctx, b.items, b.res.data_ptr(), 0) == gbu.GBU_OK
            _run(ctx, b, gbu.gbu_batch_launch, times=1)
            _run(ctx, b, gbu.gbu_batch_launch_graph, times=1)
            check_u8(ctx, t8.data)
            check_u8(ctx, bad8)
            check_u16(ctx, t16.data)
    finally:
        assert gbu.gbu_set_tune(ctx, 1, 0) == gbu.GBU_OK
    torch.cuda.synchronize()


def test_tune_rejects_bad_values(ctx):
    assert gbu.gbu_set_tune(ctx, 5, 0) == gbu.GBU_INVALID_ARG
    assert gbu.gbu_set_tune(ctx, 8, -1) == gbu.GBU_INVALID_ARG
    assert gbu.gbu_set_tune(ctx, 8, 1000) == gbu.GBU_INVALID_ARG
    assert gbu.gbu_set_tune(ctx, 8, 0, 8, 12288, 128) == gbu.GBU_INVALID_ARG   # not compiled
    assert gbu.gbu_set_tune(ctx, 8, 0, 8, 4096, 0) == gbu.GBU_INVALID_ARG
    assert gbu.gbu_set_tune(ctx, 8, 2, 8, 16384, 512) == gbu.GBU_INVALID_ARG   # fits one per SM
    t = gbu.gbu_get_tune(ctx)
    assert (t.look_width, t.ctas_per_sm, t.chunk_bytes, t.compute_threads) == (1, 0, 0, 0)


def test_autotune_and_cache(ctx, tmp_path):
    rng = np.random.default_rng(85)
    cases = [_case(rng, 800 + i) for i in range(40)]
    b = Batch(cases, rng)
    assert gbu.gbu_batch_plan(ctx, b.items, b.res.data_ptr(), 0) == gbu.GBU_OK
    cache = str(tmp_path / "tune.txt")
    try:
        st, t = gbu.gbu_batch_autotune(ctx, 0, cache)
        assert st == gbu.GBU_OK and t.look_width in (1, 2, 4, 8, 16) and 1 <= t.ctas_per_sm <= 3
        assert (t.chunk_bytes, t.compute_threads) in SHAPES
        chosen = [str(x) for x in (t.look_width, t.ctas_per_sm, t.chunk_bytes, t.compute_threads)]
        lines = [l for l in open(cache) if l.strip()]
        assert len(lines) == 1 and lines[0].split()[1:5] == chosen
        _run(ctx, b, gbu.gbu_batch_launch_graph)    # on the chosen shape
        # a cached key is taken without timing and without a new line
        assert gbu.gbu_set_tune(ctx, 1, 0) == gbu.GBU_OK
        st2, t2 = gbu.gbu_batch_autotune(ctx, 0, cache)
        assert st2 == gbu.GBU_OK
        assert [str(x) for x in (t2.look_width, t2.ctas_per_sm, t2.chunk_bytes, t2.compute_threads)] == chosen
        assert len([l for l in open(cache) if l.strip()]) == 1
        _run(ctx, b, gbu.gbu_batch_launch_graph)
    finally:
        assert gbu.gbu_set_tune(ctx, 1, 0) == gbu.GBU_OK


def test_batch_big_endian_ops(ctx):
    """UTF-16BE operations in a batch next to UTF-16LE ones."""
    import torch
    rng = np.random.default_rng(90)
    items, checks, keep = [], [], []
    res = torch.zeros(24 * 12, dtype=torch.uint8, device="cuda")
    for i in range(12):
        prof = list(textgen.PROFILES)[i % 5]
        t8 = textgen.generate(prof, 50_000 + 977 * i, textgen.UTF8, seed=900 + i).data
        t16 = textgen.generate(prof, 2 * (40_000 + 313 * i), textgen.UTF16, seed=950 + i).data
        be16 = t16.reshape(-1, 2)[:, ::-1].reshape(-1).copy()
        if i % 4 == 3:
            be16.view(">u2")[777] = 0xD801                  # lone high
        op = [gbu.GBU_OP_UTF8_TO_UTF16BE, gbu.GBU_OP_UTF16BE_TO_UTF8,
              gbu.GBU_OP_UTF8_LENGTH_FROM_UTF16BE, gbu.GBU_OP_UTF8_TO_UTF16LE][i % 4]
        src = t8 if op in (gbu.GBU_OP_UTF8_TO_UTF16BE, gbu.GBU_OP_UTF8_TO_UTF16LE) else be16
        d_in = torch.from_numpy(src).cuda()
        n = src.size if src is t8 else src.size // 2
        cap = n if src is t8 else 3 * n
        d_out = torch.full((2 * cap + 64,), 0xA5, dtype=torch.uint8, device="cuda")
        keep += [d_in, d_out]
        writes = op != gbu.GBU_OP_UTF8_LENGTH_FROM_UTF16BE
        items.append((d_in.data_ptr(), n, d_out.data_ptr() if writes else 0, cap if writes else 0, op))
        checks.append((op, src, d_out, cap))
    assert gbu.gbu_batch_plan(ctx, items, res.data_ptr(), 0) == gbu.GBU_OK
    for launch in (gbu.gbu_batch_launch, gbu.gbu_batch_launch_graph):
        assert launch(ctx, 0) == gbu.GBU_OK
        torch.cuda.synchronize()
        got = np.frombuffer(res.cpu().numpy().tobytes(), dtype=RESULT_DTYPE)
        for i, (op, src, d_out, cap) in enumerate(checks):
            if op == gbu.GBU_OP_UTF8_TO_UTF16BE:
                ref, out = oracle.utf8_to_utf16be(src, cap)
            elif op == gbu.GBU_OP_UTF16BE_TO_UTF8:
                ref, out = oracle.utf16be_to_utf8(src, cap)
            elif op == gbu.GBU_OP_UTF8_LENGTH_FROM_UTF16BE:
                ref, out = oracle.utf8_length_from_utf16be(src), None
            else:
                ref, out = oracle.utf8_to_utf16le(src, cap)
                out = out.view(np.uint8)
            assert (int(got[i]["status"]), int(got[i]["in_offset"]), int(got[i]["out_len"])) == \
                (ref.status, ref.in_offset, ref.out_len), i
            if out is not None:
                assert np.array_equal(d_out[: out.size].cpu().numpy(), out), i


@pytest.mark.parametrize("ops", [(0, 2), (1, 3), (0,), (1,)])
def test_single_encoding_batches(ctx, ops):
    """Batches whose items all read one encoding (they run the kernel with
    that direction's code only), transcoding and length items mixed."""
    rng = np.random.default_rng(95 + ops[0] + 10 * len(ops))
    cases = []
    for i in range(40):
        op, data, cap = _case(rng, 1500 + 50 * ops[0] + i)
        want_op = ops[i % len(ops)]
        if (op in (1, 3)) != (want_op in (1, 3)):   # re-draw in the wanted encoding
            enc = textgen.UTF16 if want_op in (1, 3) else textgen.UTF8
            n = max(2, data.size)
            data = textgen.generate("emoji", n + (n & 1), enc, seed=1700 + i).data
            cap = None
        cases.append((want_op, data, cap if want_op <= 1 else None))
    b = Batch(cases, rng)
    assert gbu.gbu_batch_plan(ctx, b.items, b.res.data_ptr(), 0) == gbu.GBU_OK
    _run(ctx, b, gbu.gbu_batch_launch)
    _run(ctx, b, gbu.gbu_batch_launch_graph)


def test_large_batch_spread(ctx):
    """A batch of more than 512 MiB runs its one-chunk items in their own
    kernel and the rest as one job per input encoding: every result and output
    still equals the oracle's, with errors and small capacities in both."""
    rng = np.random.default_rng(96)
    cases = []
    for i in range(44):                       # ~14 MB each, every operation
        op = i % 4
        enc = textgen.UTF16 if op in (1, 3) else textgen.UTF8
        n = 13_000_000 + 7919 * i
        data = textgen.generate(["cjk", "emoji", "mix", "cyrillic"][i % 4], n + (n & 1), enc,
                                seed=1800 + i).data
        if i % 5 == 0:
            data = textgen.mutate(data, 1, seed=1900 + i)
        cap = int(data.size // 3) if (op <= 1 and i % 7 == 3) else None
        cases.append((op, data, cap))
    for i in range(600):                      # short items, many of one chunk, some empty
        cases.append(_case(rng, 2000 + i) if i % 3 else (i % 4, np.zeros(0, np.uint8), None))
    b = Batch(cases, rng)
    assert sum(c[1].size for c in cases) > (512 << 20)
    assert gbu.gbu_batch_plan(ctx, b.items, b.res.data_ptr(), 0) == gbu.GBU_OK
    before = gbu.gbu_kernel_launch_count()
    _run(ctx, b, gbu.gbu_batch_launch, times=1)
    assert gbu.gbu_kernel_launch_count() - before == 3   # one-chunk items + one job per encoding
    _run(ctx, b, gbu.gbu_batch_launch_graph, times=1)
