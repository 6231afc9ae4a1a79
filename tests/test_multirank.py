"""Multi-rank host logic on CPU (gloo, world size 2), no GPU:

- one buffer split across ranks at character boundaries: each rank handles
  its part (here with the oracle standing in for its GPU), the ranks exchange
  one (length, first error) record each, and the assembled output, result and
  first error equal those of the whole buffer;
- the benchmark's whole-job rate: all ranks' bytes over the slowest rank's
  time, and per-rank inputs that differ between ranks.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
import textgen
from paper_2212_05098_gb300 import shard

WORLD = 2


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _init(rank, port):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    return dist


def _cases():
    t8 = textgen.generate("mix", 200_001, textgen.UTF8, seed=0).data
    t16 = textgen.generate("emoji", 300_000, textgen.UTF16, seed=4).data
    bad8 = t8.copy()
    bad8[150_000] = 0xFF                       # error in the second half
    bad8b = t8.copy()
    bad8b[1000] = 0x80                         # stray continuation in the first half
    bad8b[170_000] = 0xC0
    bad16 = t16.copy().view("<u2")
    bad16[120_000] = 0xD800                    # lone high surrogate (second half)
    bad16[120_001] = 0x0041
    tiny = np.frombuffer("é".encode(), dtype=np.uint8).copy()   # 2 bytes: one part is empty
    return [("mix8", t8, False), ("emoji16", t16, True), ("bad8", bad8, False),
            ("bad8b", bad8b, False), ("bad16", bad16.view(np.uint8), True), ("tiny", tiny, False)]


def _whole(data, utf16):
    return oracle.utf16le_to_utf8(data) if utf16 else oracle.utf8_to_utf16le(data)


def _worker_shard(rank, port, ret):
    dist = _init(rank, port)
    try:
        out = {}
        for name, data, utf16 in _cases():
            cuts = shard.split_points(data, WORLD, utf16)
            part = data[cuts[rank]:cuts[rank + 1]]
            r, o = _whole(part, utf16)
            units = part.size // (2 if utf16 else 1)
            base, total = shard.exchange(shard.PartResult(r.status, r.in_offset, r.out_len), units)
            # every rank contributes its valid output at its base
            mine = o[: r.out_len]
            parts = [None] * WORLD
            dist.all_gather_object(parts, (base, np.asarray(mine)))
            out[name] = (total.status, total.in_offset, total.out_len, parts, cuts)
        if rank == 0:
            ret.update(out)
    finally:
        dist.destroy_process_group()


def test_sharded_buffer_equals_whole():
    mgr = mp.Manager()
    ret = mgr.dict()
    mp.spawn(_worker_shard, args=(_free_port(), ret), nprocs=WORLD, join=True)
    for name, data, utf16 in _cases():
        status, in_off, out_len, parts, cuts = ret[name]
        ref, ref_out = _whole(data, utf16)
        assert (status, in_off, out_len) == (ref.status, ref.in_offset, ref.out_len), name
        # bases are the exclusive scan of the parts' lengths
        assert parts[0][0] == 0
        # concatenated valid output = the whole buffer's valid output
        got = np.concatenate([p[1] for p in parts])
        if ref.status == 0:
            assert np.array_equal(got, ref_out[: ref.out_len]), name
        else:
            assert np.array_equal(got[: ref.out_len], ref_out[: ref.out_len]), name
        # cuts sit on character boundaries
        for c in cuts[1:-1]:
            if utf16:
                assert c % 2 == 0 and (int(data.view("<u2")[c // 2]) & 0xFC00) != 0xDC00
            elif c < data.size:
                assert (int(data[c]) & 0xC0) != 0x80


def test_combine_rules():
    P = shard.PartResult
    bases, tot = shard.combine([P(0, 10, 12), P(0, 5, 7), P(0, 3, 3)], [10, 5, 3])
    assert bases == [0, 12, 19] and (tot.status, tot.in_offset, tot.out_len) == (0, 18, 22)
    # first error: the lowest rank with one; prefix = base + local prefix
    bases, tot = shard.combine([P(0, 10, 12), P(2, 4, 5), P(7, 0, 0)], [10, 5, 3])
    assert (tot.status, tot.in_offset, tot.out_len) == (2, 14, 17)
    with pytest.raises(ValueError):
        shard.split_points(np.zeros(4, np.uint8), 0, False)
    assert shard.split_points(np.zeros(0, np.uint8), 3, False) == [0, 0, 0, 0]


def _worker_rate(rank, port, ret):
    import bench
    dist = _init(rank, port)
    try:
        # rank-specific inputs (the benchmark seeds each rank differently)
        cases = bench.gen_inputs(["latin"], 4096, rank, None)
        local_bytes = sum(c["data"].size for c in cases)
        gbs, ms = bench.job_rate(local_bytes * (rank + 1), 10.0 * (rank + 1), WORLD, "cpu")
        digest = [bytes(c["data"][:64]) for c in cases]
        objs = [None] * WORLD
        dist.all_gather_object(objs, digest)
        if rank == 0:
            ret["rate"] = (gbs, ms, local_bytes, objs)
    finally:
        dist.destroy_process_group()


def test_job_rate_and_rank_inputs():
    mgr = mp.Manager()
    ret = mgr.dict()
    mp.spawn(_worker_rate, args=(_free_port(), ret), nprocs=WORLD, join=True)
    gbs, ms, local_bytes, objs = ret["rate"]
    assert ms == 20.0                                          # the slowest rank's time
    assert abs(gbs - (local_bytes * 3) / 0.020 / 1e9) < 1e-9   # all ranks' bytes
    assert objs[0] != objs[1]                                  # ranks draw different text


def test_parallel_oracle_cuts():
    """The N-core oracle timing's cuts: at character boundaries, and the
    parts' conversions concatenate to the whole buffer's."""
    import bench
    for prof, enc in (("emoji", textgen.UTF8), ("emoji", textgen.UTF16), ("cjk", textgen.UTF8)):
        data = textgen.generate(prof, 300_002 if enc == textgen.UTF16 else 300_001, enc, seed=9).data
        u16 = enc == textgen.UTF16
        f = oracle.utf16le_to_utf8 if u16 else oracle.utf8_to_utf16le
        for parts in (1, 3, 16):
            cuts = bench._char_cuts(data, parts, u16)
            assert cuts[0] == 0 and cuts[-1] == data.size and cuts == sorted(cuts)
            outs = []
            for a, b in zip(cuts[:-1], cuts[1:]):
                r, o = f(data[a:b])
                assert r.status == 0
                outs.append(o)
            assert np.array_equal(np.concatenate(outs), f(data)[1])
