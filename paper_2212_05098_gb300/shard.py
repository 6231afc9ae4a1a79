"""Splitting one buffer across ranks (one process per GPU).

The transcoding of one buffer shards with a single exchange step: every rank
takes a contiguous part cut at a character boundary (a part starts at a UTF-8
lead byte or at a UTF-16 word that is not a low surrogate, so every character
belongs to exactly one rank), transcodes or counts it on its own GPU, and the
ranks exchange one (output length, first error) pair each. An exclusive scan
of the lengths gives every rank the output offset of its part; the first error
of the buffer is the first error of the lowest rank that has one, and the
valid prefix before it is that rank's offset plus its local prefix. This is
the decoupled look-back of the kernel lifted to ranks, with one all-gather
instead of a look-back (the paper's parallel idea of computing the segment
sizes first, Sec. 8).

Only the host-side logic lives here; the per-rank work is whatever callable
the caller passes (the library's GPU calls in a multi-GPU program).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

__all__ = ["split_points", "PartResult", "combine", "exchange"]


def split_points(data: np.ndarray, parts: int, utf16: bool) -> list[int]:
    """Byte offsets [0, s1, ..., len] cutting `data` into `parts` contiguous
    pieces of nearly equal size, each starting at a character boundary.

    UTF-8: a cut is moved forward past continuation bytes (10xxxxxx), at most
    3 of them; UTF-16LE: a cut is moved forward by one word when it would
    start at a low surrogate. Invalid input is cut the same way (an invalid
    sequence is then reported by the rank that holds its first unit)."""
    if parts < 1:
        raise ValueError("parts must be >= 1")
    n = int(data.size)
    unit = 2 if utf16 else 1
    cuts = [0]
    for k in range(1, parts):
        c = (n * k // parts) // unit * unit
        c = max(c, cuts[-1])
        if utf16:
            w = data.view("<u2")
            if c // 2 < w.size and (int(w[c // 2]) & 0xFC00) == 0xDC00:
                c += 2
        else:
            steps = 0
            while c < n and (int(data[c]) & 0xC0) == 0x80 and steps < 3:
                c += 1
                steps += 1
        cuts.append(min(c, n))
    cuts.append(n)
    return cuts


@dataclass
class PartResult:
    """What one rank reports about its part: the status of its local call
    (0 = OK), the first-error offset within the part (input units) and the
    output length (the full length on success, the valid prefix's length on
    an error)."""
    status: int
    in_offset: int
    out_len: int


def combine(results: list[PartResult], part_units: list[int]) -> tuple[list[int], PartResult]:
    """Output offset of every part, and the buffer's result (gbu_result
    semantics) from the per-part results in rank order."""
    bases, total_in, total_out = [], 0, 0
    first = None
    for r, units in zip(results, part_units):
        bases.append(total_out)
        if first is None and r.status != 0:
            first = PartResult(r.status, total_in + r.in_offset, total_out + r.out_len)
        total_in += units
        total_out += r.out_len
    if first is None:
        first = PartResult(0, total_in, total_out)
    return bases, first


def exchange(local: PartResult, local_units: int, group=None) -> tuple[int, PartResult]:
    """All-gather every rank's (status, offset, length, units) and combine:
    returns this rank's output offset and the buffer's result. Works with any
    torch.distributed backend (one 32-byte message per rank)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    mine = torch.tensor([local.status, local.in_offset, local.out_len, local_units], dtype=torch.int64)
    if dist.get_backend(group) == "nccl":
        mine = mine.cuda()
    got = [torch.zeros_like(mine) for _ in range(world)]
    dist.all_gather(got, mine, group=group)
    rows = [g.cpu().tolist() for g in got]
    results = [PartResult(int(s), int(o), int(l)) for s, o, l, _ in rows]
    bases, total = combine(results, [int(u) for *_, u in rows])
    return bases[rank], total
