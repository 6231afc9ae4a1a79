"""Seeded layouts of many independent strings (the batched workload).

Each string is a window of one of the per-(profile, encoding) corpora, cut at
character boundaries, so every string is valid text of its profile. Lengths
are log-uniform between `lo` and `hi` bytes (UTF-16 lengths rounded down to an
even count), the profile is uniform over the given corpora's profiles and the
direction is 50/50 (UTF-8 input -> UTF-16LE output, or the reverse). Pure
input generation: none of the transcoding arithmetic lives here.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import UTF8, UTF16, _rng


@dataclass
class Layout:
    corpus: np.ndarray   # int32 index into the corpus list
    start: np.ndarray    # int64 byte offset in the corpus
    nbytes: np.ndarray   # int64 byte length (even for UTF-16)

    @property
    def total_bytes(self) -> int:
        return int(self.nbytes.sum())


def draw_lengths(n: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """n lengths log-uniform over [lo, hi] bytes (int64)."""
    rng = _rng(seed, 1 << 41)
    u = rng.random(n)
    return np.floor(np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo)))).astype(np.int64)


def layout(corpora: list[tuple[str, str, np.ndarray]], n: int, lo: int, hi: int, seed: int,
           scale: float = 1.0, min_bytes: int = 2) -> Layout:
    """Windows for n strings over `corpora` = [(profile, encoding, bytes), ...].

    A string picks a profile uniformly, then a direction 50/50 (the corpus of
    that profile in that input encoding), a length (log-uniform, times `scale`,
    at least `min_bytes`) and a uniform start, then moves start and end to
    character boundaries of its corpus.
    """
    rng = _rng(seed, 1 << 42)
    profiles = sorted({p for p, _, _ in corpora})
    index = {(p, e): k for k, (p, e, _) in enumerate(corpora)}
    prof = rng.integers(0, len(profiles), size=n)
    to16 = rng.random(n) < 0.5
    enc = np.where(to16, 0, 1)   # 0: UTF-8 input, 1: UTF-16LE input
    corpus = np.array([index[(profiles[p], UTF8 if e == 0 else UTF16)] for p, e in zip(prof, enc)],
                      dtype=np.int32)
    length = np.maximum((draw_lengths(n, lo, hi, seed) * scale).astype(np.int64), min_bytes)
    sizes = np.array([c[2].size for c in corpora], dtype=np.int64)[corpus]
    length = np.minimum(length, sizes)
    length = np.where(enc == 1, length & ~1, length)
    start = (rng.random(n) * (sizes - length + 1)).astype(np.int64)
    start = np.where(enc == 1, start & ~1, start)
    end = start + length
    for k, (_, e, data) in enumerate(corpora):
        sel = np.nonzero(corpus == k)[0]
        if sel.size == 0:
            continue
        s, t = start[sel], end[sel]
        if e == UTF8:
            # a boundary is a byte that is not a continuation (10xxxxxx), or the end
            for _ in range(3):
                s = np.where((s < data.size) & ((data[np.minimum(s, data.size - 1)] & 0xC0) == 0x80),
                             s + 1, s)
                t = np.where((t < data.size) & ((data[np.minimum(t, data.size - 1)] & 0xC0) == 0x80),
                             t - 1, t)
        else:
            w = data.view("<u2")
            # do not start on a low surrogate, do not end after a high one
            s = np.where((s // 2 < w.size) & ((w[np.minimum(s // 2, w.size - 1)] & 0xFC00) == 0xDC00),
                         s + 2, s)
            t = np.where((t >= 2) & ((w[np.maximum(t // 2 - 1, 0)] & 0xFC00) == 0xD800), t - 2, t)
        t = np.maximum(t, s)
        start[sel], end[sel] = s, t
    return Layout(corpus, start, end - start)


@dataclass
class Trace:
    layout: Layout
    t_arrival: np.ndarray      # float64 seconds, non-decreasing
    error_at: np.ndarray       # int64 byte offset of the injected error in the string, -1: none


def poisson_arrivals(n: int, rate: float, seed: int) -> np.ndarray:
    """n arrival times (seconds) of a Poisson process of `rate` per second."""
    rng = _rng(seed, 1 << 43)
    return np.cumsum(rng.exponential(1.0 / rate, size=n))


def serving_trace(corpora, n: int, rate: float, seed: int, lo: int = 64, hi: int = 16 << 20,
                  error_frac: float = 0.01) -> Trace:
    """Requests of a serving run: sizes log-uniform over [lo, hi] bytes,
    profile uniform, direction 50/50 (as `layout`), Poisson arrivals at `rate`
    requests per second, and `error_frac` of them marked for one injected
    error at a uniform position (see `inject_error`)."""
    lay = layout(corpora, n, lo, hi, seed)
    rng = _rng(seed, 1 << 44)
    err = rng.random(n) < error_frac
    pos = (rng.random(n) * np.maximum(lay.nbytes, 1)).astype(np.int64)
    error_at = np.where(err & (lay.nbytes > 0), pos, -1)
    return Trace(lay, poisson_arrivals(n, rate, seed), error_at)


def inject_error(data: np.ndarray, at: int, encoding: str) -> np.ndarray:
    """A copy of `data` (one string) with an invalid unit written at byte `at`:
    0xFF in UTF-8 (a byte that never occurs in UTF-8), or a high surrogate
    followed by U+0041 in UTF-16LE (a lone high surrogate). The first error of
    the result is at or before that position."""
    out = data.copy()
    if encoding == UTF8:
        out[at] = 0xFF
    else:
        w = out.view("<u2")
        u = at // 2
        w[u] = 0xD800
        if u + 1 < w.size:
            w[u + 1] = 0x0041
    return out
