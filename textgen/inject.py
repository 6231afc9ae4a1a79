"""Seeded encoding-error injection for the validation-stress cases.

Each case replaces a window of whole characters of a valid text with U+0020
spaces followed by one malformed pattern. The pattern's first error, its kind
and the output length of the valid prefix are known by construction, so the
injector gives an expectation that is independent of both transcoders.

UTF-8 patterns (Sec. 6.4 validation rules 1-6):
  overlong2    C0/C1 + continuation                    OVERLONG    at the lead
  overlong3    E0 80-9F cont                           OVERLONG    at the lead
  overlong4    F0 80-8F cont cont                      OVERLONG    at the lead
  surrogate    ED A0-BF cont                           SURROGATE   at the lead
  too_large    F4 90-BF cont cont                      TOO_LARGE   at the lead
  short_edge   a 2/3/4-byte lead at edge-1/-2/-3 whose sequence is cut by a
               space at the edge (edges: multiples of 4..64 KiB), or by the
               end of the buffer                       TOO_SHORT   at the lead
  stray        a continuation byte after a space       TOO_LONG    at it
  header       F5-FF                                   HEADER_BITS at it
UTF-16LE patterns (Sec. 7.4 sequencing):
  lone_high    high surrogate then U+0020              LONE_HIGH   at it
  lone_low     U+0020 then low surrogate               LONE_LOW    at the low
  reversed     low then high surrogate                 LONE_LOW    at the low
  high_last    high surrogate as the last unit         LONE_HIGH   at it
  low_first    low surrogate as the first unit         LONE_LOW    at it
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import UTF8, Text, _rng

# status codes of the library's public enum
HEADER_BITS, TOO_SHORT, TOO_LONG, OVERLONG, TOO_LARGE, SURROGATE = 1, 2, 3, 4, 5, 6
LONE_HIGH_SURROGATE, LONE_LOW_SURROGATE = 7, 8

UTF8_CASES = ("overlong2", "overlong3", "overlong4", "surrogate", "too_large",
              "short_edge", "stray", "header")
UTF16_CASES = ("lone_high", "lone_low", "reversed", "high_last", "low_first")
EDGES = tuple(k * 1024 for k in (4, 8, 16, 32, 64))


@dataclass
class Patch:
    case: str
    offset: int               # byte offset of the replaced window
    data: np.ndarray          # uint8 replacement bytes (same length as the window)
    kind: int                 # expected status
    err_unit: int             # expected first-error offset, in input units
    prefix_out: int           # expected output units of the valid prefix

    def apply(self, buf: np.ndarray) -> np.ndarray:
        out = np.array(buf, copy=True)
        out[self.offset:self.offset + self.data.size] = self.data
        return out


def _cont(rng, lo=0x80, hi=0xBF):
    return int(rng.integers(lo, hi + 1))


def _utf8_pattern(case: str, rng):
    """(pattern bytes, index of the error in the pattern, kind)."""
    if case == "overlong2":
        return [int(rng.integers(0xC0, 0xC2)), _cont(rng)], 0, OVERLONG
    if case == "overlong3":
        return [0xE0, _cont(rng, 0x80, 0x9F), _cont(rng)], 0, OVERLONG
    if case == "overlong4":
        return [0xF0, _cont(rng, 0x80, 0x8F), _cont(rng), _cont(rng)], 0, OVERLONG
    if case == "surrogate":
        return [0xED, _cont(rng, 0xA0, 0xBF), _cont(rng)], 0, SURROGATE
    if case == "too_large":
        return [0xF4, _cont(rng, 0x90, 0xBF), _cont(rng), _cont(rng)], 0, TOO_LARGE
    if case == "stray":
        return [_cont(rng)], 0, TOO_LONG
    if case == "header":
        return [int(rng.integers(0xF5, 0x100))], 0, HEADER_BITS
    raise ValueError(case)


def _truncated_lead(rng, k: int):
    """A lead byte whose sequence needs more than the k-1 bytes that follow it
    before the cut; returns the bytes before the cut (lead + k-1 continuations)."""
    # sequence length strictly greater than k
    length = int(rng.integers(k + 1, 5)) if k < 4 else 4
    lead = {2: 0xD0, 3: 0xE4, 4: 0xF0}[length]
    body = [lead]
    for j in range(1, k):
        # keep the prefix free of value errors: F0 needs >= 90, E4 any
        body.append(_cont(rng, 0x90, 0xBF) if (lead == 0xF0 and j == 1) else _cont(rng))
    return body


def _window(text: Text, starts: np.ndarray, lo_unit: int, hi_unit: int):
    """Smallest window of whole characters covering units [lo_unit, hi_unit)."""
    j0 = int(np.searchsorted(starts, lo_unit, side="right")) - 1
    j1 = int(np.searchsorted(starts, hi_unit, side="left"))
    j1 = min(max(j1, j0 + 1), starts.size - 1)
    return j0, j1


def make_patch(text: Text, case_index: int, seed: int,
               starts: np.ndarray | None = None,
               out_starts: np.ndarray | None = None) -> Patch:
    """Case `case_index` (round-robin over the kinds) for `text`."""
    rng = _rng(seed * 1_000_003 + case_index)
    if starts is None:
        starts = text.char_starts()
    if out_starts is None:
        out_starts = text.out_starts()
    n = text.n_units
    ub = 1 if text.encoding == UTF8 else 2

    if text.encoding == UTF8:
        case = UTF8_CASES[case_index % len(UTF8_CASES)]
        if case == "short_edge":
            k = int(rng.integers(1, 4))                 # lead at edge - k
            at_end = case_index % 7 == 5
            if at_end:
                edge = n
            else:
                e = EDGES[int(rng.integers(0, len(EDGES)))]
                edge = e * int(rng.integers(1, max(2, n // e)))
                edge = min(edge, n - 1)
            body = _truncated_lead(rng, k)
            if not at_end:
                body = body + [0x20]                    # the cut at the edge
            pat_at = edge - k
            kind, err_in_pat = TOO_SHORT, 0
        else:
            body, err_in_pat, kind = _utf8_pattern(case, rng)
            pat_at = int(rng.integers(0, max(1, n - len(body) - 8)))
    else:
        case = UTF16_CASES[case_index % len(UTF16_CASES)]
        hi = int(rng.integers(0xD800, 0xDC00))
        lo = int(rng.integers(0xDC00, 0xE000))
        if case == "lone_high":
            body, err_in_pat, kind = [hi, 0x20], 0, LONE_HIGH_SURROGATE
        elif case == "lone_low":
            body, err_in_pat, kind = [0x20, lo], 1, LONE_LOW_SURROGATE
        elif case == "reversed":
            body, err_in_pat, kind = [lo, hi, 0x20], 0, LONE_LOW_SURROGATE
        elif case == "high_last":
            body, err_in_pat, kind = [hi], 0, LONE_HIGH_SURROGATE
        else:
            body, err_in_pat, kind = [lo], 0, LONE_LOW_SURROGATE
        if case == "high_last":
            pat_at = n - 1
        elif case == "low_first":
            pat_at = 0
        else:
            pat_at = int(rng.integers(0, max(1, n - len(body) - 8)))

    j0, j1 = _window(text, starts, pat_at, pat_at + len(body))
    w_lo, w_hi = int(starts[j0]), int(starts[j1])
    units = np.full(w_hi - w_lo, 0x20, dtype=np.uint32)
    units[pat_at - w_lo: pat_at - w_lo + len(body)] = body
    if ub == 1:
        data = units.astype(np.uint8)
    else:
        data = units.astype("<u2").view(np.uint8)
    err_unit = pat_at + err_in_pat
    # valid prefix: characters before the window, the spaces before the
    # pattern, and (lone_low) the pattern's own leading space
    prefix_out = int(out_starts[j0]) + (pat_at - w_lo) + err_in_pat
    return Patch(case, w_lo * ub, data, kind, err_unit, prefix_out)
