"""Seeded synthetic text for the transcoder's tests and benchmark.

This module holds no transcoding arithmetic. It draws code points from the
text profiles below with a counter-based generator (numpy's Philox-4x64, Salmon
et al., SC'11), and turns them into UTF-8 / UTF-16LE bytes with Python's
built-in codecs. It serves both the oracle side and the CUDA side of the tests
and is the only code they share.

Profiles (code points i.i.d.; "ASCII" means U+0020-U+007E):
  mix       60% ASCII, 25% U+0080-U+07FF, 10% U+0800-U+FFFF without
            U+D800-U+DFFF, 5% U+10000-U+10FFFF           (1 MiB parity case)
  latin     95% ASCII, 5% U+00C0-U+017F
  cyrillic  15% space/punctuation {space , . ; : ! ? - ( ) "}, 85% U+0400-U+04FF
  cjk       10% ASCII, 90% U+4E00-U+9FFF
  emoji     50% ASCII, 20% U+0080-U+07FF, 30% U+1F300-U+1FAFF

The four profiles latin/cyrillic/cjk/emoji stand in for the paper's lipsum
files (Sec. 8.1: Latin; Arabic/Hebrew/Russian; Chinese/Japanese/Korean/Hindi;
Emoji), which are not available.

Every category of a profile has a single encoded length in each encoding; the
lengths are part of the profile's data (they follow from the category's code
point range) and are used to cut text at character boundaries and to place
injected errors.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

ASCII = ((0x20, 0x7E),)
PUNCT = tuple((c, c) for c in map(ord, ' ,.;:!?-()"'))


@dataclass(frozen=True)
class Category:
    prob: float
    ranges: tuple          # inclusive (lo, hi) code point ranges
    utf8_len: int          # bytes per character in UTF-8
    utf16_len: int         # 16-bit units per character in UTF-16

    @property
    def size(self) -> int:
        return sum(hi - lo + 1 for lo, hi in self.ranges)


PROFILES = {
    "mix": (
        Category(0.60, ASCII, 1, 1),
        Category(0.25, ((0x80, 0x7FF),), 2, 1),
        Category(0.10, ((0x800, 0xD7FF), (0xE000, 0xFFFF)), 3, 1),
        Category(0.05, ((0x10000, 0x10FFFF),), 4, 2),
    ),
    "latin": (
        Category(0.95, ASCII, 1, 1),
        Category(0.05, ((0xC0, 0x17F),), 2, 1),
    ),
    "cyrillic": (
        Category(0.15, PUNCT, 1, 1),
        Category(0.85, ((0x400, 0x4FF),), 2, 1),
    ),
    "cjk": (
        Category(0.10, ASCII, 1, 1),
        Category(0.90, ((0x4E00, 0x9FFF),), 3, 1),
    ),
    "emoji": (
        Category(0.50, ASCII, 1, 1),
        Category(0.20, ((0x80, 0x7FF),), 2, 1),
        Category(0.30, ((0x1F300, 0x1FAFF),), 4, 2),
    ),
}

BENCH_PROFILES = ("latin", "cyrillic", "cjk", "emoji")
PROFILE_SEED = {"mix": 0, "latin": 1, "cyrillic": 2, "cjk": 3, "emoji": 4}

UTF8 = "utf8"
UTF16 = "utf16le"


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=int(seed)))


def _unit_bytes(encoding: str) -> int:
    return 1 if encoding == UTF8 else 2


def draw_chars(profile: str, n_chars: int, seed: int):
    """Return (code points uint32[n_chars], category index uint8[n_chars])."""
    cats = PROFILES[profile]
    rng = _rng(seed)
    cum = np.cumsum([c.prob for c in cats])
    cum[-1] = 1.0
    u = rng.random(n_chars, dtype=np.float64)
    cat = np.searchsorted(cum, u, side="right").astype(np.uint8)
    np.minimum(cat, len(cats) - 1, out=cat)
    cps = np.empty(n_chars, dtype=np.uint32)
    for k, c in enumerate(cats):
        idx = np.nonzero(cat == k)[0]
        if idx.size == 0:
            continue
        r = rng.integers(0, c.size, size=idx.size, dtype=np.int64)
        # map a uniform index into the union of the category's ranges
        vals = np.empty(idx.size, dtype=np.int64)
        base = 0
        for lo, hi in c.ranges:
            w = hi - lo + 1
            m = (r >= base) & (r < base + w)
            vals[m] = lo + (r[m] - base)
            base += w
        cps[idx] = vals.astype(np.uint32)
    return cps, cat


def encode(cps: np.ndarray, encoding: str) -> np.ndarray:
    """Encode code points with Python's codecs; returns a uint8 array."""
    s = np.ascontiguousarray(cps, dtype="<u4").tobytes().decode("utf-32-le")
    b = s.encode("utf-8" if encoding == UTF8 else "utf-16-le")
    return np.frombuffer(b, dtype=np.uint8)


@dataclass
class Text:
    profile: str
    encoding: str
    seed: int
    data: np.ndarray            # uint8 bytes in `encoding`
    cps: np.ndarray             # code points, including the U+0020 padding
    in_len: np.ndarray          # uint8 input units per character (this encoding)
    out_len: np.ndarray         # uint8 output units per character (other encoding)

    @property
    def n_units(self) -> int:
        return self.data.size // _unit_bytes(self.encoding)

    def char_starts(self) -> np.ndarray:
        """int64 input-unit offset of every character, plus the end."""
        s = np.zeros(self.in_len.size + 1, dtype=np.int64)
        np.cumsum(self.in_len, dtype=np.int64, out=s[1:])
        return s

    def out_starts(self) -> np.ndarray:
        s = np.zeros(self.out_len.size + 1, dtype=np.int64)
        np.cumsum(self.out_len, dtype=np.int64, out=s[1:])
        return s


def generate(profile: str, target_bytes: int, encoding: str, seed: int | None = None) -> Text:
    """Seeded text of exactly `target_bytes` bytes in `encoding`.

    Characters are appended until the next one would pass the target, then the
    text is padded with U+0020 to the exact size (the target must be even for
    UTF-16LE).
    """
    if seed is None:
        seed = PROFILE_SEED[profile]
    ub = _unit_bytes(encoding)
    if target_bytes % ub:
        raise ValueError("UTF-16LE text needs an even byte count")
    target_units = target_bytes // ub
    cats = PROFILES[profile]
    in_tab = np.array([c.utf8_len if encoding == UTF8 else c.utf16_len for c in cats], np.uint8)
    out_tab = np.array([c.utf16_len if encoding == UTF8 else c.utf8_len for c in cats], np.uint8)
    mean = sum(c.prob * int(in_tab[k]) for k, c in enumerate(cats))
    n_draw = int(target_units / mean * 1.02) + 64
    cps, cat = draw_chars(profile, n_draw, seed)
    in_len = in_tab[cat]
    cum = np.cumsum(in_len, dtype=np.int64)
    k = int(np.searchsorted(cum, target_units, side="right"))
    if k == n_draw and cum[-1] < target_units:
        raise RuntimeError("generator under-drew; increase the margin")
    used = int(cum[k - 1]) if k else 0
    pad = target_units - used
    cps = np.concatenate([cps[:k], np.full(pad, 0x20, np.uint32)])
    space = np.ones(pad, np.uint8)
    in_len = np.concatenate([in_len[:k], space])
    out_len = np.concatenate([out_tab[cat[:k]], space])
    data = encode(cps, encoding)
    assert data.size == target_bytes
    return Text(profile, encoding, seed, np.array(data), cps, in_len, out_len)


def random_bytes(n: int, seed: int) -> np.ndarray:
    return _rng(seed).integers(0, 256, size=n, dtype=np.uint8)


def mutate(data: np.ndarray, n_flips: int, seed: int) -> np.ndarray:
    """Copy of `data` with `n_flips` seeded random bytes overwritten."""
    out = np.array(data, copy=True)
    if out.size == 0 or n_flips <= 0:
        return out
    rng = _rng(seed)
    pos = rng.integers(0, out.size, size=n_flips)
    out[pos] = rng.integers(0, 256, size=n_flips, dtype=np.uint8)
    return out
