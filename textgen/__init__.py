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


def _rng(seed: int, block: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[int(seed), int(block)]))


def _unit_bytes(encoding: str) -> int:
    return 1 if encoding == UTF8 else 2


# Characters per independently keyed block: block b of seed s is drawn from
# Philox with key (s, b), so any block can be produced on its own and the text
# does not depend on how blocks are spread over worker processes.
BLOCK = 1 << 22


def _draw_block(profile: str, seed: int, block: int, n: int = BLOCK):
    """Code points and category indices of one block of `n` characters."""
    cats = PROFILES[profile]
    # interleaved (category, offset) pairs: the first n characters of a block
    # do not depend on how many are drawn
    u = _rng(seed, block).integers(0, 1 << 32, size=(n, 2), dtype=np.uint32)
    u1, u2 = u[:, 0], u[:, 1].astype(np.uint64)
    cat = np.zeros(n, dtype=np.uint8)
    acc = 0.0
    for c in cats[:-1]:
        acc += c.prob
        cat += (u1 >= np.uint32(min(int(acc * 2.0**32), (1 << 32) - 1))).astype(np.uint8)
    sizes = np.array([c.size for c in cats], dtype=np.uint64)
    off = (u2 * sizes[cat]) >> np.uint64(32)          # uniform in [0, size)
    cps = np.empty(n, dtype=np.uint32)
    for k, c in enumerate(cats):
        m = cat == k
        o = off[m].astype(np.int64)
        if len(c.ranges) == 1:
            cps[m] = (c.ranges[0][0] + o).astype(np.uint32)
        else:
            widths = np.array([hi - lo + 1 for lo, hi in c.ranges], dtype=np.int64)
            base = np.concatenate([[0], np.cumsum(widths)[:-1]])
            los = np.array([lo for lo, _ in c.ranges], dtype=np.int64)
            idx = np.searchsorted(base, o, side="right") - 1
            cps[m] = (los[idx] + (o - base[idx])).astype(np.uint32)
    return cps, cat


def draw_chars(profile: str, n_chars: int, seed: int):
    """Return (code points uint32[n_chars], category index uint8[n_chars])."""
    parts = [_draw_block(profile, seed, b, min(BLOCK, n_chars - b * BLOCK))
             for b in range((n_chars + BLOCK - 1) // BLOCK)]
    if not parts:
        return np.zeros(0, np.uint32), np.zeros(0, np.uint8)
    return np.concatenate([p[0] for p in parts]), np.concatenate([p[1] for p in parts])


def encode(cps: np.ndarray, encoding: str) -> np.ndarray:
    """Encode code points with Python's codecs; returns a uint8 array."""
    s = np.ascontiguousarray(cps, dtype="<u4").tobytes().decode("utf-32-le")
    b = s.encode("utf-8" if encoding == UTF8 else "utf-16-le")
    return np.frombuffer(b, dtype=np.uint8)


def _encoded_block(profile: str, seed: int, block: int, encoding: str, keep_cps: bool,
                   n: int = BLOCK, keep_cat: bool = True):
    cps, cat = _draw_block(profile, seed, block, n)
    data = encode(cps, encoding).tobytes()
    return data, (cat if keep_cat else None), (cps if keep_cps else None)


@dataclass
class Text:
    profile: str
    encoding: str
    seed: int
    data: np.ndarray            # uint8 bytes in `encoding`
    in_len: np.ndarray | None   # uint8 input units per character (this encoding)
    out_len: np.ndarray | None  # uint8 output units per character (other encoding)
    cps: np.ndarray | None = None   # code points incl. padding (when requested)

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


def generate(profile: str, target_bytes: int, encoding: str, seed: int | None = None,
             executor=None, keep_cps: bool = True, keep_lens: bool = True) -> Text:
    """Seeded text of exactly `target_bytes` bytes in `encoding`.

    Characters are appended until the next one would pass the target, then the
    text is padded with U+0020 to the exact size (the target must be even for
    UTF-16LE). `executor` (a concurrent.futures executor, e.g. a process pool
    started with "spawn") draws blocks in parallel; the text is the same either
    way. With keep_lens=False (large benchmark inputs) the per-character
    length arrays are not kept.
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
    n_blocks = int(target_units / (mean * BLOCK) * 1.01) + 1

    blocks = []
    have = 0
    b = 0
    if target_units < 0.9 * mean * BLOCK:
        # small text: the needed prefix of block 0 (the same characters)
        n0 = min(BLOCK, int(target_units / mean * 1.05) + 256)
        data, cat, cps = _encoded_block(profile, seed, 0, encoding, keep_cps, n0)
        if len(data) // ub >= target_units:
            blocks.append((data, cat, cps))
            have = target_units
    while have < target_units:
        todo = list(range(b, b + max(1, n_blocks - b)))
        if executor is not None and len(todo) > 1:
            futs = [executor.submit(_encoded_block, profile, seed, k, encoding, keep_cps,
                                    BLOCK, keep_lens) for k in todo]
            got = [f.result() for f in futs]
        else:
            got = [_encoded_block(profile, seed, k, encoding, keep_cps, BLOCK, keep_lens)
                   for k in todo]
        for data, cat, cps in got:
            if have >= target_units:
                break
            blocks.append((data, cat, cps))
            have += len(data) // ub
        b = todo[-1] + 1
        n_blocks = b + 1

    # cut inside the last block at the last character that still fits
    datas, cats_l, cps_l = [], [], []
    used = 0
    for data, cat, cps in blocks:
        units = len(data) // ub
        if used + units <= target_units:
            datas.append(np.frombuffer(data, np.uint8))
            cats_l.append(cat)
            if cps is not None:
                cps_l.append(cps)
            used += units
            continue
        if cat is None:   # redraw the last block's categories here (same key)
            cat = _draw_block(profile, seed, len(datas), BLOCK)[1]
        lens = in_tab[cat]
        cum = np.cumsum(lens, dtype=np.int64)
        k = int(np.searchsorted(cum, target_units - used, side="right"))
        take = int(cum[k - 1]) if k else 0
        datas.append(np.frombuffer(data, np.uint8)[: take * ub])
        cats_l.append(cat[:k])
        if cps is not None:
            cps_l.append(cps[:k])
        used += take
        break
    pad = target_units - used
    space = np.full(pad, 0x20, np.uint32)
    datas.append(encode(space, encoding))
    data = np.concatenate(datas)
    assert data.size == target_bytes
    in_len = out_len = None
    if keep_lens:
        cat_all = np.concatenate(cats_l) if cats_l else np.zeros(0, np.uint8)
        ones = np.ones(pad, np.uint8)
        in_len = np.concatenate([in_tab[cat_all], ones])
        out_len = np.concatenate([out_tab[cat_all], ones])
    cps_all = np.concatenate(cps_l + [space]) if keep_cps else None
    return Text(profile, encoding, seed, data, in_len, out_len, cps_all)


def process_pool(workers: int | None = None):
    """A process pool started with "spawn" (safe after CUDA initialisation)."""
    import multiprocessing
    import os
    from concurrent.futures import ProcessPoolExecutor
    if workers is None:
        workers = max(1, min(16, (os.cpu_count() or 2) - 1))
    return ProcessPoolExecutor(max_workers=workers,
                               mp_context=multiprocessing.get_context("spawn"))


def random_bytes(n: int, seed: int) -> np.ndarray:
    return _rng(seed, 1 << 40).integers(0, 256, size=n, dtype=np.uint8)


def mutate(data: np.ndarray, n_flips: int, seed: int) -> np.ndarray:
    """Copy of `data` with `n_flips` seeded random bytes overwritten."""
    out = np.array(data, copy=True)
    if out.size == 0 or n_flips <= 0:
        return out
    rng = _rng(seed, 1 << 41)
    pos = rng.integers(0, out.size, size=n_flips)
    out[pos] = rng.integers(0, 256, size=n_flips, dtype=np.uint8)
    return out
