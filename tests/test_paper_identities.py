"""Closed-form identities the paper states and the CUDA kernels rely on,
checked exhaustively with numpy (CPU only)."""
import numpy as np


def test_high_surrogate_offset_constant():
    # Sec. 6.2, footnote to the surrogate fix-up: adding 0xd7c0 applies the
    # tag bits and the surrogate plane shift in one step. The footnote writes
    # the constant as 0xd800 - 0x0020, which is 0xd7e0; the constant itself is
    # right because the plane shift seen after >> 10 is 0x10000 >> 10 = 0x40.
    assert 0xD800 - 0x0020 != 0xD7C0
    assert 0xD7C0 == 0xD800 - (0x10000 >> 10)
    cp = np.arange(0x10000, 0x110000, dtype=np.int64)
    hi = 0xD800 + ((cp - 0x10000) >> 10)
    assert np.array_equal(hi, (cp >> 10) + 0xD7C0)


def test_surrogate_join_constant_all_pairs():
    # Sec. 7.2: hi << 10 + lo + 0xfca02400 (32-bit wrap) is the code point of
    # every valid pair.
    hi = np.arange(0xD800, 0xDC00, dtype=np.uint32)[:, None]
    lo = np.arange(0xDC00, 0xE000, dtype=np.uint32)[None, :]
    joined = ((hi << np.uint32(10)) + lo + np.uint32(0xFCA02400)).astype(np.uint32)
    expect = 0x10000 + ((hi - 0xD800) << 10) + (lo - 0xDC00)
    assert np.array_equal(joined, expect.astype(np.uint32))


def test_pair_bytes_split_between_halves():
    # The UTF-16 -> UTF-8 kernel splits a pair's 4 UTF-8 bytes between its
    # halves: with U = (hi & 0x3FF) + 0x40 (= the code point >> 10, Sec. 7.2's
    # plane shift), the high surrogate gives F0 | U >> 8 and 80 | (U >> 2) & 3F,
    # the low one 80 | (hi & 3) << 4 | (lo >> 6) & F and 80 | lo & 3F. All 2^20
    # pairs against the UTF-8 encoding of the joined code point (Fig. 1(a)).
    hi = np.arange(0xD800, 0xDC00, dtype=np.int64)[:, None]
    lo = np.arange(0xDC00, 0xE000, dtype=np.int64)[None, :]
    cp = 0x10000 + ((hi - 0xD800) << 10) + (lo - 0xDC00)
    u = (hi & 0x3FF) + 0x40
    assert np.array_equal(np.broadcast_to(u, cp.shape), cp >> 10)
    b0 = np.broadcast_to(0xF0 | (u >> 8), cp.shape)
    b1 = np.broadcast_to(0x80 | ((u >> 2) & 0x3F), cp.shape)
    b2 = 0x80 | ((hi & 3) << 4) | ((lo >> 6) & 0xF)
    b3 = np.broadcast_to(0x80 | (lo & 0x3F), cp.shape)
    assert np.array_equal(b0, 0xF0 | (cp >> 18))
    assert np.array_equal(b1, 0x80 | ((cp >> 12) & 0x3F))
    assert np.array_equal(b2, 0x80 | ((cp >> 6) & 0x3F))
    assert np.array_equal(b3, 0x80 | (cp & 0x3F))
    # spot-check against the codec
    for h, l in ((0xD800, 0xDC00), (0xDBFF, 0xDFFF), (0xD83D, 0xDE00)):
        c = 0x10000 + ((h - 0xD800) << 10) + (l - 0xDC00)
        uu = (h & 0x3FF) + 0x40
        got = bytes([0xF0 | (uu >> 8), 0x80 | ((uu >> 2) & 0x3F),
                     0x80 | ((h & 3) << 4) | ((l >> 6) & 0xF), 0x80 | (l & 0x3F)])
        assert got == chr(c).encode("utf-8")
