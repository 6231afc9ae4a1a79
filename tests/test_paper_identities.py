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
