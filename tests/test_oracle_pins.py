"""Pins of the oracle to values outside itself (CPU only).

- Fig. 1(b) code points and the worked byte strings the paper prints
  (tests/golden/*.txt);
- an exhaustive round trip of every Unicode scalar value against Python's
  built-in codecs (an independent implementation);
- seeded fuzzing against Python's codecs (first-error offsets, prefix output);
- every 1-4 byte UTF-8 string and every 1-2 unit UTF-16 string against a
  matcher of the Unicode well-formed byte-sequence table (tests/brute);
- the capacity / error-precedence conventions of the library's interface.
"""
import os
import subprocess

import numpy as np
import pytest

import oracle
import textgen

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                yield [c.strip() for c in line.split("|")]


def _u16(words):
    return np.array(words, dtype="<u2")


# --- Fig. 1(b) ---------------------------------------------------------------

@pytest.mark.parametrize("row", list(_rows("fig1b_examples.txt")), ids=lambda r: r[0])
def test_fig1b_examples(row):
    cp = int(row[0][2:], 16)
    words = [int(w, 2) for w in row[1].split()]
    utf8 = bytes(int(b, 2) for b in row[2].split())
    r, out = oracle.utf8_to_utf16le(utf8)
    assert r == oracle.Result(oracle.OK, len(utf8), len(words))
    assert out.tolist() == words
    r, out = oracle.utf16le_to_utf8(_u16(words))
    assert r == oracle.Result(oracle.OK, len(words), len(utf8))
    assert out.tobytes() == utf8
    # the figure's code point column, through the surrogate rule of Sec. 2.1
    if len(words) == 1:
        assert words[0] == cp
    else:
        assert 0x10000 + ((words[0] - 0xD800) << 10) + (words[1] - 0xDC00) == cp


@pytest.mark.parametrize("row", list(_rows("worked_examples.txt")), ids=lambda r: r[0])
def test_worked_examples(row):
    utf8 = bytes.fromhex(row[1])
    r, out = oracle.utf8_to_utf16le(utf8)
    assert r.status == oracle.OK and r.in_offset == len(utf8)
    if row[2] != "-":
        words = [int(w, 16) for w in row[2].split()]
        assert out.tolist() == words
    r2, back = oracle.utf16le_to_utf8(out)
    assert r2.status == oracle.OK and back.tobytes() == utf8


# --- exhaustive scalar round trip against Python's codecs --------------------

def _all_scalars():
    return np.concatenate([np.arange(0, 0xD800), np.arange(0xE000, 0x110000)]).astype(np.uint32)


def test_all_scalars_match_python_codecs():
    cps = _all_scalars()
    assert cps.size == 1_112_064
    s = cps.astype("<u4").tobytes().decode("utf-32-le")
    u8 = s.encode("utf-8")
    u16 = np.frombuffer(s.encode("utf-16-le"), dtype="<u2")

    r, out = oracle.utf8_to_utf16le(u8)
    assert r == oracle.Result(oracle.OK, len(u8), u16.size)
    assert np.array_equal(out, u16)

    r, out = oracle.utf16le_to_utf8(u16)
    assert r == oracle.Result(oracle.OK, u16.size, len(u8))
    assert out.tobytes() == u8

    assert oracle.utf16_length_from_utf8(u8) == oracle.Result(oracle.OK, len(u8), u16.size)
    assert oracle.utf8_length_from_utf16le(u16) == oracle.Result(oracle.OK, u16.size, len(u8))


def test_each_scalar_length_matches_python():
    # per-scalar output lengths (one call per length class boundary region)
    for cp in [0, 0x7F, 0x80, 0x7FF, 0x800, 0xD7FF, 0xE000, 0xFFFF, 0x10000, 0x10FFFF]:
        c = chr(cp)
        r = oracle.utf16_length_from_utf8(c.encode("utf-8"))
        assert r.out_len == len(c.encode("utf-16-le")) // 2
        r = oracle.utf8_length_from_utf16le(c.encode("utf-16-le"))
        assert r.out_len == len(c.encode("utf-8"))


# --- fuzz against Python's codecs ------------------------------------------

def _py_utf8(data: bytes):
    try:
        s = data.decode("utf-8")
        return None, s
    except UnicodeDecodeError as e:
        return e.start, data[: e.start].decode("utf-8")


def _py_utf16(data: bytes):
    try:
        s = data.decode("utf-16-le")
        return None, s
    except UnicodeDecodeError as e:
        return e.start // 2, data[: e.start].decode("utf-16-le")


@pytest.mark.parametrize("profile", list(textgen.PROFILES))
def test_fuzz_utf8_against_python(profile):
    base = textgen.generate(profile, 4096, textgen.UTF8, seed=11)
    for i in range(60):
        data = textgen.mutate(base.data, i % 4, seed=1000 + i)
        cut = data[: 4096 - (i % 7)].tobytes()
        err, prefix = _py_utf8(cut)
        r, out = oracle.utf8_to_utf16le(cut)
        expect = prefix.encode("utf-16-le")
        if err is None:
            assert r.status == oracle.OK and r.in_offset == len(cut)
        else:
            assert r.status not in (oracle.OK, oracle.OUTPUT_TOO_SMALL)
            assert r.in_offset == err
        assert r.out_len * 2 == len(expect)
        assert out.tobytes() == expect


@pytest.mark.parametrize("profile", list(textgen.PROFILES))
def test_fuzz_utf16_against_python(profile):
    base = textgen.generate(profile, 4096, textgen.UTF16, seed=12)
    for i in range(60):
        data = base.data.copy()
        rng = np.random.Generator(np.random.Philox(key=2000 + i))
        words = data.view("<u2")
        for _ in range(i % 4):  # plant surrogates at random
            words[rng.integers(0, words.size)] = rng.integers(0xD800, 0xE000)
        cut = data[: 4096 - 2 * (i % 5)].tobytes()
        err, prefix = _py_utf16(cut)
        r, out = oracle.utf16le_to_utf8(cut)
        expect = prefix.encode("utf-8")
        if err is None:
            assert r.status == oracle.OK
        else:
            assert r.status in (oracle.LONE_HIGH_SURROGATE, oracle.LONE_LOW_SURROGATE)
            assert r.in_offset == err
        assert r.out_len == len(expect)
        assert out.tobytes() == expect


def test_random_bytes_against_python():
    for i in range(200):
        data = textgen.random_bytes(1 + i % 37, seed=3000 + i).tobytes()
        err, prefix = _py_utf8(data)
        r = oracle.utf16_length_from_utf8(data)
        assert r.in_offset == (len(data) if err is None else err)
        assert r.out_len == len(prefix.encode("utf-16-le")) // 2


# --- exhaustive table matcher (C) ----------------------------------------------

@pytest.fixture(scope="module")
def matcher(tmp_path_factory):
    lib = oracle.library_path()
    exe = str(tmp_path_factory.mktemp("brute") / "table_matcher")
    subprocess.run(["gcc", "-O2", "-pthread", "-o", exe,
                    os.path.join(HERE, "brute", "table_matcher.c"), lib,
                    "-Wl,-rpath," + os.path.dirname(lib)], check=True)
    return exe


@pytest.mark.parametrize("mode", ["utf8", "utf16"])
def test_exhaustive_short_strings_vs_table(matcher, mode):
    threads = str(max(1, min(32, os.cpu_count() or 1)))
    p = subprocess.run([matcher, mode, threads], capture_output=True, text=True)
    assert p.returncode == 0, p.stdout + p.stderr
    assert "mismatches 0" in p.stdout


# --- error kinds on hand-made cases ------------------------------------------------

KIND_CASES = [
    ("C1 BF", oracle.OVERLONG, 0),
    ("C0 41", oracle.OVERLONG, 0),
    ("41 E0 9F BF", oracle.OVERLONG, 1),
    ("F0 8F BF BF", oracle.OVERLONG, 0),
    ("ED A0 80", oracle.SURROGATE, 0),
    ("ED 9F BF 41", oracle.OK, 4),
    ("F4 90 80 80", oracle.TOO_LARGE, 0),
    ("F4 8F BF BF", oracle.OK, 4),
    ("F5 80 80 80", oracle.HEADER_BITS, 0),
    ("41 FF", oracle.HEADER_BITS, 1),
    ("41 80", oracle.TOO_LONG, 1),
    ("C3 A9 A9", oracle.TOO_LONG, 2),
    ("E2 88", oracle.TOO_SHORT, 0),
    ("E2 88 41", oracle.TOO_SHORT, 0),
    ("E0 80 41", oracle.TOO_SHORT, 0),
    ("F0 9F 98", oracle.TOO_SHORT, 0),
    ("", oracle.OK, 0),
    ("00", oracle.OK, 1),
]


@pytest.mark.parametrize("hexbytes,kind,offset", KIND_CASES)
def test_utf8_error_kinds(hexbytes, kind, offset):
    r = oracle.utf16_length_from_utf8(bytes.fromhex(hexbytes))
    assert (r.status, r.in_offset) == (kind, offset)


UTF16_KIND_CASES = [
    ([0xD800], oracle.LONE_HIGH_SURROGATE, 0),
    ([0x41, 0xDBFF, 0x41], oracle.LONE_HIGH_SURROGATE, 1),
    ([0xDC00], oracle.LONE_LOW_SURROGATE, 0),
    ([0x41, 0xDC00, 0xD800], oracle.LONE_LOW_SURROGATE, 1),
    ([0xD800, 0xD800, 0xDC00], oracle.LONE_HIGH_SURROGATE, 0),
    ([0xD800, 0xDC00, 0xDC00], oracle.LONE_LOW_SURROGATE, 2),
    ([0xFEFF, 0xFFFE, 0xFFFF], oracle.OK, 3),   # BOM / noncharacters are valid
]


@pytest.mark.parametrize("words,kind,offset", UTF16_KIND_CASES)
def test_utf16_error_kinds(words, kind, offset):
    r = oracle.utf8_length_from_utf16le(_u16(words))
    assert (r.status, r.in_offset) == (kind, offset)


# --- capacity conventions ------------------------------------------------------------

def test_capacity_too_small_reports_required_length():
    data = "héllo \U0001F600".encode("utf-8")
    full, out = oracle.utf8_to_utf16le(data)
    assert full.status == oracle.OK
    for cap in range(full.out_len):
        r, part = oracle.utf8_to_utf16le(data, cap_units=cap)
        assert r == oracle.Result(oracle.OUTPUT_TOO_SMALL, len(data), full.out_len)
        assert np.array_equal(part, out[:cap])   # first cap units are exact


def test_encoding_error_takes_precedence_over_capacity():
    data = bytes.fromhex("41 42 43 80 44")
    r, part = oracle.utf8_to_utf16le(data, cap_units=1)
    assert r == oracle.Result(oracle.TOO_LONG, 3, 3)
    assert part.tolist() == [0x41]
    r, part = oracle.utf16le_to_utf8(_u16([0x41, 0x4E00, 0xDC00]), cap_bytes=2)
    assert r == oracle.Result(oracle.LONE_LOW_SURROGATE, 2, 4)
    assert part.tobytes() == bytes([0x41, 0xE4])


def test_utf16be_matches_python_codecs():
    """UTF-16BE forms against Python's own big-endian codec on every profile,
    and errors at the same units as in UTF-16LE."""
    import textgen
    for prof in textgen.PROFILES:
        t = textgen.generate(prof, 20_000, textgen.UTF8, seed=7)
        text = t.data.tobytes().decode("utf-8")
        be = text.encode("utf-16-be")
        r, out = oracle.utf8_to_utf16be(t.data)
        assert r.status == oracle.OK and out.tobytes() == be
        r2, back = oracle.utf16be_to_utf8(np.frombuffer(be, np.uint8))
        assert r2.status == oracle.OK and back.tobytes() == t.data.tobytes()
        assert oracle.utf8_length_from_utf16be(np.frombuffer(be, np.uint8)).out_len == len(t.data)
    # a lone high surrogate: same kind and unit offset in both byte orders
    le = np.array([0x41, 0xD800, 0x42], dtype="<u2")
    be = le.astype(">u2").view(np.uint8)
    ra, _ = oracle.utf16le_to_utf8(le.view(np.uint8))
    rb, _ = oracle.utf16be_to_utf8(be)
    assert (ra.status, ra.in_offset, ra.out_len) == (rb.status, rb.in_offset, rb.out_len)
    assert rb.status == oracle.LONE_HIGH_SURROGATE and rb.in_offset == 1


# --- UTF-32LE (Sec. 2's third format) ----------------------------------------

def test_utf32_all_scalars_match_python_codecs():
    cps = _all_scalars()
    s = cps.astype("<u4").tobytes().decode("utf-32-le")
    u8 = s.encode("utf-8")
    r, out = oracle.utf8_to_utf32le(u8)
    assert r == oracle.Result(oracle.OK, len(u8), cps.size)
    assert np.array_equal(out, cps.astype(np.uint32))
    r, out = oracle.utf32le_to_utf8(cps.astype("<u4"))
    assert r == oracle.Result(oracle.OK, cps.size, len(u8))
    assert out.tobytes() == u8
    assert oracle.utf32_length_from_utf8(u8) == oracle.Result(oracle.OK, len(u8), cps.size)
    assert oracle.utf8_length_from_utf32le(cps.astype("<u4")) == \
        oracle.Result(oracle.OK, cps.size, len(u8))


def _py_utf32(data: bytes):
    try:
        return None, data.decode("utf-32-le")
    except UnicodeDecodeError as e:
        return e.start // 4, data[: e.start - e.start % 4].decode("utf-32-le")


def test_utf32_invalid_units():
    """Every surrogate value and values above U+10FFFF, alone and after a
    valid prefix: SURROGATE / TOO_LARGE at the unit, prefix transcoded; the
    position agrees with Python's UTF-32 decoder."""
    prefix = np.array([0x41, 0xE9, 0x4E2D, 0x1F600], dtype="<u4")
    plen = len("Aé中😀".encode("utf-8"))
    bad = [(u, oracle.SURROGATE) for u in range(0xD800, 0xE000)] + \
          [(u, oracle.TOO_LARGE) for u in (0x110000, 0x110001, 0x1FFFFF, 0x7FFFFFFF, 0x80000000,
                                            0xFFFFFFFF, 0x00110000 + 12345)]
    for u, kind in bad:
        data = np.concatenate([prefix, np.array([u, 0x41], dtype="<u4")])
        r, out = oracle.utf32le_to_utf8(data)
        assert (r.status, r.in_offset, r.out_len) == (kind, 4, plen), hex(u)
        assert out.tobytes() == "Aé中😀".encode("utf-8")
        err, _ = _py_utf32(data.tobytes())
        assert err == 4, hex(u)
        assert oracle.utf8_length_from_utf32le(data) == r


@pytest.mark.parametrize("profile", ["mix", "emoji"])
def test_utf8_to_utf32_errors_match_utf16_and_python(profile):
    """UTF-8 -> UTF-32 validates exactly like UTF-8 -> UTF-16 (same status and
    offset); its prefix length counts code points (Python's decode of the
    prefix)."""
    base = textgen.generate(profile, 4096, textgen.UTF8, seed=17)
    for i in range(60):
        data = textgen.mutate(base.data, i % 4, seed=3000 + i)
        cut = data[: 4096 - (i % 7)].tobytes()
        r32, out32 = oracle.utf8_to_utf32le(cut)
        r16, _ = oracle.utf8_to_utf16le(cut)
        assert (r32.status, r32.in_offset) == (r16.status, r16.in_offset)
        err, prefix = _py_utf8(cut)
        assert r32.out_len == len(prefix)
        assert np.array_equal(out32, np.frombuffer(prefix.encode("utf-32-le"), dtype="<u4"))
        assert oracle.utf32_length_from_utf8(cut) == r32


def test_utf32_random_units_against_python():
    rng = np.random.Generator(np.random.Philox(key=91))
    for i in range(200):
        n = int(rng.integers(1, 64))
        # mostly valid values, some surrogates and out-of-range ones
        u = rng.integers(0, 0x110000, size=n).astype(np.uint32)
        u[rng.random(n) < 0.02] = rng.integers(0xD800, 0xE000)
        u[rng.random(n) < 0.02] = rng.integers(0x110000, 0xFFFFFFFF, dtype=np.uint64)
        data = u.astype("<u4").tobytes()
        r, out = oracle.utf32le_to_utf8(data)
        err, prefix = _py_utf32(data)
        if err is None:
            assert (r.status, r.in_offset) == (oracle.OK, n)
        else:
            assert r.status in (oracle.SURROGATE, oracle.TOO_LARGE) and r.in_offset == err
        assert out.tobytes() == prefix.encode("utf-8")


def test_utf32_capacity():
    data = np.array([0x41, 0x4E2D, 0x1F600], dtype="<u4")        # 1 + 3 + 4 bytes
    r, out = oracle.utf32le_to_utf8(data, cap_bytes=5)
    assert (r.status, r.in_offset, r.out_len) == (oracle.OUTPUT_TOO_SMALL, 3, 8)
    r, out = oracle.utf8_to_utf32le("A中😀".encode(), cap_units=2)
    assert (r.status, r.in_offset, r.out_len) == (oracle.OUTPUT_TOO_SMALL, 8, 3)
    assert out.tolist() == [0x41, 0x4E2D]
