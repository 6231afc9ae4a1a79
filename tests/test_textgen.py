"""The seeded generators and the error injector (CPU only).

The injector's expectations (kind, offset, prefix length) are built from the
patterns, independently of any transcoder; here they are checked against the
oracle and against Python's codecs on small texts.
"""
import numpy as np
import pytest

import oracle
import textgen
from textgen import inject


@pytest.mark.parametrize("profile", list(textgen.PROFILES))
@pytest.mark.parametrize("enc", [textgen.UTF8, textgen.UTF16])
def test_exact_size_valid_and_deterministic(profile, enc):
    a = textgen.generate(profile, 50_000, enc, seed=5)
    b = textgen.generate(profile, 50_000, enc, seed=5)
    assert a.data.size == 50_000
    assert np.array_equal(a.data, b.data)
    codec = "utf-8" if enc == textgen.UTF8 else "utf-16-le"
    s = a.data.tobytes().decode(codec)          # valid text
    assert [ord(c) for c in s[:50]] == a.cps[:50].tolist()
    assert int(a.in_len.sum()) == a.n_units
    other = "utf-16-le" if enc == textgen.UTF8 else "utf-8"
    ub = 2 if other == "utf-16-le" else 1
    assert int(a.out_len.sum()) == len(s.encode(other)) // ub


def test_profile_fractions():
    for name, cats in textgen.PROFILES.items():
        cps, cat = textgen.draw_chars(name, 200_000, seed=9)
        for k, c in enumerate(cats):
            frac = float(np.mean(cat == k))
            assert abs(frac - c.prob) < 0.01, (name, k, frac)
            sel = cps[cat == k]
            inside = np.zeros(sel.size, bool)
            for lo, hi in c.ranges:
                inside |= (sel >= lo) & (sel <= hi)
            assert inside.all()
        assert not ((cps >= 0xD800) & (cps <= 0xDFFF)).any()


@pytest.mark.parametrize("enc", [textgen.UTF8, textgen.UTF16])
def test_injected_errors_match_oracle(enc):
    text = textgen.generate("cjk", 200_000, enc, seed=3)
    starts, outs = text.char_starts(), text.out_starts()
    ncases = len(inject.UTF8_CASES if enc == textgen.UTF8 else inject.UTF16_CASES)
    for i in range(4 * ncases):
        p = inject.make_patch(text, i, seed=3, starts=starts, out_starts=outs)
        data = p.apply(text.data)
        if enc == textgen.UTF8:
            r = oracle.utf16_length_from_utf8(data)
        else:
            r = oracle.utf8_length_from_utf16le(data)
        assert (r.status, r.in_offset, r.out_len) == (p.kind, p.err_unit, p.prefix_out), p.case
        codec = "utf-8" if enc == textgen.UTF8 else "utf-16-le"
        with pytest.raises(UnicodeDecodeError) as e:
            data.tobytes().decode(codec)
        assert e.value.start == p.err_unit * (1 if enc == textgen.UTF8 else 2)
