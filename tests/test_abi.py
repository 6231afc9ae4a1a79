"""The C-ABI library builds for sm_103a, loads, and exports every function
declared in include/gbutf.h (CPU only; no compute call is made)."""
import ctypes
import os
import re

import paper_2212_05098_gb300 as gbu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "gbutf.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gbu_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["gbu_create", "gbu_destroy", "gbu_utf8_to_utf16le", "gbu_utf16le_to_utf8",
                     "gbu_utf16_length_from_utf8", "gbu_utf8_length_from_utf16le"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(gbu.library_path() if os.path.exists(gbu.library_path())
                      else gbu._build.build())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    assert set(declared_functions()) == set(gbu.SIGNATURES)
    for name in gbu.SIGNATURES:
        assert hasattr(gbu, name) or name in ("gbu_status_name",)


def test_status_names_without_gpu():
    lib = gbu.load()
    assert gbu.status_name(gbu.GBU_OK) == "GBU_OK"
    assert gbu.status_name(gbu.GBU_LONE_LOW_SURROGATE) == "GBU_LONE_LOW_SURROGATE"
    assert gbu.status_name(12345) == "GBU_UNKNOWN"
    assert lib.gbu_kernel_launch_count() >= 0


def test_null_context_is_invalid_argument():
    # argument checks happen before any CUDA call
    r = gbu.gbu_utf8_to_utf16le(None, None, 0, None, 0, None)
    assert r.status == gbu.GBU_INVALID_ARG


def test_kernel_shapes_without_gpu():
    shapes = gbu.gbu_tune_shapes()
    assert shapes[0] == (12288, 256)            # the default shape first
    assert len(set(shapes)) == len(shapes) >= 2
    for chunk, threads in shapes:
        assert chunk % threads == 0 and (chunk // threads) % 16 == 0
