"""No-GPU checks of the boundary: the library builds for sm_103a, loads, and
exports every entry point that include/ladder.h declares (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "ladder.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ladder_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1810_08142_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_documented_calls():
    names = declared_symbols()
    for n in ("ladder_plan", "ladder_apply", "ladder_energy", "ladder_backward", "ladder_tau",
              "ladder_destroy", "ladder_workspace_size", "ladder_set_workspace"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_binding_wraps_every_declared_symbol():
    import paper_1810_08142_gb300 as L
    assert sorted(L.EXPORTS) == declared_symbols()
    for name in declared_symbols():
        if name != "ladder_status_string":
            assert callable(getattr(L, name)), name


def test_status_strings_and_null_arguments(lib):
    lib.ladder_status_string.restype = ctypes.c_char_p
    assert lib.ladder_status_string(0) == b"ok"
    assert lib.ladder_status_string(6).startswith(b"workspace")
    # argument checks run before any CUDA call
    assert lib.ladder_plan(4, 24, 96, 0, None) == 1
    out = ctypes.c_void_p()
    assert lib.ladder_plan(0, 24, 96, 0, ctypes.byref(out)) == 1
    assert lib.ladder_plan(4, 24, 96, 9, ctypes.byref(out)) == 1
    lib.ladder_apply.argtypes = [ctypes.c_void_p] * 5
    assert lib.ladder_apply(None, None, None, None, None) == 1


def test_triples_workspace_size_is_host_logic(lib):
    """ladder_triples_workspace_size needs no device: it covers the integrals,
    W for one (i, j) and the partial sums, and rejects bad arguments."""
    size = ctypes.c_size_t()
    f = lib.ladder_triples_workspace_size
    f.argtypes = [ctypes.c_int] * 4 + [ctypes.POINTER(ctypes.c_size_t)]
    f.restype = ctypes.c_int
    assert f(10, 120, 480, 0, ctypes.byref(size)) == 0
    b64 = size.value
    assert f(10, 120, 480, 1, ctypes.byref(size)) == 0
    b32 = size.value
    o, v = 10, 120
    floor64 = 8 * (2 * o * v ** 3 + o ** 3 * v + o ** 2 * v ** 2 + o * v ** 3)
    assert b64 >= floor64 and b32 >= floor64 // 2 and b32 < b64
    assert f(0, 120, 480, 0, ctypes.byref(size)) == 1       # LADDER_EINVAL
    assert f(10, 120, 480, 7, ctypes.byref(size)) == 1


def test_noalloc_energy_size_limit_is_host_logic(lib):
    """ladder_energy_noalloc checks its shape against the fixed array of
    524288 partial sums before it touches a pointer or the device:
    ceil(v/32)^2 o^2 = 4^2 * 182^2 = 529984 is refused (LADDER_ENOTSUP),
    4^2 * 181^2 = 524176 passes the size check and fails on the null pointers
    (LADDER_EINVAL); so does o = 256, v = 32 (65536 pairs)."""
    f = lib.ladder_energy_noalloc
    f.argtypes = [ctypes.c_int, ctypes.c_int] + [ctypes.c_void_p] * 4
    f.restype = ctypes.c_int
    assert f(182, 100, None, None, None, None) == 5
    assert f(181, 100, None, None, None, None) == 1
    assert f(256, 32, None, None, None, None) == 1
    assert f(257, 32, None, None, None, None) == 1
    assert f(120, 200, None, None, None, None) == 5


def test_ozaki_mode_and_nonfinite_status_are_exposed(lib):
    import paper_1810_08142_gb300 as lad
    lib.ladder_status_string.restype = ctypes.c_char_p
    assert lad.MODES["ozaki"] == 4
    assert lad.STATUS[7] == "LADDER_ENONFINITE"
    assert b"NaN" in lib.ladder_status_string(7)
    # the ctypes mirror of ladder_tuning lists the header's fields in order
    hdr = open(os.path.join(ROOT, "include", "ladder.h")).read()
    body = hdr[hdr.index("typedef struct {", hdr.index("Launch parameters")):hdr.index("} ladder_tuning;")]
    fields = [f.strip() for f in body.split("int", 1)[1].replace(";", "").split(",")]
    assert [f for f, _ in lad.Tuning._fields_] == fields
    assert fields[-3:] == ["oz_slices", "tile_chunk", "sym_b"]
    # mode 5 is out of range
    out = ctypes.c_void_p()
    assert lib.ladder_plan(4, 24, 96, 5, ctypes.byref(out)) == 1
