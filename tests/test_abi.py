"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/etics.h declares; argument errors are reported synchronously
(these checks run without a GPU: they return before any CUDA call)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "etics.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(etics_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1406_4254_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["etics_scf_coeffs", "etics_scf_field", "etics_mex_field",
                     "etics_leapfrog_step", "etics_workspace_bytes", "etics_get_error",
                     "etics_strerror", "etics_radial_sort"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_argument_errors_are_synchronous(lib):
    vp, i64, i32, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_size_t
    lib.etics_scf_coeffs.argtypes = [vp, i64, i32, i32, i32, vp, vp, sz, vp]
    lib.etics_scf_field.argtypes = [vp, i64, i32, i32, i32, vp, vp, i32, vp]
    lib.etics_mex_field.argtypes = [vp, i64, i32, i32, vp, i32, vp, sz, vp]
    lib.etics_strerror.argtypes = [i32]
    lib.etics_strerror.restype = ctypes.c_char_p
    fake = 1 << 20   # never dereferenced: validation fails first
    # negative N, bad precision, null output, misaligned particles
    assert lib.etics_scf_coeffs(fake, -1, 4, 2, 1, fake, fake, 0, None) == -1
    assert lib.etics_scf_coeffs(fake, 10, 4, 2, 7, fake, fake, 0, None) == -1
    assert lib.etics_scf_coeffs(fake, 10, 4, 2, 1, None, fake, 0, None) == -1
    assert lib.etics_scf_coeffs(fake + 4, 10, 4, 2, 1, fake, fake, 1 << 30, None) == -1
    # limits
    assert lib.etics_scf_coeffs(fake, 10, 17, 2, 1, fake, fake, 0, None) == -6
    assert lib.etics_scf_field(fake, 10, 4, 15, 1, fake, fake, 3, None) == -6
    assert lib.etics_mex_field(fake, 10, 11, 1, fake, 3, fake, 0, None) == -6
    # empty output mask
    assert lib.etics_scf_field(fake, 10, 4, 2, 1, fake, fake, 0, None) == -1
    assert lib.etics_strerror(-3) == b"workspace too small"
