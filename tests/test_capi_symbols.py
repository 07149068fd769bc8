"""The C-ABI library builds for sm_103a, loads on a host without a GPU, and
exports every entry point include/swr.h declares.  No compute calls."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    hdr = open(os.path.join(ROOT, "include", "swr.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[\w]+\s*\*?\s*(swr_\w+)\s*\(", hdr, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libswr():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1503_02564_gb300 import build_ext
    path = build_ext.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for f in ("swr_plan", "swr_build_interface", "swr_solve", "swr_adjoint", "swr_destroy",
              "swr_status_string", "swr_apply_R", "swr_apply_interface", "swr_get_interface",
              "swr_apply_precond", "swr_misfit"):
        assert f in names, f


def test_library_exports_every_declared_symbol(libswr):
    for name in _declared():
        assert hasattr(libswr, name), name


def test_status_strings_without_gpu(libswr):
    libswr.swr_status_string.restype = ctypes.c_char_p
    libswr.swr_status_string.argtypes = [ctypes.c_int]
    for code in range(10):
        assert libswr.swr_status_string(code).startswith(b"SWR_")


def test_plan_rejects_bad_arguments_without_touching_the_device(libswr):
    from paper_1503_02564_gb300 import swr
    h = ctypes.c_void_p()
    assert libswr.swr_plan(None, ctypes.byref(h), None) == swr.SWR_ERR_ARG
    d = swr.swr_desc()
    d.nx = 2                      # too few nodes
    assert libswr.swr_plan(ctypes.byref(d), ctypes.byref(h), None) == swr.SWR_ERR_ARG
    assert not h.value
