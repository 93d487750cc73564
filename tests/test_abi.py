"""Host-side checks of the C ABI that need no GPU: the library builds for sm_103a, loads, and
exports every function include/omp_gb300.h declares; argument errors are returned before any
device work."""
import ctypes
import os
import re

import pytest

from paper_2407_06434_gb300 import build as libbuild
from paper_2407_06434_gb300 import omp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^[A-Za-z_][\w \*]*?\b(omp_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return omp.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 10
    assert sorted(omp.EXPORTS) == names
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings(lib):
    for code, name in omp.STATUS.items():
        assert omp.omp_status_string(code) == name


def test_desc_default(lib):
    d = omp.omp_desc_default(1024, 8192)
    assert (d.M, d.N, d.max_iters, d.precision, d.rescore_topk, d.eps_relative, d.use_graph,
            d.gather24) == (1024, 8192, 64, 1, 8, 1, 1, 0)


def test_invalid_arguments_rejected_before_device_work(lib):
    h = ctypes.c_void_p()
    assert lib.omp_create(None, ctypes.byref(h)) == 1
    d = omp.omp_desc()
    lib.omp_desc_default(ctypes.byref(d), 64, 256)
    for field, bad in [("M", 0), ("N", 1), ("max_batch", 0), ("max_iters", 0),
                       ("max_iters", 300), ("precision", 7), ("rescore_topk", 9),
                       ("gather24", 2)]:
        dd = omp.omp_desc.from_buffer_copy(d)
        setattr(dd, field, bad)
        assert lib.omp_create(ctypes.byref(dd), ctypes.byref(h)) == 1, field
    assert lib.omp_solve_batch(None, None, None, 1, 1, 0.0, None, None, None) == 1
    assert lib.omp_destroy(None) == 0


def test_library_is_sm103a_only():
    assert "arch=compute_103a,code=sm_103a" in libbuild.ARCH
