"""CPU-side checks of the boundary: the library builds for sm_103a, loads, and
exports every entry point that include/pxsne.h declares.  No GPU call."""
import ctypes
import os
import re

import pytest

import paper_1611_02568_gb300 as px
from paper_1611_02568_gb300 import build as pxbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pxsne.h")


def declared_symbols():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pxsne_[A-Za-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    pxbuild.build()
    return ctypes.CDLL(pxbuild.LIB)


def test_library_exports_every_declared_symbol(lib):
    syms = declared_symbols()
    assert len(syms) >= 18
    for s in syms:
        assert hasattr(lib, s), f"{s} declared in pxsne.h but not exported"
    assert sorted(px.EXPORTED) == syms


def test_default_params_and_binding_mirror(lib):
    L = px.load()
    p = px._CParams()
    L.pxsne_default_params(ctypes.byref(p))
    d = px.Params()
    for f in px._CParams._fields_:
        name = f[0]
        assert getattr(p, name) == pytest.approx(getattr(d, name)), name


def test_create_rejects_bad_params(lib):
    L = px.load()
    for bad in (dict(log2_r=0), dict(log2_r=15), dict(theta=-1.0), dict(k=0),
                dict(perplexity=200.0), dict(momentum1=1.0), dict(centre_mode=2)):
        p = px.Params(**bad).c()
        h = ctypes.c_void_p()
        rc = L.pxsne_create(ctypes.byref(h), ctypes.byref(p), None)
        assert rc == -1, bad
        assert L.pxsne_last_error(None)


def test_null_context_is_rejected(lib):
    L = px.load()
    assert L.pxsne_step(None, 1) == -1
    assert L.pxsne_sync(None, None) == -1
    L.pxsne_destroy(None)


def test_sources_target_sm103a_only():
    assert pxbuild.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
