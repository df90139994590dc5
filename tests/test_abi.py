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
                dict(perplexity=200.0), dict(momentum1=1.0), dict(centre_mode=2),
                dict(screen_x=3000, log2_r=11), dict(knn_probe=5000), dict(dim=4),
                dict(dim=1), dict(dim=3, log2_r=10), dict(dim=3, screen_x=100),
                dict(dim=3, centre_mode=1), dict(knn_explore=2), dict(knn_probe=64, knn_explore=9),
                dict(knn_probe=64, knn_explore=-1), dict(knn_probe=1), dict(knn_probe=2, k=200)):
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


def test_kl_noalloc_rejects_bad_arguments_before_any_device_work(lib):
    vp = ctypes.c_void_p
    f = lib.pxsne_kl_noalloc
    f.argtypes = [vp, vp, vp, ctypes.c_int64, vp, ctypes.c_double, ctypes.c_double,
                  ctypes.c_double, vp, vp]
    f.restype = ctypes.c_int
    lib.pxsne_kl_noalloc_max_rows.restype = ctypes.c_int64
    big = lib.pxsne_kl_noalloc_max_rows()
    assert big == 2 ** 24
    ok = dict(rp=1, col=1, val=1, n=10, z=1, s0=1.0, s1=1.0, Z=1.0, out=1)
    for bad in (dict(rp=None), dict(col=None), dict(val=None), dict(z=None), dict(out=None),
                dict(n=0), dict(n=big + 1), dict(s0=0.0), dict(s1=-1.0), dict(Z=0.0),
                dict(Z=float("nan")), dict(Z=float("inf")), dict(s0=float("inf")),
                dict(s1=float("inf"))):
        a = ok | bad
        assert f(a["rp"], a["col"], a["val"], a["n"], a["z"], a["s0"], a["s1"], a["Z"],
                 a["out"], None) == -1, bad


def test_stateless_calls_reject_bad_arguments_before_any_device_work(lib):
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
    lib.pxsne_pca.argtypes = [vp, i64, i32, i32, vp, vp, vp, ctypes.c_int, ctypes.c_uint64]
    lib.pxsne_embed_align.argtypes = [vp, vp, i64, vp, ctypes.c_int]
    lib.pxsne_mlp_create.argtypes = [ctypes.POINTER(vp), i32, ctypes.c_uint64, vp]
    lib.pxsne_mlp_train.argtypes = [vp, vp, vp, i64, i32, i32, ctypes.c_float, ctypes.c_uint64,
                                    vp, ctypes.c_int]
    lib.pxsne_mlp_predict.argtypes = [vp, vp, i64, vp, ctypes.c_int]
    lib.pxsne_mlp_num_params.argtypes = [vp]
    lib.pxsne_mlp_num_params.restype = i64
    lib.pxsne_mlp_destroy.argtypes = [vp]
    # PCA: 2 <= n, 1 <= dout <= D, X and Xout given
    for args in [(None, 10, 4, 2), (1, 1, 4, 2), (1, 10, 4, 5), (1, 10, 4, 0), (1, 10, 0, 0)]:
        X, n, D, dout = args
        assert lib.pxsne_pca(X, n, D, dout, 1, None, None, 0, 0) == -1, args
    assert lib.pxsne_pca(1, 10, 4, 2, None, None, None, 0, 0) == -1
    # alignment: 2 <= n, Y and Yout given
    assert lib.pxsne_embed_align(None, None, 10, 1, 0) == -1
    assert lib.pxsne_embed_align(1, None, 1, 1, 0) == -1
    assert lib.pxsne_embed_align(1, None, 10, None, 0) == -1
    # MLP: 1 <= d <= 1024; *out is NULL after a failure; NULL models are rejected
    h = vp(12345)
    assert lib.pxsne_mlp_create(ctypes.byref(h), 0, 0, None) == -1 and not h.value
    h = vp(12345)
    assert lib.pxsne_mlp_create(ctypes.byref(h), 1025, 0, None) == -1 and not h.value
    assert lib.pxsne_mlp_create(None, 8, 0, None) == -1
    assert lib.pxsne_mlp_train(None, 1, 1, 10, 1, 8, 1e-3, 0, None, 0) == -1
    assert lib.pxsne_mlp_predict(None, 1, 10, 1, 0) == -1
    assert lib.pxsne_mlp_num_params(None) == 0
    lib.pxsne_mlp_destroy(None)


def test_kernel_group_names(lib):
    # the tracing groups of one iteration, in launch order, as the bench's
    # roofline and byte model name them
    import sys
    sys.path.insert(0, ROOT)
    import bench
    lib.pxsne_kernel_group_name.argtypes = [ctypes.c_int32]
    lib.pxsne_kernel_group_name.restype = ctypes.c_char_p
    names = [lib.pxsne_kernel_group_name(g) for g in range(8)]
    assert [x.decode() for x in names] == [
        "k_relabel", "k_update", "k_snap_hist", "k_pyr_pass", "k_perm_scatter",
        "k_bh_traverse", "k_attract", "k_zsum"]
    assert lib.pxsne_kernel_group_name(8) is None and lib.pxsne_kernel_group_name(-1) is None
    assert set(bench.group_bytes(100, 1000, 3)) == {x.decode() for x in names}


def test_missing_library_fails_loudly():
    """Without the compiled library every entry point raises: there is no
    CPU fallback."""
    import subprocess
    import sys
    code = ("import paper_1611_02568_gb300 as p\n"
            "p.LIB_PATH = p.LIB_PATH + '.absent'\n"
            "for f in (lambda: p.Context(), lambda: p.MLP(8), lambda: p.pca([[0.0]], 1),\n"
            "          lambda: p.embed_align([[0.0, 0.0]])):\n"
            "    try:\n"
            "        f()\n"
            "    except RuntimeError as e:\n"
            "        assert 'missing' in str(e)\n"
            "    else:\n"
            "        raise SystemExit('no error')\n"
            "print('ok')\n")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True,
                         timeout=300)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr


C_CLIENT = r"""
#include "pxsne.h"
#include <stdio.h>
int main(void) {
    pxsne_params p;
    pxsne_ctx *c = 0;
    int rc;
    pxsne_default_params(&p);
    rc = pxsne_create(&c, 0, 0);
    printf("%d %d %d\n", p.log2_r, p.k, rc);
    return !(p.log2_r == 11 && p.k == 90 && rc == PXSNE_E_ARG && c == 0 &&
             pxsne_last_error(0)[0] != 0);
}
"""


def test_header_serves_a_plain_c_client(tmp_path):
    """include/pxsne.h is plain C (C99, pedantic, no warnings) and C++; a C
    program links against the library and calls it (no device work)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None or shutil.which("g++") is None:
        pytest.skip("gcc/g++ needed")
    pxbuild.build()
    src = tmp_path / "client.c"
    src.write_text(C_CLIENT)
    exe = tmp_path / "client"
    libdir = os.path.dirname(pxbuild.LIB)
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
                    "-I", os.path.join(ROOT, "include"), str(src), "-L", libdir, "-lpxsne",
                    f"-Wl,-rpath,{libdir}", "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.split() == ["11", "90", "-1"], out
    subprocess.run(["g++", "-std=c++17", "-Wall", "-Wextra", "-Werror", "-fsyntax-only",
                    "-x", "c++", HEADER], check=True)


def test_sources_target_sm103a_only():
    assert pxbuild.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_product_and_oracle_share_nothing():
    """The CUDA path and the oracle are independent: no source of either names
    the other, the library is built from the package's own sources and
    headers only and exports none of the oracle's symbols, and importing the
    package loads no oracle module."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    pkg = os.path.join(root, "paper_1611_02568_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"\boracle\b|orc_", text), f
    for f in os.listdir(os.path.join(root, "include")):
        assert "orc_" not in open(os.path.join(root, "include", f)).read()
    src = open(os.path.join(root, "oracle", "pxsne_oracle.c")).read()
    assert "pxsne.h" not in src and "common.cuh" not in src
    assert not re.search(r"\bpxsne_[a-z]", src)
    flags = pxbuild._flags()
    incs = [flags[i + 1] for i, f in enumerate(flags) if f == "-I"]
    assert sorted(incs) == sorted([pxbuild.INCLUDE, pxbuild.CSRC])
    assert os.path.dirname(pxbuild.CSRC) == pkg
    lib = ctypes.CDLL(px.LIB_PATH)
    for sym in ("orc_run", "orc_bh_repulsion", "orc_knn", "orc_kl"):
        assert not hasattr(lib, sym)
    code = ("import sys, paper_1611_02568_gb300 as p; p.load(); "
            "print(sorted(m for m in sys.modules if m.split('.')[0] == 'oracle'))")
    out = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True,
                         text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == "[]"
