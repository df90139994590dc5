"""pxsne_kl_noalloc: the KL entry point for callers that cannot allocate
device memory (a caller-owned memory pool, or a loop that must not take the
device synchronisation of cudaMalloc/cudaFree).  Checked against the
context's pxsne_kl on the same state, on two calls in a row (the second
reuses the shared scratch left by the first), through the C ABI: once with a
single block of rows, and once over many blocks with a ragged last block (the
partials of several blocks, the ticket that picks the last one, and its reset
between calls).

Kept in a file that pytest collects last."""
import ctypes

import numpy as np
import pytest

import datagen
import oracle

pytestmark = pytest.mark.gpu

ROWS_PER_BLOCK = 2048  # rows one block of the kernel reduces


def _lib(px):
    from paper_1611_02568_gb300 import build
    build.build()
    lib = px.load()
    vp = ctypes.c_void_p
    lib.pxsne_kl_noalloc.argtypes = [vp, vp, vp, ctypes.c_int64, vp, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, vp, vp]
    lib.pxsne_kl_noalloc.restype = ctypes.c_int
    lib.pxsne_kl_noalloc_max_rows.restype = ctypes.c_int64
    return lib


def _state(px, X, L, steps):
    """P from X, `steps` iterations; the context's KL and the raw state."""
    n = X.shape[0]
    with px.Context(px.Params(log2_r=L)) as ctx:
        ctx.affinities(X)
        ctx.init(datagen.init_y0(0, n))
        ctx.step(steps)
        ref = ctx.kl()
        rp, col, val = ctx.get_P()
        z, s, _, _, _ = ctx.get_state()
        _, _, _, Z = ctx.get_forces()
    return ref, rp, col, val, z, s, Z


def _calls(lib, torch, rp, col, val, z, s, Z, times=2):
    dev = torch.device("cuda", torch.cuda.current_device())
    n = rp.shape[0] - 1
    rp_d = torch.from_numpy(rp).to(dev)
    col_d = torch.from_numpy(col).to(dev)
    val_d = torch.from_numpy(val).to(dev)
    z_d = torch.from_numpy(z.view(np.int32)).to(dev)
    out = torch.zeros(1, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info(dev)
    got = []
    for _ in range(times):
        out.fill_(-1.0)
        rc = lib.pxsne_kl_noalloc(rp_d.data_ptr(), col_d.data_ptr(), val_d.data_ptr(), n,
                                  z_d.data_ptr(), float(s[0]), float(s[1]), float(Z),
                                  out.data_ptr(), ctypes.c_void_p(stream.cuda_stream))
        stream.synchronize()
        assert rc == 0
        got.append(float(out.item()))
    free_after, _ = torch.cuda.mem_get_info(dev)
    assert free_after == free_before
    return got, (rp_d, col_d, val_d, z_d, out, stream)


def test_kl_noalloc_matches_pxsne_kl():
    torch = pytest.importorskip("torch")
    import paper_1611_02568_gb300 as px
    lib = _lib(px)

    X, _ = datagen.gauss10(0)
    n = X.shape[0]
    P, _, _, _ = oracle.affinities(X, 30.0, 90)
    with px.Context(px.Params(log2_r=9)) as ctx:
        ctx.set_P(P.row_ptr, P.col, P.val.astype(np.float32))
        ctx.init(datagen.init_y0(0, n))
        ctx.step(60)
        ref = ctx.kl()
        rp, col, val = ctx.get_P()
        z, s, _, _, _ = ctx.get_state()
        _, _, _, Z = ctx.get_forces()
    assert n < ROWS_PER_BLOCK  # one block
    got, (rp_d, col_d, val_d, z_d, out, stream) = _calls(lib, torch, rp, col, val, z, s, Z)
    for g in got:
        assert abs(g - ref) <= 1e-6 * abs(ref), (g, ref)

    # sizes beyond the fixed scratch are refused before any launch
    big = int(lib.pxsne_kl_noalloc_max_rows()) + 1
    rc = lib.pxsne_kl_noalloc(rp_d.data_ptr(), col_d.data_ptr(), val_d.data_ptr(), big,
                              z_d.data_ptr(), float(s[0]), float(s[1]), float(Z),
                              out.data_ptr(), ctypes.c_void_p(stream.cuda_stream))
    assert rc == -1


def test_kl_noalloc_many_blocks_ragged():
    # 30,001 rows: 15 blocks, the last one holding 1,361 rows
    torch = pytest.importorskip("torch")
    import paper_1611_02568_gb300 as px
    lib = _lib(px)
    X, _ = datagen.gmm128(0, n=30001)
    n = X.shape[0]
    assert n > 10 * ROWS_PER_BLOCK and n % ROWS_PER_BLOCK != 0
    ref, rp, col, val, z, s, Z = _state(px, X, 10, 120)
    got, _ = _calls(lib, torch, rp, col, val, z, s, Z, times=3)
    for g in got:
        assert abs(g - ref) <= 1e-6 * abs(ref), (g, ref)
    # every call gives the same value: the ticket was reset between calls
    assert got[0] == got[1] == got[2]


def test_kl_noalloc_out_of_range_column_gives_nan():
    # a column outside [0, n) is skipped by the kernel's bounds check (no
    # read of z) and reported as NaN; the next valid call is unaffected
    torch = pytest.importorskip("torch")
    import paper_1611_02568_gb300 as px
    lib = _lib(px)
    X, _ = datagen.gauss10(0, n=5000)
    ref, rp, col, val, z, s, Z = _state(px, X, 9, 30)
    bad = col.copy()
    e = int(rp[2500]) + 1
    assert val[e] > 0
    bad[e] = X.shape[0] + 7
    got, _ = _calls(lib, torch, rp, bad, val, z, s, Z, times=1)
    assert np.isnan(got[0])
    bad[e] = -3
    got, _ = _calls(lib, torch, rp, bad, val, z, s, Z, times=1)
    assert np.isnan(got[0])
    got, _ = _calls(lib, torch, rp, col, val, z, s, Z, times=1)
    assert abs(got[0] - ref) <= 1e-6 * abs(ref), (got, ref)
