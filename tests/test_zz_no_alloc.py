"""pxsne_kl_noalloc: the KL entry point for callers that cannot allocate
device memory (a caller-owned memory pool, or a loop that must not take the
device synchronisation of cudaMalloc/cudaFree).  Checked against the
context's pxsne_kl on the same state, on two calls in a row (the second
reuses the shared scratch left by the first), through the C ABI.

Kept in a file that pytest collects last."""
import ctypes

import numpy as np
import pytest

import datagen
import oracle

pytestmark = pytest.mark.gpu


def test_kl_noalloc_matches_pxsne_kl():
    torch = pytest.importorskip("torch")
    import paper_1611_02568_gb300 as px
    from paper_1611_02568_gb300 import build
    build.build()
    lib = px.load()
    vp = ctypes.c_void_p
    lib.pxsne_kl_noalloc.argtypes = [vp, vp, vp, ctypes.c_int64, vp, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, vp, vp]
    lib.pxsne_kl_noalloc.restype = ctypes.c_int
    lib.pxsne_kl_noalloc_max_rows.restype = ctypes.c_int64

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

    dev = torch.device("cuda", torch.cuda.current_device())
    rp_d = torch.from_numpy(rp).to(dev)
    col_d = torch.from_numpy(col).to(dev)
    val_d = torch.from_numpy(val).to(dev)
    z_d = torch.from_numpy(z.view(np.int32)).to(dev)
    out = torch.zeros(1, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info(dev)
    for _ in range(2):
        out.fill_(-1.0)
        rc = lib.pxsne_kl_noalloc(rp_d.data_ptr(), col_d.data_ptr(), val_d.data_ptr(), n,
                                  z_d.data_ptr(), float(s[0]), float(s[1]), float(Z),
                                  out.data_ptr(), ctypes.c_void_p(stream.cuda_stream))
        stream.synchronize()
        assert rc == 0
        got = float(out.item())
        assert abs(got - ref) <= 1e-6 * abs(ref), (got, ref)
    free_after, _ = torch.cuda.mem_get_info(dev)
    assert free_after == free_before

    # sizes beyond the fixed scratch are refused before any launch
    big = int(lib.pxsne_kl_noalloc_max_rows()) + 1
    rc = lib.pxsne_kl_noalloc(rp_d.data_ptr(), col_d.data_ptr(), val_d.data_ptr(), big,
                              z_d.data_ptr(), float(s[0]), float(s[1]), float(Z),
                              out.data_ptr(), ctypes.c_void_p(stream.cuda_stream))
    assert rc == -1
