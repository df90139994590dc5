"""Screens of r_1 x r_2 pixels (Sec. 4.2's per-axis r_d; the 1024 x 768 example
of Sec. 1) on the padded 2^L root, GPU against the oracle through the C ABI:
the init map and the rescale bit-exact (per-axis extent R_d = r_d 2^(32-L)),
pixels spanning exactly 0 .. r_d - 1, the tree bit-exact, forces within
1e-4, and the KL of a full run within 1 % of the oracle's run."""
import numpy as np
import pytest

import datagen
import oracle

pytestmark = pytest.mark.gpu

SCREENS = [(10, 1024, 768), (9, 384, 512), (9, 300, 200)]


@pytest.fixture(scope="module")
def px():
    import paper_1611_02568_gb300 as m
    from paper_1611_02568_gb300 import build
    build.build()
    return m


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.mark.parametrize("L,rx,ry", SCREENS)
def test_screen_map_rescale_and_tree(px, L, rx, ry):
    X, _ = datagen.gauss10(7, n=2500)
    n = X.shape[0]
    P, _, _, _ = oracle.affinities(X, 30.0, 90)
    Y0 = datagen.init_y0(7, n)
    R = oracle.screen_R(L, rx, ry)
    F = 32 - L
    with px.Context(px.Params(log2_r=L, screen_x=rx, screen_y=ry)) as ctx:
        ctx.set_P(P.row_ptr, P.col, P.val.astype(np.float32))
        ctx.init(Y0)
        z, s, _, _, _ = ctx.get_state()
        zo, so = oracle.init_fx(Y0, R)
        assert np.array_equal(z, zo) and np.array_equal(s, so)
        ctx.step(40)
        for _ in range(3):
            z, s, u, g, t = ctx.get_state()
            ctx.step(1)
            z2, s2, u2, _, _ = ctx.get_state()
            # the step as the kernel forms it: z + rint(u / s) in FP64
            zhat = z.astype(np.int64) + np.rint(u2.astype(np.float64) *
                                                (1.0 / s)[None, :]).astype(np.int64)
            zr, sr = oracle.rescale(zhat, s, R)
            assert np.array_equal(z2, zr) and np.array_equal(s2, sr)
        for d, r in enumerate((rx, ry)):
            assert (z2[:, d] >> F).min() == 0 and (z2[:, d] >> F).max() == r - 1
            assert int(z2[:, d].max()) < int(R[d])
        cnt_o, sx_o, sy_o = oracle.pyramid(z2, L)
        for lev in range(L + 1):
            cnt, sx, sy, _ = ctx.get_tree(lev, sums=(lev == L))
            off = oracle.level_offset(lev)
            assert np.array_equal(cnt, cnt_o[off:off + 4 ** lev]), lev
            if lev == L:
                assert np.array_equal(sx, sx_o[off:off + 4 ** lev])
                assert np.array_equal(sy, sy_o[off:off + 4 ** lev])
        Frep, Zi, Fattr, Z = ctx.get_forces()
    oF, oZi, _ = oracle.bh_repulsion(z2, s2, L, 0.5)
    assert rel(Frep, oF) <= 1e-4 and rel(Zi, oZi) <= 1e-4
    assert rel(Fattr, oracle.attraction(P, z2, s2)) <= 1e-4


def test_screen_full_run_kl_within_one_percent(px):
    X, _ = datagen.gauss10(0)
    n = X.shape[0]
    L, rx, ry = 9, 384, 512
    P, _, _, _ = oracle.affinities(X, 30.0, 90)
    Y0 = datagen.init_y0(0, n)
    prm = oracle.Params(L=L, rx=rx, ry=ry)
    st = oracle.State.from_y0(Y0, prm.R())
    oracle.run(P, st, prm, 500)
    kl_o = oracle.kl_of(P, st, prm)
    with px.Context(px.Params(log2_r=L, screen_x=rx, screen_y=ry)) as ctx:
        ctx.set_P(P.row_ptr, P.col, P.val.astype(np.float32))
        ctx.init(Y0)
        ctx.step(500)
        kl_g = ctx.kl()
        z, s, _, _, _ = ctx.get_state()
    assert (z[:, 0] >> (32 - L)).max() == rx - 1 and (z[:, 1] >> (32 - L)).max() == ry - 1
    assert abs(kl_g - kl_o) <= 0.01 * kl_o, (kl_g, kl_o)


def test_screen_arguments_checked(px):
    for bad in (dict(log2_r=9, screen_x=513), dict(log2_r=9, screen_y=-1)):
        with pytest.raises(px.PxsneError):
            px.Context(px.Params(**bad))
