"""3-D embeddings (dim = 3: a voxel grid of 2^L per axis and its octree, the
extension the paper's introduction names), GPU against the oracle through the
C ABI on the same seeded inputs.

Bars (written in each test):
  init map, rescale (R = 2^32 per axis)        bit-exact
  octree counts per level, leaf sums, Morton   bit-exact
  forces Frep, Zi, Fattr, Z                    <= 1e-4 relative L2
  KL of a full run                             <= 1 % of the oracle's run
"""
import numpy as np
import pytest

import datagen
import oracle

pytestmark = pytest.mark.gpu

FORCE_TOL = 1e-4


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def px():
    import paper_1611_02568_gb300 as m
    from paper_1611_02568_gb300 import build
    build.build()
    return m


@pytest.fixture(scope="module")
def gauss3():
    """2500 points of the 10-Gaussian mixture, oracle P, a 3-D start and the
    oracle's state after 60 iterations (clustered under exaggeration)."""
    X, _ = datagen.gauss10(3, n=2500)
    P, _, _, bad = oracle.affinities(X, 30.0, 90)
    assert bad == 0
    Y0 = datagen.init_y0(3, X.shape[0], dim=3)
    st = oracle.State3.from_y0(Y0)
    oracle.run3(P, st, oracle.Params(L=7), 60)
    return X, P, Y0, st


def check_tree(ctx, z, L):
    cnt_o, sx_o, sy_o, sz_o = oracle.pyramid3(z, L)
    for lev in range(L + 1):
        cnt, sx, sy, sz, _ = ctx.get_tree3(lev, sums=(lev == L))
        off = oracle.level_offset3(lev)
        assert np.array_equal(cnt, cnt_o[off:off + 8 ** lev]), lev
    off = oracle.level_offset3(L)
    for a, b in zip((sx, sy, sz), (sx_o, sy_o, sz_o)):
        assert np.array_equal(a, b[off:off + 8 ** L])
    _, _, _, _, mk = ctx.get_tree3(L, morton=True)
    vox = z >> (32 - L)
    want = np.array([oracle.morton3(*v) for v in vox], np.uint32)
    assert np.array_equal(mk, want)


def test_init_map_and_tree_bit_exact(px, gauss3):
    X, P, Y0, _ = gauss3
    L = 7
    with px.Context(px.Params(log2_r=L, dim=3)) as ctx:
        ctx.set_P(P.row_ptr, P.col, P.val.astype(np.float32))
        ctx.init(Y0)
        z, s, u, g, t = ctx.get_state()
        zo, so = oracle.init_fx3(Y0)
        assert z.shape == (P.n, 3) and s.shape == (3,)
        assert np.array_equal(z, zo) and np.array_equal(s, so)
        assert not u.any() and (g == 1).all() and t == 0
        check_tree(ctx, z, L)
        Y, pix = ctx.get_Y(want_pix=True)
        assert np.array_equal(pix, (z >> (32 - L)).astype(np.int32))


@pytest.mark.parametrize("theta", [0.5, 0.0, 1.0])
def test_forces_match_oracle(px, gauss3, theta):
    X, P, Y0, st = gauss3
    L = 7
    with px.Context(px.Params(log2_r=L, theta=theta, dim=3)) as ctx:
        ctx.set_P(P.row_ptr, P.col, P.val.astype(np.float32))
        ctx.set_state(st.z, st.s, st.u.astype(np.float32), st.gains.astype(np.float32), st.t)
        check_tree(ctx, st.z, L)
        Frep, Zi, Fattr, Z = ctx.get_forces()
    oF, oZi, _ = oracle.bh_repulsion3(st.z, st.s, L, theta)
    oA = oracle.attraction3(P, st.z, st.s)
    assert Frep.shape == (P.n, 3)
    assert rel(Frep, oF) <= FORCE_TOL
    assert rel(Zi, oZi) <= FORCE_TOL
    assert rel(Fattr, oA) <= FORCE_TOL
    assert abs(Z - oZi.sum()) / oZi.sum() <= FORCE_TOL


def test_rescale_bit_exact_and_tree_after_steps(px, gauss3):
    X, P, Y0, _ = gauss3
    L = 6
    with px.Context(px.Params(log2_r=L, dim=3)) as ctx:
        ctx.set_P(P.row_ptr, P.col, P.val.astype(np.float32))
        ctx.init(Y0)
        ctx.step(30)
        for _ in range(3):
            z, s, u, g, t = ctx.get_state()
            ctx.step(1)
            z2, s2, u2, _, t2 = ctx.get_state()
            assert t2 == t + 1
            # the step as the kernel forms it: z + rint(u / s) in FP64
            zhat = z.astype(np.int64) + np.rint(u2.astype(np.float64) *
                                                (1.0 / s)[None, :]).astype(np.int64)
            zr, sr = oracle.rescale3(zhat, s)
            assert np.array_equal(z2, zr) and np.array_equal(s2, sr)
            vox = z2 >> (32 - L)
            assert (vox.min(0) == 0).all() and (vox.max(0) == 2 ** L - 1).all()
        check_tree(ctx, z2, L)
        assert ctx.sync() == 0


def test_run_kl_within_one_percent(px, gauss3):
    X, P, Y0, _ = gauss3
    L, iters = 7, 400
    prm = oracle.Params(L=L)
    st = oracle.State3.from_y0(Y0)
    oracle.run3(P, st, prm, iters)
    kl_o = oracle.kl_of3(P, st, prm)
    with px.Context(px.Params(log2_r=L, dim=3)) as ctx:
        ctx.set_P(P.row_ptr, P.col, P.val.astype(np.float32))
        ctx.init(Y0)
        ctx.step(iters)
        kl = ctx.kl()
        assert ctx.sync() == 0
        Y, _ = ctx.get_Y()
    print(f"3-D KL after {iters}: GPU {kl:.5f}, oracle {kl_o:.5f}")
    assert Y.shape == (P.n, 3) and np.isfinite(Y).all()
    assert abs(kl - kl_o) <= 0.01 * kl_o


def test_calls_without_a_3d_form_are_refused(px, gauss3):
    X, P, Y0, _ = gauss3
    with px.Context(px.Params(log2_r=6, dim=3)) as ctx:
        ctx.set_P(P.row_ptr, P.col, P.val.astype(np.float32))
        ctx.init(Y0)
        for call in (lambda: ctx.get_tree(2), lambda: ctx.step_profiled(1),
                     lambda: ctx.nbr_precision(10, np.zeros((P.n, 10), np.int32))):
            with pytest.raises(px.PxsneError):
                call()
        ctx.step(2)
        assert ctx.sync() == 0


def test_octree_rebuilt_from_cleared_leaves(px, gauss3):
    # the first reduction clears the leaves it read: a second state's octree
    # has no trace of the first's
    X, P, Y0, st = gauss3
    L = 6
    rng = np.random.default_rng(47)
    z2 = rng.integers(0, 2 ** 32, st.z.shape, dtype=np.uint64).astype(np.uint32)
    with px.Context(px.Params(log2_r=L, dim=3)) as ctx:
        ctx.set_P(P.row_ptr, P.col, P.val.astype(np.float32))
        for z in (st.z, z2, st.z):
            ctx.set_state(z, st.s)
            check_tree(ctx, z, L)
            Frep, Zi, _, _ = ctx.get_forces()
            oF, oZi, _ = oracle.bh_repulsion3(z, st.s, L, 0.5)
            assert rel(Frep, oF) <= FORCE_TOL and rel(Zi, oZi) <= FORCE_TOL
        assert ctx.sync() == 0
