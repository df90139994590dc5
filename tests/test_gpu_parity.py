"""GPU path vs the CPU oracle, through the C ABI, on the same seeded inputs.

Bars (written in each test):
  tree (pixels, Morton keys, counts, exact coordinate sums)  bit-exact
  forces Frep, Zi, Fattr, Z                                  <= 1e-4 relative L2
  final KL of a full run                                     <= 1 % of the oracle's
  fixed-point init / rescale                                  bit-exact
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
def gauss():
    """The 2000-point mixture (10 Gaussians in D = 50): oracle P and an oracle state after 60 iterations
    (clustered under exaggeration)."""
    X, lab = datagen.gauss10(0)
    P, idx, d2, bad = oracle.affinities(X, 30.0, 90)
    assert bad == 0
    Y0 = datagen.init_y0(0, X.shape[0])
    st = oracle.State.from_y0(Y0)
    oracle.run(P, st, oracle.Params(L=9), 60)
    return X, P, Y0, st


def make_ctx(px, L=9, **kw):
    return px.Context(px.Params(log2_r=L, **kw))


def inject(ctx, P, st):
    ctx.set_P(P.row_ptr, P.col, P.val.astype(np.float32))
    ctx.set_state(st.z, st.s, st.u.astype(np.float32), st.gains.astype(np.float32), st.t)


def check_tree(ctx, z, L):
    cnt_o, sx_o, sy_o = oracle.pyramid(z, L)
    for l in range(L + 1):
        cnt, sx, sy, _ = ctx.get_tree(l, sums=(l == L))
        off = oracle.level_offset(l)
        assert np.array_equal(cnt, cnt_o[off:off + 4 ** l]), f"level {l} counts"
        if l == L:
            assert np.array_equal(sx, sx_o[off:off + 4 ** l])
            assert np.array_equal(sy, sy_o[off:off + 4 ** l])
    _, _, _, mk = ctx.get_tree(0, morton=True)
    _, _, mo = oracle.leaf_keys(z, L)
    assert np.array_equal(mk, mo)


def test_init_maps_y0_bit_exact(px):
    n = 1537
    Y0 = datagen.init_y0(3, n)
    X = np.random.default_rng(0).standard_normal((n, 4)).astype(np.float32)
    with make_ctx(px, L=10, k=5, perplexity=3.0) as ctx:
        ctx.affinities(X)
        ctx.init(Y0)
        z, s, u, g, t = ctx.get_state()
        zo, so = oracle.init_fx(Y0.astype(np.float64))
        assert np.array_equal(z, zo) and np.array_equal(s, so)
        assert t == 0 and np.all(u == 0) and np.all(g == 1)
        check_tree(ctx, z, 10)


@pytest.mark.parametrize("L", [1, 4, 5, 6, 9, 11, 12, 13])
def test_tree_bit_exact(px, gauss, L):
    X, P, Y0, st = gauss
    rng = np.random.default_rng(L)
    n = P.n
    z = st.z.copy()
    z[:300] = z[0]                      # one very hot pixel
    z[300:310] = rng.integers(0, 2 ** 32, (10, 2), dtype=np.uint64).astype(np.uint32)
    z[310, :] = 0
    z[311, :] = 0xFFFFFFFF             # screen corners
    with make_ctx(px, L=L) as ctx:
        ctx.set_P(P.row_ptr, P.col, P.val.astype(np.float32))
        ctx.set_state(z, st.s)
        check_tree(ctx, z, L)


@pytest.mark.slow
def test_largest_screen(px, gauss):
    # L = 14 (a 16384^2 screen, the largest; 268M pixels, about 12 GB of
    # tree): counts at the root, the middle and the two deepest levels, the
    # leaf sums, and the forces of every point
    X, P, Y0, st = gauss
    L = 14
    with make_ctx(px, L=L) as ctx:
        inject(ctx, P, st)
        cnt_o, sx_o, sy_o = oracle.pyramid(st.z, L)
        for l in (0, 1, 7, 13, 14):
            cnt, sx, sy, _ = ctx.get_tree(l, sums=(l == L))
            off = oracle.level_offset(l)
            assert np.array_equal(cnt, cnt_o[off:off + 4 ** l]), l
        assert np.array_equal(sx, sx_o[off:off + 4 ** L])
        assert np.array_equal(sy, sy_o[off:off + 4 ** L])
        del cnt_o, sx_o, sy_o
        Frep, Zi, Fattr, Z = ctx.get_forces()
        assert ctx.sync() == 0
    oF, oZi, _ = oracle.bh_repulsion(st.z, st.s, L, 0.5)
    assert rel(Frep, oF) <= FORCE_TOL and rel(Zi, oZi) <= FORCE_TOL


@pytest.mark.parametrize("L,cm", [(4, 0), (11, 0), (13, 0), (11, 1)])
def test_tree_rebuilt_from_cleared_leaves(px, gauss, L, cm):
    # the pyramid clears the leaves it read: a second state's tree (both
    # pyramid kernels, and the count-only tree) has no trace of the first's
    X, P, Y0, st = gauss
    rng = np.random.default_rng(100 + L)
    z1 = st.z.copy()
    z2 = rng.integers(0, 2 ** 32, st.z.shape, dtype=np.uint64).astype(np.uint32)
    z2[:50] = z2[0]
    with make_ctx(px, L=L, centre_mode=cm) as ctx:
        ctx.set_P(P.row_ptr, P.col, P.val.astype(np.float32))
        for z in (z1, z2, z1):
            ctx.set_state(z, st.s)
            if cm == 0:
                check_tree(ctx, z, L)
            else:
                cnt_o, _, _ = oracle.pyramid(z, L)
                for l in range(L + 1):
                    cnt, _, _, _ = ctx.get_tree(l)
                    off = oracle.level_offset(l)
                    assert np.array_equal(cnt, cnt_o[off:off + 4 ** l]), l
        assert ctx.sync() == 0


@pytest.mark.parametrize("theta", [0.5, 0.0, 0.25, 1.0])
def test_forces_match_oracle(px, gauss, theta):
    X, P, Y0, st = gauss
    L = 9
    with make_ctx(px, L=L, theta=theta) as ctx:
        inject(ctx, P, st)
        Frep, Zi, Fattr, Z = ctx.get_forces()
        n_acc = ctx.counters()[0]
    oF, oZi, oacc = oracle.bh_repulsion(st.z, st.s, L, theta)
    oA = oracle.attraction(P, st.z, st.s)
    # the same (point, cell) interactions, up to FP32 d^2 at the criterion's
    # boundary
    assert n_acc == pytest.approx(int(oacc.sum()), rel=1e-4)
    assert rel(Frep, oF) <= FORCE_TOL
    assert rel(Zi, oZi) <= FORCE_TOL
    assert rel(Fattr, oA) <= FORCE_TOL
    assert abs(Z - oZi.sum()) / oZi.sum() <= FORCE_TOL


def test_forces_geometric_centre_mode(px, gauss):
    X, P, Y0, st = gauss
    with make_ctx(px, L=9, centre_mode=1) as ctx:
        inject(ctx, P, st)
        Frep, Zi, _, _ = ctx.get_forces()
    oF, oZi, _ = oracle.bh_repulsion(st.z, st.s, 9, 0.5, centre_mode=1)
    assert rel(Frep, oF) <= FORCE_TOL
    assert rel(Zi, oZi) <= FORCE_TOL


@pytest.mark.parametrize("L", [4, 9, 13])
def test_geometric_centre_mode_keeps_counts_only(px, gauss, L):
    """The geometric-centre tree (counts only, no coordinate sums): counts
    bit-exact at every level, through iterations (rescale, relabel) on both
    pyramid paths; forces still match the oracle's geometric-centre mode."""
    X, P, Y0, st = gauss
    with make_ctx(px, L=L, centre_mode=1) as ctx:
        ctx.set_P(P.row_ptr, P.col, P.val.astype(np.float32))
        ctx.init(Y0)
        ctx.step(30)
        z, s, _, _, _ = ctx.get_state()
        cnt_o = oracle.pyramid(z, L)[0]
        for lev in range(L + 1):
            cnt, _, _, _ = ctx.get_tree(lev)
            off = oracle.level_offset(lev)
            assert np.array_equal(cnt, cnt_o[off:off + 4 ** lev]), f"level {lev}"
        with pytest.raises(px.PxsneError) as ei:
            ctx.get_tree(L, sums=True)
        assert ei.value.code == -6
        ctx.set_state(*ctx.get_state())
        Frep, Zi, _, _ = ctx.get_forces()
        assert ctx.sync() == 0
    oF, oZi, _ = oracle.bh_repulsion(z, s, L, 0.5, centre_mode=1)
    assert rel(Frep, oF) <= FORCE_TOL
    assert rel(Zi, oZi) <= FORCE_TOL


def test_one_step_matches_oracle(px, gauss):
    X, P, Y0, st = gauss
    L = 9
    params = oracle.Params(L=L)
    with make_ctx(px, L=L) as ctx:
        inject(ctx, P, st)
        ctx.step(1)
        z, s, u, g, t = ctx.get_state()
    so = st.copy()
    oracle.run(P, so, params, 1)
    assert t == so.t
    assert np.allclose(s, so.s, rtol=1e-6)
    # positions after one step: the FP32 forces move points by < 1e-4 of a step
    y, yo = z * s, so.z * so.s
    step = np.abs(so.u).max()
    assert np.abs((y - y.mean(0)) - (yo - yo.mean(0))).max() <= 1e-3 * step + 4 * so.s.max()
    assert rel(u, so.u) <= 1e-3


def test_full_run_kl_within_one_percent(px, gauss):
    """The 2000-point mixture (512^2, 500 iterations): injected oracle P, same Y0."""
    X, P, Y0, _ = gauss
    params = oracle.Params(L=9)
    st = oracle.State.from_y0(Y0)
    oracle.run(P, st, params, 500)
    kl_o = oracle.kl_of(P, st, params)
    with make_ctx(px, L=9) as ctx:
        ctx.set_P(P.row_ptr, P.col, P.val.astype(np.float32))
        ctx.init(Y0)
        ctx.step(500)
        kl_g = ctx.kl()
        z, s, _, _, t = ctx.get_state()
    assert t == 500
    # the GPU's own KL evaluation against the oracle's on the GPU's final state
    kl_o_on_g = oracle.kl_of(P, oracle.State(z, s, None, None), params)
    assert abs(kl_g - kl_o_on_g) <= 1e-4 * kl_o_on_g
    assert abs(kl_g - kl_o) <= 0.01 * kl_o, (kl_g, kl_o)


def check_knn_rows(X, rows, idx_o, d2_o, idx, d2, tol=2e-5):
    """What is unique must match (neighbours closer than the true k-th distance
    by more than the FP32 error); every returned neighbour must be within the
    tolerance of the true k-th distance."""
    for q, i in enumerate(rows):
        dk = d2_o[q, -1]
        must = set(idx_o[q][d2_o[q] < dk * (1 - tol)])
        got = set(idx[i])
        assert len(got) == idx.shape[1], i       # k distinct neighbours
        assert must <= got, i
        dd = ((X[idx[i]].astype(np.float64) - X[i].astype(np.float64)) ** 2).sum(1)
        assert np.all(dd <= dk * (1 + tol)), i
        assert i not in got
        np.testing.assert_allclose(d2[i], np.sort(dd), rtol=1e-5)


@pytest.fixture(params=["tc", "fp32"])
def knn_path(request, monkeypatch):
    """Run the neighbour search on the tensor cores (default) or the FP32 path."""
    if request.param == "fp32":
        monkeypatch.setenv("PXSNE_KNN", "fp32")
    else:
        monkeypatch.delenv("PXSNE_KNN", raising=False)
    return request.param


def test_affinities_match_oracle(px, knn_path):
    X, _ = datagen.gauss10(1, n=1500)
    X[7] = X[3]                       # duplicate rows: distance 0, tie on index
    X[900] = X[3]
    k, u = 90, 30.0
    P, idx_o, d2_o, bad = oracle.affinities(X, u, k)
    with make_ctx(px, L=9, k=k, perplexity=u) as ctx:
        ctx.affinities(X)
        idx, d2, beta = ctx.get_knn()
        rp, col, val = ctx.get_P()
    n = X.shape[0]
    check_knn_rows(X, np.arange(n), idx_o, d2_o, idx, d2)
    assert idx[3][0] == 7 and idx[3][1] == 900
    # perplexity of each GPU row, evaluated in FP64 from its own d2 and beta
    e = np.exp(-beta[:, None].astype(np.float64) * (d2 - d2[:, :1]))
    p = e / e.sum(1, keepdims=True)
    H = -(p * np.log(p)).sum(1)
    assert np.abs(H - np.log(u)).max() < 1e-4
    # symmetric P: same pattern, values within the bisection tolerance
    assert np.array_equal(rp, P.row_ptr) and np.array_equal(col, P.col)
    np.testing.assert_allclose(val, P.val, rtol=2e-3, atol=1e-9)
    assert abs(val.astype(np.float64).sum() - 1.0) < 1e-5


@pytest.mark.parametrize("n,k", [(130, 5), (129, 90), (200, 90), (257, 33)])
def test_knn_small_sizes(px, knn_path, n, k):
    """Small searches: a few tiles, the last one ragged (129 rows: one row in
    it), k close to n, a small k (short lists, odd row strides)."""
    X, _ = datagen.gauss10(4, n=n)
    idx_o, d2_o = oracle.knn(X, k)
    with make_ctx(px, L=9, k=k, perplexity=min(30.0, k / 3.0)) as ctx:
        ctx.affinities(X)
        idx, d2, _ = ctx.get_knn()
    check_knn_rows(X, np.arange(n), idx_o, d2_o, idx, d2)


def test_knn_many_duplicates(px, knn_path):
    """300 identical rows: each one's list is decided by the tie rule alone
    (distance 0, then the lower index), whatever order the survivors are
    inserted in.  Those rows' k neighbours all lie at distance 0, so no
    bandwidth gives them perplexity 30: the call reports the bisection flag,
    as documented, and the lists are still there."""
    X, _ = datagen.gauss10(5, n=1000)
    X[100:400] = X[100]
    k = 90
    idx_o, d2_o = oracle.knn(X, k)
    with make_ctx(px, L=9, k=k, perplexity=30.0) as ctx:
        with pytest.raises(px.PxsneError, match="bisection"):
            ctx.affinities(X)
        idx, d2, _ = ctx.get_knn()
        assert ctx.sync() == 0
    check_knn_rows(X, np.arange(X.shape[0]), idx_o, d2_o, idx, d2)
    for i in (100, 150, 399):
        want = [j for j in range(100, 400) if j != i][:k]
        assert list(idx[i]) == want, i
        assert not d2[i].any()


def test_knn_far_from_origin(px, knn_path):
    """Points far from the origin next to their spread (the 10-Gaussian
    mixture moved by 500 on every axis: |x| about 3,500 against neighbour
    distances about 10), where the FP16 copies' rounding errors are a
    sizeable part of the distances: the lists must stay exact."""
    X, _ = datagen.gauss10(2, n=3000)
    X = (X.astype(np.float64) + 500.0).astype(np.float32)
    k = 90
    rows = np.arange(X.shape[0])
    idx_o, d2_o = oracle.knn(X, k)
    with make_ctx(px, L=9, k=k, perplexity=30.0) as ctx:
        ctx.affinities(X)
        idx, d2, _ = ctx.get_knn()
    check_knn_rows(X, rows, idx_o, d2_o, idx, d2)


def test_affinities_with_hub_rows(px):
    """Rows of the symmetric P longer than a warp's staging buffer (1,024
    entries): points spread over a shell (radii 8 to 12) around two central
    points, which are in nearly every other point's neighbour list."""
    rng = np.random.default_rng(5)
    n, D, k, u = 2500, 50, 90, 30.0
    X = rng.standard_normal((n, D))
    X *= rng.uniform(8.0, 12.0, (n, 1)) / np.linalg.norm(X, axis=1, keepdims=True)
    X = X.astype(np.float32)
    X[0] = 0.0
    X[1] = 0.05
    P, idx_o, d2_o, bad = oracle.affinities(X, u, k)
    assert np.diff(P.row_ptr)[:2].min() > 1024
    with make_ctx(px, L=9, k=k, perplexity=u) as ctx:
        ctx.affinities(X)
        rp, col, val = ctx.get_P()
    assert np.array_equal(rp, P.row_ptr) and np.array_equal(col, P.col)
    np.testing.assert_allclose(val, P.val, rtol=2e-3, atol=1e-9)


def test_knn_d128_sampled_rows(px, knn_path):
    """The bench's data shape (D = 128 anisotropic mixture) at n = 20,000 with a
    ragged last tile; exact FP64 neighbours of 300 sampled rows."""
    n, k = 20011, 90
    X, _ = datagen.gmm128(seed=3, n=n)
    rows = np.random.default_rng(0).choice(n, 300, replace=False)
    rows = np.concatenate([rows, [0, n - 1]])
    idx_o, d2_o = oracle.knn(X, k, rows=rows)
    with make_ctx(px, L=11, k=k, perplexity=30.0) as ctx:
        ctx.affinities(X)
        idx, d2, _ = ctx.get_knn()
    check_knn_rows(X, rows, idx_o, d2_o, idx, d2)


def test_full_gpu_path_kl(px):
    """Whole GPU path (P built on the GPU) vs the oracle's whole path."""
    X, _ = datagen.gauss10(0)
    Y0 = datagen.init_y0(0, X.shape[0])
    params = oracle.Params(L=9)
    P, _, _, _ = oracle.affinities(X, 30.0, 90)
    st = oracle.State.from_y0(Y0)
    oracle.run(P, st, params, 500)
    kl_o = oracle.kl_of(P, st, params)
    with make_ctx(px, L=9) as ctx:
        ctx.affinities(X)
        ctx.init(Y0)
        ctx.step(500)
        kl_g = ctx.kl()
    assert abs(kl_g - kl_o) <= 0.01 * kl_o, (kl_g, kl_o)


def test_get_Y_and_pixels(px, gauss):
    X, P, Y0, st = gauss
    with make_ctx(px, L=9) as ctx:
        inject(ctx, P, st)
        Y, pix = ctx.get_Y()
        pix_only = np.empty_like(pix)
        ctx.get_Y(None, pix_only)          # pixels alone (no centring pass)
    assert np.array_equal(pix, (st.z >> (32 - 9)).astype(np.int32))
    assert np.array_equal(pix_only, pix)
    y = st.y()
    np.testing.assert_allclose(Y, y - y.mean(0), rtol=0, atol=1e-6 * np.abs(y).max())


def test_get_Y_without_synchronising(px, gauss):
    # the frame enqueued on the context's stream (device buffers, no host
    # wait) equals the synchronised one once the stream has reached it, also
    # with steps enqueued behind it
    import torch
    X, P, Y0, st = gauss
    s = torch.cuda.Stream()
    n = P.n
    with px.Context(px.Params(log2_r=9), stream=s.cuda_stream) as ctx:
        inject(ctx, P, st)
        Yd = torch.empty((n, 2), dtype=torch.float32, device="cuda")
        Pd = torch.empty((n, 2), dtype=torch.int32, device="cuda")
        ctx.get_Y(Yd, Pd, blocking=False)
        ctx.step(3)
        s.synchronize()
        Y2, pix2 = ctx.get_Y()            # after the three steps
        z2 = ctx.get_state()[0]
        assert np.array_equal(Pd.cpu().numpy(), (st.z >> (32 - 9)).astype(np.int32))
        y = st.y()
        np.testing.assert_allclose(Yd.cpu().numpy(), y - y.mean(0), rtol=0,
                                   atol=1e-6 * np.abs(y).max())
        assert np.array_equal(pix2, (z2 >> (32 - 9)).astype(np.int32))
        with pytest.raises(ValueError):
            ctx.get_Y(np.empty((n, 2), np.float32), None, blocking=False)
        assert ctx.sync() == 0


def test_edge_cases(px):
    # two points (k = 1), both in one pixel, then apart
    P = oracle.CSR(np.array([0, 1, 2]), np.array([1, 0], np.int32), np.array([0.5, 0.5]))
    with make_ctx(px, L=3, k=1, perplexity=1.0) as ctx:
        ctx.set_P(P.row_ptr, P.col, P.val.astype(np.float32))
        for z in (np.array([[5, 5], [5, 5]], np.uint32),
                  np.array([[0, 0], [2 ** 32 - 1, 2 ** 32 - 1]], np.uint32)):
            s = np.array([1e-9, 2e-9])
            ctx.set_state(z, s)
            Frep, Zi, Fattr, Z = ctx.get_forces()
            oF, oZi, _ = oracle.bh_repulsion(z, s, 3, 0.5)
            np.testing.assert_allclose(Frep, oF, rtol=1e-5, atol=1e-30)
            np.testing.assert_allclose(Zi, oZi, rtol=1e-6)
            ctx.step(3)
            assert np.isfinite(ctx.kl())
    # ragged n (not a multiple of the warp or CTA), all points in one pixel
    n = 1001
    rng = np.random.default_rng(5)
    X = rng.standard_normal((n, 3)).astype(np.float32)
    Po, _, _, _ = oracle.affinities(X, 5.0, 15)
    z = np.full((n, 2), 123456789, np.uint32)
    z[:, 0] += np.arange(n, dtype=np.uint32)
    s = np.array([1e-6, 1e-6])
    with make_ctx(px, L=11, k=15, perplexity=5.0) as ctx:
        ctx.set_P(Po.row_ptr, Po.col, Po.val.astype(np.float32))
        ctx.set_state(z, s)
        check_tree(ctx, z, 11)
        Frep, Zi, Fattr, Z = ctx.get_forces()
        oF, oZi, _ = oracle.bh_repulsion(z, s, 11, 0.5)
        assert rel(Frep, oF) <= FORCE_TOL and rel(Zi, oZi) <= FORCE_TOL
        ctx.step(5)
        assert ctx.sync() == 0


def test_invalid_calls(px):
    with make_ctx(px, L=9) as ctx:
        with pytest.raises(px.PxsneError):
            ctx.step(1)                     # no state
        with pytest.raises(px.PxsneError):
            ctx.init(np.zeros((10, 2), np.float32))   # no P
        X = np.zeros((50, 3), np.float32)
        X[3, 1] = np.nan
        with pytest.raises(px.PxsneError):
            ctx.affinities(X)
        with pytest.raises(px.PxsneError):
            ctx.affinities(np.zeros((50, 300), np.float32))   # D > 256


def test_P_with_empty_rows(px, gauss):
    # points that nothing attracts: the first, a middle and the last row of P
    # emptied, and every entry pointing at them removed; checked at the
    # injected state and after 120 iterations (across the attraction's
    # relabel at t = 100)
    X, P, Y0, st = gauss
    n, L = P.n, 9
    params = oracle.Params(L=L)
    gone = np.array([0, 777, n - 1])
    keep_row = np.ones(n, bool)
    keep_row[gone] = False
    rows = np.repeat(np.arange(n), np.diff(P.row_ptr))
    keep = keep_row[rows] & keep_row[P.col]
    rp = np.concatenate([[0], np.cumsum(np.bincount(rows[keep], minlength=n))]).astype(np.int64)
    Pe = oracle.CSR(rp, P.col[keep].astype(np.int32), P.val[keep])
    assert all(rp[i] == rp[i + 1] for i in gone)
    with make_ctx(px, L=L) as ctx:
        ctx.set_P(Pe.row_ptr, Pe.col, Pe.val.astype(np.float32))
        ctx.set_state(st.z, st.s, st.u.astype(np.float32), st.gains.astype(np.float32), st.t)
        for it in (0, 120):
            if it:
                ctx.step(it)
            z, s, _, _, t = ctx.get_state()
            assert t == st.t + it
            Frep, Zi, Fattr, Z = ctx.get_forces()
            assert not Fattr[gone].any()
            assert rel(Fattr, oracle.attraction(Pe, z, s)) <= FORCE_TOL
            oF, oZi, _ = oracle.bh_repulsion(z, s, L, 0.5)
            assert rel(Frep, oF) <= FORCE_TOL
            kl_o = oracle.kl_of(Pe, oracle.State(z, s, None, None), params)
            assert abs(ctx.kl() - kl_o) <= 1e-4 * kl_o
        assert ctx.sync() == 0


def test_nonfinite_X_refused_and_context_kept(px, gauss):
    # the check runs on the device, for host and device X alike, before any
    # state is replaced: a refused call leaves P and the embedding as they were
    import torch
    X, P, Y0, _ = gauss
    with make_ctx(px, L=9) as ctx:
        ctx.affinities(X)
        ctx.init(Y0)
        ctx.step(3)
        before = ctx.get_state()
        rp, col, val = ctx.get_P()
        for bad in (np.inf, -np.inf, np.nan):
            Xb = X.copy()
            Xb[X.shape[0] - 1, X.shape[1] - 1] = bad   # the last value of X
            for src in (Xb, torch.from_numpy(Xb).cuda()):
                with pytest.raises(px.PxsneError):
                    ctx.affinities(src)
        for a, b in zip(ctx.get_state(), before):
            assert np.array_equal(a, b)
        rp2, col2, val2 = ctx.get_P()
        assert np.array_equal(rp, rp2) and np.array_equal(col, col2) and np.array_equal(val, val2)
        ctx.step(2)
        assert ctx.sync() == 0
        # a finite X passed on the device is taken
        ctx.affinities(torch.from_numpy(X).cuda())
        assert np.array_equal(ctx.get_P()[1], col)


@pytest.mark.parametrize("k", [1, 10, 32])
def test_nbr_precision_matches_oracle(px, gauss, k):
    X, P, Y0, st = gauss
    kh = 90
    idx, _ = oracle.knn(X, kh)
    z = st.z.copy()
    z[10] = z[11]                 # coinciding points: ties to the lower index
    z[12] = z[11]
    with make_ctx(px, L=9) as ctx:
        ctx.set_P(P.row_ptr, P.col, P.val.astype(np.float32))
        ctx.set_state(z, st.s)
        prec, hits = ctx.nbr_precision(k=k, knn_hd=idx, per_point=True)
    prec_o, hits_o = oracle.nbr_precision(idx, k, z, st.s, per_row=True)
    assert np.array_equal(hits, hits_o)
    assert prec == pytest.approx(prec_o, abs=1e-15)


def test_pca_matches_oracle(px):
    """MNIST-shaped workload (784-D, 10 classes) at 8,000 rows, 50 components."""
    X, _ = datagen.protos784(seed=4, n=8000)
    Z, V, lam = px.pca(X, 50, seed=1)
    Zo, Vo, lamo = oracle.pca(X, 50)
    # the leading, well separated eigenpairs agree; the 50-dim subspace keeps the
    # same variance
    np.testing.assert_allclose(lam[:10], lamo[:10], rtol=1e-4)
    P10 = V[:, :10].astype(np.float64) @ V[:, :10].T
    Po10 = Vo[:, :10] @ Vo[:, :10].T
    assert np.linalg.norm(P10 - Po10) < 1e-3
    assert abs(lam.sum() - lamo.sum()) <= 2e-3 * lamo.sum()
    np.testing.assert_allclose(V.T.astype(np.float64) @ V, np.eye(50), atol=1e-4)
    # projections agree up to the (fixed) signs of the leading components
    rel = np.linalg.norm(Z[:, :10] - Zo[:, :10]) / np.linalg.norm(Zo[:, :10])
    assert rel < 1e-3


def test_profiled_run_and_work_counters(px, gauss):
    """pxsne_step_profiled times the iteration's own kernels and counts each
    iteration's state by one more traversal afterwards: its counters are the
    sums over those states, equal to the counters of the same states set
    again one by one, and the accepted pairs equal the oracle's count."""
    X, P, Y0, _ = gauss
    with make_ctx(px, L=9) as ctx, make_ctx(px, L=9) as ref:
        ctx.set_P(P.row_ptr, P.col, P.val.astype(np.float32))
        ref.set_P(P.row_ptr, P.col, P.val.astype(np.float32))
        ctx.init(Y0)
        states = []
        for _ in range(7):
            ctx.step(1)
            states.append(ctx.get_state())
        ctx.init(Y0)
        groups, total = ctx.step_profiled(7)
        assert list(groups) == ["k_relabel", "k_update", "k_snap_hist", "k_pyr_pass",
                                "k_perm_scatter", "k_bh_traverse", "k_attract", "k_zsum"]
        assert all(v >= 0.0 for v in groups.values()) and groups["k_bh_traverse"] > 0.0
        assert sum(groups.values()) <= total * 1.001 + 1e-3
        c1 = ctx.counters()
        lv = ctx.level_counters()
        # by level of the tested cell: they add up to the totals
        assert (int(lv[:, 1].sum()), int(lv[:, 0].sum()), int(lv[:, 2].sum())) == c1[:3]
        assert lv[0].sum() == 0 and lv[9, 0] > 0
        F1 = ctx.get_forces()
        z, s, u, g, t = ctx.get_state()
        for a, b in zip((z, s, u, g, t), states[-1]):
            assert np.array_equal(a, b)
        sums = np.zeros(4, np.int64)
        acc_oracle = 0
        for st in states:
            ref.set_state(*st)
            sums += np.array(ref.counters(), np.int64)
            _, _, acc = oracle.bh_repulsion(st[0], st[1], 9, 0.5)
            acc_oracle += int(acc.sum())
        # per-point counts are the same; warp steps and nodes depend on how
        # points within a pixel are grouped into warps, which follows the
        # order of the previous tree (identity order after set_state)
        assert tuple(sums[:2]) == c1[:2]
        assert c1[2] == pytest.approx(sums[2], rel=0.01)
        assert c1[3] == pytest.approx(sums[3], rel=0.01)
        F2 = ref.get_forces()
        for a, b in zip(F1[:3], F2[:3]):
            assert np.array_equal(a, b)
    assert c1[0] == pytest.approx(acc_oracle, rel=1e-4)
    assert c1[1] >= c1[0] and c1[2] > 0 and c1[3] > 0
