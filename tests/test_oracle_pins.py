"""Pins of the CPU oracle against things other than itself.

Each oracle function is checked against what the paper and the mathematics
fix, so that a dropped term, a wrong sign or index, or a transposed operand
fails at least one test:

  knn            brute force by a full stable argsort of the FP64 distance matrix
  perplexity     definitional invariants of the output (entropy of the returned
                 row = ln u, p proportional to exp(-beta d2), rows sum to 1),
                 closed form for equal distances, scale invariance
  symmetrize     dense (P_cond + P_cond^T) / 2n construction, sum 1, symmetry
  init_fx        extremes map to 0 and R-1, affine within one ulp; the floor
                 of the exact rational map
  morton         recursive quadtree child numbering (child = 2*ybit + xbit)
  pyramid        per-level bincount of the shifted pixel pairs; sums
  exact forces   scikit-learn's exact t-SNE KL and gradient; hand-derived
                 closed forms (tests/golden/kl_closed_forms.txt); finite
                 differences of the KL; net force zero; stored zeros of P
                 add nothing to the KL; sampled rows equal the full rows
  bh_repulsion   theta = 0 with <= 1 point per pixel equals the exact sum;
                 theta = 0 in general equals a tree-free brute force over pixels
                 (centres of mass; pixel midpoints in geometric-centre mode);
                 the acceptance threshold on a hand-built tree sits at
                 r_c / d = theta (r_c the cell diagonal, d the distance to the
                 centre of mass; r_c / d^2 in the printed form); at a huge
                 theta exactly the siblings of a point's own cells; error
                 falls with theta
  rescale        Python big-integer arithmetic; pixel range exactly 0..r-1
  update         hand cases of the gains rule; the step rounded half to even
  run            one step is the composition of the pinned parts, bit for
                 bit; the fixed-point + rescale + beta run equals plain y-space
                 t-SNE (scikit-learn gradient) up to translation (Sec. 4.2's
                 claimed equivalence)
  kl             scikit-learn, closed forms, KL >= 0, a stored value written
                 by tests/golden/make_kl_target.py
  nbr_precision  per-row brute force by a full stable argsort; identity cases
                 (precision 1 for the same geometry, ~k/n for an unrelated one)
  gelu, mlp      the erf definition and central differences; a closed-form
                 forward pass; finite differences of the loss
  pca            SVD of the centred matrix
  philox_y0      the generator's published known-answer vectors; the draw's
                 mean, scale, one-sigma mass and independence

tests/test_oracle_mutants.py plants one such mistake at a time in a copy of
the oracle and checks that these pins fail.
"""
import json
import math
import os
import sys

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
R = 2 ** 32


# ------------------------------------------------------------------ kNN
def test_knn_matches_full_sort():
    rng = np.random.default_rng(1)
    X = rng.standard_normal((257, 7)).astype(np.float32)
    X[10] = X[3]           # duplicate points: distance 0, tie on index
    X[200] = X[3]
    X[50] = X[51]
    k = 12
    idx, d2 = oracle.knn(X, k)
    Xd = X.astype(np.float64)
    Dm = ((Xd[:, None, :] - Xd[None, :, :]) ** 2).sum(-1)
    np.fill_diagonal(Dm, np.inf)
    ref = np.argsort(Dm, axis=1, kind="stable")[:, :k]
    assert np.array_equal(idx, ref)
    np.testing.assert_allclose(d2, np.take_along_axis(Dm, ref, 1), rtol=1e-12, atol=0)
    # sampled rows give the same answer as the full run
    rows = np.array([0, 3, 256, 10])
    idx2, d22 = oracle.knn(X, k, rows=rows)
    assert np.array_equal(idx2, idx[rows])
    assert idx[3][0] in (10, 200) and idx[3][0] == 10  # lower index wins the tie


def test_knn_rejects_k_ge_n():
    X = np.zeros((5, 3), np.float32)
    with pytest.raises(ValueError):
        oracle.knn(X, 5)


# ------------------------------------------------------------------ perplexity
def test_perplexity_invariants():
    rng = np.random.default_rng(2)
    d2 = np.sort(rng.gamma(3.0, 20.0, (300, 90)), axis=1)
    u = 30.0
    p, beta, H, bad = oracle.perplexity(d2, u)
    assert bad == 0
    assert np.all(beta > 0)
    np.testing.assert_allclose(p.sum(1), 1.0, rtol=0, atol=1e-12)
    Hdef = -(p * np.log(p)).sum(1)            # entropy of the returned rows
    assert np.max(np.abs(Hdef - math.log(u))) < 1e-5
    np.testing.assert_allclose(Hdef, H, rtol=0, atol=1e-10)
    # Gaussian kernel: p_j / p_0 = exp(-beta (d_j - d_0))
    ratio = p / p[:, :1]
    np.testing.assert_allclose(ratio, np.exp(-beta[:, None] * (d2 - d2[:, :1])),
                               rtol=1e-10, atol=1e-300)
    # ascending distances give non-increasing p
    assert np.all(np.diff(p, axis=1) <= 1e-15)


def test_perplexity_equal_distances_closed_form():
    # all k distances equal: p = 1/k for every beta and H = ln k
    d2 = np.full((4, 30), 7.25)
    p, beta, H, bad = oracle.perplexity(d2, 30.0)
    assert bad == 0
    np.testing.assert_allclose(p, 1.0 / 30, rtol=1e-14)
    np.testing.assert_allclose(H, math.log(30), rtol=1e-14)


def test_perplexity_unreachable_target():
    # all k distances tied but a perplexity below k: H = ln k whatever beta,
    # so no beta reaches the target; every row is reported and keeps the
    # uniform weights 1/k
    d2 = np.zeros((3, 90))
    d2[1] = 4.0
    p, beta, H, bad = oracle.perplexity(d2, 30.0)
    assert bad == 3
    np.testing.assert_allclose(p, 1.0 / 90, rtol=1e-14)
    np.testing.assert_allclose(H, math.log(90), rtol=1e-14)


def test_perplexity_scale_invariance():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((400, 10)).astype(np.float32)
    idx1, d1 = oracle.knn(X, 30)
    idx2, d2 = oracle.knn(X * np.float32(4.0), 30)
    assert np.array_equal(idx1, idx2)
    p1, b1, _, _ = oracle.perplexity(d1, 10.0)
    p2, b2, _, _ = oracle.perplexity(d2, 10.0)
    # beta absorbs the scale (c^2 = 16) up to the bisection tolerance
    np.testing.assert_allclose(p1, p2, rtol=2e-3, atol=1e-6)


# ------------------------------------------------------------------ symmetrize
def test_symmetrize_dense():
    rng = np.random.default_rng(4)
    X = rng.standard_normal((150, 5)).astype(np.float32)
    k = 9
    idx, d2 = oracle.knn(X, k)
    p, _, _, _ = oracle.perplexity(d2, 3.0)
    P = oracle.symmetrize(idx, p)
    n = X.shape[0]
    C = np.zeros((n, n))
    for i in range(n):
        C[i, idx[i]] = p[i]
    ref = (C + C.T) / (2 * n)
    D = P.dense()
    np.testing.assert_allclose(D, ref, rtol=1e-14, atol=0)
    assert abs(D.sum() - 1.0) < 1e-12
    assert np.array_equal(D != 0, ref != 0)
    for i in range(n):  # columns strictly ascending in each row, no self
        c = P.col[P.row_ptr[i]:P.row_ptr[i + 1]]
        assert np.all(np.diff(c) > 0) and i not in c


# ------------------------------------------------------------------ fixed point
def test_init_fx_extremes_and_affine():
    rng = np.random.default_rng(5)
    Y = rng.standard_normal((500, 2)) * 1e-4
    z, s = oracle.init_fx(Y)
    for d in range(2):
        assert z[:, d].min() == 0 and z[:, d].max() == R - 1
        mn, mx = Y[:, d].min(), Y[:, d].max()
        assert s[d] == (mx - mn) / R
        back = z[:, d].astype(np.float64) * s[d] + mn
        assert np.max(np.abs(back - Y[:, d])) <= s[d] * 1.0000001
    # degenerate axis
    Y2 = np.stack([np.arange(4.0), np.full(4, 3.0)], 1)
    z2, s2 = oracle.init_fx(Y2)
    assert np.all(z2[:, 1] == 0) and s2[1] == 1.0 / R


def _morton_rec(px, py):
    if px == 0 and py == 0:
        return 0
    return 4 * _morton_rec(px >> 1, py >> 1) + ((py & 1) << 1 | (px & 1))


def test_morton_recursive_child_numbering():
    rng = np.random.default_rng(6)
    for px, py in rng.integers(0, 2 ** 15, (300, 2)):
        assert oracle.morton(px, py) == _morton_rec(int(px), int(py))
    assert [oracle.morton(x, y) for (x, y) in [(0, 0), (1, 0), (0, 1), (1, 1)]] == [0, 1, 2, 3]
    # an aligned 2^k x 2^k block is a contiguous Morton range
    k = 3
    block = sorted(oracle.morton(8 + x, 16 + y) for x in range(8) for y in range(8))
    assert block == list(range(block[0], block[0] + 64))


def test_pyramid_counts_and_sums():
    rng = np.random.default_rng(7)
    L = 5
    n = 3000
    z = rng.integers(0, R, (n, 2), dtype=np.uint64)
    z[:500] = z[0]          # a hot pixel
    z = z.astype(np.uint32)
    cnt, sx, sy = oracle.pyramid(z, L)
    assert cnt.shape[0] == (4 ** (L + 1) - 1) // 3
    F = 32 - L
    px = (z[:, 0] >> F).astype(np.int64)
    py = (z[:, 1] >> F).astype(np.int64)
    for l in range(L + 1):
        off = (4 ** l - 1) // 3
        cx, cy = px >> (L - l), py >> (L - l)
        m = np.array([_morton_rec(int(a), int(b)) for a, b in zip(cx, cy)])
        ref_cnt = np.bincount(m, minlength=4 ** l)
        assert np.array_equal(cnt[off:off + 4 ** l], ref_cnt)
        ref_sx = np.zeros(4 ** l, dtype=object)
        ref_sy = np.zeros(4 ** l, dtype=object)
        for i in range(n):
            ref_sx[m[i]] += int(z[i, 0])
            ref_sy[m[i]] += int(z[i, 1])
        assert [int(v) for v in sx[off:off + 4 ** l]] == list(ref_sx)
        assert [int(v) for v in sy[off:off + 4 ** l]] == list(ref_sy)
        assert int(cnt[off:off + 4 ** l].sum()) == n
    _, _, mk = oracle.leaf_keys(z, L)
    assert np.array_equal(mk, [_morton_rec(int(a), int(b)) for a, b in zip(px, py)])


# ------------------------------------------------------------------ forces / KL
def _dense_csr(Pd):
    n = Pd.shape[0]
    rows, cols = np.nonzero(Pd)
    rp = np.zeros(n + 1, np.int64)
    np.add.at(rp, rows + 1, 1)
    rp = np.cumsum(rp)
    return oracle.CSR(rp, cols.astype(np.int32), Pd[rows, cols].astype(np.float64))


def _random_state(n, seed, sigma=3.0):
    rng = np.random.default_rng(seed)
    Y = rng.standard_normal((n, 2)) * sigma
    return oracle.init_fx(Y)


def _oracle_grad(P, z, s, alpha=1.0):
    Frep, Zi = oracle.exact_repulsion(z, s)
    Fattr = oracle.attraction(P, z, s)
    Z = Zi.sum()
    return 4.0 * (alpha * Fattr - Frep / Z), Z, Fattr, Frep


def test_exact_gradient_and_kl_match_sklearn():
    tsne = pytest.importorskip("sklearn.manifold._t_sne")
    from scipy.spatial.distance import squareform
    n = 40
    rng = np.random.default_rng(8)
    A = rng.random((n, n))
    A = A + A.T
    np.fill_diagonal(A, 0)
    Pd = A / A.sum()
    P = _dense_csr(Pd)
    z, s = _random_state(n, 9)
    y = z.astype(np.float64) * s
    g, Z, _, _ = _oracle_grad(P, z, s)
    kl_ref, g_ref = tsne._kl_divergence(y.ravel(), squareform(Pd, checks=False), 1, n, 2)
    np.testing.assert_allclose(g.ravel(), g_ref, rtol=1e-9, atol=1e-12 * np.abs(g_ref).max())
    assert abs(oracle.kl(P, z, s, Z) - kl_ref) < 1e-10 * max(1.0, kl_ref)
    # exaggerated gradient = gradient of the KL with alpha * P in the first term
    g4, _, _, _ = _oracle_grad(P, z, s, alpha=4.0)
    _, g4_ref = tsne._kl_divergence(y.ravel(), 4.0 * squareform(Pd, checks=False), 1, n, 2)
    np.testing.assert_allclose(g4.ravel(), g4_ref, rtol=1e-9,
                               atol=1e-12 * np.abs(g4_ref).max())


def test_gradient_finite_differences():
    n = 25
    rng = np.random.default_rng(10)
    A = rng.random((n, n)) ** 3
    A = A + A.T
    np.fill_diagonal(A, 0)
    P = _dense_csr(A / A.sum())
    z, s = _random_state(n, 11)
    g, _, _, _ = _oracle_grad(P, z, s)

    def C(zz):
        _, Zi = oracle.exact_repulsion(zz, s)
        return oracle.kl(P, zz, s, Zi.sum())

    h = 2 ** 18  # ulps
    for i, d in [(0, 0), (3, 1), (17, 0), (24, 1)]:
        zp = z.astype(np.int64).copy()
        zm = z.astype(np.int64).copy()
        zp[i, d] += h
        zm[i, d] -= h
        fd = (C(zp.astype(np.uint32)) - C(zm.astype(np.uint32))) / (2 * h * s[d])
        assert abs(fd - g[i, d]) < 1e-6 * np.abs(g).max()


def _golden_cases():
    out = []
    with open(os.path.join(GOLDEN, "kl_closed_forms.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            t = line.split()
            n = int(t[1])
            xs = [float(v) for v in t[2:2 + n]]
            kl = float(t[2 + n])
            gx = [float(v) for v in t[3 + n:3 + 2 * n]]
            out.append((t[0], n, xs, kl, gx))
    return out


@pytest.mark.parametrize("case", _golden_cases(), ids=lambda c: c[0])
def test_closed_form_kl_and_gradient(case):
    name, n, xs, kl_ref, gx_ref = case
    # y_x = s_x * z_x exactly with s_x = 2^-20; y_y = 0
    s = np.array([2.0 ** -20, 1.0])
    z = np.zeros((n, 2), np.uint32)
    z[:, 0] = [int(round(x * 2 ** 20)) for x in xs]
    Pd = np.zeros((n, n))
    Pd[0, 1] = Pd[1, 0] = 0.5
    P = _dense_csr(Pd)
    g, Z, _, _ = _oracle_grad(P, z, s)
    assert abs(oracle.kl(P, z, s, Z) - kl_ref) < 1e-14
    np.testing.assert_allclose(g[:, 0], gx_ref, rtol=0, atol=1e-14)
    np.testing.assert_allclose(g[:, 1], 0.0, atol=0)


def test_net_forces_vanish():
    n = 120
    rng = np.random.default_rng(12)
    A = (rng.random((n, n)) < 0.1) * rng.random((n, n))
    A = A + A.T
    np.fill_diagonal(A, 0)
    P = _dense_csr(A / A.sum())
    z, s = _random_state(n, 13)
    Frep, Zi = oracle.exact_repulsion(z, s)
    Fattr = oracle.attraction(P, z, s)
    assert np.abs(Fattr.sum(0)).max() < 1e-12 * np.abs(Fattr).sum()
    assert np.abs(Frep.sum(0)).max() < 1e-12 * np.abs(Frep).sum()


def test_sampled_rows_equal_the_full_rows():
    # the row-sampled forms (used at full sizes, where only a sample of rows
    # is affordable) give row rows[q] of the full result, in the listed order,
    # repeats included
    n, L = 300, 6
    rng = np.random.default_rng(26)
    A = (rng.random((n, n)) < 0.05) * rng.random((n, n))
    A = A + A.T
    np.fill_diagonal(A, 0)
    P = _dense_csr(A / A.sum())
    z, s = _random_state(n, 27)
    rows = np.array([299, 0, 17, 17, 150, 3])
    Fe, Ze = oracle.exact_repulsion(z, s)
    Fr, Zr = oracle.exact_repulsion(z, s, rows=rows)
    assert np.array_equal(Fr, Fe[rows]) and np.array_equal(Zr, Ze[rows])
    Fa = oracle.attraction(P, z, s)
    assert np.array_equal(oracle.attraction(P, z, s, rows=rows), Fa[rows])
    for cm in (0, 1):
        Fb, Zb, ab = oracle.bh_repulsion(z, s, L, 0.5, centre_mode=cm)
        Fq, Zq, aq = oracle.bh_repulsion(z, s, L, 0.5, rows=rows, centre_mode=cm)
        assert np.array_equal(Fq, Fb[rows]) and np.array_equal(Zq, Zb[rows])
        assert np.array_equal(aq, ab[rows])
    idx, _ = oracle.knn(rng.standard_normal((n, 3)).astype(np.float32), 8)
    _, hits = oracle.nbr_precision(idx, 8, z, s, per_row=True)
    p_r, hits_r = oracle.nbr_precision(idx[rows], 8, z, s, rows=rows, per_row=True)
    assert np.array_equal(hits_r, hits[rows])
    assert p_r == hits[rows].sum() / (8 * len(rows))


def test_Z_of_the_run_is_the_sum_of_its_repulsion():
    # the KL's normalisation: Z = sum_i Z_i of the run's own repulsion, the
    # tree's at the run's theta and centre mode, the exact sum when exact
    n, L = 400, 7
    z, s = _random_state(n, 32)
    st = oracle.State(z, s, np.zeros((n, 2)), np.ones((n, 2)))
    for theta, cm in ((0.5, 0), (0.8, 1), (0.0, 0)):
        _, Zi, _ = oracle.bh_repulsion(z, s, L, theta, centre_mode=cm)
        Z = oracle.Z_of(st, oracle.Params(L=L, theta=theta, centre_mode=cm))
        assert Z == pytest.approx(Zi.sum(), rel=1e-12)
    _, Ze = oracle.exact_repulsion(z, s)
    assert oracle.Z_of(st, oracle.Params(L=L, exact=1)) == pytest.approx(Ze.sum(), rel=1e-12)
    _, Zb, _ = oracle.bh_repulsion(z, s, L, 0.5)
    assert abs(Zb.sum() - Ze.sum()) > 1e-9 * Ze.sum()     # the two differ here


def test_kl_ignores_explicit_zeros():
    # a stored zero of P (0 ln 0 = 0) adds nothing to Eq. cost_func
    n = 30
    rng = np.random.default_rng(28)
    A = (rng.random((n, n)) < 0.3) * rng.random((n, n))
    A = A + A.T
    np.fill_diagonal(A, 0)
    Pd = A / A.sum()
    P = _dense_csr(Pd)
    z, s = _random_state(n, 29)
    _, Zi = oracle.exact_repulsion(z, s)
    Z = Zi.sum()
    # the same P with every absent off-diagonal pair of row 0 stored as 0
    rp, col, val = [0], [], []
    for i in range(n):
        for j in range(n):
            if j != i and (Pd[i, j] > 0 or i == 0):
                col.append(j)
                val.append(Pd[i, j])
        rp.append(len(col))
    P0 = oracle.CSR(np.array(rp, np.int64), np.array(col, np.int32), np.array(val))
    assert P0.nnz > P.nnz
    # (equal up to the order in which the threads' partial sums are added)
    assert oracle.kl(P0, z, s, Z) == pytest.approx(oracle.kl(P, z, s, Z), rel=1e-13)


def _unique_pixel_state(n, L, seed):
    rng = np.random.default_rng(seed)
    F = 32 - L
    pix = rng.choice(4 ** L, size=n, replace=False)
    px, py = pix % (2 ** L), pix // (2 ** L)
    z = np.stack([(px << F) | rng.integers(0, 2 ** F, n),
                  (py << F) | rng.integers(0, 2 ** F, n)], 1).astype(np.uint32)
    s = np.array([3e-9, 2e-9])
    return z, s


def test_bh_theta0_one_point_per_pixel_is_exact():
    L = 9
    z, s = _unique_pixel_state(180, L, 14)
    Fb, Zb, acc = oracle.bh_repulsion(z, s, L, 0.0)
    Fe, Ze = oracle.exact_repulsion(z, s)
    np.testing.assert_allclose(Fb, Fe, rtol=1e-12, atol=1e-14 * np.abs(Fe).max())
    np.testing.assert_allclose(Zb, Ze, rtol=1e-12)
    assert np.all(acc == 179)   # every other point is its own leaf


def test_bh_theta0_equals_pixel_bruteforce():
    L = 4
    F = 32 - L
    rng = np.random.default_rng(15)
    n = 240
    centres = rng.integers(2, 14, (12, 2))
    pix = centres[rng.integers(0, 12, n)] + rng.integers(-2, 3, (n, 2))
    z = ((pix.astype(np.int64) << F) + rng.integers(0, 2 ** F, (n, 2))).astype(np.uint32)
    z[5] = z[6]               # an exact duplicate
    s = np.array([1.1e-9, 0.7e-9])
    Fb, Zb, _ = oracle.bh_repulsion(z, s, L, 0.0)
    # tree-free brute force: every other pixel's centre of mass with weight N,
    # the own pixel without i
    key = (z[:, 0] >> F).astype(np.int64) * 4096 + (z[:, 1] >> F)
    groups = {}
    for i, kk in enumerate(key):
        groups.setdefault(int(kk), []).append(i)
    Fr = np.zeros((n, 2))
    Zr = np.zeros(n)
    for i in range(n):
        for kk, members in groups.items():
            mem = [j for j in members if j != i]
            if not mem:
                continue
            N = len(mem)
            cx = sum(int(z[j, 0]) for j in mem) / N
            cy = sum(int(z[j, 1]) for j in mem) / N
            dx = s[0] * (int(z[i, 0]) - cx)
            dy = s[1] * (int(z[i, 1]) - cy)
            w = 1.0 / (1.0 + dx * dx + dy * dy)
            Zr[i] += N * w
            Fr[i] += N * w * w * np.array([dx, dy])
    np.testing.assert_allclose(Fb, Fr, rtol=1e-9, atol=1e-12 * np.abs(Fr).max())
    np.testing.assert_allclose(Zb, Zr, rtol=1e-12)


def test_bh_theta0_geometric_equals_pixel_midpoint_bruteforce():
    # Sec. 4.1's geometric-centre approximation at theta = 0: every leaf is
    # reached, and each stands for its points at the pixel's midpoint; the
    # own pixel counts its other points, still at the midpoint
    L = 5
    F = 32 - L
    rng = np.random.default_rng(25)
    n = 300
    pix = rng.integers(0, 2 ** L, (n, 2))
    pix[:40] = pix[40:80]       # shared pixels
    z = ((pix.astype(np.int64) << F) + rng.integers(0, 2 ** F, (n, 2))).astype(np.uint32)
    s = np.array([0.9e-9, 1.3e-9])
    Fb, Zb, _ = oracle.bh_repulsion(z, s, L, 0.0, centre_mode=1)
    groups = {}
    for i in range(n):
        groups.setdefault((int(pix[i, 0]), int(pix[i, 1])), []).append(i)
    Fr = np.zeros((n, 2))
    Zr = np.zeros(n)
    half = 2.0 ** (F - 1)
    for i in range(n):
        for (px, py), members in groups.items():
            N = sum(1 for j in members if j != i)
            if N == 0:
                continue
            dx = s[0] * (int(z[i, 0]) - (px * 2.0 ** F + half))
            dy = s[1] * (int(z[i, 1]) - (py * 2.0 ** F + half))
            w = 1.0 / (1.0 + dx * dx + dy * dy)
            Zr[i] += N * w
            Fr[i] += N * w * w * np.array([dx, dy])
    np.testing.assert_allclose(Fb, Fr, rtol=1e-9, atol=1e-12 * np.abs(Fr).max())
    np.testing.assert_allclose(Zb, Zr, rtol=1e-12)
    # and it differs from the centre-of-mass tree (the two modes are distinct)
    Fc, _, _ = oracle.bh_repulsion(z, s, L, 0.0)
    assert np.abs(Fc - Fb).max() > 1e-3 * np.abs(Fb).max()


@pytest.mark.parametrize("crit_mode", [0, 1])
def test_bh_acceptance_threshold_is_the_cell_diagonal(crit_mode):
    # Eq. bh_criteria on a hand-built tree (L = 3): point i alone in pixel
    # (0, 0), three points in the level-1 cell x, y in [4, 8), one per
    # level-2 child.  That cell is summarised by one interaction when
    # r_c / d (crit_mode 0; r_c / d^2, the printed form, in crit_mode 1) is
    # below theta, with r_c the diagonal of a level-1 cell and d the distance
    # to its centre of mass; otherwise it is opened and its three points come
    # back as three interactions.  Theta one part in 1e9 either side of the
    # threshold must land on either side.
    L = 3
    F = 32 - L
    s = np.array([1.3e-9, 0.8e-9])
    pix = [(0, 0), (4, 4), (6, 5), (5, 7)]
    sub = [(12345, 777), (2 ** 28, 3), (99, 2 ** 27), (5, 6)]
    z = np.array([[(px << F) + a, (py << F) + b] for (px, py), (a, b) in zip(pix, sub)],
                 dtype=np.uint32)
    Wc = 2.0 ** 31            # width of a level-1 cell in ulps
    rc = math.hypot(s[0] * Wc, s[1] * Wc)
    cx = sum(int(v) for v in z[1:, 0]) / 3
    cy = sum(int(v) for v in z[1:, 1]) / 3
    d = math.hypot(s[0] * (int(z[0, 0]) - cx), s[1] * (int(z[0, 1]) - cy))
    th_star = rc / d if crit_mode == 0 else rc / d ** 2
    _, _, acc_hi = oracle.bh_repulsion(z, s, L, th_star * (1 + 1e-9), rows=[0],
                                       crit_mode=crit_mode)
    _, _, acc_lo = oracle.bh_repulsion(z, s, L, th_star * (1 - 1e-9), rows=[0],
                                       crit_mode=crit_mode)
    assert acc_hi[0] == 1
    assert acc_lo[0] == 3


def test_bh_own_cells_are_always_opened():
    # with theta so large that every other cell is accepted at its first test,
    # point i interacts exactly with the non-empty siblings of each of its
    # ancestors (one level at a time) and with the others of its own pixel:
    # a tree-free count and sum over pixel coordinates
    L = 4
    F = 32 - L
    rng = np.random.default_rng(31)
    n = 200
    pix = rng.integers(0, 2 ** L, (n, 2))
    pix[:30] = pix[30:60]
    z = ((pix.astype(np.int64) << F) + rng.integers(0, 2 ** F, (n, 2))).astype(np.uint32)
    s = np.array([1.0e-9, 1.5e-9])
    Fb, Zb, acc = oracle.bh_repulsion(z, s, L, 1e6)
    zi64 = z.astype(np.int64)
    for i in range(n):
        cnt, fx, fy, zs = 0, 0.0, 0.0, 0.0
        for l in range(1, L + 1):
            cell = pix >> (L - l)
            mine = cell[i]
            sib = np.all((cell >> 1) == (mine >> 1), axis=1) & ~np.all(cell == mine, axis=1)
            groups = {}
            for j in np.nonzero(sib)[0]:
                groups.setdefault((int(cell[j, 0]), int(cell[j, 1])), []).append(j)
            if l == L:
                others = [j for j in np.nonzero(np.all(cell == mine, axis=1))[0] if j != i]
                if others:
                    groups["own"] = others
            for mem in groups.values():
                N = len(mem)
                dx = s[0] * (int(zi64[i, 0]) - zi64[mem, 0].sum() / N)
                dy = s[1] * (int(zi64[i, 1]) - zi64[mem, 1].sum() / N)
                w = 1.0 / (1.0 + dx * dx + dy * dy)
                cnt += 1
                zs += N * w
                fx += N * w * w * dx
                fy += N * w * w * dy
        assert acc[i] == cnt, i
        assert Zb[i] == pytest.approx(zs, rel=1e-12)
        assert Fb[i, 0] == pytest.approx(fx, rel=1e-9, abs=1e-12 * abs(Fb).max())
        assert Fb[i, 1] == pytest.approx(fy, rel=1e-9, abs=1e-12 * abs(Fb).max())


def test_bh_theta_half_close_to_exact():
    rng = np.random.default_rng(16)
    L = 9
    Y = np.concatenate([rng.standard_normal((400, 2)) * 2 + c for c in ([0, 0], [15, 3], [-6, 12])])
    z, s = oracle.init_fx(Y)
    Fe, Ze = oracle.exact_repulsion(z, s)
    errs = []
    for th in (0.8, 0.5, 0.25):
        Fb, Zb, acc = oracle.bh_repulsion(z, s, L, th)
        errs.append(np.linalg.norm(Fb - Fe) / np.linalg.norm(Fe))
        assert abs(Zb.sum() - Ze.sum()) / Ze.sum() < 0.02
    assert errs[0] > errs[1] > errs[2]
    assert errs[1] < 0.05
    # the geometric-centre variant (Sec. 4.1's printed approximation) is coarser
    Fg, _, _ = oracle.bh_repulsion(z, s, L, 0.5, centre_mode=1)
    assert np.linalg.norm(Fg - Fe) / np.linalg.norm(Fe) < 0.5


# ------------------------------------------------------------------ update / rescale
def test_rescale_big_integer_arithmetic():
    rng = np.random.default_rng(17)
    n = 500
    zhat = np.stack([rng.integers(-2 ** 34, 2 ** 35, n), rng.integers(-7, 2 ** 20, n)], 1)
    s = np.array([1e-9, 3e-8])
    z, s2 = oracle.rescale(zhat, s)
    for d in range(2):
        mn, mx = int(zhat[:, d].min()), int(zhat[:, d].max())
        gamma = mx - mn + 1
        ref = [((int(v) - mn) << 32) // gamma for v in zhat[:, d]]
        assert [int(v) for v in z[:, d]] == ref
        assert s2[d] == s[d] * (gamma / 2 ** 32)
    for L in (9, 11):  # Sec. 4.2: pixel coordinates span exactly 0 .. r-1
        F = 32 - L
        for d in range(2):
            assert (z[:, d] >> F).min() == 0 and (z[:, d] >> F).max() == 2 ** L - 1
    # the widest range a step can produce (steps are clamped to 2^58 ulps):
    # (zhat - min) 2^32 overflows 64 bits and must still be exact
    zw = np.array([[-(2 ** 58), 0], [2 ** 32 - 1 + 2 ** 58, 1], [12345, 2 ** 58],
                   [2 ** 57 + 3, 7]], np.int64)
    z, _ = oracle.rescale(zw, s)
    for d in range(2):
        mn, mx = int(zw[:, d].min()), int(zw[:, d].max())
        gamma = mx - mn + 1
        assert [int(v) for v in z[:, d]] == [((int(v) - mn) << 32) // gamma for v in zw[:, d]]


@pytest.mark.parametrize("mode", [dict(), dict(centre_mode=1), dict(crit_mode=1, theta=2.0),
                                  dict(exact=1)])
def test_run_step_is_the_composition_of_its_parts(mode):
    # one iteration of the run = tree, repulsion (the run's theta, criterion
    # and centre mode, or the exact sum), attraction, update with Z = sum Z_i
    # and the schedule's alpha and mu, then the rescale: each part pinned above
    n = 300
    rng = np.random.default_rng(33)
    A = (rng.random((n, n)) < 0.05) * rng.random((n, n))
    A = A + A.T
    np.fill_diagonal(A, 0)
    P = _dense_csr(A / A.sum())
    z, s = _random_state(n, 34)
    prm = oracle.Params(L=7, **mode)
    for t0 in (0, prm.exag_iters):
        st = oracle.State(z.copy(), s.copy(), rng.standard_normal((n, 2)) * 1e-3,
                          rng.uniform(0.5, 2.0, (n, 2)), t0)
        ref = st.copy()
        oracle.run(P, st, prm, 1)
        if prm.exact:
            Fr, Zi = oracle.exact_repulsion(ref.z, ref.s)
        else:
            Fr, Zi, _ = oracle.bh_repulsion(ref.z, ref.s, prm.L, prm.theta,
                                            crit_mode=prm.crit_mode, centre_mode=prm.centre_mode)
        Fa = oracle.attraction(P, ref.z, ref.s)
        alpha = prm.exag if t0 < prm.exag_iters else 1.0
        mu = prm.mom0 if t0 < prm.mom_switch else prm.mom1
        Z = float(np.cumsum(Zi)[-1])     # summed in point order, as the run does
        zhat, _ = oracle.update(ref.z, ref.s, Fa, Fr, Z, alpha, mu, prm.eta, ref.u,
                                ref.gains, min_gain=prm.min_gain)
        zr, sr = oracle.rescale(zhat, ref.s)
        assert np.array_equal(st.z, zr) and np.array_equal(st.s, sr)
        assert np.array_equal(st.u, ref.u) and np.array_equal(st.gains, ref.gains)
        assert st.t == t0 + 1


def test_update_rule_cases():
    # g = 4 (alpha Fattr - Frep / Z); gains compare sign(g) with sign(u), sign(0) = 0
    z = np.array([[1000, 1000]] * 4, np.uint32)
    s = np.array([0.5, 0.25])
    Fattr = np.array([[1.0, -1.0], [1.0, -1.0], [0.0, 0.0], [1.0, 1.0]])
    Frep = np.zeros((4, 2))
    u = np.array([[0.0, 0.0], [2.0, 2.0], [1.0, -1.0], [-3.0, 5.0]])
    gains = np.array([[1.0, 1.0], [1.0, 1.0], [0.011, 1.0], [1.0, 1.0]])
    zhat, g = oracle.update(z, s, Fattr, Frep, 1.0, 2.0, 0.5, 10.0, u, gains)
    np.testing.assert_array_equal(g, [[8, -8], [8, -8], [0, 0], [8, 8]])
    # u = 0: always different sign -> +0.2; same sign -> *0.8; g = 0 vs u != 0 -> +0.2
    np.testing.assert_allclose(gains, [[1.2, 1.2], [0.8, 1.2], [0.211, 1.2], [1.2, 0.8]])
    np.testing.assert_allclose(u[0], [-96.0, 96.0])
    assert zhat[0, 0] == 1000 + round(-96.0 / 0.5) and zhat[0, 1] == 1000 + round(96 / 0.25)
    # min gain clamp
    gains2 = np.array([[0.01, 0.01]])
    u2 = np.array([[1.0, 1.0]])
    oracle.update(z[:1], s, np.array([[1.0, 1.0]]), np.zeros((1, 2)), 1.0, 1.0, 0.5, 1.0,
                  u2, gains2, min_gain=0.01)
    np.testing.assert_allclose(gains2, [[0.01, 0.01]])


def test_update_rounds_the_step_half_to_even():
    # zhat = z + rint(u / s): nearest ulp, ties to even (2.5 -> 2, 3.5 -> 4,
    # -2.5 -> -2), not truncation (2.7 -> 3, -2.7 -> -3)
    want = np.array([2.5, 3.5, -2.5, 2.7, -2.7, 0.49])
    m = want.shape[0]
    z = np.full((m, 2), 1000, np.uint32)
    s = np.array([1.0, 1.0])
    # u = 0, gains 0.8 -> 1.0 (the signs differ), mu = 0, eta = 1: u' = -g = -4 Fattr
    Fattr = np.stack([-want / 4, -want / 4], 1)
    u = np.zeros((m, 2))
    gains = np.full((m, 2), 0.8)
    zhat, _ = oracle.update(z, s, Fattr, np.zeros((m, 2)), 1.0, 1.0, 0.0, 1.0, u, gains)
    np.testing.assert_allclose(u[:, 0], want, rtol=1e-15)
    assert list(zhat[:, 0] - 1000) == [2, 4, -2, 3, -3, 0]


def test_init_fx_is_the_floor_of_the_exact_map():
    # Eq. z1: z = floor((y - min) 2^32 / (max - min)); against exact rational
    # arithmetic on the same float64 inputs (the FP64 evaluation may differ
    # only where the exact value lies within a few 2^-20 of an integer)
    from fractions import Fraction
    rng = np.random.default_rng(30)
    Y = rng.standard_normal((3000, 2)) * 3.0 + 1.0
    z, _ = oracle.init_fx(Y)
    for d in range(2):
        mn, mx = Fraction(Y[:, d].min()), Fraction(Y[:, d].max())
        off = 0
        for i in range(Y.shape[0]):
            t = (Fraction(Y[i, d]) - mn) * 2 ** 32 / (mx - mn)
            exact = min(2 ** 32 - 1, t.numerator // t.denominator)
            if int(z[i, d]) != exact:
                frac = t - (t.numerator // t.denominator)
                assert min(frac, 1 - frac) < Fraction(1, 2 ** 18), (i, d)
                off += 1
        assert off <= 3


def test_fixed_point_run_equals_y_space_tsne():
    """Sec. 4.2: with the rescale compensated (Eq. q_wrt_z, Eq. beta_scaling), each
    PixelSNE step is a plain t-SNE step in y-space (scikit-learn's exact
    gradient) up to translation and the 2^-32 quantisation of the screen.
    Checked step by step along a 20-step trajectory; the free-running
    trajectories separate only at the chaotic rate of the dynamics."""
    tsne = pytest.importorskip("sklearn.manifold._t_sne")
    from scipy.spatial.distance import squareform
    n = 50
    rng = np.random.default_rng(18)
    X = np.concatenate([rng.standard_normal((25, 4)), rng.standard_normal((25, 4)) + 4])
    idx, d2 = oracle.knn(X.astype(np.float32), 15)
    p, _, _, _ = oracle.perplexity(d2, 5.0)
    P = oracle.symmetrize(idx, p)
    Pc = squareform(P.dense(), checks=False)
    Y0 = rng.standard_normal((n, 2)) * 1e-2
    params = oracle.Params(L=9, exact=1, exag=4.0, exag_iters=10, mom_switch=10,
                           eta=50.0)
    st = oracle.State.from_y0(Y0)
    for t in range(20):
        y, u, gains = st.y(), st.u.copy(), st.gains.copy()
        alpha = params.exag if t < params.exag_iters else 1.0
        mu = params.mom0 if t < params.mom_switch else params.mom1
        _, g = tsne._kl_divergence(y.ravel(), alpha * Pc, 1, n, 2)
        g = g.reshape(n, 2)
        gains = np.where(np.sign(g) != np.sign(u), gains + 0.2, gains * 0.8)
        gains = np.maximum(gains, params.min_gain)
        u = mu * u - params.eta * gains * g
        y = y + u
        s_old = st.s.copy()
        oracle.run(P, st, params, 1)
        np.testing.assert_allclose(st.u, u, rtol=1e-9, atol=1e-12 * np.abs(u).max())
        np.testing.assert_array_equal(st.gains, gains)
        a = st.y() - st.y().mean(0)
        b = y - y.mean(0)
        # half an old ulp from rint(u/s) plus one new ulp from the floor
        tol = 0.5 * s_old + st.s + 1e-12 * np.abs(b).max()
        assert np.all(np.abs(a - b).max(0) <= 2 * tol)


def test_run_lowers_kl_and_keeps_screen():
    import datagen
    X, _ = datagen.gauss10(0, n=600)
    P, _, _, bad = oracle.affinities(X, 30, 90)
    assert bad == 0
    st = oracle.State.from_y0(datagen.init_y0(0, 600))
    params = oracle.Params(L=9)
    kl0 = oracle.kl_of(P, st, params)
    oracle.run(P, st, params, 300)
    kl1 = oracle.kl_of(P, st, params)
    assert 0 < kl1 < kl0
    F = 32 - 9
    for d in range(2):
        assert (st.z[:, d] >> F).min() == 0 and (st.z[:, d] >> F).max() == 511


# ------------------------------------------------------------------ quality metric
def test_nbr_precision_identity_cases():
    rng = np.random.default_rng(19)
    n, k = 300, 10
    Y = rng.standard_normal((n, 2))
    z, s = oracle.init_fx(Y)
    idx, _ = oracle.knn((z.astype(np.float64) * s).astype(np.float32), k)
    # high-D neighbours computed on the same geometry: precision ~ 1 (ties and
    # the fp32 copy may swap a few boundary neighbours)
    assert oracle.nbr_precision(idx, k, z, s) > 0.97
    # unrelated geometry: precision ~ k / n
    z2, s2 = oracle.init_fx(rng.standard_normal((n, 2)))
    assert oracle.nbr_precision(idx, k, z2, s2) < 0.15


# ------------------------------------------------------------------ seeded start
def test_philox_known_answers():
    # the generator's published known-answer vectors
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        rows = [[int(w, 16) for w in line.split()] for line in f
                if line.strip() and not line.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        out = oracle.philox4x32_10([r[0:4]], (r[4], r[5]))[0]
        assert [int(v) for v in out] == r[6:10]


def test_philox_y0_is_a_gaussian_draw():
    sigma = 1e-4
    Y = oracle.philox_y0(7, 400_000, sigma).astype(np.float64)
    assert np.array_equal(Y, oracle.philox_y0(7, 400_000, sigma))
    # N(0, sigma^2 I): mean, scale, the one-sigma mass, no correlation
    assert np.abs(Y.mean(0)).max() < 5 * sigma / math.sqrt(400_000)
    assert np.abs(Y.std(0) / sigma - 1).max() < 0.005
    assert abs((np.abs(Y) < sigma).mean() - math.erf(1 / math.sqrt(2))) < 0.003
    assert abs(np.corrcoef(Y[:, 0], Y[:, 1])[0, 1]) < 0.005
    # Box-Muller: the angle is uniform and independent of the radius
    r = np.hypot(Y[:, 0], Y[:, 1])
    a = np.arctan2(Y[:, 1], Y[:, 0])
    assert abs(np.corrcoef(r, a)[0, 1]) < 0.005
    assert abs(np.corrcoef(r, np.abs(a))[0, 1]) < 0.005
    # both halves of the 64-bit seed matter; the draw is a prefix of a longer one
    assert not np.array_equal(oracle.philox_y0(1, 10), oracle.philox_y0(1 + 2 ** 32, 10))
    assert np.array_equal(oracle.philox_y0(3, 10), oracle.philox_y0(3, 1000)[:10])


# ------------------------------------------------------------------ MLP warm start
def _gelu_ref(z):
    return 0.5 * z * (1.0 + math.erf(z / math.sqrt(2.0)))


def test_gelu_against_erf_definition():
    for z in (-6.0, -1.3, -0.2, 0.0, 0.7, 2.5, 8.0):
        assert abs(oracle.gelu(z) - _gelu_ref(z)) < 1e-15
        h = 1e-6
        fd = (_gelu_ref(z + h) - _gelu_ref(z - h)) / (2 * h)
        assert abs(oracle.gelu_d(z) - fd) < 1e-8


def test_mlp_forward_closed_form():
    # identity weights, zero biases: y = g(g(x)) component-wise (d = H = 2)
    I = np.eye(2)
    net = oracle.MLP(I.copy(), np.zeros(2), I.copy(), np.zeros(2), I.copy(), np.array([0.5, -1.0]))
    X = np.array([[0.3, -1.7], [2.0, 0.0]], np.float32)
    _, Y, _ = oracle.mlp(net, X)
    for r in range(2):
        for o in range(2):
            ref = _gelu_ref(_gelu_ref(float(X[r, o]))) + net.b3[o]
            assert abs(Y[r, o] - ref) < 1e-14


def test_mlp_gradient_finite_differences():
    rng = np.random.default_rng(21)
    d, H, m = 5, 7, 9
    net = oracle.MLP(rng.standard_normal((H, d)) * 0.5, rng.standard_normal(H) * 0.1,
                     rng.standard_normal((H, H)) * 0.4, rng.standard_normal(H) * 0.1,
                     rng.standard_normal((2, H)) * 0.5, rng.standard_normal(2) * 0.1)
    X = rng.standard_normal((m, d)).astype(np.float32)
    T = rng.standard_normal((m, 2)).astype(np.float32)
    L, _, g = oracle.mlp(net, X, T, grad=True)
    v = net.flat()
    h = 1e-6
    for q in rng.choice(v.size, 40, replace=False):
        vp, vm = v.copy(), v.copy()
        vp[q] += h
        vm[q] -= h
        Lp, _, _ = oracle.mlp(oracle.MLP.from_flat(vp, d, H), X, T)
        Lm, _, _ = oracle.mlp(oracle.MLP.from_flat(vm, d, H), X, T)
        assert abs((Lp - Lm) / (2 * h) - g[q]) < 1e-7 * max(1.0, abs(g[q]))
    # the loss is the mean squared error of the outputs
    _, Y, _ = oracle.mlp(net, X)
    assert abs(L - ((Y - T) ** 2).sum() / m) < 1e-12


def test_nbr_precision_bruteforce_per_row():
    rng = np.random.default_rng(22)
    n, k, kh = 400, 10, 15
    z = rng.integers(0, 2 ** 20, (n, 2)).astype(np.uint32)
    z[5] = z[6]                 # duplicate positions: ties go to the lower index
    z[100] = z[6]
    s = np.array([2e-6, 3e-6])
    knn_hd = np.stack([rng.choice(n, kh, replace=False) for _ in range(n)]).astype(np.int32)
    prec, hits = oracle.nbr_precision(knn_hd, k, z, s, per_row=True)
    y = z.astype(np.float64) * s
    dd = ((y[:, None, :] - y[None, :, :]) ** 2).sum(-1)
    np.fill_diagonal(dd, np.inf)
    nn2 = np.argsort(dd, axis=1, kind="stable")[:, :k]
    ref = np.array([len(set(nn2[i]) & set(knn_hd[i, :k])) for i in range(n)])
    assert np.array_equal(hits, ref)
    assert abs(prec - ref.sum() / (k * n)) < 1e-15


def test_pca_against_svd():
    rng = np.random.default_rng(23)
    X = rng.standard_normal((500, 12)) @ rng.standard_normal((12, 12)) + 3.0
    Z, V, lam = oracle.pca(X, 5)
    Xc = X - X.mean(0)
    U, S, Vt = np.linalg.svd(Xc, full_matrices=False)       # a different routine
    np.testing.assert_allclose(lam, S[:5] ** 2 / (X.shape[0] - 1), rtol=1e-10)
    for c in range(5):
        assert abs(abs(V[:, c] @ Vt[c]) - 1.0) < 1e-8
    np.testing.assert_allclose(V.T @ V, np.eye(5), atol=1e-12)
    np.testing.assert_allclose(Z.var(0, ddof=1), lam, rtol=1e-10)


def test_stored_kl_target_matches_the_oracle():
    # the time-to-target measurement's stored target is the oracle's own value
    sys.path.insert(0, GOLDEN)
    import make_kl_target
    with open(os.path.join(GOLDEN, "kl_target_gauss10.json")) as f:
        stored = json.load(f)
    fresh = make_kl_target.compute()
    assert stored["kl"] == pytest.approx(fresh["kl"], rel=1e-9)
    assert {k: v for k, v in stored.items() if k != "kl"} == \
        {k: v for k, v in fresh.items() if k != "kl"}


def test_stored_large_kl_targets_describe_their_workloads():
    """The stored oracle KL of the larger workloads (hours of CPU to recompute
    at n = 1M, minutes at 70k and 200k) carry the workload the script names,
    a KL that falls along the schedule, and a P whose size fits k = 90."""
    sys.path.insert(0, GOLDEN)
    import make_kl_target
    for name, (gen, n, L, iters, dpca) in make_kl_target.WORKLOADS.items():
        path = os.path.join(GOLDEN, f"kl_target_{name}.json")
        if name == "gauss10" or not os.path.exists(path):
            continue
        with open(path) as f:
            g = json.load(f)
        assert (g["workload"], g["n"], g["log2_r"], g["iterations"], g["pca"]) == \
            (gen, n, L, iters, dpca)
        assert g["k"] == 90 and g["perplexity"] == 30.0 and g["theta"] == 0.5
        assert g["unconverged_rows"] == 0
        q = g["kl_quarters"]
        assert len(q) == 4 and q[-1] == g["kl"] and all(a > b > 0 for a, b in zip(q, q[1:]))
        assert 90 * n <= g["nnz"] <= 2 * 90 * n


SCREENS = [(10, 768, 1024), (9, 300, 512), (7, 128, 96), (11, 2048, 2048)]


@pytest.mark.parametrize("L,rx,ry", SCREENS)
def test_screen_rescale_big_integer_arithmetic(L, rx, ry):
    """Sec. 4.2 on an r_x x r_y screen (per-axis r_d, the padded 2^L root):
    z_d = floor((zhat_d - min) R_d / gamma_d), R_d = r_d 2^(32-L), exactly;
    s_d <- (s_d gamma_d) / R_d; pixels span exactly 0 .. r_d - 1."""
    rng = np.random.default_rng(L + rx)
    n = 400
    zhat = np.stack([rng.integers(-2 ** 40, 2 ** 41, n), rng.integers(-9, 2 ** 26, n)], 1)
    zhat[0] = (-(2 ** 58), 2 ** 58)            # the widest range a clamped step makes
    R = oracle.screen_R(L, rx, ry)
    assert list(R) == [rx * 2 ** (32 - L), ry * 2 ** (32 - L)]
    s = np.array([1e-9, 3e-8])
    z, s2 = oracle.rescale(zhat, s, R)
    F = 32 - L
    for d, r in enumerate((rx, ry)):
        Rd = r << F
        mn, mx = int(zhat[:, d].min()), int(zhat[:, d].max())
        gamma = mx - mn + 1
        assert [int(v) for v in z[:, d]] == [(int(v) - mn) * Rd // gamma for v in zhat[:, d]]
        assert s2[d] == (s[d] * float(gamma)) / float(Rd)
        assert (z[:, d] >> F).min() == 0 and (z[:, d] >> F).max() == r - 1
        assert int(z[:, d].max()) < Rd


@pytest.mark.parametrize("L,rx,ry", SCREENS[:3])
def test_screen_init_is_the_floor_of_the_exact_map(L, rx, ry):
    # Eq. z1 with R_d = r_d 2^(32-L): extremes at 0 and R_d - 1, pixels 0 .. r_d - 1
    from fractions import Fraction
    rng = np.random.default_rng(31)
    Y = rng.standard_normal((1500, 2)) * 2.0 - 0.5
    R = oracle.screen_R(L, rx, ry)
    z, s = oracle.init_fx(Y, R)
    F = 32 - L
    for d, r in enumerate((rx, ry)):
        Rd = r << F
        mn, mx = Fraction(Y[:, d].min()), Fraction(Y[:, d].max())
        assert s[d] == (Y[:, d].max() - Y[:, d].min()) / Rd
        assert int(z[:, d].min()) == 0 and int(z[:, d].max()) == Rd - 1
        assert (z[:, d] >> F).max() == r - 1
        off = 0
        for i in range(0, Y.shape[0], 3):
            t = (Fraction(Y[i, d]) - mn) * Rd / (mx - mn)
            exact = min(Rd - 1, t.numerator // t.denominator)
            if int(z[i, d]) != exact:
                frac = t - (t.numerator // t.denominator)
                assert min(frac, 1 - frac) < Fraction(1, 2 ** 18), (i, d)
                off += 1
        assert off <= 3


def test_square_screen_is_the_default_extent():
    rng = np.random.default_rng(32)
    Y = rng.standard_normal((300, 2))
    zhat = rng.integers(-2 ** 33, 2 ** 33, (300, 2))
    for L in (5, 11):
        R = oracle.screen_R(L)
        assert list(R) == [2.0 ** 32, 2.0 ** 32]
        for a, b in zip(oracle.init_fx(Y), oracle.init_fx(Y, R)):
            assert np.array_equal(a, b)
        for a, b in zip(oracle.rescale(zhat, [1e-3, 2e-3]), oracle.rescale(zhat, [1e-3, 2e-3], R)):
            assert np.array_equal(a, b)


def test_screen_run_step_is_the_composition_of_its_parts():
    # the run on a 100 x 128 screen of the padded 2^7 root: one step = the
    # pinned parts with the screen's per-axis extents in the rescale
    n = 300
    rng = np.random.default_rng(35)
    A = (rng.random((n, n)) < 0.05) * rng.random((n, n))
    A = A + A.T
    np.fill_diagonal(A, 0)
    P = _dense_csr(A / A.sum())
    prm = oracle.Params(L=7, rx=100, ry=128)
    Y = rng.standard_normal((n, 2))
    st = oracle.State.from_y0(Y, prm.R())
    ref = st.copy()
    oracle.run(P, st, prm, 1)
    Fr, Zi, _ = oracle.bh_repulsion(ref.z, ref.s, prm.L, prm.theta)
    Fa = oracle.attraction(P, ref.z, ref.s)
    zhat, _ = oracle.update(ref.z, ref.s, Fa, Fr, float(np.cumsum(Zi)[-1]), prm.exag, prm.mom0,
                            prm.eta, ref.u, ref.gains, min_gain=prm.min_gain)
    zr, sr = oracle.rescale(zhat, ref.s, prm.R())
    assert np.array_equal(st.z, zr) and np.array_equal(st.s, sr)
    # and a longer run keeps every point on the 100 x 128 pixels, spanning them
    oracle.run(P, st, prm, 40)
    px, py = st.z[:, 0] >> 25, st.z[:, 1] >> 25
    assert px.min() == 0 and px.max() == 99 and py.min() == 0 and py.max() == 127


# ---------------------------------------------------------------- 3-D embedding
def _kl3_y(Pd, Y):
    """Eq. cost_func from its definition on a dense P and 3-D y (numpy)."""
    D2 = ((Y[:, None, :] - Y[None, :, :]) ** 2).sum(-1)
    W = 1.0 / (1.0 + D2)
    np.fill_diagonal(W, 0.0)
    Q = W / W.sum()
    m = Pd > 0
    return float((Pd[m] * np.log(Pd[m] / Q[m])).sum())


def test_morton3_is_the_octree_child_numbering():
    rng = np.random.default_rng(40)
    L = 7
    for _ in range(200):
        px, py, pz = (int(v) for v in rng.integers(0, 2 ** L, 3))
        m = 0
        for b in range(L - 1, -1, -1):       # root to leaf: child = 4 z + 2 y + x
            m = 8 * m + 4 * ((pz >> b) & 1) + 2 * ((py >> b) & 1) + ((px >> b) & 1)
        assert oracle.morton3(px, py, pz) == m
    assert [oracle.level_offset3(l) for l in range(4)] == [0, 1, 9, 73]


def test_pyramid3_counts_and_sums():
    rng = np.random.default_rng(41)
    L = 4
    z = rng.integers(0, 2 ** 32, (500, 3), dtype=np.uint64).astype(np.uint32)
    z[:50] = z[50]                            # one crowded voxel
    cnt, sx, sy, sz = oracle.pyramid3(z, L)
    vox = z >> (32 - L)
    for l in range(L + 1):
        key = [oracle.morton3(*(v >> (L - l))) for v in vox]
        off = oracle.level_offset3(l)
        ref = np.bincount(key, minlength=8 ** l)
        assert np.array_equal(cnt[off:off + 8 ** l], ref)
        for ax, S in enumerate((sx, sy, sz)):
            acc = {}
            for k, v in zip(key, z[:, ax]):
                acc[k] = acc.get(k, 0) + int(v)
            for k, v in acc.items():
                assert int(S[off + k]) == v


def test_bh3_theta0_and_the_exact_sum():
    rng = np.random.default_rng(42)
    z, s = oracle.init_fx3(rng.standard_normal((300, 3)))
    Fe, Ze = oracle.exact_repulsion3(z, s)
    # one point per voxel (L = 8, checked): theta = 0 is the exact sum
    assert len({tuple(v) for v in (z >> 24)}) == len(z)
    F, Zi, _ = oracle.bh_repulsion3(z, s, 8, 0.0)
    assert np.abs(F - Fe).max() <= 1e-12 * np.abs(Fe).max()
    assert np.abs(Zi - Ze).max() <= 1e-12 * Ze.max()
    # Newton's third law on the exact sum
    assert np.abs(Fe.sum(0)).max() <= 1e-10 * np.abs(Fe).sum()
    # the error falls with theta
    errs = [np.linalg.norm(oracle.bh_repulsion3(z, s, 8, th)[0] - Fe) / np.linalg.norm(Fe)
            for th in (0.25, 0.5, 1.0)]
    assert errs[0] < errs[1] < errs[2] < 0.05


def test_bh3_theta0_is_the_voxel_bruteforce():
    # with several points per voxel, theta = 0 sums every other voxel's centre
    # of mass (weight N) and the own voxel without the point itself
    rng = np.random.default_rng(43)
    L = 4
    z, s = oracle.init_fx3(rng.standard_normal((400, 3)))
    F, Zi, _ = oracle.bh_repulsion3(z, s, L, 0.0)
    vox = [tuple(v) for v in (z >> (32 - L))]
    groups = {}
    for i, v in enumerate(vox):
        groups.setdefault(v, []).append(i)
    zz = z.astype(np.float64)
    for i in range(0, 400, 37):
        f = np.zeros(3)
        zs = 0.0
        for v, mem in groups.items():
            mem = [j for j in mem if j != i]
            if not mem:
                continue
            c = zz[mem].mean(0)
            d = s * (zz[i] - c)
            w = 1.0 / (1.0 + d @ d)
            zs += len(mem) * w
            f += len(mem) * w * w * d
        np.testing.assert_allclose(F[i], f, rtol=1e-9, atol=1e-14)
        assert Zi[i] == pytest.approx(zs, rel=1e-10)


def test_gradient3_is_the_derivative_of_the_kl():
    # 4 (Fattr - Frep / Z) (exact repulsion) against central differences of
    # the KL written from its definition in y-space
    rng = np.random.default_rng(44)
    n = 40
    A = rng.random((n, n)) * (rng.random((n, n)) < 0.3)
    A = A + A.T
    np.fill_diagonal(A, 0)
    Pd = A / A.sum()
    P = _dense_csr(Pd)
    z, s = oracle.init_fx3(rng.standard_normal((n, 3)))
    Y = z.astype(np.float64) * s
    Fa = oracle.attraction3(P, z, s)
    Fr, Zi = oracle.exact_repulsion3(z, s)
    g = 4.0 * (Fa - Fr / Zi.sum())
    h = 1e-5
    for i in range(0, n, 7):
        for d in range(3):
            Yp, Ym = Y.copy(), Y.copy()
            Yp[i, d] += h
            Ym[i, d] -= h
            fd = (_kl3_y(Pd, Yp) - _kl3_y(Pd, Ym)) / (2 * h)
            assert g[i, d] == pytest.approx(fd, rel=1e-5, abs=1e-9)
    assert oracle.kl3(P, z, s, Zi.sum()) == pytest.approx(_kl3_y(Pd, Y), rel=1e-10)


def test_update3_and_rescale3_per_coordinate():
    # the optimiser acts per coordinate: a 3-D step equals the 2-D one on the
    # same coordinates; the rescale is exact per axis (big integers)
    rng = np.random.default_rng(45)
    n = 300
    z = rng.integers(0, 2 ** 32, (n, 3), dtype=np.uint64).astype(np.uint32)
    s = np.array([1e-6, 2e-6, 3e-7])
    Fa, Fr = rng.standard_normal((n, 3)), rng.standard_normal((n, 3))
    u, g = rng.standard_normal((n, 3)) * 1e-3, rng.uniform(0.5, 2, (n, 3))
    u3, g3 = u.copy(), g.copy()
    zh3, gr3 = oracle.update3(z, s, Fa, Fr, 3.5, 12.0, 0.5, 200.0, u3, g3)
    for cols in ((0, 1), (2, 2)):
        c = list(cols)
        u2, g2 = np.ascontiguousarray(u[:, c]), np.ascontiguousarray(g[:, c])
        zh2, gr2 = oracle.update(np.ascontiguousarray(z[:, c]), s[c], Fa[:, c], Fr[:, c], 3.5,
                                 12.0, 0.5, 200.0, u2, g2)
        assert np.array_equal(zh3[:, c], zh2) and np.array_equal(u3[:, c], u2)
        assert np.array_equal(g3[:, c], g2) and np.array_equal(gr3[:, c], gr2)
    zhat = np.stack([rng.integers(-2 ** 40, 2 ** 40, n), rng.integers(5, 2 ** 20, n),
                     rng.integers(-(2 ** 58), 2 ** 58, n)], 1)
    zr, sr = oracle.rescale3(zhat, s)
    for d in range(3):
        mn, mx = int(zhat[:, d].min()), int(zhat[:, d].max())
        gamma = mx - mn + 1
        assert [int(v) for v in zr[:, d]] == [((int(v) - mn) << 32) // gamma for v in zhat[:, d]]
        assert sr[d] == (s[d] * float(gamma)) / 2.0 ** 32


def test_run3_step_is_the_composition_of_its_parts():
    n = 250
    rng = np.random.default_rng(46)
    A = (rng.random((n, n)) < 0.05) * rng.random((n, n))
    A = A + A.T
    np.fill_diagonal(A, 0)
    P = _dense_csr(A / A.sum())
    prm = oracle.Params(L=5)
    st = oracle.State3.from_y0(rng.standard_normal((n, 3)))
    ref = st.copy()
    oracle.run3(P, st, prm, 1)
    Fr, Zi, _ = oracle.bh_repulsion3(ref.z, ref.s, prm.L, prm.theta)
    Fa = oracle.attraction3(P, ref.z, ref.s)
    zhat, _ = oracle.update3(ref.z, ref.s, Fa, Fr, float(np.cumsum(Zi)[-1]), prm.exag, prm.mom0,
                             prm.eta, ref.u, ref.gains, min_gain=prm.min_gain)
    zr, sr = oracle.rescale3(zhat, ref.s)
    assert np.array_equal(st.z, zr) and np.array_equal(st.s, sr)
    assert np.array_equal(st.u, ref.u) and np.array_equal(st.gains, ref.gains)
    # without exaggeration a run lowers the KL from its start, and keeps every
    # voxel axis spanned
    plain = oracle.Params(L=5, exag=1.0)
    kl0 = oracle.kl_of3(P, st, plain)
    oracle.run3(P, st, plain, 60)
    assert oracle.kl_of3(P, st, plain) < kl0
    vox = st.z >> (32 - prm.L)
    assert vox.min() == 0 and vox.max() == 2 ** prm.L - 1


def test_bh3_acceptance_threshold_is_the_cell_diagonal():
    # Eq. bh_criteria in 3-D on a hand-built tree: A near the origin, B1 and B2
    # in the far octant (level 1) but in different level-2 cells.  Just above
    # theta* = r_c / d (r_c = W sqrt(s0^2 + s1^2 + s2^2), W = 2^31, d from A to
    # the octant's centre of mass) the octant is accepted as one body; just
    # below it is opened and A meets B1 and B2 one by one.
    L = 5
    z = np.array([[1 << 27, 3 << 26, 5 << 25],
                  [(3 << 30) + 12345, (3 << 30) + 777, (3 << 30) + 99],
                  [(2 << 30) + 4321, (2 << 30) + 55, (2 << 30) + 8]], np.uint32)
    s = np.array([1.3e-9, 0.7e-9, 2.1e-9])
    zz = z.astype(np.float64)
    com = zz[1:].mean(0)
    dA = s * (zz[0] - com)
    rc = 2.0 ** 31 * np.sqrt((s ** 2).sum())
    th = rc / np.sqrt(dA @ dA)
    w = 1.0 / (1.0 + dA @ dA)
    one_body = 2.0 * w * w * dA
    each = np.zeros(3)
    for j in (1, 2):
        d = s * (zz[0] - zz[j])
        wj = 1.0 / (1.0 + d @ d)
        each += wj * wj * d
    assert np.abs(one_body - each).max() > 1e-6 * np.abs(each).max()
    F_hi, _, _ = oracle.bh_repulsion3(z, s, L, th * (1 + 1e-9), rows=[0])
    F_lo, _, _ = oracle.bh_repulsion3(z, s, L, th * (1 - 1e-9), rows=[0])
    np.testing.assert_allclose(F_hi[0], one_body, rtol=1e-10)
    np.testing.assert_allclose(F_lo[0], each, rtol=1e-10)
