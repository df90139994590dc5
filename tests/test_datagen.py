"""The seeded input generators follow their stated recipes (shapes, class
and component structure, value ranges) and are reproducible by seed."""
import numpy as np
import pytest

import datagen


def test_zipf_sizes_sum_and_ratios():
    for n, k, s in [(1_000_000, 100, 1.1), (990_000, 256, 1.2), (7, 5, 1.0), (0, 3, 1.1)]:
        sz = datagen.zipf_sizes(n, k, s)
        assert sz.sum() == n and sz.shape == (k,) and np.all(sz >= 0)
        raw = n / np.arange(1, k + 1) ** s / (1.0 / np.arange(1, k + 1) ** s).sum()
        assert np.all(np.abs(sz - raw) < 1.0)      # largest-remainder rounding
    sz = datagen.zipf_sizes(1_000_000, 100, 1.1)
    assert np.all(np.diff(sz) <= 0)
    assert abs(sz[0] / sz[9] - 10 ** 1.1) < 0.01 * 10 ** 1.1


def test_reproducible_by_seed_and_distinct_across_seeds():
    for name, n in [("gauss10", 500), ("protos784", 300), ("gmm128", 2000), ("gmm64out", 3000)]:
        X0, l0 = datagen.make(name, 0, n)
        X0b, l0b = datagen.make(name, 0, n)
        X1, _ = datagen.make(name, 1, n)
        assert X0.dtype == np.float32 and X0.flags.c_contiguous
        assert np.array_equal(X0, X0b) and np.array_equal(l0, l0b)
        assert not np.array_equal(X0, X1)
    Y = datagen.init_y0(3, 1000)
    assert Y.shape == (1000, 2) and Y.dtype == np.float32
    assert np.array_equal(Y, datagen.init_y0(3, 1000))
    assert 0.9e-4 < Y.std() < 1.1e-4 and abs(Y.mean()) < 1e-5


def test_gauss10_recipe():
    X, lab = datagen.gauss10(0)
    assert X.shape == (2000, 50)
    assert np.array_equal(np.bincount(lab), np.full(10, 200))
    # unit variance around each class mean; means spread with std 5
    within = np.concatenate([X[lab == c] - X[lab == c].mean(0) for c in range(10)])
    assert abs(within.std() - 1.0) < 0.02
    means = np.stack([X[lab == c].mean(0) for c in range(10)])
    assert 4.0 < means.std() < 6.0


def test_protos784_recipe():
    X, lab = datagen.protos784(0, n=2000)
    assert X.shape == (2000, 784) and X.min() >= 0.0 and X.max() <= 1.0
    assert np.array_equal(np.bincount(lab), np.full(10, 200))
    # entries off the prototype are pure U(0, 0.2) noise: about 80 % of them
    # lie below 0.2
    assert 0.7 < (X < 0.2).mean() < 0.85


def test_gmm_recipes():
    X, lab = datagen.gmm128(0, n=20000)
    assert X.shape == (20000, 128)
    cnt = np.bincount(lab, minlength=100)
    assert np.array_equal(cnt, datagen.zipf_sizes(20000, 100, 1.1))
    # the anisotropic covariance: eigenvalues of the largest component in
    # [0.1, 2] (up to sampling error)
    big = X[lab == 0].astype(np.float64)
    ev = np.linalg.eigvalsh(np.cov(big.T))
    assert 0.05 < ev.min() and ev.max() < 2.6
    # the same world: another seed draws the same components
    X2, lab2 = datagen.gmm128(1, n=20000)
    m1 = X[lab == 0].mean(0)
    m2 = X2[lab2 == 0].mean(0)
    assert np.linalg.norm(m1 - m2) < 1.0       # sampling error ~0.25; other means ~80 away
    Xo, labo = datagen.gmm64out(0, n=50000)
    assert Xo.shape == (50000, 64)
    out = labo == -1
    assert out.sum() == 500
    assert np.abs(Xo[out]).max() <= 50.0 and np.abs(Xo[out]).max() > 45.0
    assert np.array_equal(np.bincount(labo[~out], minlength=256),
                          datagen.zipf_sizes(49500, 256, 1.2))


@pytest.mark.parametrize("name", list(datagen.WORKLOADS))
def test_workload_table(name):
    gen, n0, L, T = datagen.WORKLOADS[name]
    assert callable(gen) and n0 >= 2000 and 9 <= L <= 12 and T in (500, 1000)


def test_lowdim_recipe():
    # rank d_latent up to the noise: the centred data's singular values drop
    # by orders of magnitude after the d_latent-th
    X = datagen.lowdim(seed=1, n=3000, d_latent=4, D=32)
    assert X.shape == (3000, 32) and X.dtype == np.float32
    assert np.array_equal(X, datagen.lowdim(seed=1, n=3000, d_latent=4, D=32))
    assert not np.array_equal(X, datagen.lowdim(seed=2, n=3000, d_latent=4, D=32))
    sv = np.linalg.svd(X - X.mean(0), compute_uv=False)
    assert sv[3] > 100 * sv[4]
