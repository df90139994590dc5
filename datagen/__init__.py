"""Seeded synthetic inputs for the PixelSNE workloads.

This module is shared by the CUDA path's tests/bench and by the CPU oracle's
tests. It holds no arithmetic of the method itself (no distances, affinities,
trees, forces or updates): only random draws that produce the input matrix X,
class labels, and the random initial embedding Y0 that t-SNE starts from.

The paper's datasets (MNIST, Yelp, NewsAgg, ...; Sec. 5.1.1) are not
available; each workload below stands in for one of them with the same
shape (n, D) and a cluster structure of the kind the paper's data has.

Workloads (names used across tests and the bench):

* ``gauss10``   n=2,000, D=50: 10 isotropic unit-variance Gaussians, means
  drawn from N(0, 25 I), 200 points each.
* ``protos784`` n=70,000, D=784 in [0,1]: 10 classes of 7,000; each class has
  a non-negative prototype with ~20% non-zero entries; an item keeps each
  prototype entry with probability 0.9, adds U(0, 0.2) noise, and is clipped
  to [0,1].  (MNIST-shaped stand-in, reduced to 50 dims by PCA before kNN.)
* ``gmm128``    n=1,000,000, D=128: 100-component Gaussian mixture with
  Zipf(s=1.1) component sizes, means from N(0, 25 I) and per-component
  covariance Q^T diag(U[0.1, 2]) Q with Q a Haar-random rotation.
  (Yelp-sized stand-in.)
* ``gmm64out``  n=10,000,000, D=64: 256 components, Zipf(s=1.2) sizes, plus 1%
  uniform outliers in [-50, 50]^64.

Every generator takes ``n`` so that the same recipe can be drawn at a smaller
size for tests; the structure parameters (component count, Zipf exponent,
dimension) stay those of the named workload.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "WORKLOADS",
    "zipf_sizes",
    "gauss10",
    "protos784",
    "gmm",
    "gmm128",
    "gmm64out",
    "init_y0",
    "make",
]


def zipf_sizes(n: int, k: int, s: float) -> np.ndarray:
    """Component sizes proportional to 1/c^s, c = 1..k, summing exactly to n
    (largest-remainder rounding, ties to the lower component index)."""
    w = 1.0 / np.arange(1, k + 1, dtype=np.float64) ** s
    raw = w / w.sum() * n
    base = np.floor(raw).astype(np.int64)
    rem = int(n - base.sum())
    order = np.argsort(-(raw - base), kind="stable")
    base[order[:rem]] += 1
    return base


def _shuffle(rng, X, labels):
    perm = rng.permutation(X.shape[0])
    return np.ascontiguousarray(X[perm]), np.ascontiguousarray(labels[perm])


def gauss10(seed: int = 0, n: int = 2000, D: int = 50, n_classes: int = 10):
    """10 isotropic unit-variance Gaussians, means ~ N(0, 25 I)."""
    rng = np.random.default_rng([seed, 1])
    means = rng.standard_normal((n_classes, D)) * 5.0
    sizes = np.full(n_classes, n // n_classes, dtype=np.int64)
    sizes[: n - sizes.sum()] += 1
    labels = np.repeat(np.arange(n_classes, dtype=np.int32), sizes)
    X = means[labels] + rng.standard_normal((n, D))
    return _shuffle(rng, X.astype(np.float32), labels)


def protos784(seed: int = 0, n: int = 70000, D: int = 784, n_classes: int = 10):
    """Sparse non-negative prototypes with Bernoulli dropout and uniform noise."""
    rng = np.random.default_rng([seed, 2])
    protos = np.where(rng.random((n_classes, D)) < 0.2,
                      rng.uniform(0.3, 1.0, (n_classes, D)), 0.0)
    sizes = np.full(n_classes, n // n_classes, dtype=np.int64)
    sizes[: n - sizes.sum()] += 1
    labels = np.repeat(np.arange(n_classes, dtype=np.int32), sizes)
    X = np.empty((n, D), dtype=np.float32)
    step = 8192
    for a in range(0, n, step):
        b = min(n, a + step)
        keep = rng.random((b - a, D)) < 0.9
        x = protos[labels[a:b]] * keep + rng.uniform(0.0, 0.2, (b - a, D))
        X[a:b] = np.clip(x, 0.0, 1.0)
    return _shuffle(rng, X, labels)


def _haar_rotation(rng, D):
    A = rng.standard_normal((D, D))
    Q, R = np.linalg.qr(A)
    return Q * np.sign(np.diag(R))[None, :]


def gmm(seed: int, n: int, D: int, n_comp: int, zipf_s: float,
        outlier_frac: float = 0.0, outlier_box: float = 50.0,
        world_seed: int = 12345):
    """Anisotropic Gaussian mixture with Zipf component sizes.

    The mixture parameters (means, rotations, eigenvalues) come from
    ``world_seed``; only the sampling of points depends on ``seed``, so
    independent draws of the same world share their clusters."""
    wrng = np.random.default_rng([world_seed, n_comp, D])
    means = wrng.standard_normal((n_comp, D)) * 5.0
    n_out = int(round(n * outlier_frac))
    sizes = zipf_sizes(n - n_out, n_comp, zipf_s)
    rng = np.random.default_rng([seed, 3, n_comp, D])
    X = np.empty((n, D), dtype=np.float32)
    labels = np.empty(n, dtype=np.int32)
    o = 0
    for c in range(n_comp):
        Q = _haar_rotation(wrng, D)
        ev = wrng.uniform(0.1, 2.0, D)
        m = int(sizes[c])
        if m == 0:
            continue
        step = 65536
        for a in range(0, m, step):
            b = min(m, a + step)
            g = rng.standard_normal((b - a, D)) * np.sqrt(ev)[None, :]
            X[o + a:o + b] = (g @ Q.T + means[c]).astype(np.float32)
        labels[o:o + m] = c
        o += m
    if n_out:
        X[o:] = rng.uniform(-outlier_box, outlier_box, (n_out, D)).astype(np.float32)
        labels[o:] = -1
    return _shuffle(rng, X, labels)


def gmm128(seed: int = 0, n: int = 1_000_000):
    return gmm(seed, n, 128, 100, 1.1)


def gmm64out(seed: int = 0, n: int = 10_000_000):
    return gmm(seed, n, 64, 256, 1.2, outlier_frac=0.01)


def lowdim(seed: int = 0, n: int = 1_000_000, d_latent: int = 4, D: int = 64,
           noise: float = 1e-3):
    """Points near a d_latent-dimensional linear manifold of R^D: latent
    coordinates uniform in the unit cube, mapped by a fixed Gaussian D x
    d_latent matrix, plus isotropic noise of std ``noise``.  The stand-in for
    data of low intrinsic dimension, where a neighbour's neighbours are likely
    neighbours (the premise of Sec. 4.3's neighbour exploring); the Gaussian
    mixtures above are full-rank and have none of that structure."""
    wrng = np.random.default_rng([12345, d_latent, D])
    A = wrng.standard_normal((d_latent, D))
    rng = np.random.default_rng([seed, 5, d_latent, D])
    Z = rng.random((n, d_latent))
    return (Z @ A + noise * rng.standard_normal((n, D))).astype(np.float32)


def init_y0(seed: int, n: int, sigma: float = 1e-4, dim: int = 2) -> np.ndarray:
    """The random initial embedding Y0 ~ N(0, sigma^2 I), shape (n, dim),
    float32 (the random draw that t-SNE starts from; passed to both sides)."""
    rng = np.random.default_rng([seed, 7])
    return (rng.standard_normal((n, dim)) * sigma).astype(np.float32)


# name -> (generator, default n, screen log2 resolution L, iterations T)
WORKLOADS = {
    "gauss10": (gauss10, 2000, 9, 500),
    "protos784": (protos784, 70000, 10, 1000),
    "gmm128": (gmm128, 1_000_000, 11, 1000),
    "gmm64out": (gmm64out, 10_000_000, 12, 1000),
}


def make(name: str, seed: int = 0, n: int | None = None):
    gen, n0, _, _ = WORKLOADS[name]
    return gen(seed=seed, n=n0 if n is None else n)
