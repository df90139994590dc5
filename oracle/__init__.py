"""PixelSNE CPU oracle: ctypes front-end of ``pxsne_oracle.c``.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package.  It is a
plain FP64 statement of the method (arXiv 1611.02568), independent of the CUDA
library: it neither imports nor links anything from it.

Parity pins: every function here is pinned in ``tests/test_oracle_pins.py``
against closed forms, invariants, finite differences or brute force; see the
header of that file for the mapping.  ``tests/test_oracle_mutants.py`` checks
that planted mistakes in this package fail those pins.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pxsne_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

R = 2.0 ** 32


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP) into oracle/_build/liboracle.so."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-Wall", "-Wextra",
           "-fno-fast-math", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


def _P(a, t):
    return a.ctypes.data_as(C.POINTER(t))


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        i64, i32, u32, dbl = C.c_int64, C.c_int32, C.c_uint32, C.c_double
        pf = C.POINTER(C.c_float)
        pd = C.POINTER(dbl)
        pi64 = C.POINTER(i64)
        pi32 = C.POINTER(i32)
        pu32 = C.POINTER(u32)
        pu64 = C.POINTER(C.c_uint64)
        L.orc_knn.argtypes = [pf, i64, i32, i32, pi64, i64, pi32, pd]
        L.orc_knn.restype = C.c_int
        L.orc_perplexity.argtypes = [pd, i64, i32, dbl, dbl, i32, pd, pd, pd]
        L.orc_perplexity.restype = i64
        L.orc_symmetrize.argtypes = [pi32, pd, i64, i32, pi64, pi32, pd]
        L.orc_symmetrize.restype = i64
        L.orc_init_fx.argtypes = [pd, i64, pu32, pd]
        L.orc_init_fx_screen.argtypes = [pd, i64, pd, pu32, pd]
        L.orc_morton.argtypes = [u32, u32]
        L.orc_morton.restype = u32
        L.orc_level_offset.argtypes = [i32]
        L.orc_level_offset.restype = i64
        L.orc_leaf_keys.argtypes = [pu32, i64, i32, pu32, pu32, pu32]
        L.orc_pyramid.argtypes = [pu32, i64, i32, pu32, pu64, pu64]
        L.orc_bh_repulsion.argtypes = [pu32, pd, i64, i32, dbl, i32, i32, pu32, pu64,
                                       pu64, pi64, i64, pd, pd, pi64]
        L.orc_exact_repulsion.argtypes = [pu32, pd, i64, pi64, i64, pd, pd]
        L.orc_attraction.argtypes = [pi64, pi32, pd, pu32, pd, pi64, i64, pd]
        L.orc_update.argtypes = [i64, pu32, pd, pd, pd, dbl, dbl, dbl, dbl, dbl, pd, pd,
                                 pd, pi64]
        L.orc_rescale.argtypes = [i64, pi64, pu32, pd]
        L.orc_rescale_screen.argtypes = [i64, pi64, pd, pu32, pd]
        L.orc_init_fx_dim.argtypes = [pd, i64, i32, pd, pu32, pd]
        L.orc_update_dim.argtypes = [i64, i32, pu32, pd, pd, pd, dbl, dbl, dbl, dbl, dbl, pd, pd,
                                     pd, pi64]
        L.orc_rescale_dim.argtypes = [i64, i32, pi64, pd, pu32, pd]
        L.orc_morton3.argtypes = [u32, u32, u32]
        L.orc_morton3.restype = u32
        L.orc_level_offset3.argtypes = [i32]
        L.orc_level_offset3.restype = i64
        L.orc_pyramid3.argtypes = [pu32, i64, i32, pu32, pu64, pu64, pu64]
        L.orc_bh_repulsion3.argtypes = [pu32, pd, i64, i32, dbl, pu32, pu64, pu64, pu64, pi64,
                                        i64, pd, pd, pi64]
        L.orc_exact_repulsion3.argtypes = [pu32, pd, i64, pi64, i64, pd, pd]
        L.orc_attraction3.argtypes = [pi64, pi32, pd, pu32, pd, pi64, i64, pd]
        L.orc_kl3.argtypes = [pi64, pi32, pd, i64, pu32, pd, dbl]
        L.orc_kl3.restype = dbl
        L.orc_run3.argtypes = [C.c_void_p, pi64, pi32, pd, i64, pu32, pd, pd, pd, i32, i32]
        L.orc_run3.restype = C.c_int
        L.orc_Z3.argtypes = [C.c_void_p, i64, pu32, pd]
        L.orc_Z3.restype = dbl
        L.orc_kl.argtypes = [pi64, pi32, pd, i64, pu32, pd, dbl]
        L.orc_kl.restype = dbl
        L.orc_run.argtypes = [C.c_void_p, pi64, pi32, pd, i64, pu32, pd, pd, pd, i32, i32,
                              pd]
        L.orc_run.restype = C.c_int
        L.orc_Z.argtypes = [C.c_void_p, i64, pu32, pd]
        L.orc_Z.restype = dbl
        L.orc_nbr_precision.argtypes = [pi32, i32, i32, i64, pu32, pd, pi64, i64, pi32]
        L.orc_nbr_precision.restype = dbl
        L.orc_mlp.argtypes = [C.c_int32, C.c_int32, pd, pd, pd, pd, pd, pd, pf, pf, i64, pd, pd]
        L.orc_mlp.restype = dbl
        L.orc_gelu.argtypes = [dbl]
        L.orc_gelu.restype = dbl
        L.orc_gelu_d.argtypes = [dbl]
        L.orc_gelu_d.restype = dbl
        L.orc_num_threads.restype = C.c_int
        L.orc_set_num_threads.argtypes = [C.c_int]
        _lib = L
    return _lib


def num_threads() -> int:
    return lib().orc_num_threads()


def set_num_threads(t: int) -> None:
    lib().orc_set_num_threads(int(t))


def _rows(rows, n):
    if rows is None:
        return None, n
    r = np.ascontiguousarray(rows, dtype=np.int64)
    return r, r.shape[0]


def _ptr_or_null(a, t):
    return None if a is None else _P(a, t)


# ---------------------------------------------------------------- affinities
def knn(X, k, rows=None):
    """Exact kNN (FP64 from FP32 X), self excluded, ties to the lower index."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    n, D = X.shape
    r, m = _rows(rows, n)
    idx = np.empty((m, k), dtype=np.int32)
    d2 = np.empty((m, k), dtype=np.float64)
    rc = lib().orc_knn(_P(X, C.c_float), n, D, k, _ptr_or_null(r, C.c_int64), m,
                       _P(idx, C.c_int32), _P(d2, C.c_double))
    if rc != 0:
        raise ValueError(f"orc_knn failed ({rc})")
    return idx, d2


def perplexity(d2, u, tol=1e-5, max_iter=200):
    """Per-row bisection on beta; returns (pcond, beta, H, n_unconverged)."""
    d2 = np.ascontiguousarray(d2, dtype=np.float64)
    n, k = d2.shape
    p = np.empty_like(d2)
    beta = np.empty(n)
    H = np.empty(n)
    bad = lib().orc_perplexity(_P(d2, C.c_double), n, k, float(u), float(tol),
                               int(max_iter), _P(p, C.c_double), _P(beta, C.c_double),
                               _P(H, C.c_double))
    return p, beta, H, int(bad)


@dataclass
class CSR:
    row_ptr: np.ndarray  # int64 [n+1]
    col: np.ndarray      # int32 [nnz]
    val: np.ndarray      # float64 [nnz]

    @property
    def n(self):
        return self.row_ptr.shape[0] - 1

    @property
    def nnz(self):
        return self.col.shape[0]

    def dense(self):
        n = self.n
        M = np.zeros((n, n))
        rows = np.repeat(np.arange(n), np.diff(self.row_ptr))
        M[rows, self.col] = self.val
        return M


def symmetrize(idx, pcond):
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    pcond = np.ascontiguousarray(pcond, dtype=np.float64)
    n, k = idx.shape
    rp = np.empty(n + 1, dtype=np.int64)
    nnz = lib().orc_symmetrize(_P(idx, C.c_int32), _P(pcond, C.c_double), n, k,
                               _P(rp, C.c_int64), None, None)
    if nnz < 0:
        raise MemoryError("orc_symmetrize")
    col = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=np.float64)
    lib().orc_symmetrize(_P(idx, C.c_int32), _P(pcond, C.c_double), n, k,
                         _P(rp, C.c_int64), _P(col, C.c_int32), _P(val, C.c_double))
    return CSR(rp, col, val)


def affinities(X, perplexity_u, k):
    idx, d2 = knn(X, k)
    p, _, _, bad = perplexity(d2, perplexity_u)
    return symmetrize(idx, p), idx, d2, bad


# ---------------------------------------------------------------- tree / forces
def screen_R(L, rx=0, ry=0):
    """Per-axis extent R_d = r_d 2^(32 - L) in ulps of an r_x x r_y screen
    (0: 2^L pixels) whose quadtree root is the padded 2^L x 2^L square."""
    return np.array([float(r) * 2.0 ** (32 - L) if r else 2.0 ** 32 for r in (rx, ry)])


def init_fx(Y0, R=None):
    """Eq. z1/z2 onto [0, R_d) ulps per axis (R: screen_R; None: 2^32)."""
    Y0 = np.ascontiguousarray(Y0, dtype=np.float64)
    n = Y0.shape[0]
    z = np.empty((n, 2), dtype=np.uint32)
    s = np.empty(2)
    if R is None:
        lib().orc_init_fx(_P(Y0, C.c_double), n, _P(z, C.c_uint32), _P(s, C.c_double))
    else:
        R = np.ascontiguousarray(R, dtype=np.float64)
        lib().orc_init_fx_screen(_P(Y0, C.c_double), n, _P(R, C.c_double), _P(z, C.c_uint32),
                                 _P(s, C.c_double))
    return z, s


def morton(px, py):
    return int(lib().orc_morton(int(px), int(py)))


def level_offset(l):
    return int(lib().orc_level_offset(int(l)))


def leaf_keys(z, L):
    z = np.ascontiguousarray(z, dtype=np.uint32)
    n = z.shape[0]
    px = np.empty(n, dtype=np.uint32)
    py = np.empty(n, dtype=np.uint32)
    m = np.empty(n, dtype=np.uint32)
    lib().orc_leaf_keys(_P(z, C.c_uint32), n, L, _P(px, C.c_uint32), _P(py, C.c_uint32),
                        _P(m, C.c_uint32))
    return px, py, m


def pyramid(z, L):
    """Flattened pyramid: (cnt u32, sx u64, sy u64), level l at offset (4^l-1)/3."""
    z = np.ascontiguousarray(z, dtype=np.uint32)
    n = z.shape[0]
    cells = level_offset(L + 1)
    cnt = np.empty(cells, dtype=np.uint32)
    sx = np.empty(cells, dtype=np.uint64)
    sy = np.empty(cells, dtype=np.uint64)
    lib().orc_pyramid(_P(z, C.c_uint32), n, L, _P(cnt, C.c_uint32), _P(sx, C.c_uint64),
                      _P(sy, C.c_uint64))
    return cnt, sx, sy


def bh_repulsion(z, s, L, theta, rows=None, crit_mode=0, centre_mode=0, tree=None):
    """(Frep [m,2], Zi [m], n_accepted [m]) for the listed rows (all if None)."""
    z = np.ascontiguousarray(z, dtype=np.uint32)
    s = np.ascontiguousarray(s, dtype=np.float64)
    n = z.shape[0]
    cnt, sx, sy = pyramid(z, L) if tree is None else tree
    r, m = _rows(rows, n)
    F = np.empty((m, 2))
    Zi = np.empty(m)
    acc = np.empty(m, dtype=np.int64)
    lib().orc_bh_repulsion(_P(z, C.c_uint32), _P(s, C.c_double), n, L, float(theta),
                           crit_mode, centre_mode, _P(cnt, C.c_uint32), _P(sx, C.c_uint64),
                           _P(sy, C.c_uint64), _ptr_or_null(r, C.c_int64), m,
                           _P(F, C.c_double), _P(Zi, C.c_double), _P(acc, C.c_int64))
    return F, Zi, acc


def exact_repulsion(z, s, rows=None):
    z = np.ascontiguousarray(z, dtype=np.uint32)
    s = np.ascontiguousarray(s, dtype=np.float64)
    n = z.shape[0]
    r, m = _rows(rows, n)
    F = np.empty((m, 2))
    Zi = np.empty(m)
    lib().orc_exact_repulsion(_P(z, C.c_uint32), _P(s, C.c_double), n,
                              _ptr_or_null(r, C.c_int64), m, _P(F, C.c_double),
                              _P(Zi, C.c_double))
    return F, Zi


def attraction(P: CSR, z, s, rows=None):
    z = np.ascontiguousarray(z, dtype=np.uint32)
    s = np.ascontiguousarray(s, dtype=np.float64)
    r, m = _rows(rows, P.n)
    F = np.empty((m, 2))
    lib().orc_attraction(_P(P.row_ptr, C.c_int64), _P(P.col, C.c_int32),
                         _P(P.val, C.c_double), _P(z, C.c_uint32), _P(s, C.c_double),
                         _ptr_or_null(r, C.c_int64), m, _P(F, C.c_double))
    return F


def update(z, s, Fattr, Frep, Z, alpha, mu, eta, u, gains, min_gain=0.01):
    """One optimiser step; u and gains are updated in place. Returns (zhat, grad)."""
    z = np.ascontiguousarray(z, dtype=np.uint32)
    s = np.ascontiguousarray(s, dtype=np.float64)
    Fattr = np.ascontiguousarray(Fattr, dtype=np.float64)
    Frep = np.ascontiguousarray(Frep, dtype=np.float64)
    assert u.dtype == np.float64 and u.flags.c_contiguous
    assert gains.dtype == np.float64 and gains.flags.c_contiguous
    n = z.shape[0]
    zhat = np.empty((n, 2), dtype=np.int64)
    g = np.empty((n, 2))
    lib().orc_update(n, _P(z, C.c_uint32), _P(s, C.c_double), _P(Fattr, C.c_double),
                     _P(Frep, C.c_double), float(Z), float(alpha), float(mu), float(eta),
                     float(min_gain), _P(u, C.c_double), _P(gains, C.c_double),
                     _P(g, C.c_double), _P(zhat, C.c_int64))
    return zhat, g


def rescale(zhat, s, R=None):
    """Returns (z u32 [n,2], s_new); R: per-axis screen extent (None: 2^32)."""
    zhat = np.ascontiguousarray(zhat, dtype=np.int64)
    s2 = np.array(s, dtype=np.float64)
    n = zhat.shape[0]
    z = np.empty((n, 2), dtype=np.uint32)
    if R is None:
        lib().orc_rescale(n, _P(zhat, C.c_int64), _P(z, C.c_uint32), _P(s2, C.c_double))
    else:
        R = np.ascontiguousarray(R, dtype=np.float64)
        lib().orc_rescale_screen(n, _P(zhat, C.c_int64), _P(R, C.c_double), _P(z, C.c_uint32),
                                 _P(s2, C.c_double))
    return z, s2


def kl(P: CSR, z, s, Z):
    z = np.ascontiguousarray(z, dtype=np.uint32)
    s = np.ascontiguousarray(s, dtype=np.float64)
    return float(lib().orc_kl(_P(P.row_ptr, C.c_int64), _P(P.col, C.c_int32),
                              _P(P.val, C.c_double), P.n, _P(z, C.c_uint32),
                              _P(s, C.c_double), float(Z)))


class _Params(C.Structure):
    _fields_ = [("L", C.c_int32), ("theta", C.c_double), ("eta", C.c_double),
                ("exag", C.c_double), ("exag_iters", C.c_int32), ("mom0", C.c_double),
                ("mom1", C.c_double), ("mom_switch", C.c_int32),
                ("min_gain", C.c_double), ("crit_mode", C.c_int32),
                ("centre_mode", C.c_int32), ("exact", C.c_int32), ("rx", C.c_int32),
                ("ry", C.c_int32)]


@dataclass
class Params:
    """Optimiser schedule and tree parameters of one run."""
    L: int = 9
    theta: float = 0.5
    eta: float = 200.0
    exag: float = 12.0
    exag_iters: int = 250
    mom0: float = 0.5
    mom1: float = 0.8
    mom_switch: int = 250
    min_gain: float = 0.01
    crit_mode: int = 0
    centre_mode: int = 0
    exact: int = 0
    rx: int = 0        # screen pixels per axis (0: 2^L)
    ry: int = 0

    def c(self):
        return _Params(self.L, self.theta, self.eta, self.exag, self.exag_iters, self.mom0,
                       self.mom1, self.mom_switch, self.min_gain, self.crit_mode,
                       self.centre_mode, self.exact, self.rx, self.ry)

    def R(self):
        return screen_R(self.L, self.rx, self.ry)


@dataclass
class State:
    z: np.ndarray       # uint32 [n,2]
    s: np.ndarray       # float64 [2]
    u: np.ndarray       # float64 [n,2]
    gains: np.ndarray   # float64 [n,2]
    t: int = 0

    @classmethod
    def from_y0(cls, Y0, R=None):
        z, s = init_fx(Y0, R)
        n = z.shape[0]
        return cls(z, s, np.zeros((n, 2)), np.ones((n, 2)), 0)

    def copy(self):
        return State(self.z.copy(), self.s.copy(), self.u.copy(), self.gains.copy(), self.t)

    def y(self):
        return self.z.astype(np.float64) * self.s[None, :]


def run(P: CSR, state: State, params: Params, iters: int, Z_trace=False):
    """Advance ``state`` in place by ``iters`` iterations."""
    n = P.n
    pc = params.c()
    zt = np.empty(max(iters, 1)) if Z_trace else None
    rc = lib().orc_run(C.byref(pc), _P(P.row_ptr, C.c_int64), _P(P.col, C.c_int32),
                       _P(P.val, C.c_double), n, _P(state.z, C.c_uint32),
                       _P(state.s, C.c_double), _P(state.u, C.c_double),
                       _P(state.gains, C.c_double), state.t, iters,
                       None if zt is None else _P(zt, C.c_double))
    if rc != 0:
        raise MemoryError("orc_run")
    state.t += iters
    return zt[:iters] if Z_trace else None


def Z_of(state: State, params: Params):
    pc = params.c()
    return float(lib().orc_Z(C.byref(pc), state.z.shape[0], _P(state.z, C.c_uint32),
                             _P(state.s, C.c_double)))


def kl_of(P: CSR, state: State, params: Params):
    return kl(P, state.z, state.s, Z_of(state, params))


def nbr_precision(knn_hd, k, z, s, rows=None, per_row=False):
    """Eq. nei_prec over the listed rows; with per_row also the hit counts."""
    knn_hd = np.ascontiguousarray(knn_hd, dtype=np.int32)
    z = np.ascontiguousarray(z, dtype=np.uint32)
    s = np.ascontiguousarray(s, dtype=np.float64)
    n = z.shape[0]
    r, m = _rows(rows, n)
    assert knn_hd.shape[0] == m and knn_hd.shape[1] >= k
    hits = np.empty(m, dtype=np.int32)
    v = float(lib().orc_nbr_precision(_P(knn_hd, C.c_int32), knn_hd.shape[1], k, n,
                                      _P(z, C.c_uint32), _P(s, C.c_double),
                                      _ptr_or_null(r, C.c_int64), m, _P(hits, C.c_int32)))
    return (v, hits) if per_row else v


# ---------------------------------------------------------------- seeded start
# The random initial embedding drawn when the caller gives none (t-SNE starts
# from a random layout, Sec. 3.2; Sec. 4.2 draws it from an isotropic
# Gaussian, here of a chosen scale sigma).  The draw is not part of the
# method's arithmetic, so both sides implement the same
# published counter-based generator: Philox4x32-10 (Salmon, Moraes, Dror and
# Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC 2011), followed by
# the Box-Muller transform (Box and Muller, 1958).
_PHILOX_M = (0xD2511F53, 0xCD9E8D57)   # round multipliers
_PHILOX_W = (0x9E3779B9, 0xBB67AE85)   # key schedule (Weyl) increments


def philox4x32_10(ctr, key):
    """Philox4x32 with 10 rounds: ctr uint32 [m, 4], key (k0, k1) -> uint32
    [m, 4].  Each round multiplies words 0 and 2 by the round multipliers
    into 64-bit products; the new words are (hi(w2 M1) ^ w1 ^ k0, lo(w2 M1),
    hi(w0 M0) ^ w3 ^ k1, lo(w0 M0)); the key advances by the Weyl increments
    between rounds."""
    c = np.array(ctr, dtype=np.uint64).reshape(-1, 4)
    k0, k1 = np.uint64(key[0]), np.uint64(key[1])
    mask = np.uint64(0xFFFFFFFF)
    for r in range(10):
        if r:
            k0 = (k0 + np.uint64(_PHILOX_W[0])) & mask
            k1 = (k1 + np.uint64(_PHILOX_W[1])) & mask
        p0 = c[:, 0] * np.uint64(_PHILOX_M[0])
        p1 = c[:, 2] * np.uint64(_PHILOX_M[1])
        c = np.stack([((p1 >> np.uint64(32)) ^ c[:, 1] ^ k0) & mask, p1 & mask,
                      ((p0 >> np.uint64(32)) ^ c[:, 3] ^ k1) & mask, p0 & mask], 1)
    return c.astype(np.uint32)


def philox_y0(seed, n, sigma=1e-4):
    """Y0 [n, 2] float32 ~ N(0, sigma^2 I): point i takes counter (i, 0, 0, 0)
    and key (low, high 32 bits of seed); its first two output words give the
    uniforms u = (w + 1/2) 2^-32, and Box-Muller gives
    (sigma r cos a, sigma r sin a) with r = sqrt(-2 ln u1), a = 2 pi u2, in
    FP64, rounded to float32 (sigma is taken as a float32 value)."""
    ctr = np.zeros((n, 4), np.uint64)
    ctr[:, 0] = np.arange(n, dtype=np.uint64)
    seed = int(seed)
    w = philox4x32_10(ctr, (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)).astype(np.float64)
    u1 = (w[:, 0] + 0.5) * 2.0 ** -32
    u2 = (w[:, 1] + 0.5) * 2.0 ** -32
    rad = np.sqrt(-2.0 * np.log(u1))
    ang = 6.283185307179586 * u2
    sg = float(np.float32(sigma))
    return np.stack([sg * rad * np.cos(ang), sg * rad * np.sin(ang)], 1).astype(np.float32)


# ---------------------------------------------------------------- MLP warm start
@dataclass
class MLP:
    """Weights of d -> H -> H -> 2 (row-major, FP64)."""
    W1: np.ndarray
    b1: np.ndarray
    W2: np.ndarray
    b2: np.ndarray
    W3: np.ndarray
    b3: np.ndarray

    @property
    def d(self):
        return self.W1.shape[1]

    @property
    def H(self):
        return self.W1.shape[0]

    def flat(self):
        return np.concatenate([a.ravel() for a in (self.W1, self.b1, self.W2, self.b2,
                                                    self.W3, self.b3)])

    @classmethod
    def from_flat(cls, v, d, H):
        sizes = [H * d, H, H * H, H, 2 * H, 2]
        parts = np.split(np.asarray(v, dtype=np.float64), np.cumsum(sizes)[:-1])
        return cls(parts[0].reshape(H, d), parts[1], parts[2].reshape(H, H), parts[3],
                   parts[4].reshape(2, H), parts[5])


def gelu(z):
    return float(lib().orc_gelu(float(z)))


def gelu_d(z):
    return float(lib().orc_gelu_d(float(z)))


def mlp(net: MLP, X, T=None, grad=False):
    """(loss, Y [m,2], flat gradient or None) of the MLP on rows X with targets T."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    m = X.shape[0]
    w = [np.ascontiguousarray(a, dtype=np.float64) for a in (net.W1, net.b1, net.W2, net.b2,
                                                            net.W3, net.b3)]
    Tc = None if T is None else np.ascontiguousarray(T, dtype=np.float32)
    Y = np.empty((m, 2))
    g = np.empty(net.flat().size) if grad else None
    L = lib().orc_mlp(net.d, net.H, *[_P(a, C.c_double) for a in w], _P(X, C.c_float),
                      None if Tc is None else _P(Tc, C.c_float), m, _P(Y, C.c_double),
                      None if g is None else _P(g, C.c_double))
    return float(L), Y, g


# ---------------------------------------------------------------- PCA (Sec. 5.1.1)
def pca(X, dout):
    """(projection, components [D, dout], eigenvalues) from the FP64 sample
    covariance and numpy's symmetric eigensolver; each component's largest
    entry is positive."""
    Xd = np.asarray(X, dtype=np.float64)
    mu = Xd.mean(0)
    Xc = Xd - mu
    Cv = Xc.T @ Xc / (Xd.shape[0] - 1)
    lam, V = np.linalg.eigh(Cv)
    order = np.argsort(-lam, kind="stable")[:dout]
    lam, V = lam[order], V[:, order]
    sg = np.sign(V[np.argmax(np.abs(V), axis=0), np.arange(dout)])
    V = V * sg
    return Xc @ V, V, lam


# ---------------------------------------------------------------- 3-D embedding
# Sec. 1's footnote: the method on a voxel grid of 2^L per axis, the octree of
# eight children per cell (Morton bits x, y, z from the least significant).
def init_fx3(Y0):
    """Eq. z1/z2 per axis of a 3-D start (n x 3) onto [0, 2^32) ulps."""
    Y0 = np.ascontiguousarray(Y0, dtype=np.float64)
    n = Y0.shape[0]
    z = np.empty((n, 3), dtype=np.uint32)
    s = np.empty(3)
    R = np.full(3, 2.0 ** 32)
    lib().orc_init_fx_dim(_P(Y0, C.c_double), n, 3, _P(R, C.c_double), _P(z, C.c_uint32),
                          _P(s, C.c_double))
    return z, s


def morton3(px, py, pz):
    return int(lib().orc_morton3(int(px), int(py), int(pz)))


def level_offset3(l):
    return int(lib().orc_level_offset3(int(l)))


def pyramid3(z, L):
    z = np.ascontiguousarray(z, dtype=np.uint32)
    cells = level_offset3(L + 1)
    cnt = np.empty(cells, np.uint32)
    sx, sy, sz = (np.empty(cells, np.uint64) for _ in range(3))
    lib().orc_pyramid3(_P(z, C.c_uint32), z.shape[0], L, _P(cnt, C.c_uint32),
                       _P(sx, C.c_uint64), _P(sy, C.c_uint64), _P(sz, C.c_uint64))
    return cnt, sx, sy, sz


def bh_repulsion3(z, s, L, theta, rows=None, tree=None):
    z = np.ascontiguousarray(z, dtype=np.uint32)
    s = np.ascontiguousarray(s, dtype=np.float64)
    n = z.shape[0]
    cnt, sx, sy, sz = tree if tree is not None else pyramid3(z, L)
    r, m = _rows(rows, n)
    F = np.empty((m, 3))
    Zi = np.empty(m)
    acc = np.empty(m, np.int64)
    lib().orc_bh_repulsion3(_P(z, C.c_uint32), _P(s, C.c_double), n, L, float(theta),
                            _P(cnt, C.c_uint32), _P(sx, C.c_uint64), _P(sy, C.c_uint64),
                            _P(sz, C.c_uint64), _ptr_or_null(r, C.c_int64), m, _P(F, C.c_double),
                            _P(Zi, C.c_double), _P(acc, C.c_int64))
    return F, Zi, acc


def exact_repulsion3(z, s, rows=None):
    z = np.ascontiguousarray(z, dtype=np.uint32)
    s = np.ascontiguousarray(s, dtype=np.float64)
    n = z.shape[0]
    r, m = _rows(rows, n)
    F = np.empty((m, 3))
    Zi = np.empty(m)
    lib().orc_exact_repulsion3(_P(z, C.c_uint32), _P(s, C.c_double), n,
                               _ptr_or_null(r, C.c_int64), m, _P(F, C.c_double),
                               _P(Zi, C.c_double))
    return F, Zi


def attraction3(P: CSR, z, s, rows=None):
    z = np.ascontiguousarray(z, dtype=np.uint32)
    s = np.ascontiguousarray(s, dtype=np.float64)
    r, m = _rows(rows, P.n)
    F = np.empty((m, 3))
    lib().orc_attraction3(_P(P.row_ptr, C.c_int64), _P(P.col, C.c_int32), _P(P.val, C.c_double),
                          _P(z, C.c_uint32), _P(s, C.c_double), _ptr_or_null(r, C.c_int64), m,
                          _P(F, C.c_double))
    return F


def update3(z, s, Fattr, Frep, Z, alpha, mu, eta, u, gains, min_gain=0.01):
    """One optimiser step of a 3-D state; u and gains updated in place."""
    z = np.ascontiguousarray(z, dtype=np.uint32)
    s = np.ascontiguousarray(s, dtype=np.float64)
    Fattr = np.ascontiguousarray(Fattr, dtype=np.float64)
    Frep = np.ascontiguousarray(Frep, dtype=np.float64)
    assert u.dtype == np.float64 and u.flags.c_contiguous
    assert gains.dtype == np.float64 and gains.flags.c_contiguous
    n = z.shape[0]
    zhat = np.empty((n, 3), dtype=np.int64)
    g = np.empty((n, 3))
    lib().orc_update_dim(n, 3, _P(z, C.c_uint32), _P(s, C.c_double), _P(Fattr, C.c_double),
                         _P(Frep, C.c_double), float(Z), float(alpha), float(mu), float(eta),
                         float(min_gain), _P(u, C.c_double), _P(gains, C.c_double),
                         _P(g, C.c_double), _P(zhat, C.c_int64))
    return zhat, g


def rescale3(zhat, s):
    zhat = np.ascontiguousarray(zhat, dtype=np.int64)
    s2 = np.array(s, dtype=np.float64)
    n = zhat.shape[0]
    z = np.empty((n, 3), dtype=np.uint32)
    R = np.full(3, 2.0 ** 32)
    lib().orc_rescale_dim(n, 3, _P(zhat, C.c_int64), _P(R, C.c_double), _P(z, C.c_uint32),
                          _P(s2, C.c_double))
    return z, s2


def kl3(P: CSR, z, s, Z):
    z = np.ascontiguousarray(z, dtype=np.uint32)
    s = np.ascontiguousarray(s, dtype=np.float64)
    return float(lib().orc_kl3(_P(P.row_ptr, C.c_int64), _P(P.col, C.c_int32),
                               _P(P.val, C.c_double), P.n, _P(z, C.c_uint32),
                               _P(s, C.c_double), float(Z)))


@dataclass
class State3:
    z: np.ndarray       # uint32 [n,3]
    s: np.ndarray       # float64 [3]
    u: np.ndarray       # float64 [n,3]
    gains: np.ndarray   # float64 [n,3]
    t: int = 0

    @classmethod
    def from_y0(cls, Y0):
        z, s = init_fx3(Y0)
        n = z.shape[0]
        return cls(z, s, np.zeros((n, 3)), np.ones((n, 3)), 0)

    def copy(self):
        return State3(self.z.copy(), self.s.copy(), self.u.copy(), self.gains.copy(), self.t)


def run3(P: CSR, state: State3, params: Params, iters: int):
    """Advance a 3-D state in place by ``iters`` iterations (L <= 10)."""
    pc = params.c()
    rc = lib().orc_run3(C.byref(pc), _P(P.row_ptr, C.c_int64), _P(P.col, C.c_int32),
                        _P(P.val, C.c_double), P.n, _P(state.z, C.c_uint32),
                        _P(state.s, C.c_double), _P(state.u, C.c_double),
                        _P(state.gains, C.c_double), state.t, iters)
    if rc != 0:
        raise MemoryError("orc_run3")
    state.t += iters


def Z_of3(state: State3, params: Params):
    pc = params.c()
    return float(lib().orc_Z3(C.byref(pc), state.z.shape[0], _P(state.z, C.c_uint32),
                              _P(state.s, C.c_double)))


def kl_of3(P: CSR, state: State3, params: Params):
    return kl3(P, state.z, state.s, Z_of3(state, params))
