"""GB300-native PixelSNE (arXiv 1611.02568): Python binding of ``libpxsne.so``.

Argument marshalling only: every step of the method runs in the CUDA kernels
behind the C ABI of ``include/pxsne.h``.  There is no CPU fallback; importing
works without a GPU, but every call needs the compiled library and a CUDA
device.

Names follow the C ABI::

    ctx = Context(Params(log2_r=11))
    ctx.affinities(X)            # pxsne_affinities
    ctx.init(Y0)                 # pxsne_init (Y0=None draws from the seed)
    ctx.step(1000)               # pxsne_step
    ctx.kl()                     # pxsne_kl
    Y, pix = ctx.get_Y()         # pxsne_get_Y
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, fields

import numpy as np

from . import build as _build

LIB_PATH = _build.LIB
_lib = None

PXSNE_OK = 0
ERRORS = {-1: "E_ARG", -2: "E_OOM", -3: "E_CUDA", -4: "E_STATE", -5: "E_DEVICE",
          -6: "E_UNSUPPORTED"}
DEVERR = {1: "NONFINITE", 2: "STACK", 4: "BISECT", 8: "RANGE", 16: "TIMEOUT"}


class PxsneError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"pxsne {ERRORS.get(code, code)}: {msg}")
        self.code = code


class _CParams(C.Structure):
    _fields_ = [("log2_r", C.c_int32), ("theta", C.c_float), ("eta", C.c_float),
                ("exaggeration", C.c_float), ("exag_iters", C.c_int32),
                ("momentum0", C.c_float), ("momentum1", C.c_float),
                ("momentum_switch", C.c_int32), ("min_gain", C.c_float), ("k", C.c_int32),
                ("perplexity", C.c_float), ("init_sigma", C.c_float),
                ("centre_mode", C.c_int32), ("screen_x", C.c_int32), ("screen_y", C.c_int32),
                ("knn_probe", C.c_int32), ("dim", C.c_int32), ("knn_explore", C.c_int32)]


@dataclass
class Params:
    """Mirror of ``pxsne_params`` (defaults of ``pxsne_default_params``)."""
    log2_r: int = 11
    theta: float = 0.5
    eta: float = 200.0
    exaggeration: float = 12.0
    exag_iters: int = 250
    momentum0: float = 0.5
    momentum1: float = 0.8
    momentum_switch: int = 250
    min_gain: float = 0.01
    k: int = 90
    perplexity: float = 30.0
    init_sigma: float = 1e-4
    centre_mode: int = 0
    screen_x: int = 0      # pixels of the screen's width (0: 2^log2_r)
    screen_y: int = 0      # pixels of its height (0: 2^log2_r)
    knn_probe: int = 0     # 0: exact neighbour search; W: approximate, W tiles per tile
    dim: int = 2           # embedding dimension: 2, or 3 (voxel grid and octree)
    knn_explore: int = 0   # rounds of neighbour exploring after an approximate search

    def c(self):
        return _CParams(*[getattr(self, f.name) for f in fields(self)])


def load(path: str | None = None):
    """Load the compiled library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is missing: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = C.CDLL(p)
    vp, i32, i64, u64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64
    L.pxsne_default_params.argtypes = [C.POINTER(_CParams)]
    L.pxsne_create.argtypes = [C.POINTER(vp), C.POINTER(_CParams), vp]
    L.pxsne_destroy.argtypes = [vp]
    L.pxsne_destroy.restype = None
    L.pxsne_last_error.argtypes = [vp]
    L.pxsne_last_error.restype = C.c_char_p
    L.pxsne_affinities.argtypes = [vp, vp, i64, i32, C.c_float, C.c_int]
    L.pxsne_init.argtypes = [vp, vp, C.c_int, u64]
    L.pxsne_step.argtypes = [vp, i32]
    L.pxsne_kl.argtypes = [vp, C.POINTER(C.c_double)]
    L.pxsne_get_Y.argtypes = [vp, vp, vp, C.c_int]
    L.pxsne_sync.argtypes = [vp, C.POINTER(C.c_uint32)]
    L.pxsne_get_sizes.argtypes = [vp, C.POINTER(i64), C.POINTER(i64)]
    L.pxsne_get_P.argtypes = [vp, vp, vp, vp]
    L.pxsne_set_P.argtypes = [vp, i64, vp, vp, vp]
    L.pxsne_get_knn.argtypes = [vp, vp, vp, vp]
    L.pxsne_set_state.argtypes = [vp, vp, vp, vp, vp, i32]
    L.pxsne_get_state.argtypes = [vp, vp, vp, vp, vp, vp]
    L.pxsne_get_tree.argtypes = [vp, i32, vp, vp, vp, vp]
    L.pxsne_get_forces.argtypes = [vp, vp, vp, vp, vp]
    L.pxsne_step_profiled.argtypes = [vp, i32, C.POINTER(C.c_double), i32,
                                      C.POINTER(C.c_double)]
    L.pxsne_kernel_group_name.argtypes = [i32]
    L.pxsne_kernel_group_name.restype = C.c_char_p
    L.pxsne_get_counters.argtypes = [vp, C.POINTER(u64), C.POINTER(u64), C.POINTER(u64),
                                     C.POINTER(u64)]
    L.pxsne_get_knn_counters.argtypes = [vp, C.POINTER(u64), C.POINTER(u64), C.POINTER(i32)]
    L.pxsne_get_knn_time.argtypes = [vp, C.POINTER(C.c_double)]
    L.pxsne_get_knn_pruning.argtypes = [vp, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]
    L.pxsne_test_bounded_wait.argtypes = [vp, i32, C.POINTER(C.c_uint32)]
    L.pxsne_set_schedule.argtypes = [vp, C.POINTER(_CParams)]
    L.pxsne_nbr_precision.argtypes = [vp, i32, vp, i32, C.c_int, C.POINTER(C.c_double), vp]
    L.pxsne_mlp_create.argtypes = [C.POINTER(vp), i32, u64, vp]
    L.pxsne_mlp_destroy.argtypes = [vp]
    L.pxsne_mlp_destroy.restype = None
    L.pxsne_mlp_last_error.argtypes = [vp]
    L.pxsne_mlp_last_error.restype = C.c_char_p
    L.pxsne_mlp_num_params.argtypes = [vp]
    L.pxsne_mlp_num_params.restype = i64
    L.pxsne_mlp_set_params.argtypes = [vp, vp]
    L.pxsne_mlp_get_params.argtypes = [vp, vp]
    L.pxsne_mlp_loss_grad.argtypes = [vp, vp, vp, i64, vp, C.POINTER(C.c_double), C.c_int]
    L.pxsne_mlp_train.argtypes = [vp, vp, vp, i64, i32, i32, C.c_float, u64,
                                  C.POINTER(C.c_double), C.c_int]
    L.pxsne_mlp_predict.argtypes = [vp, vp, i64, vp, C.c_int]
    L.pxsne_embed_align.argtypes = [vp, vp, i64, vp, C.c_int]
    L.pxsne_pca.argtypes = [vp, i64, i32, i32, vp, vp, vp, C.c_int, u64]
    L.pxsne_device_bytes.argtypes = [vp]
    L.pxsne_device_bytes.restype = i64
    L.pxsne_get_level_counters.argtypes = [vp, C.POINTER(u64), i32]
    L.pxsne_save.argtypes = [vp, C.c_char_p]
    L.pxsne_test_stack_limit.argtypes = [vp, i32]
    L.pxsne_load.argtypes = [C.POINTER(vp), C.c_char_p, vp]
    L.pxsne_get_params.argtypes = [vp, C.POINTER(_CParams)]
    L.pxsne_get_tree3.argtypes = [vp, i32, vp, vp, vp, vp, vp]
    L.pxsne_measure_peaks.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                      C.POINTER(C.c_double), C.POINTER(i32), C.POINTER(i64)]
    _lib = L
    return L


def _buf(a, dtype, shape, name):
    """(pointer, on_device) of a C-contiguous numpy array or torch tensor (or
    None) of exactly this element type and shape; a None entry in ``shape``
    matches any extent.  Raises instead of handing the library a buffer it
    would read or write past.  A CUDA tensor's current stream is synchronised
    first (the library works on its own stream)."""
    if a is None:
        return None, 0
    dt = np.dtype(dtype)
    if isinstance(a, np.ndarray):
        got, contiguous, ptr, dev = a.dtype, a.flags.c_contiguous, a.ctypes.data, 0
    else:
        try:
            import torch
        except ImportError:
            torch = None
        if torch is None or not isinstance(a, torch.Tensor):
            raise TypeError(f"{name}: unsupported buffer type {type(a).__name__}")
        try:
            got = np.dtype(str(a.dtype).replace("torch.", ""))
        except TypeError:
            got = None
        contiguous, ptr, dev = a.is_contiguous(), a.data_ptr(), int(a.is_cuda)
    if got is None or got != dt:
        raise TypeError(f"{name}: element type {got if got is not None else a.dtype}, "
                        f"expected {dt}")
    if len(a.shape) != len(shape) or any(w is not None and g != w
                                         for g, w in zip(a.shape, shape)):
        want = "(" + ", ".join("*" if w is None else str(w) for w in shape) + ")"
        raise ValueError(f"{name}: shape {tuple(a.shape)}, expected {want}")
    if not contiguous:
        raise ValueError(f"{name}: not C-contiguous")
    if dev:
        import torch
        torch.cuda.current_stream(a.device).synchronize()
    return ptr, dev


def _f32(a):
    """numpy input as C-contiguous float32 (tensors pass through unchanged)."""
    return np.ascontiguousarray(a, np.float32) if isinstance(a, np.ndarray) else a


class Context:
    """One embedding problem on the current CUDA device (``pxsne_ctx``)."""

    def __init__(self, params: Params | None = None, stream=None):
        self.L = load()
        self.params = params or Params()
        self._p = self.params.c()
        h = C.c_void_p()
        rc = self.L.pxsne_create(C.byref(h), C.byref(self._p), stream)
        if rc != PXSNE_OK:
            raise PxsneError(rc, self.L.pxsne_last_error(None).decode())
        self.h = h

    def _ck(self, rc):
        if rc != PXSNE_OK:
            raise PxsneError(rc, self.L.pxsne_last_error(self.h).decode())

    @classmethod
    def load(cls, path, stream=None):
        """A context resumed from a checkpoint file (``pxsne_load``)."""
        L = load()
        h = C.c_void_p()
        rc = L.pxsne_load(C.byref(h), os.fsencode(path), stream)
        if rc != PXSNE_OK:
            raise PxsneError(rc, L.pxsne_last_error(None).decode())
        self = cls.__new__(cls)
        self.L, self.h = L, h
        cp = _CParams()
        self._ck(L.pxsne_get_params(h, C.byref(cp)))
        self.params = Params(**{f: getattr(cp, f) for f, _ in _CParams._fields_})
        self._p = self.params.c()
        return self

    def save(self, path):
        """Write P, the state and the schedule to a checkpoint file
        (``pxsne_save``)."""
        self._ck(self.L.pxsne_save(self.h, os.fsencode(path)))

    def close(self):
        if getattr(self, "h", None):
            self.L.pxsne_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---------------------------------------------------------------- the method
    def affinities(self, X, perplexity: float = 0.0):
        X = _f32(X)
        p, dev = _buf(X, np.float32, (None, None), "X")
        n, D = X.shape
        self._ck(self.L.pxsne_affinities(self.h, p, n, D, float(perplexity), dev))

    def init(self, Y0=None, seed: int = 0):
        Y0 = _f32(Y0)
        n = self.sizes()[0] or None   # without P the library reports the order error
        p, dev = _buf(Y0, np.float32, (n, self.dim), "Y0")
        self._ck(self.L.pxsne_init(self.h, p, dev, int(seed)))

    def step(self, iters: int = 1):
        self._ck(self.L.pxsne_step(self.h, int(iters)))

    def kl(self) -> float:
        out = C.c_double()
        self._ck(self.L.pxsne_kl(self.h, C.byref(out)))
        return out.value

    def get_Y(self, Y=None, pix=None, want_pix=True, blocking=True):
        """Centred y-space coordinates and pixels; fills Y/pix if given
        (numpy, or CUDA tensors), else returns new numpy arrays.  With
        blocking=False (CUDA tensors only) the frame is enqueued on the
        context's stream and the call returns at once."""
        n, d = self.sizes()[0], self.dim
        if Y is None and pix is None:
            Y = np.empty((n, d), np.float32)
            pix = np.empty((n, d), np.int32) if want_pix else None
        py, dy = _buf(Y, np.float32, (n, d), "Y")
        pp, dp = _buf(pix, np.int32, (n, d), "pix")
        if Y is not None and pix is not None and dy != dp:
            raise ValueError("Y and pix must both be host or both be device buffers")
        dev = dy or dp
        if not blocking and not dev:
            raise ValueError("blocking=False needs device buffers")
        self._ck(self.L.pxsne_get_Y(self.h, py, pp, dev if blocking else 2))
        return Y, pix

    def sync(self):
        f = C.c_uint32()
        rc = self.L.pxsne_sync(self.h, C.byref(f))
        self._ck(rc)
        return f.value

    # ---------------------------------------------------------------- inspection
    def sizes(self):
        n, nnz = C.c_int64(), C.c_int64()
        self._ck(self.L.pxsne_get_sizes(self.h, C.byref(n), C.byref(nnz)))
        return n.value, nnz.value

    def get_P(self):
        n, nnz = self.sizes()
        rp = np.empty(n + 1, np.int64)
        col = np.empty(nnz, np.int32)
        val = np.empty(nnz, np.float32)
        self._ck(self.L.pxsne_get_P(self.h, rp.ctypes.data, col.ctypes.data, val.ctypes.data))
        return rp, col, val

    def set_P(self, row_ptr, col, val):
        row_ptr = np.ascontiguousarray(row_ptr, np.int64)
        col = np.ascontiguousarray(col, np.int32)
        val = np.ascontiguousarray(val, np.float32)
        if row_ptr.ndim != 1 or row_ptr.shape[0] < 1:
            raise ValueError("row_ptr: expected a 1-D array of n + 1 offsets")
        nnz = int(row_ptr[-1])
        _buf(col, np.int32, (nnz,), "col")
        _buf(val, np.float32, (nnz,), "val")
        self._ck(self.L.pxsne_set_P(self.h, row_ptr.shape[0] - 1, row_ptr.ctypes.data,
                                    col.ctypes.data, val.ctypes.data))

    def get_knn(self):
        n, _ = self.sizes()
        k = self.params.k
        idx = np.empty((n, k), np.int32)
        d2 = np.empty((n, k), np.float32)
        beta = np.empty(n, np.float32)
        self._ck(self.L.pxsne_get_knn(self.h, idx.ctypes.data, d2.ctypes.data, beta.ctypes.data))
        return idx, d2, beta

    def set_state(self, z, s, u=None, gains=None, t=0):
        n = self.sizes()[0] or None   # without P the library reports the order error
        z = np.ascontiguousarray(z, np.uint32)
        s = np.ascontiguousarray(s, np.float64)
        u = None if u is None else np.ascontiguousarray(u, np.float32)
        gains = None if gains is None else np.ascontiguousarray(gains, np.float32)
        d = self.dim
        pz, _ = _buf(z, np.uint32, (n, d), "z")
        ps, _ = _buf(s, np.float64, (d,), "s")
        pu, _ = _buf(u, np.float32, (n, d), "u")
        pg, _ = _buf(gains, np.float32, (n, d), "gains")
        self._ck(self.L.pxsne_set_state(self.h, pz, ps, pu, pg, int(t)))

    def get_state(self):
        n, _ = self.sizes()
        d = self.dim
        z = np.empty((n, d), np.uint32)
        s = np.empty(d, np.float64)
        u = np.empty((n, d), np.float32)
        g = np.empty((n, d), np.float32)
        t = C.c_int32()
        self._ck(self.L.pxsne_get_state(self.h, z.ctypes.data, s.ctypes.data, u.ctypes.data,
                                        g.ctypes.data, C.byref(t)))
        return z, s, u, g, t.value

    def get_tree(self, level, sums=False, morton=False):
        n, _ = self.sizes()
        cells = 4 ** level
        cnt = np.empty(cells, np.uint32)
        sx = np.empty(cells, np.uint64) if sums else None
        sy = np.empty(cells, np.uint64) if sums else None
        mk = np.empty(n, np.uint32) if morton else None
        self._ck(self.L.pxsne_get_tree(self.h, int(level), cnt.ctypes.data,
                                       None if sx is None else sx.ctypes.data,
                                       None if sy is None else sy.ctypes.data,
                                       None if mk is None else mk.ctypes.data))
        return cnt, sx, sy, mk

    def get_tree3(self, level, sums=False, morton=False):
        """The octree of a 3-D state at one level (``pxsne_get_tree3``)."""
        n, _ = self.sizes()
        cells = 8 ** level
        cnt = np.empty(cells, np.uint32)
        sx, sy, sz = ((np.empty(cells, np.uint64) if sums else None) for _ in range(3))
        mk = np.empty(n, np.uint32) if morton else None
        ptr = [None if a is None else a.ctypes.data for a in (sx, sy, sz, mk)]
        self._ck(self.L.pxsne_get_tree3(self.h, int(level), cnt.ctypes.data, *ptr))
        return cnt, sx, sy, sz, mk

    @property
    def dim(self):
        return 3 if self.params.dim == 3 else 2

    def get_forces(self):
        n, _ = self.sizes()
        Frep = np.empty((n, self.dim), np.float32)
        Zi = np.empty(n, np.float32)
        Fattr = np.empty((n, self.dim), np.float32)
        Z = C.c_double()
        self._ck(self.L.pxsne_get_forces(self.h, Frep.ctypes.data, Zi.ctypes.data,
                                         Fattr.ctypes.data, C.byref(Z)))
        return Frep, Zi, Fattr, Z.value

    def step_profiled(self, iters: int):
        """Run iterations with CUDA events around each kernel group; returns
        ({group name: summed ms}, total ms)."""
        g = (C.c_double * 16)()
        tot = C.c_double()
        self._ck(self.L.pxsne_step_profiled(self.h, int(iters), g, 16, C.byref(tot)))
        out = {}
        for k in range(16):
            name = self.L.pxsne_kernel_group_name(k)
            if name is None:
                break
            out[name.decode()] = g[k]
        return out, tot.value

    def counters(self):
        """(accepted pairs, tested pairs, warp steps, nodes) of the last
        counted traversal."""
        a, t, w, nd = C.c_uint64(), C.c_uint64(), C.c_uint64(), C.c_uint64()
        self._ck(self.L.pxsne_get_counters(self.h, C.byref(a), C.byref(t), C.byref(w),
                                           C.byref(nd)))
        return a.value, t.value, w.value, nd.value

    def level_counters(self):
        """(tested, accepted, warp steps) by level of the tested cell, rows
        0 .. L (``pxsne_get_level_counters``)."""
        lv = self.params.log2_r + 1
        buf = (C.c_uint64 * (3 * lv))()
        self._ck(self.L.pxsne_get_level_counters(self.h, buf, lv))
        return np.array(buf[:], dtype=np.int64).reshape(lv, 3)

    def nbr_precision(self, k=10, knn_hd=None, per_point=False):
        """Eq. nei_prec of the current embedding (high-D lists from the last
        affinities call unless knn_hd [n x kh] is given)."""
        n = self.sizes()[0]
        prec = C.c_double()
        hits = np.empty(n, np.int32) if per_point else None
        if knn_hd is None:
            rc = self.L.pxsne_nbr_precision(self.h, int(k), None, 0, 0, C.byref(prec),
                                            None if hits is None else hits.ctypes.data)
        else:
            kd = np.ascontiguousarray(knn_hd, np.int32)
            _buf(kd, np.int32, (n, None), "knn_hd")
            rc = self.L.pxsne_nbr_precision(self.h, int(k), kd.ctypes.data, kd.shape[1], 0,
                                            C.byref(prec),
                                            None if hits is None else hits.ctypes.data)
        self._ck(rc)
        return (prec.value, hits) if per_point else prec.value

    def set_schedule(self, **kw):
        """Change optimiser fields (eta, exaggeration, exag_iters, momentum0,
        momentum1, momentum_switch, min_gain) of this context."""
        for k, v in kw.items():
            setattr(self.params, k, v)
        self._p = self.params.c()
        self._ck(self.L.pxsne_set_schedule(self.h, C.byref(self._p)))

    def knn_counters(self):
        """(exact distances, insertions, path) of the last neighbour search."""
        a, b, p = C.c_uint64(), C.c_uint64(), C.c_int32()
        self._ck(self.L.pxsne_get_knn_counters(self.h, C.byref(a), C.byref(b), C.byref(p)))
        return a.value, b.value, p.value

    def test_bounded_wait(self, polls):
        """(status code, device error flags) of the bounded-wait test hook."""
        f = C.c_uint32()
        rc = self.L.pxsne_test_bounded_wait(self.h, int(polls), C.byref(f))
        return rc, f.value

    def test_stack_limit(self, entries):
        """Lower the traversal's stack room (test hook; 0 restores it)."""
        self._ck(self.L.pxsne_test_stack_limit(self.h, int(entries)))

    def knn_pruning(self):
        """(skipped (query tile, candidate tile) pairs, all pairs) of the last
        tensor-core neighbour search."""
        a, b = C.c_uint64(), C.c_uint64()
        self._ck(self.L.pxsne_get_knn_pruning(self.h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def knn_time_ms(self):
        """Device time of the last neighbour-search kernel (ms)."""
        ms = C.c_double()
        self._ck(self.L.pxsne_get_knn_time(self.h, C.byref(ms)))
        return ms.value

    def device_bytes(self):
        return int(self.L.pxsne_device_bytes(self.h))


class MLP:
    """The learned warm start (``pxsne_mlp``): d -> 256 -> 256 -> 2, GELU."""

    def __init__(self, d: int, seed: int = 0, stream=None):
        self.L = load()
        h = C.c_void_p()
        rc = self.L.pxsne_mlp_create(C.byref(h), int(d), int(seed), stream)
        if rc != PXSNE_OK:
            raise PxsneError(rc, "pxsne_mlp_create")
        self.h = h
        self.d = d
        self.np = int(self.L.pxsne_mlp_num_params(h))

    def _ck(self, rc):
        if rc != PXSNE_OK:
            raise PxsneError(rc, self.L.pxsne_mlp_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.L.pxsne_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def get_params(self):
        w = np.empty(self.np, np.float32)
        self._ck(self.L.pxsne_mlp_get_params(self.h, w.ctypes.data))
        return w

    def set_params(self, w):
        w = np.ascontiguousarray(w, np.float32).reshape(-1)
        _buf(w, np.float32, (self.np,), "w")
        self._ck(self.L.pxsne_mlp_set_params(self.h, w.ctypes.data))

    def loss_grad(self, X, T):
        X = np.ascontiguousarray(X, np.float32)
        T = np.ascontiguousarray(T, np.float32)
        _buf(X, np.float32, (None, self.d), "X")
        _buf(T, np.float32, (X.shape[0], 2), "T")
        g = np.empty(self.np, np.float32)
        loss = C.c_double()
        self._ck(self.L.pxsne_mlp_loss_grad(self.h, X.ctypes.data, T.ctypes.data, X.shape[0],
                                            g.ctypes.data, C.byref(loss), 0))
        return loss.value, g

    def train(self, X, T, epochs=10, batch=4096, lr=1e-3, seed=0):
        X, T = _f32(X), _f32(T)
        Xp, dx = _buf(X, np.float32, (None, self.d), "X")
        n = X.shape[0]
        Tp, dt = _buf(T, np.float32, (n, 2), "T")
        if dx != dt:
            raise ValueError("X and T must both be host or both be device buffers")
        loss = C.c_double()
        self._ck(self.L.pxsne_mlp_train(self.h, Xp, Tp, n, int(epochs), int(batch), float(lr),
                                        int(seed), C.byref(loss), dx))
        return loss.value

    def predict(self, X, Y=None):
        X = _f32(X)
        Xp, dx = _buf(X, np.float32, (None, self.d), "X")
        n = X.shape[0]
        if Y is None:
            Y = np.empty((n, 2), np.float32)
        Yp, dy = _buf(Y, np.float32, (n, 2), "Y")
        if dx != dy:
            raise ValueError("X and Y must both be host or both be device buffers")
        self._ck(self.L.pxsne_mlp_predict(self.h, Xp, n, Yp, dx))
        return Y


def embed_align(Y, Yref=None):
    """Centre, scale to unit RMS and (with Yref, whose row i is the same point
    as row i of Y) orthogonally align Y (numpy)."""
    L = load()
    Y = np.ascontiguousarray(Y, np.float32)
    out = np.empty_like(Y)
    _buf(Y, np.float32, (None, 2), "Y")
    R = None if Yref is None else np.ascontiguousarray(Yref, np.float32)
    _buf(R, np.float32, Y.shape, "Yref")
    rc = L.pxsne_embed_align(Y.ctypes.data, None if R is None else R.ctypes.data, Y.shape[0],
                             out.ctypes.data, 0)
    if rc != PXSNE_OK:
        raise PxsneError(rc, "pxsne_embed_align")
    return out


def pca(X, dout=50, seed=0):
    """(projection [n, dout], components [D, dout], eigenvalues [dout])."""
    L = load()
    X = np.ascontiguousarray(X, np.float32)
    _buf(X, np.float32, (None, None), "X")
    n, D = X.shape
    out = np.empty((n, dout), np.float32)
    V = np.empty((D, dout), np.float32)
    lam = np.empty(dout, np.float32)
    rc = L.pxsne_pca(X.ctypes.data, n, D, int(dout), out.ctypes.data, V.ctypes.data,
                     lam.ctypes.data, 0, int(seed))
    if rc != PXSNE_OK:
        raise PxsneError(rc, "pxsne_pca")
    return out, V, lam


def measure_peaks(stream=None):
    """Measured L2 read bandwidth (GB/s), FP32 FMA rate scalar and packed
    (TFLOP/s), SM count and L2 size of the current device
    (``pxsne_measure_peaks``)."""
    L = load()
    l2, f1, f2 = C.c_double(), C.c_double(), C.c_double()
    sms, l2b = C.c_int32(), C.c_int64()
    rc = L.pxsne_measure_peaks(stream, C.byref(l2), C.byref(f1), C.byref(f2), C.byref(sms),
                               C.byref(l2b))
    if rc != PXSNE_OK:
        raise PxsneError(rc, "pxsne_measure_peaks")
    return {"l2_read_gbs": l2.value, "fp32_tflops": f1.value, "fp32_packed_tflops": f2.value,
            "sm_count": sms.value, "l2_bytes": l2b.value}


EXPORTED = ["pxsne_default_params", "pxsne_create", "pxsne_destroy", "pxsne_last_error",
            "pxsne_affinities", "pxsne_init", "pxsne_step", "pxsne_kl", "pxsne_get_Y",
            "pxsne_sync", "pxsne_get_sizes", "pxsne_get_P", "pxsne_set_P", "pxsne_get_knn",
            "pxsne_set_state", "pxsne_get_state", "pxsne_get_tree", "pxsne_get_forces",
            "pxsne_device_bytes", "pxsne_step_profiled", "pxsne_kernel_group_name",
            "pxsne_get_knn_time", "pxsne_test_bounded_wait", "pxsne_get_knn_pruning",
            "pxsne_get_counters", "pxsne_kl_noalloc", "pxsne_kl_noalloc_max_rows",
            "pxsne_get_knn_counters", "pxsne_set_schedule", "pxsne_mlp_create",
            "pxsne_mlp_destroy", "pxsne_mlp_last_error", "pxsne_mlp_num_params",
            "pxsne_mlp_set_params", "pxsne_mlp_get_params", "pxsne_mlp_loss_grad",
            "pxsne_mlp_train", "pxsne_mlp_predict", "pxsne_embed_align",
            "pxsne_nbr_precision", "pxsne_pca", "pxsne_measure_peaks",
            "pxsne_get_level_counters", "pxsne_save", "pxsne_load", "pxsne_get_params",
            "pxsne_test_stack_limit", "pxsne_get_tree3"]
