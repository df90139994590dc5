"""Argument marshalling of the Python binding, on the CPU (no library call):
buffers are accepted only with the element type, shape and layout the C ABI
reads or writes, so that a wrong buffer raises instead of being overrun."""
import numpy as np
import pytest

import paper_1611_02568_gb300 as px


def test_numpy_buffers():
    a = np.zeros((7, 2), np.float32)
    p, dev = px._buf(a, np.float32, (7, 2), "Y")
    assert p == a.ctypes.data and dev == 0
    assert px._buf(None, np.float32, (7, 2), "Y") == (None, 0)
    assert px._buf(a, np.float32, (None, 2), "Y")[0] == a.ctypes.data
    with pytest.raises(TypeError, match="element type"):
        px._buf(a.astype(np.float64), np.float32, (7, 2), "Y")
    with pytest.raises(TypeError, match="element type"):
        px._buf(a.astype(np.int32), np.float32, (7, 2), "Y")
    with pytest.raises(ValueError, match="shape"):
        px._buf(a, np.float32, (8, 2), "Y")
    with pytest.raises(ValueError, match="shape"):
        px._buf(a.reshape(-1), np.float32, (None, 2), "Y")
    with pytest.raises(ValueError, match="contiguous"):
        px._buf(np.zeros((2, 7), np.float32).T, np.float32, (7, 2), "Y")
    with pytest.raises(TypeError, match="unsupported"):
        px._buf([[0.0, 0.0]], np.float32, (1, 2), "Y")


def test_torch_cpu_tensors():
    torch = pytest.importorskip("torch")
    t = torch.zeros((5, 2), dtype=torch.int32)
    p, dev = px._buf(t, np.int32, (5, 2), "pix")
    assert p == t.data_ptr() and dev == 0
    with pytest.raises(TypeError, match="element type"):
        px._buf(t.to(torch.int64), np.int32, (5, 2), "pix")
    with pytest.raises(TypeError, match="element type"):
        px._buf(torch.zeros((5, 2), dtype=torch.bfloat16), np.float64, (5, 2), "s")
    with pytest.raises(ValueError, match="shape"):
        px._buf(t[:4], np.int32, (5, 2), "pix")
    with pytest.raises(ValueError, match="contiguous"):
        px._buf(torch.zeros((2, 5), dtype=torch.int32).t(), np.int32, (5, 2), "pix")


def test_f32_converts_numpy_only():
    a = np.arange(6, dtype=np.float64).reshape(3, 2)
    b = px._f32(a)
    assert b.dtype == np.float32 and b.flags.c_contiguous and np.array_equal(a, b)
    sentinel = object()
    assert px._f32(sentinel) is sentinel


class _FakeLib:
    """Stands in for libpxsne.so: records each call's arguments and returns
    PXSNE_OK; pxsne_get_sizes reports n points."""

    def __init__(self, n):
        self.n = n
        self.calls = []

    def pxsne_get_sizes(self, h, n_ref, nnz_ref):
        n_ref._obj.value = self.n
        nnz_ref._obj.value = 0
        return 0

    def __getattr__(self, name):
        def call(*args):
            self.calls.append((name, args))
            return 0
        return call


def _ctx(n):
    ctx = object.__new__(px.Context)
    ctx.L = _FakeLib(n)
    ctx.h = None
    ctx.params = px.Params()
    return ctx


def test_context_marshalling_without_a_gpu():
    ctx = _ctx(6)
    X = np.zeros((6, 3), np.float64)
    ctx.affinities(X)
    name, args = ctx.L.calls[-1]
    assert name == "pxsne_affinities" and args[2:] == (6, 3, 0.0, 0)
    ctx.init(np.zeros((6, 2)))
    assert ctx.L.calls[-1][0] == "pxsne_init" and ctx.L.calls[-1][1][2] == 0
    ctx.init(None, seed=5)
    assert ctx.L.calls[-1][1][1:] == (None, 0, 5)
    with pytest.raises(ValueError, match="Y0: shape"):
        ctx.init(np.zeros((5, 2)))
    Y, pix = ctx.get_Y()
    assert Y.shape == (6, 2) and Y.dtype == np.float32 and pix.dtype == np.int32
    assert ctx.L.calls[-1][0] == "pxsne_get_Y" and ctx.L.calls[-1][1][3] == 0
    with pytest.raises(TypeError, match="pix: element type"):
        ctx.get_Y(None, np.zeros((6, 2), np.int64))
    with pytest.raises(ValueError, match="Y: shape"):
        ctx.get_Y(np.zeros((7, 2), np.float32))
    z = np.zeros((6, 2), np.uint32)
    ctx.set_state(z, [1e-9, 1e-9])
    assert ctx.L.calls[-1][0] == "pxsne_set_state"
    with pytest.raises(ValueError, match="z: shape"):
        ctx.set_state(z[:5], [1e-9, 1e-9])
    with pytest.raises(ValueError, match="s: shape"):
        ctx.set_state(z, [1e-9])
    with pytest.raises(ValueError, match="col: shape"):
        ctx.set_P(np.array([0, 2, 3]), np.array([1, 0]), np.ones(3))
    with pytest.raises(ValueError, match="knn_hd: shape"):
        ctx.nbr_precision(k=2, knn_hd=np.zeros((5, 4), np.int32))


def test_order_errors_are_left_to_the_library():
    # without P the library reports E_STATE; the binding must not pre-empt it
    ctx = _ctx(0)
    ctx.init(np.zeros((10, 2), np.float32))
    assert ctx.L.calls[-1][0] == "pxsne_init"
    ctx.set_state(np.zeros((10, 2), np.uint32), [1.0, 1.0])
    assert ctx.L.calls[-1][0] == "pxsne_set_state"


def test_mlp_marshalling_without_a_gpu():
    net = object.__new__(px.MLP)
    net.L = _FakeLib(0)
    net.h = None
    net.d = 4
    net.np = 10
    Y = net.predict(np.zeros((3, 4)))
    assert Y.shape == (3, 2) and net.L.calls[-1][0] == "pxsne_mlp_predict"
    assert net.L.calls[-1][1][2] == 3
    with pytest.raises(ValueError, match="X: shape"):
        net.predict(np.zeros((3, 5), np.float32))
    with pytest.raises(ValueError, match="T: shape"):
        net.train(np.zeros((3, 4)), np.zeros((2, 2)))
    net.train(np.zeros((3, 4)), np.zeros((3, 2)), epochs=1)
    assert net.L.calls[-1][0] == "pxsne_mlp_train" and net.L.calls[-1][1][3] == 3
    with pytest.raises(ValueError, match="w: shape"):
        net.set_params(np.zeros(9))
    with pytest.raises(ValueError, match="T: shape"):
        net.loss_grad(np.zeros((3, 4)), np.zeros((3, 3)))
    with pytest.raises(ValueError, match="Yref: shape"):
        px.embed_align(np.zeros((4, 2)), np.zeros((3, 2)))
