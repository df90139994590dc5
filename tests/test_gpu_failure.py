"""Failure detection on the GPU without a GPU fault: each device error flag is
raised by an input that reaches it through ordinary arithmetic (or, for the
time-out, by a bounded wait on an mbarrier that nothing arrives at), comes back
as PXSNE_E_DEVICE from the next synchronising call, and leaves the context
usable.

Bars: the returned status and flag bits exactly; the oracle's P (within the
bisection tolerance of the affinity tests) for rows whose perplexity target is
out of reach."""
import numpy as np
import pytest

import datagen
import oracle

pytestmark = pytest.mark.gpu

E_ARG, E_DEVICE = -1, -5
NONFINITE, STACK, BISECT, RANGE, TIMEOUT = 1, 2, 4, 8, 16


@pytest.fixture(scope="module")
def px():
    import paper_1611_02568_gb300 as m
    from paper_1611_02568_gb300 import build
    build.build()
    return m


def small_run(px, ctx, X):
    ctx.affinities(X)
    ctx.init(datagen.init_y0(0, X.shape[0]))
    ctx.step(20)
    assert ctx.sync() == 0
    assert np.isfinite(ctx.kl())


def test_bounded_wait_times_out(px):
    X, _ = datagen.gauss10(2, n=1200)
    with px.Context(px.Params(log2_r=9)) as ctx:
        rc, flags = ctx.test_bounded_wait(2000)
        assert rc == E_DEVICE and flags == TIMEOUT
        assert "timeout" in ctx.L.pxsne_last_error(ctx.h).decode()
        assert ctx.sync() == 0                 # the flag was read and cleared
        assert ctx.test_bounded_wait(0)[0] == E_ARG
        small_run(px, ctx, X)                  # the context is still usable
        rc, flags = ctx.test_bounded_wait(1)
        assert rc == E_DEVICE and flags == TIMEOUT


@pytest.mark.parametrize("value, flag, word", [(np.nan, NONFINITE, "non-finite"),
                                               (np.inf, NONFINITE, "non-finite"),
                                               (1e30, RANGE, "step-range")])
def test_bad_velocity_flagged(px, value, flag, word):
    X, _ = datagen.gauss10(3, n=1500)
    with px.Context(px.Params(log2_r=9)) as ctx:
        ctx.affinities(X)
        ctx.init(datagen.init_y0(1, X.shape[0]))
        ctx.step(5)
        z, s, u, g, t = ctx.get_state()
        u[17, 1] = value
        ctx.set_state(z, s, u, g, t)           # no update runs here
        ctx.step(1)
        with pytest.raises(px.PxsneError) as ei:
            ctx.sync()
        assert ei.value.code == E_DEVICE and word in str(ei.value)
        z2, s2, u2, _, t2 = ctx.get_state()
        assert t2 == t + 1 and np.all(np.isfinite(s2)) and np.all(s2 > 0)
        if flag == NONFINITE:
            # the bad coordinate's velocity is reset and nothing else moves
            # out of range: the next iterations run clean
            assert u2[17, 1] == 0.0 and np.all(np.isfinite(u2))
            ctx.step(10)
            assert ctx.sync() == 0
            assert np.isfinite(ctx.kl())
        else:
            # the step was clamped to 2^58 ulps and the velocity kept
            assert np.isfinite(u2[17, 1]) and abs(u2[17, 1]) > 1e29


@pytest.mark.parametrize("value", [np.nan, -np.inf])
def test_nonfinite_start_flagged(px, value):
    X, _ = datagen.gauss10(4, n=1100)
    Y0 = datagen.init_y0(2, X.shape[0])
    Y0[40, 0] = value
    with px.Context(px.Params(log2_r=9)) as ctx:
        ctx.affinities(X)
        with pytest.raises(px.PxsneError) as ei:
            ctx.init(Y0)
        assert ei.value.code == E_DEVICE and "non-finite" in str(ei.value)
        ctx.init(datagen.init_y0(2, X.shape[0]))     # a clean start runs
        ctx.step(10)
        assert ctx.sync() == 0


def test_unreachable_perplexity_flagged(px, monkeypatch):
    """Clusters of 100 identical rows with k = 90: every neighbour of every row
    is at distance 0, so the entropy is ln 90 for any beta and the target ln 30
    cannot be met. Both kNN paths; P must equal the oracle's uniform weights."""
    rng = np.random.default_rng(9)
    centres = rng.standard_normal((20, 8)).astype(np.float32) * 10
    X = np.repeat(centres, 100, axis=0)
    k, u = 90, 30.0
    P, idx_o, d2_o, bad = oracle.affinities(X, u, k)
    assert bad == X.shape[0]
    for path in ("tc", "fp32"):
        if path == "fp32":
            monkeypatch.setenv("PXSNE_KNN", "fp32")
        with px.Context(px.Params(log2_r=9, k=k, perplexity=u)) as ctx:
            with pytest.raises(px.PxsneError) as ei:
                ctx.affinities(X)
            assert ei.value.code == E_DEVICE and "bisection" in str(ei.value)
            idx, d2, beta = ctx.get_knn()
            assert np.all(d2 == 0.0)
            # ties on distance go to the lower index, as in the oracle
            assert np.array_equal(idx, idx_o)
            rp, col, val = ctx.get_P()
            assert np.array_equal(rp, P.row_ptr) and np.array_equal(col, P.col)
            np.testing.assert_allclose(val, P.val, rtol=2e-3, atol=1e-9)
            # the context runs on with this P
            ctx.init(datagen.init_y0(0, X.shape[0]))
            ctx.step(10)
            assert ctx.sync() == 0


def test_stack_overflow_flagged(px):
    """The traversal's stack guard: with room for 4 entries (a 512^2 screen
    needs 3 L - 2 = 25) a warp stops its walk, sets the flag and skips the
    push; the next synchronising call reports it, and with the full stack
    back the same state gives the oracle's forces."""
    X, _ = datagen.gauss10(5, n=1800)
    with px.Context(px.Params(log2_r=9)) as ctx:
        ctx.affinities(X)
        ctx.init(datagen.init_y0(3, X.shape[0]))
        ctx.step(30)
        assert ctx.sync() == 0
        z, s, u, g, t = ctx.get_state()
        assert ctx.L.pxsne_test_stack_limit(ctx.h, 3) == E_ARG
        ctx.test_stack_limit(4)
        ctx.step(1)
        with pytest.raises(px.PxsneError) as ei:
            ctx.sync()
        assert ei.value.code == E_DEVICE and "stack" in str(ei.value)
        assert ctx.sync() == 0                 # read and cleared
        ctx.test_stack_limit(0)
        ctx.set_state(z, s, u, g, t)
        Frep, Zi, _, _ = ctx.get_forces()
        oF, oZi, _ = oracle.bh_repulsion(z, s, 9, 0.5)
        assert np.linalg.norm(Frep - oF) / np.linalg.norm(oF) < 1e-4
        ctx.step(10)
        assert ctx.sync() == 0


def test_clamped_step_rescales_exactly(px):
    """A step clamped to 2^58 ulps makes the rescale's range gamma about 2^59
    (Sec. 4.2's gamma_d at its widest): the GPU's new z and s equal the
    oracle's exact-integer rescale of the same zhat, bit for bit.  zhat is
    rebuilt on the host from the GPU's own new velocities, exactly as the
    step forms it: z + rint(u / s) in FP64, clamped to +-2^58."""
    X, _ = datagen.gauss10(6, n=1300)
    with px.Context(px.Params(log2_r=9)) as ctx:
        ctx.affinities(X)
        ctx.init(datagen.init_y0(4, X.shape[0]))
        ctx.step(12)
        z, s, u, g, t = ctx.get_state()
        u[5, 0] = 1e30
        u[77, 1] = -3e29
        ctx.set_state(z, s, u, g, t)
        ctx.step(1)
        with pytest.raises(px.PxsneError):
            ctx.sync()                         # RANGE, as expected
        z2, s2, u2, _, _ = ctx.get_state()
    lim = 2.0 ** 58
    st = np.rint(u2.astype(np.float64) * (1.0 / s)[None, :])
    assert abs(st[5, 0]) > lim and abs(st[77, 1]) > lim
    st = np.clip(st, -lim, lim)
    zhat = z.astype(np.int64) + st.astype(np.int64)
    assert zhat[:, 0].max() - zhat[:, 0].min() > 2 ** 58
    zo, so = oracle.rescale(zhat, s)
    assert np.array_equal(z2, zo)
    assert np.array_equal(s2, so)
