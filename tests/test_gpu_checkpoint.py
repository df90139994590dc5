"""Checkpoint and resume on the GPU: a run stopped at t = 137 and saved, then
loaded into a fresh context, continues exactly as the run that wrote it -- z,
s, u, gains, t and the KL bit-identical after 50 more iterations (the
attraction's relabelled copy of P and the traversal order are rebuilt on load;
neither enters the values)."""
import numpy as np
import pytest

import datagen

pytestmark = pytest.mark.gpu


def test_resume_from_checkpoint_is_bit_exact(tmp_path):
    import paper_1611_02568_gb300 as px
    from paper_1611_02568_gb300 import build
    build.build()
    X, _ = datagen.gmm128(2, n=20011)
    n = X.shape[0]
    path = str(tmp_path / "run.pxck")
    with px.Context(px.Params(log2_r=10)) as a:
        a.affinities(X)
        a.set_schedule(exag_iters=120, momentum_switch=130)
        a.init(datagen.init_y0(2, n))
        a.step(137)
        a.save(path)
        before = a.get_state()
        a.step(50)
        ref = a.get_state()
        kl_ref = a.kl()
        Pa = a.get_P()
    with px.Context.load(path) as b:
        assert b.params.log2_r == 10 and b.params.exag_iters == 120
        assert b.params.momentum_switch == 130
        for x, y in zip(b.get_state(), before):
            assert np.array_equal(x, y)
        for x, y in zip(b.get_P(), Pa):
            assert np.array_equal(x, y)
        b.step(50)
        got = b.get_state()
        kl = b.kl()
    assert got[4] == ref[4] == 187
    for x, y in zip(got[:4], ref[:4]):
        assert np.array_equal(x, y)
    assert kl == kl_ref
