"""pxsne_init without a caller Y0 draws the start from its seed with
Philox4x32-10 and Box-Muller.  The oracle implements the same published
generator (pinned to its known-answer vectors); the state the library maps
that draw to must equal the oracle's map of the oracle's draw.

The device's FP64 log, sin and cos may differ from the host's in the last
bit, which moves a float32 coordinate by one ulp about once in 10^8 draws;
the comparison allows for that (a moved extreme shifts every fixed-point
coordinate by about a hundred ulps)."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed", [0, 12345, 2 ** 40 + 7])
def test_seeded_init_matches_the_oracle_draw(seed):
    import paper_1611_02568_gb300 as px
    from paper_1611_02568_gb300 import build
    build.build()
    n = 5000
    X = np.random.default_rng(1).standard_normal((n, 4)).astype(np.float32)
    with px.Context(px.Params(log2_r=10, k=5, perplexity=3.0, init_sigma=1e-4)) as ctx:
        ctx.affinities(X)
        ctx.init(None, seed=seed)
        z, s, u, g, t = ctx.get_state()
    zo, so = oracle.init_fx(oracle.philox_y0(seed, n, 1e-4).astype(np.float64))
    assert t == 0 and np.all(u == 0) and np.all(g == 1)
    np.testing.assert_allclose(s, so, rtol=1e-6)
    dz = np.abs(z.astype(np.int64) - zo.astype(np.int64))
    assert dz.max() <= 1024
    if np.array_equal(s, so):
        # the extremes agree, so the map is the same: every point agrees
        # exactly but for a rare one-ulp coordinate
        assert (dz == 0).mean() >= 0.999
