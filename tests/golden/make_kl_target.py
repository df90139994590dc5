"""Write kl_target_gauss10.json: the oracle's KL after the full schedule on the
small isotropic-mixture workload (10 Gaussians in D = 50, 200 points each,
seed 0; perplexity 30, k = 90, 512^2 screen, theta 0.5, 500 iterations from
datagen.init_y0(0, 2000)).  The KL is that of Eq. cost_func with the
Barnes-Hut Z of the final state, as the method's own evaluation (Sec. 5,
Table 5) reports it.  A time-to-target measurement takes 1.01 times this
value as its target.  Calls only the oracle and the seeded input generators.

    python tests/golden/make_kl_target.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import datagen  # noqa: E402
import oracle  # noqa: E402

SEED, ITERS, L, U, K = 0, 500, 9, 30.0, 90


def compute():
    X, _ = datagen.gauss10(SEED)
    P, _, _, bad = oracle.affinities(X, U, K)
    st = oracle.State.from_y0(datagen.init_y0(SEED, X.shape[0]))
    params = oracle.Params(L=L)
    oracle.run(P, st, params, ITERS)
    return {"workload": "gauss10", "n": int(X.shape[0]), "D": int(X.shape[1]), "seed": SEED,
            "perplexity": U, "k": K, "log2_r": L, "theta": 0.5, "iterations": ITERS,
            "unconverged_rows": int(bad), "kl": float(oracle.kl_of(P, st, params))}


if __name__ == "__main__":
    out = compute()
    with open(os.path.join(HERE, "kl_target_gauss10.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(out)
