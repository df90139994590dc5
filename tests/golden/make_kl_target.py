"""Write the stored KL targets: the oracle's KL of Eq. cost_func (Barnes-Hut Z
of the state, as the method's own evaluation in Sec. 5, Table 5 reports it)
after the full schedule of a workload, started from datagen.init_y0(seed, n).

Workloads (name -> file kl_target_<name>.json):

- gauss10         10 Gaussians in D = 50, n = 2,000; 512^2, 500 iterations.
- protos784_n70k  784-D prototype data, n = 70,000, reduced to 50 dims by the
                  oracle's PCA (Sec. 5.1.1); 1024^2, 1,000 iterations.
- gmm128_n200k    the 128-D, 100-component Zipf mixture at n = 200,000;
                  2048^2, 1,000 iterations.
- gmm128_n1M      the same recipe at n = 1,000,000 (the bench workload).

Every workload takes perplexity 30, k = 90, theta 0.5 and the default
schedule (exaggeration 12 for 250 iterations, momentum 0.5 then 0.8, eta
200).  Besides the final KL the file keeps the KL after every quarter of the
schedule and the size of P.  A time-to-target measurement takes 1.01 times
the final value as its target; the GPU parity tests hold the whole GPU path
within 1 % of it.  Calls only the oracle and the seeded input generators.

    python tests/golden/make_kl_target.py [name ...] [--cache DIR]

--cache keeps the oracle's neighbour lists of a workload in DIR (.npz), so
that a rerun skips the exact neighbour search (hours at n = 1M).
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import datagen  # noqa: E402
import oracle  # noqa: E402

U, K, THETA = 30.0, 90, 0.5

# name: (generator, n, log2 r, iterations, PCA dims or None)
WORKLOADS = {
    "gauss10": ("gauss10", 2000, 9, 500, None),
    "protos784_n70k": ("protos784", 70000, 10, 1000, 50),
    "gmm128_n200k": ("gmm128", 200000, 11, 1000, None),
    "gmm128_n1M": ("gmm128", 1000000, 11, 1000, None),
}
SEED = 0


def inputs(name):
    """The X both sides build P from (after the oracle's PCA where the workload
    asks for it), as float32, and Y0."""
    gen, n, _, _, dpca = WORKLOADS[name]
    X, _ = getattr(datagen, gen)(SEED, n=n)
    if dpca:
        X = oracle.pca(X, dpca)[0].astype(np.float32)
    return np.ascontiguousarray(X), datagen.init_y0(SEED, n)


def compute(name="gauss10", cache=None, log=None):
    gen, n, L, iters, dpca = WORKLOADS[name]
    X, Y0 = inputs(name)
    t0 = time.time()
    path = os.path.join(cache, f"knn_{name}.npz") if cache else None
    if path and os.path.exists(path):
        f = np.load(path)
        idx, d2 = f["idx"], f["d2"]
    else:
        idx, d2 = oracle.knn(X, K)
        if path:
            np.savez(path, idx=idx, d2=d2)
    t_knn = time.time() - t0
    pcond, _, _, bad = oracle.perplexity(d2, U)
    P = oracle.symmetrize(idx, pcond)
    st = oracle.State.from_y0(Y0)
    params = oracle.Params(L=L, theta=THETA)
    quarters = []
    t1 = time.time()
    for q in range(4):
        oracle.run(P, st, params, iters // 4)
        quarters.append(float(oracle.kl_of(P, st, params)))
        if log:
            log(f"{name}: t = {st.t}, KL {quarters[-1]:.6f}, {time.time() - t1:.0f} s")
    out = {"workload": gen, "n": int(n), "D": int(X.shape[1]), "seed": SEED,
           "pca": dpca, "perplexity": U, "k": K, "log2_r": L, "theta": THETA,
           "iterations": iters, "unconverged_rows": int(bad), "nnz": int(P.nnz),
           "kl_quarters": quarters, "kl": quarters[-1]}
    if name == "gauss10":
        # the first stored target kept only these fields
        out = {k: out[k] for k in ("workload", "n", "D", "seed", "perplexity", "k", "log2_r",
                                   "theta", "iterations", "unconverged_rows", "kl")}
    if log:
        log(f"{name}: knn {t_knn:.0f} s, iterations {time.time() - t1:.0f} s")
    return out


def _target_file(name):
    return os.path.join(HERE, f"kl_target_{name}.json")


if __name__ == "__main__":
    argv = sys.argv[1:]
    cache = None
    if "--cache" in argv:
        i = argv.index("--cache")
        cache = argv[i + 1]
        del argv[i:i + 2]
        os.makedirs(cache, exist_ok=True)
    for name in argv or ["gauss10"]:
        out = compute(name, cache, log=lambda s: print(s, flush=True))
        with open(_target_file(name), "w") as f:
            json.dump(out, f, indent=1)
            f.write("\n")
        print(out, flush=True)
