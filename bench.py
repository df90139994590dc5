"""PixelSNE iterations/s on one GB300 (n = 1,000,000, D = 128, 2048^2 screen).

Workload ``gmm128``: 100-component anisotropic Gaussian mixture with Zipf(1.1)
sizes, k = 90 neighbours, perplexity 30, theta 0.5, 2^11 x 2^11 screen.
A step is one gradient iteration of the method (tree, Barnes-Hut repulsion,
attraction, Z, update with screen rescale).  P is built once before timing
(its time is reported separately, like the paper's P / Coord split).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  Timed region: K iterations from t = 0 of the schedule
(exaggeration 12 for 250 iterations), CUDA events on the library's stream,
barrier + synchronize on both sides, max over ranks.  Every iteration streams
P (about 1 GB), so the inputs exceed the 129 MB L2.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# The headline workload (the default) and the scale workload (100-component
# 128-D mixture at n = 1M on 2048^2; 256-component 64-D mixture with 1 %
# outliers at n = 10M on 4096^2).
WORKLOADS = {
    "gmm128": (dict(workload="gmm128", n=1_000_000, D=128, k=90, perplexity=30.0, log2_r=11,
                    theta=0.5, iterations=1000),
               "t-SNE iterations/sec at n=1M, 2048^2 screen"),
    "gmm64out": (dict(workload="gmm64out", n=10_000_000, D=64, k=90, perplexity=30.0,
                      log2_r=12, theta=0.5, iterations=1000),
                 "t-SNE iterations/sec at n=10M, 4096^2 screen (scale workload)"),
}
WORKLOAD, METRIC = WORKLOADS["gmm128"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="gmm128", choices=sorted(WORKLOADS))
    ap.add_argument("--n", type=int, default=None, help="points (debug only)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-studies", action="store_true",
                    help="skip the time-to-KL-target and screen-size studies")
    ap.add_argument("--no-warmstart", action="store_true",
                    help="skip the learned warm-start experiment")
    ap.add_argument("--warm-seeds", type=int, default=20)
    ap.add_argument("--warm-n", type=int, default=50000)
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x, dist, device):
    """The largest of the ranks' values of x (x itself without a process
    group): the job's time is its slowest replica's."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, seconds, ws):
    """Whole-job throughput of ws replicas that each processed units_per_rank
    units, timed as the slowest replica's seconds."""
    return ws * units_per_rank / seconds


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
            out, _ = self.p.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- workload
def draw(seed, n):
    import datagen
    return getattr(datagen, WORKLOAD["workload"])(seed=seed, n=n)[0]


def make_inputs(n, seed=0):
    import datagen
    return draw(seed, n), datagen.init_y0(seed, n)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# Algorithmic bytes (HBM) per launch of each kernel group, and FLOPs of the
# traversal per tested / accepted (point, cell) pair.
RELABEL_EVERY = 100  # the library refreshes the attraction's relabelled P this often


def group_bytes(n, nnz, L, nonempty=None, occupied=None):
    """Bytes each kernel group must move per launch.  `nonempty`: cells of
    the tree holding at least one point (only their 16-byte records are
    written; every cell's count is), all cells when not given.  `occupied`:
    leaves holding at least one point (the histogram writes their count and
    sums, 20 B, and the pyramid clears them again), min(n, 4^L) when not
    given."""
    leaves = 4 ** L
    cells = (4 ** (L + 1) - 1) // 3
    nonempty = cells if nonempty is None else nonempty
    occupied = min(n, leaves) if occupied is None else occupied
    return {
        # per iteration on average: P read and written once per relabel, plus
        # the maps, row lengths, scan and positions
        "k_relabel": (nnz * 16 + n * (4 + 8 + 4 + 4 + 4 + 8 + 8 + 8 + 8)) / RELABEL_EVERY,
        "k_update": n * (8 + 8 + 8 + 8 + 8 + 8 + 8 + 16),      # z,Frep,Fattr,u,gains r; u,gains w; zhat w
        # perm, zhat, ainv r; z, rank, zp w; the occupied leaves' count and sums w
        "k_snap_hist": n * (4 + 16 + 8 + 4 + 4 + 8) + occupied * 20,
        # every leaf's count and sums r, leaf_start w, recn w, records of the
        # non-empty cells w, the occupied leaves cleared
        "k_pyr_pass": leaves * (20 + 4) + cells * 4 + nonempty * 16 + occupied * 20,
        "k_perm_scatter": n * (8 + 4 + 4 + 4),
        "k_bh_traverse": n * (4 + 8 + 8 + 4) + cells * 20,    # perm, z r; Frep, Zi w; rec + recn r
        "k_attract": nnz * 8 + (n + 1) * 8 + n * (8 + 4 + 8),
        "k_zsum": n * 4,
    }


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from an
# ncu capture of the current kernels, by (workload, n); emptied whenever a
# kernel changes, until the capture is taken again
TRAFFIC_BYTES = {("gmm128", 1_000_000): {"k_bh_traverse": 45.49e6 + 2.10e6}}
TRAFFIC_SOURCE = ("profiles/traversal_gmm128_n1M_dram.md (one-pass ncu capture of the "
                  "9th launch, t about 2)")

FLOP_TEST = 10    # offset, d^2 and criterion of one tested cell
FLOP_ACCEPT = 10  # kernel value, N w, N w^2 and the three accumulations
RECORD_BYTES = 20  # a cell's record: centre of mass (16 B) + count (4 B)


def synthetic_P(n, seed=0, per=135):
    """A P of the workload's shape for timing the oracle: `per` entries per row
    (90 neighbours + about 45 reverse edges at k = 90), uniform columns other
    than the row, values 1/(2 n 90).  The workload's exact P would need the
    oracle's O(n^2 D) neighbour search (hours at n = 1M)."""
    import oracle
    rng = np.random.default_rng(seed + 99)
    rp = np.arange(n + 1, dtype=np.int64) * per
    rows = np.repeat(np.arange(n, dtype=np.int64), per)
    col = ((rows + 1 + rng.integers(0, n - 1, size=n * per)) % n).astype(np.int32)
    val = np.full(n * per, 1.0 / (2 * n * 90))
    return oracle.CSR(rp, col, val)


def oracle_iterations(P, Y0, L, theta, min_seconds, max_iters, warmup=0):
    """Whole iterations of the oracle (tree, Barnes-Hut repulsion and
    attraction of every row, Z, update, rescale) from Y0, one at a time until
    min_seconds of CPU work or max_iters are done (after `warmup` untimed
    ones).  Returns (it/s, iterations, seconds)."""
    import oracle
    st = oracle.State.from_y0(Y0)
    params = oracle.Params(L=L, theta=theta)
    for _ in range(warmup):
        oracle.run(P, st, params, 1)
    wall, its = 0.0, 0
    while its < max(max_iters, 1) and (its == 0 or wall < min_seconds):
        t0 = time.perf_counter()
        oracle.run(P, st, params, 1)
        wall += time.perf_counter() - t0
        its += 1
    return its / wall, its, wall


def iterate_to_kl(ctx, target, chunk, max_iters, stream, torch):
    """Iterations and device seconds of pxsne_step until the KL (evaluated
    every `chunk` iterations, outside the timed region) is at most `target`."""
    ms, it, kl = 0.0, 0, float("inf")
    while it < max_iters:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.step(chunk)
        e1.record(stream)
        e1.synchronize()
        ms += e0.elapsed_time(e1)
        it += chunk
        kl = ctx.kl()
        if kl <= target:
            break
    return {"target": target, "reached": bool(kl <= target), "iterations": it,
            "seconds": ms / 1e3, "kl": kl, "checked_every": chunk}


def kl_target_study(px, ctx, Y0, kl_final, steps, stream, torch):
    """Wall time to a fixed KL target.

    - gauss10 (n = 2000, 512^2): the target is 1.01 x the oracle's KL after
      the full 500-iteration schedule, stored in tests/golden by a script that
      calls only the oracle.
    - the bench workload: 1.01 x the oracle's KL after its full schedule when
      it is stored (tests/golden/kl_target_gmm128_n1M.json, written by a
      script that calls only the oracle), else 1.01 x this run's own KL after
      the timed iterations.
    The GPU path runs from the same Y0 through the public calls."""
    import datagen
    with open(os.path.join(ROOT, "tests", "golden", "kl_target_gauss10.json")) as f:
        tgt = json.load(f)
    Xs, _ = datagen.gauss10(tgt["seed"])
    Ys = datagen.init_y0(tgt["seed"], Xs.shape[0])
    p = px.Params(log2_r=tgt["log2_r"], theta=tgt["theta"], k=tgt["k"],
                  perplexity=tgt["perplexity"])
    with px.Context(p, stream=stream.cuda_stream) as c:
        c.affinities(Xs)
        c.init(Ys)
        c.step(3)
        c.sync()
        c.init(Ys)
        small = iterate_to_kl(c, 1.01 * tgt["kl"], 10, 2 * tgt["iterations"], stream, torch)
    small.update({"workload": f"gauss10 n={tgt['n']} {1 << tgt['log2_r']}^2",
                  "target_from": f"1.01 x oracle KL after {tgt['iterations']} iterations "
                                 f"({tgt['kl']:.6f}, tests/golden/kl_target_gauss10.json)"})
    big = None
    n = Y0.shape[0]
    gold = os.path.join(ROOT, "tests", "golden",
                        f"kl_target_{WORKLOAD['workload']}_n{n // 1000000}M.json")
    if os.path.exists(gold) and n % 1000000 == 0:
        # the oracle's KL of the same workload and seed after the full schedule
        with open(gold) as f:
            g = json.load(f)
        ctx.init(Y0)
        big = iterate_to_kl(ctx, 1.01 * g["kl"], 25, 2 * g["iterations"], stream, torch)
        big.update({"workload": WORKLOAD["workload"],
                    "target_from": f"1.01 x oracle KL after {g['iterations']} iterations "
                                   f"({g['kl']:.6f}, tests/golden/{os.path.basename(gold)})"})
    elif steps >= WORKLOAD["iterations"]:
        # (only for a run of the whole schedule: early in it the KL is not
        # yet a convergence measure)
        ctx.init(Y0)
        big = iterate_to_kl(ctx, 1.01 * kl_final, 25, steps, stream, torch)
        big.update({"workload": WORKLOAD["workload"],
                    "target_from": f"1.01 x this run's KL after {steps} timed iterations "
                                   f"({kl_final:.6f})"})
    return {"small": small, "bench_workload": big}


def screen_sweep(px, X, Y0, params_kw, levels, iters, stream, torch):
    """Iterations/s of the same data and start on 2^L x 2^L screens (the tree
    is L levels deep, so a traversal costs O(n L)): t = 0 .. iters-1."""
    out = {}
    for L in levels:
        with px.Context(px.Params(log2_r=L, **params_kw), stream=stream.cuda_stream) as c:
            c.affinities(X)
            c.init(Y0)
            c.step(3)
            c.sync()
            c.init(Y0)
            c.sync()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            c.step(iters)
            e1.record(stream)
            e1.synchronize()
            c.sync()
            out[str(L)] = {"screen": f"{1 << L}^2", "it_per_s": iters / (e0.elapsed_time(e1) / 1e3),
                           "iterations": iters}
    return out


# The smaller workloads: (generator, n, screen, iterations, PCA dims)
SMALL_CONFIGS = {"gauss10": ("gauss10", 2000, 9, 500, None),
                 "protos784": ("protos784", 70000, 10, 1000, 50)}


def small_configs_study(px, stream, torch):
    """The whole method on the smaller workloads through the public calls: the
    10-Gaussian mixture (n = 2000, 512^2, 500 iterations) and the 784-D
    prototype data (n = 70,000, PCA to 50 on the GPU, 1024^2, 1000
    iterations): P construction time, iterations/s of the full schedule
    (CUDA events), final KL."""
    import datagen
    out = {}
    for name, (gen, n, L, iters, dpca) in SMALL_CONFIGS.items():
        X, _ = getattr(datagen, gen)(0, n=n)
        Y0 = datagen.init_y0(0, n)
        p = px.Params(log2_r=L, theta=0.5, k=90, perplexity=30.0)
        with px.Context(p, stream=stream.cuda_stream) as c:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            Xin = px.pca(X, dpca)[0] if dpca else X
            c.affinities(Xin)
            t_p = time.perf_counter() - t0
            c.init(Y0)
            c.step(3)
            c.sync()
            c.init(Y0)
            c.sync()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            c.step(iters)
            e1.record(stream)
            e1.synchronize()
            c.sync()
            out[name] = {"n": n, "screen": f"{1 << L}^2", "iterations": iters,
                         "pca": dpca, "p_construction_s": t_p,
                         "it_per_s": iters / (e0.elapsed_time(e1) / 1e3), "kl": c.kl()}
    return out


def geometric_centre_study(px, X, Y0, params_kw, steps, com, stream, torch):
    """The paper's own approximation of a cell by its geometric centre (Sec.
    4.1; the tree keeps counts only) on the same data, start and schedule as
    the timed centre-of-mass run `com` ({it_per_s, kl, precision_k10}): speed,
    final KL and neighbourhood precision, and the tree kernels' times."""
    with px.Context(px.Params(centre_mode=1, **params_kw), stream=stream.cuda_stream) as c:
        c.affinities(X)
        c.init(Y0)
        c.step(3)
        c.sync()
        c.init(Y0)
        c.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        c.step(steps)
        e1.record(stream)
        e1.synchronize()
        c.sync()
        out = {"it_per_s": steps / (e0.elapsed_time(e1) / 1e3), "kl": c.kl(),
               "precision_k10": c.nbr_precision(k=10), "iterations": steps}
        c.init(Y0)
        groups, _ = c.step_profiled(100)
        out["tree_ms_per_iteration"] = {g: groups[g] / 100 for g in ("k_snap_hist", "k_pyr_pass")}
    out["centre_of_mass"] = com
    return out


def variant_study(px, P3, Y0, params, steps, stream, torch):
    """The bench workload's P (row_ptr, col, val from the timed context) under
    other parameters: the same start, the same schedule length; iterations/s
    by CUDA events and the final KL."""
    with px.Context(params, stream=stream.cuda_stream) as c:
        c.set_P(*P3)
        c.init(Y0)
        c.step(3)
        c.sync()
        c.init(Y0)
        c.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        c.step(steps)
        e1.record(stream)
        e1.synchronize()
        assert c.sync() == 0
        return {"it_per_s": steps / (e0.elapsed_time(e1) / 1e3), "kl": c.kl(),
                "iterations": steps}


def approx_knn_study(px, ctx, X, params, n, probes=(256, 1024, (256, 2)), sample=20000):
    """P construction with the approximate neighbour search (knn_probe = W
    candidate tiles per query tile, optionally followed by R rounds of
    neighbour exploring, (W, R)) beside the exact one of ctx: P time, search
    time and the recall of the exact lists on a row sample."""
    import dataclasses
    rows = np.random.default_rng(5).choice(n, min(sample, n), replace=False)
    idx_e, _, _ = ctx.get_knn()
    exact = idx_e[rows]
    out = {"exact": {"knn_ms": ctx.knn_time_ms()}}
    for W in probes:
        W, R = W if isinstance(W, tuple) else (W, 0)
        p = dataclasses.replace(params, knn_probe=W, knn_explore=R)
        with px.Context(p) as c:
            import torch
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            c.affinities(X)
            tp = time.perf_counter() - t0
            idx, _, _ = c.get_knn()
            got = idx[rows]
            hits = sum(len(np.intersect1d(a, b, assume_unique=True)) for a, b in zip(got, exact))
            out[str(W) if R == 0 else f"{W}+explore{R}"] = {
                "p_construction_s": tp, "knn_ms": c.knn_time_ms(),
                "recall_vs_exact": hits / exact.size}
    out["sample_rows"] = int(len(rows))
    return out


def warmstart_experiment(px, ctx, X, Y0, args, torch):
    """Learned warm start, on ctx's P (the bench workload).

    Training data: embeddings the method produced for independent draws of the
    same mixture (args.warm_seeds draws of args.warm_n rows).  The first is the
    plain method from a random start; a network fitted to it predicts a start
    for every later draw, which the method refines without exaggeration, so all
    training layouts share one arrangement.  Each layout is normalised
    (centred, unit RMS) and rotated onto the network's prediction for the same
    points.  The final network, trained on all of them, predicts the start for
    this draw at the training layouts' RMS; the method refines it (no
    exaggeration) until the plain run's final KL.  Reports iterations and wall
    time (inference + refinement) against the plain run's, with KL and
    neighbourhood precision for both."""
    import datagen
    W = WORKLOAD
    n = X.shape[0]
    xs = np.float32(0.1)  # input scale of the network
    epochs = 30
    params = px.Params(log2_r=W["log2_r"], theta=W["theta"], k=W["k"],
                       perplexity=W["perplexity"])
    # plain run: 1,000 iterations of the full schedule from Y0
    ctx.set_schedule(exaggeration=12.0, exag_iters=250, momentum0=0.5, momentum1=0.8,
                     momentum_switch=250)
    ctx.init(Y0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx.step(1000)
    kl_plain = ctx.kl()
    t_plain = time.perf_counter() - t0
    prec_plain = ctx.nbr_precision(10)

    def rms(Y):
        Y = Y.astype(np.float64)
        Y = Y - Y.mean(0)
        return float(np.sqrt((Y ** 2).sum() / (2 * len(Y))))

    # training embeddings (chained through the first network)
    t0 = time.perf_counter()
    Xs, Ts, rr = [], [], []
    first = None
    for k in range(args.warm_seeds):
        sd = 1000 + k
        Xk = draw(sd, args.warm_n)
        with px.Context(params) as c2:
            c2.affinities(Xk)
            if first is None:
                c2.init(datagen.init_y0(sd, args.warm_n))
                c2.step(1000)
                Yk, _ = c2.get_Y(want_pix=False)
                Tk = px.embed_align(Yk)
                first = px.MLP(X.shape[1], seed=1)
                first.train(Xk * xs, Tk, epochs=epochs, batch=4096, lr=1e-3, seed=2)
            else:
                Pk = px.embed_align(first.predict(Xk * xs))
                c2.set_schedule(exag_iters=0, momentum_switch=0)
                c2.init((Pk * np.float32(rr[0])).astype(np.float32))
                c2.step(500)
                Yk, _ = c2.get_Y(want_pix=False)
                Tk = px.embed_align(Yk, Pk)
        rr.append(rms(Yk))
        Xs.append(Xk * xs)
        Ts.append(Tk)
    first.close()
    scale = float(np.mean(rr))
    t_data = time.perf_counter() - t0
    t0 = time.perf_counter()
    with px.MLP(X.shape[1], seed=3) as net:
        train_loss = net.train(np.concatenate(Xs), np.concatenate(Ts), epochs=epochs,
                               batch=4096, lr=1e-3, seed=2)
        t_train = time.perf_counter() - t0
        torch.cuda.synchronize()
        # warm start: inference + refinement until the plain run's final KL
        t0 = time.perf_counter()
        Yw = net.predict(X * xs) * np.float32(scale)
        ctx.set_schedule(exag_iters=0, momentum_switch=0)
        ctx.init(Yw.astype(np.float32))
        kl0 = ctx.kl()
        it, kl = 0, kl0
        while kl > kl_plain and it < 1000:
            ctx.step(25)
            it += 25
            kl = ctx.kl()
        t_warm = time.perf_counter() - t0
    reached = kl <= kl_plain
    prec_warm = ctx.nbr_precision(10)
    # and where a further 250 refinement iterations take it
    ctx.step(250)
    kl_more = ctx.kl()
    prec_more = ctx.nbr_precision(10)
    return {"plain": {"iterations": 1000, "kl": kl_plain, "wall_s": t_plain,
                      "precision_k10": prec_plain},
            "warm": {"iterations_to_plain_kl": it if reached else None, "reached": reached,
                     "kl_at_start": kl0, "kl": kl, "wall_s_to_plain_kl": t_warm,
                     "precision_k10": prec_warm, "kl_after_250_more": kl_more,
                     "precision_k10_after_250_more": prec_more,
                     "wall_ratio_plain_over_warm": t_plain / t_warm if reached else None},
            "training": {"embeddings": args.warm_seeds, "rows_each": args.warm_n,
                         "epochs": epochs, "data_s": t_data, "train_s": t_train,
                         "final_mse": train_loss, "start_rms": scale},
            "schedule": "warm: no exaggeration, momentum 0.8, eta 200, gains reset; start "
                        "at the training layouts' RMS"}


REF_BUDGET_S = 120.0  # the reference arm's timed CPU work, whatever K is


def run_reference(args):
    """The oracle (plain FP64 C, OpenMP) as the reference arm on the host
    cores, on a synthetic P of the workload's shape.  Each step is one whole
    iteration when K of them fit in REF_BUDGET_S; otherwise each step is the
    per-row work of an iteration (Barnes-Hut repulsion and attraction) for a
    block of rows of the current state, sized so that the K steps fit, and the
    line's value counts the rows done as whole-iteration equivalents (rows
    processed / n per second)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    import datagen
    n = args.n
    Y0 = datagen.init_y0(0, n)
    L = WORKLOAD["log2_r"]
    P = synthetic_P(n)
    st = oracle.State.from_y0(Y0)
    params = oracle.Params(L=L, theta=WORKLOAD["theta"])
    t_iter = None
    for w in range(max(args.warmup, 1)):
        t0 = time.perf_counter()
        oracle.run(P, st, params, 1)
        t_iter = time.perf_counter() - t0
    steps = max(args.steps, 1)
    if steps * t_iter <= REF_BUDGET_S:
        t0 = time.perf_counter()
        oracle.run(P, st, params, steps)
        wall = time.perf_counter() - t0
        value = steps / wall
        rows = n
        sample = (f"{steps} whole iterations at n={n} from Y0 after {max(args.warmup, 1)} "
                  f"untimed ones (tree, Barnes-Hut and attraction of every row, Z, update, "
                  f"rescale), on a synthetic P of the workload's shape (135 uniform columns "
                  f"per row)")
    else:
        rows = max(256, min(n, int(n * REF_BUDGET_S / (steps * t_iter))))
        order = np.random.default_rng(9).permutation(n).astype(np.int64)
        tree = oracle.pyramid(st.z, L)
        t0 = time.perf_counter()
        for k in range(steps):
            a = (k * rows) % n
            r = order[a:a + rows] if a + rows <= n else np.concatenate(
                [order[a:], order[:a + rows - n]])
            oracle.bh_repulsion(st.z, st.s, L, WORKLOAD["theta"], rows=r, tree=tree)
            oracle.attraction(P, st.z, st.s, rows=r)
        wall = time.perf_counter() - t0
        value = steps * rows / n / wall
        sample = (f"{steps} steps, each the Barnes-Hut repulsion and attraction of {rows} "
                  f"rows of n={n} (a whole iteration's per-row work, {100.0 * rows / n:.1f} "
                  f"% of the rows; the tree of the state after {max(args.warmup, 1)} whole "
                  f"iterations built once, untimed); value = rows processed / n per "
                  f"second; a whole iteration took {t_iter:.2f} s")
    cores = oracle.num_threads()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "it/s",
            "n_gpus": args.gpus, "steps": steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * wall / steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {k: WORKLOAD[k] for k in WORKLOAD} | {"n": n},
            "cpu_baseline": {"value": value, "unit": "it/s", "cores": cores, "kind": "oracle",
                             "sample": sample, "rows_per_step": rows},
            "e2e": {"value": value, "unit": "it/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args):
    import torch
    ws, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_1611_02568_gb300 as px
    from paper_1611_02568_gb300 import build as pxbuild
    if rank == 0 or ws == 1:
        pxbuild.build()
    if dist:
        dist.barrier()

    n = args.n
    W = WORKLOAD
    X, Y0 = make_inputs(n, seed=rank)
    stream = torch.cuda.Stream()
    # the L2 and FP32 peaks of this GPU, measured before anything else runs
    mpeaks = px.measure_peaks(stream.cuda_stream)
    params = px.Params(log2_r=W["log2_r"], theta=W["theta"], k=W["k"],
                       perplexity=W["perplexity"])
    ctx = px.Context(params, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx.affinities(X)
    p_seconds = time.perf_counter() - t0
    n_, nnz = ctx.sizes()
    # the one dense contraction: q.c for every (query, candidate) pair on the
    # tensor cores, 2 n^2 D FLOP, against the measured dense bf16 peak (FP16 and
    # bf16 share the tensor rate)
    knn_ms = ctx.knn_time_ms()
    kx, ki, kpath = ctx.knn_counters()
    kskip, kpairs = ctx.knn_pruning()
    # the products the tensor cores actually formed: the (query tile,
    # candidate tile) pairs of 128 x 128 rows not skipped by the tile bound,
    # 2 * 128 * 128 * Dp FLOP each (rows padded to the tiles, D to Dp)
    Dp = (X.shape[1] + 63) // 64 * 64
    knn_dense = 2.0 * n * n * X.shape[1]
    knn_flop = (kpairs - kskip) * 2.0 * 128 * 128 * Dp if kpairs else knn_dense
    pk, pk_kind = measured_peaks()
    knn = {"kernel": "k_knn_tc" if kpath == 1 else "k_knn_tile", "ms": knn_ms,
           "bound": "tensor", "achieved": knn_flop / (knn_ms / 1e3) / 1e12,
           "peak": pk["bf16_tflops"], "unit": "TFLOP/s",
           "frac": knn_flop / (knn_ms / 1e3) / 1e12 / pk["bf16_tflops"],
           "dense_equivalent_tflops": knn_dense / (knn_ms / 1e3) / 1e12,
           "peak_source": f"bf16_tflops of MEASURED_PEAKS.json ({pk_kind})",
           "exact_rerank_per_row": kx / n, "insertions_per_row": ki / n,
           "tile_pairs_skipped": kskip / kpairs if kpairs else None}
    knn_approx = None
    if rank == 0 and not args.no_studies:
        knn_approx = approx_knn_study(px, ctx, X, params, n)
    ctx.init(Y0)
    ctx.step(max(args.warmup, 3) if args.warmup >= 0 else 3)  # graph capture + warm-up
    ctx.sync()
    ctx.init(Y0)                                              # timed run starts at t = 0
    ctx.sync()

    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    # events every 100 iterations as well (recorded on the same stream between
    # graph launches): the cost of an iteration along the schedule
    chunk = 100
    marks = [torch.cuda.Event(enable_timing=True)]
    marks[0].record(stream)
    done = 0
    while done < args.steps:
        c = min(chunk, args.steps - done)
        ctx.step(c)
        done += c
        marks.append(torch.cuda.Event(enable_timing=True))
        marks[-1].record(stream)
    marks[-1].synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = marks[0].elapsed_time(marks[-1])
    along = [{"t": f"{chunk * q}..{min(chunk * (q + 1), args.steps) - 1}",
              "ms_per_iteration": marks[q].elapsed_time(marks[q + 1]) /
              (min(chunk * (q + 1), args.steps) - chunk * q)} for q in range(len(marks) - 1)]
    ctx.sync()
    ms = max_over_ranks(ms, dist, "cuda")
    value = job_rate(args.steps, ms / 1000.0, ws)
    kl_after = ctx.kl()
    prec_after = ctx.nbr_precision(k=10)

    # per-kernel breakdown: the same K iterations again from t = 0, with CUDA
    # events around each kernel group on the library's stream
    ctx.init(Y0)
    groups, prof_total = ctx.step_profiled(args.steps)
    # (the traversal's work counters: sums over the K profiled iterations)
    acc, tst, wsteps, nodes = ctx.counters()
    lvc = ctx.level_counters()
    peaks, peak_kind = measured_peaks()
    # non-empty cells of the final state (only their records are written)
    occ = [int(np.count_nonzero(ctx.get_tree(l)[0])) for l in range(W["log2_r"] + 1)]
    gb = group_bytes(n, nnz, W["log2_r"], sum(occ), occ[-1])
    traffic = TRAFFIC_BYTES.get((W["workload"], n), {})
    top = max(groups, key=groups.get)
    avg_ms = {g: v / args.steps for g, v in groups.items()}
    if top == "k_bh_traverse":
        # FLOPs of the tested and accepted (point, cell) pairs of all K
        # iterations over the traversal's summed time, against the FP32 rate
        # measured in this process (packed pairs, the traversal's form)
        flops = FLOP_TEST * tst + FLOP_ACCEPT * acc
        sec = groups[top] / 1e3
        achieved = flops / sec / 1e12
        fp32 = max(mpeaks["fp32_tflops"], mpeaks["fp32_packed_tflops"])
        l2_alg = RECORD_BYTES * tst / sec / 1e9
        roof = {"kernel": top, "bound": "alu", "achieved": achieved, "peak": fp32,
                "unit": "TFLOP/s", "frac": achieved / fp32,
                "traffic": traffic.get(top),
                "peak_source": "measured in this run by pxsne_measure_peaks (FP32 FMA "
                               "chains, packed pairs; see measured_peaks)",
                "work": f"{FLOP_TEST} FLOP per tested + {FLOP_ACCEPT} per accepted "
                        f"(point, cell) pair, summed over the {args.steps} profiled "
                        f"iterations",
                "l2": {"achieved": l2_alg, "peak": mpeaks["l2_read_gbs"], "unit": "GB/s",
                       "frac": l2_alg / mpeaks["l2_read_gbs"],
                       "work": f"{RECORD_BYTES} B of cell record per tested (point, cell) "
                               f"pair (the per-pair record model, n I x 20 B; a warp loads each "
                               f"record once for all its points, so the loads it issues "
                               f"are the warp steps' records, below)",
                       "warp_loads_GBps": nodes * 80 / sec / 1e9,
                       "warp_loads_work": "80 B per node popped (the four children's "
                                          "records and counts, one load each per warp)"}}
    else:
        achieved = gb[top] / (avg_ms[top] / 1e3) / 1e9
        roof = {"kernel": top, "bound": "hbm", "achieved": achieved,
                "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": traffic.get(top),
                "peak_source": f"hbm_gbs of MEASURED_PEAKS.json ({peak_kind})"}
    roof["traffic_source"] = (TRAFFIC_SOURCE if roof["traffic"] is not None else
                              "no ncu capture of the current kernel at this size")
    kernels = {g: {"ms_per_launch": avg_ms[g], "share": groups[g] / sum(groups.values()),
                   "alg_GBps": gb[g] / (avg_ms[g] / 1e3) / 1e9 if avg_ms[g] > 0 else None,
                   "hbm_frac": gb[g] / (avg_ms[g] / 1e3) / 1e9 / peaks["hbm_gbs"]
                   if avg_ms[g] > 0 else None}
               for g in groups}

    # end to end through the public API with host buffers: P from pinned host
    # X, init from host Y0, then every iteration pxsne_step(1) and the frame a
    # screen would draw (the pixel coordinates) read back to pinned host
    # memory: the frame is written into one of two device buffers without a
    # host synchronisation, and copied to one of two pinned host buffers on a
    # copy stream while the next iteration runs; the host waits for frame t's
    # copy before it reuses that buffer two iterations later, and for the last
    # one before the clock stops
    e2e = None
    if not args.no_e2e:
        Xp = torch.from_numpy(X).pin_memory()
        Y0p = torch.from_numpy(Y0).pin_memory()
        Ph = [torch.empty((n, 2), dtype=torch.int32).pin_memory() for _ in range(2)]
        Pd = [torch.empty((n, 2), dtype=torch.int32, device="cuda") for _ in range(2)]
        copy_stream = torch.cuda.Stream()
        done = [None, None]
        ctx2 = px.Context(params, stream=stream.cuda_stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        ctx2.affinities(Xp)
        ctx2.init(Y0p)
        for it in range(args.steps):
            b = it & 1
            if done[b] is not None:
                done[b].synchronize()     # frame it - 2 is on the host
            ctx2.step(1)
            ctx2.get_Y(None, Pd[b], blocking=False)
            ready = torch.cuda.Event()
            ready.record(stream)
            copy_stream.wait_event(ready)
            with torch.cuda.stream(copy_stream):
                Ph[b].copy_(Pd[b], non_blocking=True)
                done[b] = torch.cuda.Event()
                done[b].record(copy_stream)
        for ev in done:
            if ev is not None:
                ev.synchronize()
        assert ctx2.sync() == 0
        t1 = time.perf_counter()
        el = max_over_ranks(t1 - t0, dist, "cuda")
        ctx2.close()
        e2e = {"value": job_rate(args.steps, el, ws), "unit": "it/s",
               "h2d_bytes_per_step": int((X.nbytes + Y0.nbytes) / args.steps),
               "d2h_bytes_per_step": int(Ph[0].numel() * 4),
               "wall_s": el, "includes": "P construction + init + K x (step + the pixel "
                                         "coordinates read back to pinned host memory, "
                                         "each copy overlapping the next step)"}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        cores = oracle.num_threads()

        Pc = synthetic_P(n)
        # whole iterations from Y0 until about 10 s of CPU work (at least one)
        v, its, w = oracle_iterations(Pc, Y0, W["log2_r"], W["theta"], 10.0, 50)
        cpu = {"value": v, "unit": "it/s", "cores": cores, "kind": "oracle",
               "sample": (f"{its} whole iterations from Y0 at n={n} (tree, Barnes-Hut and "
                          f"attraction of every row, Z, update, rescale; {w:.1f} s of CPU "
                          f"work) on a synthetic P of the workload's shape (135 uniform "
                          f"columns per row)")}
        # the same on one thread (the paper times its CPU code single-threaded)
        oracle.set_num_threads(1)
        try:
            v1, its1, w1 = oracle_iterations(Pc, Y0, W["log2_r"], W["theta"], 8.0, 50)
        finally:
            oracle.set_num_threads(cores)
        del Pc
        # the oracle on the smaller workloads, whole iterations the same way
        import datagen
        cpu["small_configs"] = {}
        for name, (gen, nn, LL, _, _) in SMALL_CONFIGS.items():
            Ys = datagen.init_y0(0, nn)
            vv, itv, _ = oracle_iterations(synthetic_P(nn), Ys, LL, W["theta"], 3.0, 200)
            cpu["small_configs"][name] = {"value": vv, "unit": "it/s", "cores": cores,
                                          "n": nn, "iterations": itv}
        cpu["one_thread"] = {"value": v1, "unit": "it/s", "cores": 1,
                             "sample": f"{its1} whole iterations from Y0 at n={n} ({w1:.1f} s "
                                       f"of CPU work), same synthetic P"}

    studies = None
    if rank == 0 and not args.no_studies:
        studies = {
            "time_to_kl": kl_target_study(px, ctx, Y0, kl_after, args.steps, stream, torch),
            "geometric_centre": geometric_centre_study(
                px, X, Y0, dict(log2_r=W["log2_r"], theta=W["theta"], k=W["k"],
                                perplexity=W["perplexity"]), args.steps,
                {"it_per_s": value, "kl": kl_after, "precision_k10": prec_after,
                 "tree_ms_per_iteration": {g: avg_ms[g] for g in ("k_snap_hist", "k_pyr_pass")}},
                stream, torch) if n <= 2_000_000 else None,
            "small_configs": small_configs_study(px, stream, torch),
            # (P is rebuilt for every screen: skipped for the 10M scale workload)
            "screen_sweep": screen_sweep(
                px, X, Y0, dict(theta=W["theta"], k=W["k"], perplexity=W["perplexity"]),
                [W["log2_r"] - 2, W["log2_r"] - 1, W["log2_r"], W["log2_r"] + 1,
                 W["log2_r"] + 2], 300, stream, torch) if n <= 2_000_000 else None}
        if n <= 2_000_000:
            import datagen
            P3 = ctx.get_P()
            kw = dict(theta=W["theta"], k=W["k"], perplexity=W["perplexity"])
            L = W["log2_r"]
            # an r_1 x r_2 screen of 4:3 on the same 2^L root (Sec. 4.2's r_d)
            rx, ry = 1 << L, 3 << (L - 2)
            studies["nonsquare_screen"] = dict(
                screen=f"{rx}x{ry}", square_it_per_s=value, square_kl=kl_after,
                **variant_study(px, P3, Y0, px.Params(log2_r=L, screen_x=rx, screen_y=ry, **kw),
                                args.steps, stream, torch))
            # the 3-D embedding on a 256^3 voxel grid (octree), its own 3-D start
            studies["dim3"] = dict(
                grid="256^3", kl_2d=kl_after,
                **variant_study(px, P3, datagen.init_y0(0, n, dim=3),
                                px.Params(log2_r=8, dim=3, **kw), args.steps, stream, torch))

    warm = None
    if rank == 0 and not args.no_warmstart:
        try:
            warm = warmstart_experiment(px, ctx, X, Y0, args, torch)
        except Exception as ex:  # the experiment must not take the bench line down
            warm = {"error": repr(ex)}

    ctx.close()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "it/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {k: W[k] for k in W} | {"n": n, "nnz": nnz,
                                              "parallelism": "replicas" if ws > 1 else "single",
                                              "l2": f"inputs larger than L2 (P "
                                                    f"{nnz * 8 / 1e9:.1f} GB read per iteration)",
                                              "timed_iterations": f"t = 0..{args.steps - 1}"},
            "roofline": roof, "kernels": kernels, "measured_peaks": mpeaks,
            "traversal": {"accepted_pairs": acc, "tested_pairs": tst,
                          "accepted_per_point": acc / n / args.steps,
                          "tested_per_point": tst / n / args.steps,
                          "warp_steps": wsteps, "nodes": nodes,
                          "lanes_per_step": tst / wsteps if wsteps else None,
                          "iterations": args.steps,
                          "by_level": {str(l): {"tested_per_point": int(lvc[l, 0]) / n / args.steps,
                                                "accepted_per_point": int(lvc[l, 1]) / n / args.steps,
                                                "lanes_per_step": int(lvc[l, 0]) / int(lvc[l, 2])}
                                       for l in range(1, lvc.shape[0]) if lvc[l, 2]}},
            "profiled_total_ms": prof_total, "p_construction_s": p_seconds, "knn": knn,
            "knn_approx": knn_approx,
            "along_schedule": along,
            "kl_after_timed": kl_after,
            "clocks": ck, "e2e": e2e, "cpu_baseline": cpu, "warmstart": warm,
            "studies": studies,
            # per iteration: update, snap_hist, the pyramid (one launch for
            # 5 <= L <= 12), perm_scatter, traverse, attract, zsum; per relabel
            # (before every RELABEL_EVERY-th iteration): maps, three scan
            # kernels, rows
            "gpu_launches": args.steps * 7 + 5 * ((args.steps - 1) // RELABEL_EVERY),
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    global WORKLOAD, METRIC
    args = parse()
    WORKLOAD, METRIC = WORKLOADS[args.workload]
    if args.n is None:
        args.n = WORKLOAD["n"]
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
