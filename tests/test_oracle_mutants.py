"""Planted mistakes in the oracle are caught by its pins.

Each case below plants one plausible mistake in a scratch copy of the oracle:
a dropped term, a wrong sign, index or operand, a swapped axis, a missing
normalisation.  The copy is built, and ``tests/test_oracle_pins.py`` is run
against it in a child process.  At least one pin must fail, as a reported
test failure and not as a crash.  An unmodified copy must pass the same run.
The oracle in the repository is never modified.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
C_SRC = "oracle/pxsne_oracle.c"
PY_SRC = "oracle/__init__.py"

# (what the mistake is, file, text in the oracle, text planted instead)
MUTANTS = [
    # kNN (Sec. 3.3)
    ("knn: ties broken towards the higher index", C_SRC,
     "da < db || (da == db && ja < jb)", "da < db || (da == db && ja > jb)"),
    ("knn: the point itself not excluded", C_SRC,
     "if (j == i) continue;\n            const float *xj", "const float *xj"),
    ("knn: first coordinate dropped from the distance", C_SRC,
     "for (int32_t d = 0; d < D; d++) {", "for (int32_t d = 1; d < D; d++) {"),
    ("knn: absolute differences summed, not squares", C_SRC,
     "s += t * t;", "s += fabs(t);"),
    ("knn: sampled rows ignored", C_SRC,
     "int64_t i = rows ? rows[q] : q;\n        if (i < 0", "int64_t i = q;\n        if (i < 0"),
    # perplexity bisection (Sec. 3.2)
    ("perplexity: entropy with the wrong sign on the mean term", C_SRC,
     "H = log(sum) + beta * hs / sum;", "H = log(sum) - beta * hs / sum;"),
    ("perplexity: target entropy in bits", C_SRC,
     "const double target = log(perplexity);", "const double target = log2(perplexity);"),
    ("perplexity: bracket moved the wrong way", C_SRC,
     "if (H > target) { /* too flat: sharpen */", "if (H < target) { /* too flat: sharpen */"),
    ("perplexity: bisection started at beta = 0", C_SRC,
     "double beta = 1.0, lo = 0.0, hi = 0.0;", "double beta = 0.0, lo = 0.0, hi = 0.0;"),
    ("perplexity: row minimum left in the mean term", C_SRC,
     "hs += (d[j] - dmin) * e;", "hs += d[j] * e;"),
    ("perplexity: stop test a hundred times too loose", C_SRC,
     "if (fabs(H - target) < tol) { ok = 1; break; }",
     "if (fabs(H - target) < 100 * tol) { ok = 1; break; }"),
    ("perplexity: rows not normalised", C_SRC,
     "for (int32_t j = 0; j < k; j++) p[j] /= sum;", ""),
    # symmetrisation (Sec. 3.3)
    ("symmetrize: divided by n instead of 2n", C_SRC,
     "val[nnz] = v / (2.0 * (double)n);", "val[nnz] = v / (double)n;"),
    ("symmetrize: columns left unsorted within a row", C_SRC,
     "    if (x->c != y->c) return x->c < y->c ? -1 : 1;\n", ""),
    ("symmetrize: transposed entry not added", C_SRC,
     "t[o].r = j; t[o].c = (int32_t)i;", "t[o].r = i; t[o].c = j;"),
    # screen map (Eq. z1/z2)
    ("init: extremes taken over the other axis", C_SRC,
     "double v = Y0[dim * i + d];", "double v = Y0[dim * i + (1 - d)];"),
    ("init: ceiling in place of the floor", C_SRC,
     "double q = floor((Y0[dim * i + d] - mn) * Rd / range);",
     "double q = ceil((Y0[dim * i + d] - mn) * Rd / range);"),
    ("init: extent of the other axis", C_SRC,
     "const double Rd = R[d];", "const double Rd = R[1 - d];"),
    ("init: zero-extent axis off the origin", C_SRC,
     "for (int64_t i = 0; i < n; i++) z[dim * i + d] = 0u;",
     "for (int64_t i = 0; i < n; i++) z[dim * i + d] = 1u;"),
    # tree (Sec. 4.1)
    ("morton: x and y bits swapped", C_SRC,
     "m |= ((px >> b) & 1u) << (2 * b);\n        m |= ((py >> b) & 1u) << (2 * b + 1);",
     "m |= ((py >> b) & 1u) << (2 * b);\n        m |= ((px >> b) & 1u) << (2 * b + 1);"),
    ("leaf keys: x and y pixels swapped", C_SRC,
     "uint32_t x = z[2 * i] >> F, y = z[2 * i + 1] >> F;",
     "uint32_t y = z[2 * i] >> F, x = z[2 * i + 1] >> F;"),
    ("level offsets shifted by one", C_SRC,
     "return (((int64_t)1 << (2 * l)) - 1) / 3;", "return (((int64_t)1 << (2 * l)) + 2) / 3;"),
    ("pyramid: root level left empty", C_SRC,
     "for (int32_t l = 0; l <= L; l++) {\n            int64_t c = orc_level_offset(l)",
     "for (int32_t l = 1; l <= L; l++) {\n            int64_t c = orc_level_offset(l)"),
    ("pyramid: y sums accumulate x", C_SRC, "sy[c] += z[2 * i + 1];", "sy[c] += z[2 * i];"),
    ("pyramid: leaves one level too coarse", C_SRC,
     "uint32_t m = orc_morton(z[2 * i] >> F, z[2 * i + 1] >> F);",
     "uint32_t m = orc_morton(z[2 * i] >> (F + 1), z[2 * i + 1] >> (F + 1));"),
    # Barnes-Hut repulsion (Sec. 3.3, Eq. bh_criteria)
    ("bh: centre of mass without its remainder", C_SRC,
     "uint64_t q = S / N, r = S % N;", "uint64_t q = S / N, r = 0;"),
    ("bh: distance along x only", C_SRC,
     "double dd = dx * dx + dy * dy;\n            if (!leaf", "double dd = dx * dx;\n            if (!leaf"),
    ("bh: centre-of-mass remainder added, not subtracted", C_SRC,
     "- (double)r / (double)N;", "+ (double)r / (double)N;"),
    ("bh: own point left in the x sum of its leaf", C_SRC,
     "Sx -= zx;\n                Sy -= zy;\n            }", "Sy -= zy;\n            }"),
    ("bh: own point counted in its leaf", C_SRC,
     "N -= 1;\n                if (N == 0) continue;\n                Sx -= zx;\n                Sy -= zy;\n            }",
     "if (N == 0) continue;\n                Sx -= zx;\n                Sy -= zy;\n            }"),
    ("bh: own cells above the leaves left to the criterion", C_SRC,
     "int contains = ((mi >> (2 * (L - l))) == mc);",
     "int contains = leaf && ((mi >> (2 * (L - l))) == mc);"),
    ("bh: force missing one kernel factor", C_SRC,
     "fx += Nw * w * dx;\n            fy += Nw * w * dy;\n            acc++;",
     "fx += Nw * dx;\n            fy += Nw * w * dy;\n            acc++;"),
    ("bh: acceptance test reversed", C_SRC, "crit_mode == 0 ? (rc2 < th2 * dd)",
     "crit_mode == 0 ? (rc2 > th2 * dd)"),
    ("bh: cell size of the child level", C_SRC,
     "double rc2 = (s0 * W) * (s0 * W) + (s1 * W) * (s1 * W);",
     "double rc2 = 0.25 * ((s0 * W) * (s0 * W) + (s1 * W) * (s1 * W));"),
    ("bh: cell width along x instead of the diagonal", C_SRC,
     "double rc2 = (s0 * W) * (s0 * W) + (s1 * W) * (s1 * W);",
     "double rc2 = (s0 * W) * (s0 * W);"),
    ("bh: sampled rows ignored", C_SRC,
     "int64_t i = rows ? rows[q] : q;\n        const uint32_t zx = z[2 * i]",
     "int64_t i = q;\n        const uint32_t zx = z[2 * i]"),
    ("bh geometric: centre at the cell's corner", C_SRC,
     "((double)cx * W + 0.5 * W)", "((double)cx * W)"),
    ("bh geometric: x and y cell bits swapped", C_SRC,
     "cx |= ((mc >> (2 * b)) & 1u) << b;\n                    cy |= ((mc >> (2 * b + 1)) & 1u) << b;",
     "cy |= ((mc >> (2 * b)) & 1u) << b;\n                    cx |= ((mc >> (2 * b + 1)) & 1u) << b;"),
    # exact repulsion and attraction (Eq. grad)
    ("exact repulsion: w instead of w^2", C_SRC,
     "fx += w * w * dx;\n            fy += w * w * dy;\n        }",
     "fx += w * dx;\n            fy += w * w * dy;\n        }"),
    ("exact repulsion: a point counted against itself", C_SRC,
     "if (j == i) continue;\n            double dx = s0 * (double)((int64_t)z[2 * i] - (int64_t)z[2 * j]);\n"
     "            double dy = s1 * (double)((int64_t)z[2 * i + 1] - (int64_t)z[2 * j + 1]);\n"
     "            double w = 1.0 / (1.0 + dx * dx + dy * dy);\n            zs += w;",
     "double dx = s0 * (double)((int64_t)z[2 * i] - (int64_t)z[2 * j]);\n"
     "            double dy = s1 * (double)((int64_t)z[2 * i + 1] - (int64_t)z[2 * j + 1]);\n"
     "            double w = 1.0 / (1.0 + dx * dx + dy * dy);\n            zs += w;"),
    ("exact repulsion: sampled rows ignored", C_SRC,
     "int64_t i = rows ? rows[q] : q;\n        double fx = 0.0, fy = 0.0, zs = 0.0;",
     "int64_t i = q;\n        double fx = 0.0, fy = 0.0, zs = 0.0;"),
    ("attraction: sampled rows ignored", C_SRC,
     "int64_t i = rows ? rows[q] : q;\n        double fx = 0.0, fy = 0.0;\n",
     "int64_t i = q;\n        double fx = 0.0, fy = 0.0;\n"),
    ("attraction: kernel without the y offset", C_SRC,
     "double w = 1.0 / (1.0 + dx * dx + dy * dy);\n            fx += val[e]",
     "double w = 1.0 / (1.0 + dx * dx);\n            fx += val[e]"),
    ("exact repulsion: kernel without the y offset", C_SRC,
     "double w = 1.0 / (1.0 + dx * dx + dy * dy);\n            zs += w;",
     "double w = 1.0 / (1.0 + dx * dx);\n            zs += w;"),
    ("attraction: wrong sign", C_SRC,
     "fx += val[e] * w * dx;\n            fy += val[e] * w * dy;\n        }",
     "fx -= val[e] * w * dx;\n            fy += val[e] * w * dy;\n        }"),
    ("attraction: kernel squared", C_SRC,
     "fx += val[e] * w * dx;\n            fy += val[e] * w * dy;\n        }",
     "fx += val[e] * w * w * dx;\n            fy += val[e] * w * w * dy;\n        }"),
    # optimiser step (Eq. grad, BH-SNE's gains and momentum)
    ("update: exaggeration applied to repulsion too", C_SRC,
     "double g = 4.0 * (alpha * Fattr[k] - Frep[k] / Z);",
     "double g = 4.0 * alpha * (Fattr[k] - Frep[k] / Z);"),
    ("update: repulsion not normalised by Z", C_SRC,
     "double g = 4.0 * (alpha * Fattr[k] - Frep[k] / Z);",
     "double g = 4.0 * (alpha * Fattr[k] - Frep[k]);"),
    ("update: gains rule inverted", C_SRC, "(sgn(g) != sgn(u[k]))", "(sgn(g) == sgn(u[k]))"),
    ("update: minimum gain not applied", C_SRC, "if (gn < min_gain) gn = min_gain;", ""),
    ("update: step truncated, not rounded", C_SRC,
     "zhat[k] = (int64_t)z[k] + llrint(u[k] / s[d]);",
     "zhat[k] = (int64_t)z[k] + (int64_t)(u[k] / s[d]);"),
    ("update: momentum with the wrong sign", C_SRC,
     "u[k] = mu * u[k] - eta * gn * g;", "u[k] = -mu * u[k] - eta * gn * g;"),
    # the run's schedule (exaggeration and momentum phases)
    ("run: exaggeration one iteration too long", C_SRC,
     "orc_attraction(row_ptr, col, val, z, s, NULL, n, Fattr);\n        double alpha = t < p->exag_iters",
     "orc_attraction(row_ptr, col, val, z, s, NULL, n, Fattr);\n        double alpha = t <= p->exag_iters"),
    ("run: momentum phases swapped", C_SRC,
     "double mu = t < p->mom_switch ? p->mom0 : p->mom1;\n        orc_update(",
     "double mu = t < p->mom_switch ? p->mom1 : p->mom0;\n        orc_update("),
    ("run: centre mode not passed to the repulsion", C_SRC,
     "p->theta, p->crit_mode, p->centre_mode,\n                             cnt, sx, sy",
     "p->theta, p->crit_mode, 0,\n                             cnt, sx, sy"),
    ("run: criterion form not passed to the repulsion", C_SRC,
     "p->theta, p->crit_mode, p->centre_mode,\n                             cnt, sx, sy",
     "p->theta, 0, p->centre_mode,\n                             cnt, sx, sy"),
    ("run: screen rescale skipped", C_SRC, "        orc_rescale_screen(n, zhat, R, z, s);\n    }",
     "    }"),
    ("run: screen extent of y used for both axes", C_SRC,
     "const int32_t r[2] = {p->rx, p->ry};", "const int32_t r[2] = {p->ry, p->ry};"),
    ("run: screen extent a level too fine", C_SRC,
     "ldexp((double)r[d], 32 - p->L)", "ldexp((double)r[d], 31 - p->L)"),
    # screen rescale (Sec. 4.2, Eq. beta_scaling)
    ("rescale: compensation of s not applied", C_SRC,
     "s[d] = (s[d] * (double)gamma) / R[d];", ""),
    ("rescale: compensation by 2^32 whatever the screen", C_SRC,
     "s[d] = (s[d] * (double)gamma) / R[d];", "s[d] = (s[d] * (double)gamma) / 4294967296.0;"),
    ("rescale: extent of the other axis", C_SRC,
     "const uint64_t Rd = (uint64_t)R[d];", "const uint64_t Rd = (uint64_t)R[1 - d];"),
    ("rescale: both axes' extremes from x", C_SRC,
     "int64_t mn = zhat[d], mx = zhat[d];", "int64_t mn = zhat[0], mx = zhat[0];"),
    ("rescale: offset from the maximum", C_SRC,
     "(uint64_t)(zhat[dim * i + d] - mn) * Rd", "(uint64_t)(mx - zhat[dim * i + d]) * Rd"),
    # the 3-D embedding (octree)
    ("morton3: x bits taken from z", C_SRC,
     "m |= ((px >> b) & 1u) << (3 * b);", "m |= ((pz >> b) & 1u) << (3 * b);"),
    ("level_offset3: levels of four cells", C_SRC, "o += p; p *= 8; }", "o += p; p *= 4; }"),
    ("pyramid3: z sums accumulate y", C_SRC, "sz[c] += z[3 * i + 2];", "sz[c] += z[3 * i + 1];"),
    ("bh3: cell diagonal without the z axis", C_SRC,
     "double rc2 = (s0 * W) * (s0 * W) + (s1 * W) * (s1 * W) + (s2 * W) * (s2 * W);",
     "double rc2 = (s0 * W) * (s0 * W) + (s1 * W) * (s1 * W);"),
    ("bh3: distance along x and y only", C_SRC,
     "double dd = dx * dx + dy * dy + dz * dz;", "double dd = dx * dx + dy * dy;"),
    ("bh3: own voxel keeps the point's z", C_SRC, "                Sz -= zz;\n", ""),
    ("attraction3: z force from the y difference", C_SRC,
     "            fz += val[e] * w * dz;", "            fz += val[e] * w * dy;"),
    ("kl3: distance along x and y only", C_SRC,
     "double q = 1.0 / ((1.0 + dx * dx + dy * dy + dz * dz) * Z);",
     "double q = 1.0 / ((1.0 + dx * dx + dy * dy) * Z);"),
    ("update: coordinates strided by two whatever the dimension", C_SRC,
     "int64_t k = dim * i + d;", "int64_t k = 2 * i + d;"),
    ("rescale: extremes strided by two whatever the dimension", C_SRC,
     "int64_t v = zhat[dim * i + d];", "int64_t v = zhat[2 * i + d];"),
    # KL (Eq. cost_func)
    ("kl: q not normalised by Z", C_SRC,
     "double q = 1.0 / ((1.0 + dx * dx + dy * dy) * Z);",
     "double q = 1.0 / (1.0 + dx * dx + dy * dy);"),
    ("kl: distance along x only", C_SRC,
     "double q = 1.0 / ((1.0 + dx * dx + dy * dy) * Z);", "double q = 1.0 / ((1.0 + dx * dx) * Z);"),
    ("kl: ratio inverted", C_SRC,
     "double q = 1.0 / ((1.0 + dx * dx + dy * dy) * Z);\n            c += p * log(p / q);",
     "double q = 1.0 / ((1.0 + dx * dx + dy * dy) * Z);\n            c += p * log(q / p);"),
    ("kl: stored zeros of P not skipped", C_SRC,
     "if (p <= 0.0) continue;\n            int64_t j = col[e];\n            double dx = s0 * (double)((int64_t)z[2 * i]",
     "if (p < 0.0) continue;\n            int64_t j = col[e];\n            double dx = s0 * (double)((int64_t)z[2 * i]"),
    ("kl: Z of the tree replaced by the exact sum", C_SRC,
     "    if (p->exact) {\n        orc_exact_repulsion(z, s, n, NULL, n, Frep, Zi);\n    } else {",
     "    if (1) {\n        orc_exact_repulsion(z, s, n, NULL, n, Frep, Zi);\n    } else {"),
    # neighbourhood precision (Eq. nei_prec)
    ("nbr_precision: distance along x only", C_SRC,
     "double dd = dx * dx + dy * dy;\n            int32_t p;",
     "double dd = dx * dx;\n            int32_t p;"),
    ("nbr_precision: sampled rows ignored", C_SRC,
     "int64_t i = rows ? rows[q] : q;\n        int32_t *I", "int64_t i = q;\n        int32_t *I"),
    ("nbr_precision: all kh listed neighbours used, not the first k", C_SRC,
     "for (int32_t b = 0; b < k; b++)\n                if (knn_hd",
     "for (int32_t b = 0; b < kh; b++)\n                if (knn_hd"),
    ("nbr_precision: not divided by k", C_SRC,
     "return (double)hits / ((double)k * (double)m);", "return (double)hits / (double)m;"),
    # warm-start MLP
    ("gelu: Phi with the wrong scale", C_SRC,
     "return 0.5 * z * (1.0 + erf(z / sqrt(2.0))); }", "return 0.5 * z * (1.0 + erf(z / 2.0)); }"),
    ("mlp: bias b1 left out", C_SRC, "double s = b1[a];", "double s = 0.0;"),
    ("mlp: gradient of b3 missing", C_SRC, "gb3[o] += dy[o];", ""),
    ("gelu': missing factor z", C_SRC,
     "+ z * exp(-0.5 * z * z) / sqrt(2.0 * M_PI);", "+ exp(-0.5 * z * z) / sqrt(2.0 * M_PI);"),
    ("mlp: first layer's derivative taken at the second layer's input", C_SRC,
     "dz1[c] = dh * gelu_d(z1[c]);", "dz1[c] = dh * gelu_d(z2[c]);"),
    ("mlp: W2 not transposed in the backward pass", C_SRC,
     "dh += dz2[a] * W2[(size_t)a * H + c];", "dh += dz2[a] * W2[(size_t)c * H + a];"),
    ("mlp: loss gradient without the factor 2", C_SRC,
     "dy[o] = 2.0 * e / (double)m;", "dy[o] = e / (double)m;"),
    ("mlp: bias b2 left out", C_SRC, "double s = b2[a];", "double s = 0.0;"),
    # seeded start (Philox4x32-10 and Box-Muller)
    ("philox: key increments swapped", PY_SRC,
     "_PHILOX_W = (0x9E3779B9, 0xBB67AE85)", "_PHILOX_W = (0xBB67AE85, 0x9E3779B9)"),
    ("philox: high word of a product where the low one belongs", PY_SRC,
     "p1 & mask,", "(p1 >> np.uint64(32)) & mask,"),
    ("philox_y0: both uniforms from the first word", PY_SRC,
     "u2 = (w[:, 1] + 0.5)", "u2 = (w[:, 0] + 0.5)"),
    ("philox_y0: radius without its factor 2", PY_SRC,
     "rad = np.sqrt(-2.0 * np.log(u1))", "rad = np.sqrt(-np.log(u1))"),
    ("philox_y0: high half of the seed ignored", PY_SRC,
     "(seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)", "(seed & 0xFFFFFFFF, 0)"),
    # PCA (Sec. 5.1.1 pre-processing)
    ("pca: data not centred", PY_SRC, "Xc = Xd - mu\n", "Xc = Xd\n"),
    ("pca: smallest eigenvalues kept", PY_SRC,
     'order = np.argsort(-lam, kind="stable")[:dout]',
     'order = np.argsort(lam, kind="stable")[:dout]'),
]

COPY = ["oracle/__init__.py", C_SRC, "tests/conftest.py", "tests/test_oracle_pins.py",
        "tests/golden", "datagen"]


def _scratch(base, name):
    d = os.path.join(base, name)
    for rel in COPY:
        src, dst = os.path.join(ROOT, rel), os.path.join(d, rel)
        os.makedirs(os.path.dirname(dst), exist_ok=True)
        if os.path.isdir(src):
            shutil.copytree(src, dst, ignore=shutil.ignore_patterns("__pycache__", "_build"))
        else:
            shutil.copy(src, dst)
    return d


def _run_pins(d):
    env = dict(os.environ, OMP_NUM_THREADS="2", PYTHONDONTWRITEBYTECODE="1")
    env.pop("PYTHONPATH", None)
    p = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        "tests/test_oracle_pins.py"], cwd=d, env=env, capture_output=True,
                       text=True, timeout=900)
    return p.returncode, p.stdout[-3000:] + p.stderr[-2000:]


def test_pins_catch_planted_mistakes(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc is needed to build the oracle")
    pytest.importorskip("sklearn")
    jobs = [("control", None)]
    for i, (what, rel, old, new) in enumerate(MUTANTS):
        with open(os.path.join(ROOT, rel)) as f:
            text = f.read()
        assert text.count(old) == 1, f"{what}: the planted text must occur once in {rel}"
        jobs.append((what, (rel, text.replace(old, new))))
    dirs = []
    for i, (what, edit) in enumerate(jobs):
        d = _scratch(str(tmp_path), f"m{i:02d}")
        if edit is not None:
            rel, text = edit
            with open(os.path.join(d, rel), "w") as f:
                f.write(text)
        dirs.append(d)
    workers = max(1, min(8, (os.cpu_count() or 2) // 2))
    with ThreadPoolExecutor(workers) as ex:
        results = list(ex.map(_run_pins, dirs))
    rc0, out0 = results[0]
    assert rc0 == 0, "the unmodified copy must pass its pins:\n" + out0
    missed = [(what, rc, out) for (what, _), (rc, out) in zip(jobs[1:], results[1:])
              if rc != 1 or "failed" not in out]
    assert not missed, "\n\n".join(f"{w} (exit {rc}):\n{o[-1500:]}" for w, rc, o in missed)
