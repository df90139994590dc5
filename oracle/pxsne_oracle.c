/*
 * PixelSNE CPU oracle (FP64, plain C).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * statement of what the CUDA path computes.  Only the test-suite, the smoke
 * check and the bench's CPU-baseline leg load it.  It shares no code, header,
 * table or constant with the CUDA library, and it includes none of it.
 *
 * Every function follows the paper (Kim et al., "PixelSNE: Visualizing Fast
 * with Just Enough Precision via Pixel-Aligned Stochastic Neighbor
 * Embedding", arXiv 1611.02568) and cites the passage it follows.
 *
 * Conventions (the readings of the paper that this oracle implements):
 *  - Screen r_1 x r_2 pixels with r_d <= 2^L (Sec. 4.2's per-axis r_d): the
 *    quadtree's root is the padded square of 2^L x 2^L pixels.  Positions are
 *    fixed point: z_d is a u32 in [0, R_d) ulps with R_d = r_d 2^F, F = 32 - L,
 *    and the pixel is z_d >> F (Eq. z1/z2); a square 2^L screen has
 *    R_d = 2^32.
 *  - y-space (t-SNE's own coordinates) is y_d = s_d * z_d (+ an offset that no
 *    quantity depends on).  s_d is the product of the per-iteration rescale
 *    factors, i.e. sqrt(beta_d) of Eq. beta_scaling, carried directly.
 *  - Morton index of a cell: x bits at even positions, y bits at odd ones.
 *    Cell (l, m) at level l covers the pixels whose top l bits of x and y
 *    give m; level offsets in a flattened pyramid are (4^l - 1) / 3.
 *  - Barnes-Hut criterion (Eq. bh_criteria) read as r_c / ||y_i - y_c|| < theta
 *    with r_c the cell's diagonal in y-units (the printed squared distance is
 *    kept as crit_mode 1).
 *  - The cell that contains point i is always opened; at a leaf, i is removed
 *    from its own cell's count and sums (Sec. 4.1 "leaf termination").
 */
#define _GNU_SOURCE
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_R 4294967296.0 /* 2^32 ulps per axis */

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.3 (sparse P, exact neighbour sets as the vantage-point tree gives):
 * the k nearest neighbours of x_i by squared Euclidean distance, self
 * excluded by index, ties broken towards the lower index.  Brute force over
 * all j in FP64 from the FP32 inputs.  rows == NULL means all n rows;
 * otherwise the m query rows listed.  Output rows are ascending. */
static int knn_before(double da, int32_t ja, double db, int32_t jb)
{
    return da < db || (da == db && ja < jb);
}

int orc_knn(const float *X, int64_t n, int32_t D, int32_t k,
            const int64_t *rows, int64_t m, int32_t *idx, double *d2)
{
    if (k < 1 || (int64_t)k >= n) return -1;
    int64_t err = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(| : err)
    for (int64_t q = 0; q < m; q++) {
        int64_t i = rows ? rows[q] : q;
        if (i < 0 || i >= n) { err |= 1; continue; }
        int32_t *I = idx + q * k;
        double *Dd = d2 + q * k;
        int32_t cnt = 0;
        const float *xi = X + i * (int64_t)D;
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            const float *xj = X + j * (int64_t)D;
            double s = 0.0;
            for (int32_t d = 0; d < D; d++) {
                double t = (double)xi[d] - (double)xj[d];
                s += t * t;
            }
            int32_t p;
            if (cnt < k) {
                p = cnt++;
            } else if (knn_before(s, (int32_t)j, Dd[k - 1], I[k - 1])) {
                p = k - 1;
            } else {
                continue;
            }
            while (p > 0 && knn_before(s, (int32_t)j, Dd[p - 1], I[p - 1])) {
                Dd[p] = Dd[p - 1];
                I[p] = I[p - 1];
                p--;
            }
            Dd[p] = s;
            I[p] = (int32_t)j;
        }
    }
    return err ? -2 : 0;
}

/* Sec. 3.2: the conditional p_{j|i} = exp(-beta_i d2_ij) / sum_j' exp(-beta_i d2_ij')
 * over the k neighbours, with beta_i found by bisection so that the entropy
 * H_i = -sum_j p_{j|i} ln p_{j|i} equals ln(perplexity).  Exponents are shifted
 * by the row's minimum distance (p is unchanged).  Start beta = 1; double or
 * halve until the target is bracketed, then bisect; stop when
 * |H - ln u| < tol or after max_iter evaluations.  Returns the number of
 * rows that did not converge. */
int64_t orc_perplexity(const double *d2, int64_t n, int32_t k, double perplexity,
                       double tol, int32_t max_iter, double *pcond,
                       double *beta_out, double *H_out)
{
    const double target = log(perplexity);
    int64_t bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad)
    for (int64_t i = 0; i < n; i++) {
        const double *d = d2 + i * k;
        double *p = pcond + i * k;
        double dmin = d[0];
        for (int32_t j = 1; j < k; j++)
            if (d[j] < dmin) dmin = d[j];
        double beta = 1.0, lo = 0.0, hi = 0.0;
        int has_lo = 0, has_hi = 0, ok = 0;
        double H = 0.0;
        for (int32_t it = 0; it < max_iter; it++) {
            double sum = 0.0, hs = 0.0;
            for (int32_t j = 0; j < k; j++) {
                double e = exp(-beta * (d[j] - dmin));
                sum += e;
                hs += (d[j] - dmin) * e;
            }
            H = log(sum) + beta * hs / sum;
            if (fabs(H - target) < tol) { ok = 1; break; }
            if (H > target) { /* too flat: sharpen */
                lo = beta; has_lo = 1;
                beta = has_hi ? 0.5 * (beta + hi) : 2.0 * beta;
            } else {
                hi = beta; has_hi = 1;
                beta = has_lo ? 0.5 * (beta + lo) : 0.5 * beta;
            }
        }
        double sum = 0.0, hs = 0.0;
        for (int32_t j = 0; j < k; j++) {
            p[j] = exp(-beta * (d[j] - dmin));
            sum += p[j];
            hs += (d[j] - dmin) * p[j];
        }
        for (int32_t j = 0; j < k; j++) p[j] /= sum;
        if (beta_out) beta_out[i] = beta;
        if (H_out) H_out[i] = log(sum) + beta * hs / sum;
        if (!ok) bad++;
    }
    return bad;
}

/* Sec. 3.3: the symmetric joint p_ij = (p_{j|i} + p_{i|j}) / (2n) on the union
 * of the kNN patterns, as CSR with columns ascending in each row.
 * Call with col == NULL to get nnz (row_ptr is then also filled). */
typedef struct { int64_t r; int32_t c; double v; } orc_trip;

static int trip_cmp(const void *a, const void *b)
{
    const orc_trip *x = (const orc_trip *)a, *y = (const orc_trip *)b;
    if (x->r != y->r) return x->r < y->r ? -1 : 1;
    if (x->c != y->c) return x->c < y->c ? -1 : 1;
    return 0;
}

int64_t orc_symmetrize(const int32_t *idx, const double *pcond, int64_t n, int32_t k,
                       int64_t *row_ptr, int32_t *col, double *val)
{
    int64_t m = 2 * n * (int64_t)k;
    orc_trip *t = (orc_trip *)malloc((size_t)m * sizeof(orc_trip));
    if (!t) return -1;
    int64_t o = 0;
    for (int64_t i = 0; i < n; i++)
        for (int32_t a = 0; a < k; a++) {
            int32_t j = idx[i * k + a];
            double v = pcond[i * k + a];
            t[o].r = i; t[o].c = j; t[o].v = v; o++;          /* p_{j|i} into (i,j) */
            t[o].r = j; t[o].c = (int32_t)i; t[o].v = v; o++; /* p_{j|i} into (j,i) */
        }
    qsort(t, (size_t)m, sizeof(orc_trip), trip_cmp);
    int64_t nnz = 0;
    for (int64_t i = 0; i <= n; i++) row_ptr[i] = 0;
    for (int64_t a = 0; a < m;) {
        int64_t b = a;
        double v = 0.0;
        while (b < m && t[b].r == t[a].r && t[b].c == t[a].c) v += t[b++].v;
        if (col) {
            col[nnz] = t[a].c;
            val[nnz] = v / (2.0 * (double)n);
        }
        row_ptr[t[a].r + 1]++;
        nnz++;
        a = b;
    }
    for (int64_t i = 0; i < n; i++) row_ptr[i + 1] += row_ptr[i];
    free(t);
    return nnz;
}

/* Eq. z1/z2: map an initial embedding Y0 (n x 2, y-units) onto the fixed-point
 * screen: z_d = min(R_d-1, floor((y_d - min_d) * R_d / (max_d - min_d))),
 * s_d = (max_d - min_d) / R_d, with R_d = r_d 2^F the axis' extent in ulps
 * (R[d]).  An axis with zero extent maps to z_d = 0 and s_d = 1/R_d. */
void orc_init_fx_dim(const double *Y0, int64_t n, int32_t dim, const double *R, uint32_t *z,
                     double *s)
{
    for (int d = 0; d < dim; d++) {
        const double Rd = R[d];
        double mn = Y0[d], mx = Y0[d];
        for (int64_t i = 1; i < n; i++) {
            double v = Y0[dim * i + d];
            if (v < mn) mn = v;
            if (v > mx) mx = v;
        }
        double range = mx - mn;
        if (!(range > 0.0)) {
            for (int64_t i = 0; i < n; i++) z[dim * i + d] = 0u;
            s[d] = 1.0 / Rd;
            continue;
        }
        for (int64_t i = 0; i < n; i++) {
            double q = floor((Y0[dim * i + d] - mn) * Rd / range);
            z[dim * i + d] = q >= Rd - 1.0 ? (uint32_t)(Rd - 1.0) : (uint32_t)q;
        }
        s[d] = range / Rd;
    }
}

/* The 2-D screen of r_1 x r_2 pixels. */
void orc_init_fx_screen(const double *Y0, int64_t n, const double *R, uint32_t *z, double *s)
{
    orc_init_fx_dim(Y0, n, 2, R, z, s);
}

/* The square 2^L screen: R_d = 2^32 on both axes. */
void orc_init_fx(const double *Y0, int64_t n, uint32_t *z, double *s)
{
    const double R[2] = {ORC_R, ORC_R};
    orc_init_fx_screen(Y0, n, R, z, s);
}

/* ------------------------------------------------------------------------ */
/* Sec. 4.1 P-Quadtree.  Morton index of pixel (px, py), bit by bit. */
uint32_t orc_morton(uint32_t px, uint32_t py)
{
    uint32_t m = 0;
    for (int b = 0; b < 16; b++) {
        m |= ((px >> b) & 1u) << (2 * b);
        m |= ((py >> b) & 1u) << (2 * b + 1);
    }
    return m;
}

int64_t orc_level_offset(int32_t l)
{
    return (((int64_t)1 << (2 * l)) - 1) / 3;
}

/* Pixel of each point (Eq. z1: floor of the screen coordinate) and the Morton
 * index of its leaf cell. */
void orc_leaf_keys(const uint32_t *z, int64_t n, int32_t L, uint32_t *px,
                   uint32_t *py, uint32_t *morton)
{
    int F = 32 - L;
    for (int64_t i = 0; i < n; i++) {
        uint32_t x = z[2 * i] >> F, y = z[2 * i + 1] >> F;
        if (px) px[i] = x;
        if (py) py[i] = y;
        morton[i] = orc_morton(x, y);
    }
}

/* Eq. ycell / ctrofmass on the fixed tree: for every cell of every level
 * l = 0..L, N_c = number of points whose pixel lies in the cell and the exact
 * integer sums of their z (the centre of mass is sum / N_c).  Each point is
 * added directly to the cell that contains it at every level. */
void orc_pyramid(const uint32_t *z, int64_t n, int32_t L, uint32_t *cnt,
                 uint64_t *sx, uint64_t *sy)
{
    int64_t cells = orc_level_offset(L + 1);
    memset(cnt, 0, (size_t)cells * sizeof(uint32_t));
    memset(sx, 0, (size_t)cells * sizeof(uint64_t));
    memset(sy, 0, (size_t)cells * sizeof(uint64_t));
    int F = 32 - L;
    for (int64_t i = 0; i < n; i++) {
        uint32_t m = orc_morton(z[2 * i] >> F, z[2 * i + 1] >> F);
        for (int32_t l = 0; l <= L; l++) {
            int64_t c = orc_level_offset(l) + (m >> (2 * (L - l)));
            cnt[c] += 1u;
            sx[c] += z[2 * i];
            sy[c] += z[2 * i + 1];
        }
    }
}

/* Offset, in ulps, of a point from a centre of mass S / N: z - S/N computed as
 * (z - floor(S/N)) - (S mod N)/N so that no precision is lost for large S. */
static double com_offset(uint32_t zi, uint64_t S, uint64_t N)
{
    uint64_t q = S / N, r = S % N;
    return (double)((int64_t)zi - (int64_t)q) - (double)r / (double)N;
}

/* Eq. grad second term with Eq. bh_criteria on the pixel-aligned tree
 * (Sec. 3.3, Sec. 4.1).  For each point i (rows == NULL: all; else the m
 * listed ones), depth-first over the cells with N_c > 0, starting at the root:
 *   - the cell containing i's pixel is opened; at a leaf, i is taken out
 *     (N' = N_c - 1, S' = S - z_i) and the rest is used if N' > 0;
 *   - another cell is accepted if it is a leaf (bounded depth, Sec. 4.1) or if
 *     r_c / ||y_i - y_c|| < theta (crit_mode 0; crit_mode 1 is the printed
 *     r_c / ||y_i - y_c||^2 < theta), else its four children are visited;
 *   - an accepted cell adds N w to Z_i and N w^2 (y_i - y_c) to Frep_i with
 *     w = 1 / (1 + ||y_i - y_c||^2).
 * y_c is the centre of mass (centre_mode 0) or the cell's geometric centre
 * (centre_mode 1, the approximation printed in Sec. 4.1).
 * Frep is the un-normalised sum (the gradient divides it by Z = sum_i Z_i).
 * n_inter (optional) gets the number of accepted cells per listed row. */
void orc_bh_repulsion(const uint32_t *z, const double *s, int64_t n, int32_t L,
                      double theta, int32_t crit_mode, int32_t centre_mode,
                      const uint32_t *cnt, const uint64_t *sx, const uint64_t *sy,
                      const int64_t *rows, int64_t m, double *Frep, double *Zi,
                      int64_t *n_inter)
{
    const int F = 32 - L;
    const double th2 = theta * theta;
    const double s0 = s[0], s1 = s[1];
    (void)n;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t q = 0; q < m; q++) {
        int64_t i = rows ? rows[q] : q;
        const uint32_t zx = z[2 * i], zy = z[2 * i + 1];
        const uint32_t mi = orc_morton(zx >> F, zy >> F);
        int32_t stk_l[64 * 4];
        uint32_t stk_m[64 * 4];
        int sp = 0;
        double fx = 0.0, fy = 0.0, zsum = 0.0;
        int64_t acc = 0;
        stk_l[sp] = 0; stk_m[sp] = 0; sp++;
        while (sp > 0) {
            sp--;
            int32_t l = stk_l[sp];
            uint32_t mc = stk_m[sp];
            int64_t c = orc_level_offset(l) + mc;
            uint64_t N = cnt[c];
            if (N == 0) continue;
            int leaf = (l == L);
            int contains = ((mi >> (2 * (L - l))) == mc);
            uint64_t Sx = sx[c], Sy = sy[c];
            if (contains) {
                if (!leaf) {
                    for (uint32_t ch = 0; ch < 4; ch++) {
                        stk_l[sp] = l + 1; stk_m[sp] = 4 * mc + ch; sp++;
                    }
                    continue;
                }
                N -= 1;
                if (N == 0) continue;
                Sx -= zx;
                Sy -= zy;
            }
            double dx, dy;
            if (centre_mode == 0) {
                dx = s0 * com_offset(zx, Sx, N);
                dy = s1 * com_offset(zy, Sy, N);
            } else {
                /* geometric centre of cell (l, mc): origin + W/2 */
                uint32_t cx = 0, cy = 0;
                for (int b = 0; b < l; b++) {
                    cx |= ((mc >> (2 * b)) & 1u) << b;
                    cy |= ((mc >> (2 * b + 1)) & 1u) << b;
                }
                double W = ldexp(1.0, 32 - l);
                dx = s0 * ((double)zx - ((double)cx * W + 0.5 * W));
                dy = s1 * ((double)zy - ((double)cy * W + 0.5 * W));
            }
            double dd = dx * dx + dy * dy;
            if (!leaf && !contains) {
                double W = ldexp(1.0, 32 - l);
                double rc2 = (s0 * W) * (s0 * W) + (s1 * W) * (s1 * W);
                int accept = crit_mode == 0 ? (rc2 < th2 * dd) : (rc2 < th2 * dd * dd);
                if (!accept) {
                    for (uint32_t ch = 0; ch < 4; ch++) {
                        stk_l[sp] = l + 1; stk_m[sp] = 4 * mc + ch; sp++;
                    }
                    continue;
                }
            }
            double w = 1.0 / (1.0 + dd);
            double Nw = (double)N * w;
            zsum += Nw;
            fx += Nw * w * dx;
            fy += Nw * w * dy;
            acc++;
        }
        Frep[2 * q] = fx;
        Frep[2 * q + 1] = fy;
        Zi[q] = zsum;
        if (n_inter) n_inter[q] = acc;
    }
}

/* Eq. q and Eq. grad second term without any approximation: for each listed
 * i, sum over all j != i of w_ij and w_ij^2 (y_i - y_j), w_ij = 1/(1+||y_i-y_j||^2).
 * Differences of fixed-point positions are exact integers before scaling. */
void orc_exact_repulsion(const uint32_t *z, const double *s, int64_t n,
                         const int64_t *rows, int64_t m, double *Frep, double *Zi)
{
    const double s0 = s[0], s1 = s[1];
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t q = 0; q < m; q++) {
        int64_t i = rows ? rows[q] : q;
        double fx = 0.0, fy = 0.0, zs = 0.0;
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            double dx = s0 * (double)((int64_t)z[2 * i] - (int64_t)z[2 * j]);
            double dy = s1 * (double)((int64_t)z[2 * i + 1] - (int64_t)z[2 * j + 1]);
            double w = 1.0 / (1.0 + dx * dx + dy * dy);
            zs += w;
            fx += w * w * dx;
            fy += w * w * dy;
        }
        Frep[2 * q] = fx;
        Frep[2 * q + 1] = fy;
        Zi[q] = zs;
    }
}

/* Eq. grad first term over the sparse P (Sec. 3.3):
 * Fattr_i = sum_j p_ij w_ij (y_i - y_j), un-exaggerated. */
void orc_attraction(const int64_t *row_ptr, const int32_t *col, const double *val,
                    const uint32_t *z, const double *s, const int64_t *rows,
                    int64_t m, double *Fattr)
{
    const double s0 = s[0], s1 = s[1];
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t q = 0; q < m; q++) {
        int64_t i = rows ? rows[q] : q;
        double fx = 0.0, fy = 0.0;
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; e++) {
            int64_t j = col[e];
            double dx = s0 * (double)((int64_t)z[2 * i] - (int64_t)z[2 * j]);
            double dy = s1 * (double)((int64_t)z[2 * i + 1] - (int64_t)z[2 * j + 1]);
            double w = 1.0 / (1.0 + dx * dx + dy * dy);
            fx += val[e] * w * dx;
            fy += val[e] * w * dy;
        }
        Fattr[2 * q] = fx;
        Fattr[2 * q + 1] = fy;
    }
}

/* Eq. grad assembled, then one gradient-descent step with momentum and
 * per-coordinate gains (the BH-SNE optimiser the paper keeps):
 *   g = 4 (alpha Fattr - Frep / Z)
 *   gain = (sign(g) != sign(u)) ? gain + 0.2 : gain * 0.8, at least min_gain,
 *          with sign(0) = 0 (so the first step, u = 0, always gains 0.2)
 *   u = mu u - eta gain g                       (y-units)
 *   zhat = z + rint(u / s)                      (ulps, int64)
 * zhat is the un-normalised update of Sec. 4.2, before screen rescaling. */
static int sgn(double x) { return x > 0.0 ? 1 : (x < 0.0 ? -1 : 0); }

void orc_update_dim(int64_t n, int32_t dim, const uint32_t *z, const double *s,
                    const double *Fattr, const double *Frep, double Z, double alpha, double mu,
                    double eta, double min_gain, double *u, double *gains, double *grad,
                    int64_t *zhat)
{
    for (int64_t i = 0; i < n; i++)
        for (int d = 0; d < dim; d++) {
            int64_t k = dim * i + d;
            double g = 4.0 * (alpha * Fattr[k] - Frep[k] / Z);
            if (grad) grad[k] = g;
            double gn = (sgn(g) != sgn(u[k])) ? gains[k] + 0.2 : gains[k] * 0.8;
            if (gn < min_gain) gn = min_gain;
            gains[k] = gn;
            u[k] = mu * u[k] - eta * gn * g;
            zhat[k] = (int64_t)z[k] + llrint(u[k] / s[d]);
        }
}

void orc_update(int64_t n, const uint32_t *z, const double *s, const double *Fattr,
                const double *Frep, double Z, double alpha, double mu, double eta,
                double min_gain, double *u, double *gains, double *grad, int64_t *zhat)
{
    orc_update_dim(n, 2, z, s, Fattr, Frep, Z, alpha, mu, eta, min_gain, u, gains, grad, zhat);
}

/* Sec. 4.2 screen-driven scaling to the r_d pixels of axis d, in exact
 * integer arithmetic:
 *   z_d = floor((zhat_d - min_d) * R_d / gamma_d),  gamma_d = (max_d - min_d) + 1
 * (the "+ epsilon" of gamma is one ulp; R_d = r_d 2^F, R[d]), and the
 * compensation of Eq. beta_scaling carried as s_d <- (s_d * gamma_d) / R_d
 * (two FP64 roundings; one when R_d = 2^32). */
void orc_rescale_dim(int64_t n, int32_t dim, const int64_t *zhat, const double *R, uint32_t *z,
                     double *s)
{
    for (int d = 0; d < dim; d++) {
        const uint64_t Rd = (uint64_t)R[d];
        int64_t mn = zhat[d], mx = zhat[d];
        for (int64_t i = 1; i < n; i++) {
            int64_t v = zhat[dim * i + d];
            if (v < mn) mn = v;
            if (v > mx) mx = v;
        }
        uint64_t gamma = (uint64_t)(mx - mn) + 1u;
        for (int64_t i = 0; i < n; i++) {
            unsigned __int128 num = (unsigned __int128)(uint64_t)(zhat[dim * i + d] - mn) * Rd;
            z[dim * i + d] = (uint32_t)(num / gamma);
        }
        s[d] = (s[d] * (double)gamma) / R[d];
    }
}

/* The 2-D screen of r_1 x r_2 pixels. */
void orc_rescale_screen(int64_t n, const int64_t *zhat, const double *R, uint32_t *z, double *s)
{
    orc_rescale_dim(n, 2, zhat, R, z, s);
}

/* The square 2^L screen. */
void orc_rescale(int64_t n, const int64_t *zhat, uint32_t *z, double *s)
{
    const double R[2] = {ORC_R, ORC_R};
    orc_rescale_screen(n, zhat, R, z, s);
}

/* Eq. cost_func: C = sum_ij p_ij ln(p_ij / q_ij) with q_ij = w_ij / Z, over the
 * non-zeros of P (zero entries contribute nothing). */
double orc_kl(const int64_t *row_ptr, const int32_t *col, const double *val,
              int64_t n, const uint32_t *z, const double *s, double Z)
{
    const double s0 = s[0], s1 = s[1];
    double C = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : C)
    for (int64_t i = 0; i < n; i++) {
        double c = 0.0;
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; e++) {
            double p = val[e];
            if (p <= 0.0) continue;
            int64_t j = col[e];
            double dx = s0 * (double)((int64_t)z[2 * i] - (int64_t)z[2 * j]);
            double dy = s1 * (double)((int64_t)z[2 * i + 1] - (int64_t)z[2 * j + 1]);
            double q = 1.0 / ((1.0 + dx * dx + dy * dy) * Z);
            c += p * log(p / q);
        }
        C += c;
    }
    return C;
}

/* ------------------------------------------------------------------------ */
/* One full PixelSNE run (Fig. 1(c), Sec. 4): for t = t0 .. t0+iters-1
 *   P-Quadtree assignment, BH repulsion, attraction, Z, gradient step,
 *   screen rescale.
 * Schedule: alpha = exag for t < exag_iters else 1; mu = mom0 for
 * t < mom_switch else mom1.  exact != 0 replaces the tree by the O(n^2)
 * repulsion.  Z_trace (optional, length iters) gets the Z used at each step. */
typedef struct {
    int32_t L;
    double theta;
    double eta;
    double exag;
    int32_t exag_iters;
    double mom0, mom1;
    int32_t mom_switch;
    double min_gain;
    int32_t crit_mode;
    int32_t centre_mode;
    int32_t exact;
    int32_t rx, ry;  /* screen pixels per axis (0: 2^L) */
} orc_params;

/* R_d = r_d 2^(32 - L) of a run's screen. */
static void screen_extent(const orc_params *p, double *R)
{
    const int32_t r[2] = {p->rx, p->ry};
    for (int d = 0; d < 2; d++)
        R[d] = r[d] > 0 ? ldexp((double)r[d], 32 - p->L) : ORC_R;
}

int orc_run(const orc_params *p, const int64_t *row_ptr, const int32_t *col,
            const double *val, int64_t n, uint32_t *z, double *s, double *u,
            double *gains, int32_t t0, int32_t iters, double *Z_trace)
{
    int64_t cells = orc_level_offset(p->L + 1);
    uint32_t *cnt = NULL;
    uint64_t *sx = NULL, *sy = NULL;
    if (!p->exact) {
        cnt = (uint32_t *)malloc((size_t)cells * sizeof(uint32_t));
        sx = (uint64_t *)malloc((size_t)cells * sizeof(uint64_t));
        sy = (uint64_t *)malloc((size_t)cells * sizeof(uint64_t));
    }
    double *Frep = (double *)malloc((size_t)n * 2 * sizeof(double));
    double *Fattr = (double *)malloc((size_t)n * 2 * sizeof(double));
    double *Zi = (double *)malloc((size_t)n * sizeof(double));
    int64_t *zhat = (int64_t *)malloc((size_t)n * 2 * sizeof(int64_t));
    if ((!p->exact && (!cnt || !sx || !sy)) || !Frep || !Fattr || !Zi || !zhat) {
        free(cnt); free(sx); free(sy); free(Frep); free(Fattr); free(Zi); free(zhat);
        return -1;
    }
    double R[2];
    screen_extent(p, R);
    for (int32_t t = t0; t < t0 + iters; t++) {
        if (p->exact) {
            orc_exact_repulsion(z, s, n, NULL, n, Frep, Zi);
        } else {
            orc_pyramid(z, n, p->L, cnt, sx, sy);
            orc_bh_repulsion(z, s, n, p->L, p->theta, p->crit_mode, p->centre_mode,
                             cnt, sx, sy, NULL, n, Frep, Zi, NULL);
        }
        double Z = 0.0;
        for (int64_t i = 0; i < n; i++) Z += Zi[i];
        if (Z_trace) Z_trace[t - t0] = Z;
        orc_attraction(row_ptr, col, val, z, s, NULL, n, Fattr);
        double alpha = t < p->exag_iters ? p->exag : 1.0;
        double mu = t < p->mom_switch ? p->mom0 : p->mom1;
        orc_update(n, z, s, Fattr, Frep, Z, alpha, mu, p->eta, p->min_gain, u, gains,
                   NULL, zhat);
        orc_rescale_screen(n, zhat, R, z, s);
    }
    free(cnt); free(sx); free(sy); free(Frep); free(Fattr); free(Zi); free(zhat);
    return 0;
}

/* Z of the current state (BH with the run's theta, or exact), for the KL. */
double orc_Z(const orc_params *p, int64_t n, const uint32_t *z, const double *s)
{
    double *Zi = (double *)malloc((size_t)n * sizeof(double));
    double *Frep = (double *)malloc((size_t)n * 2 * sizeof(double));
    double Z = -1.0;
    if (!Zi || !Frep) goto out;
    if (p->exact) {
        orc_exact_repulsion(z, s, n, NULL, n, Frep, Zi);
    } else {
        int64_t cells = orc_level_offset(p->L + 1);
        uint32_t *cnt = (uint32_t *)malloc((size_t)cells * sizeof(uint32_t));
        uint64_t *sx = (uint64_t *)malloc((size_t)cells * sizeof(uint64_t));
        uint64_t *sy = (uint64_t *)malloc((size_t)cells * sizeof(uint64_t));
        if (!cnt || !sx || !sy) { free(cnt); free(sx); free(sy); goto out; }
        orc_pyramid(z, n, p->L, cnt, sx, sy);
        orc_bh_repulsion(z, s, n, p->L, p->theta, p->crit_mode, p->centre_mode, cnt, sx,
                         sy, NULL, n, Frep, Zi, NULL);
        free(cnt); free(sx); free(sy);
    }
    Z = 0.0;
    for (int64_t i = 0; i < n; i++) Z += Zi[i];
out:
    free(Zi);
    free(Frep);
    return Z;
}

/* Eq. nei_prec: (1/(k m)) sum_i |N_D^k(i) intersect N_d^k(i)| over the listed
 * rows, with N_d^k(i) the k nearest neighbours of y_i in the 2-D embedding
 * (brute force, FP64, ties to the lower index) and N_D^k(i) given (knn_hd,
 * row q holds the neighbours of rows[q], at least k per row, stride kh). */
double orc_nbr_precision(const int32_t *knn_hd, int32_t kh, int32_t k, int64_t n,
                         const uint32_t *z, const double *s, const int64_t *rows,
                         int64_t m, int32_t *hits_out)
{
    const double s0 = s[0], s1 = s[1];
    int64_t hits = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : hits)
    for (int64_t q = 0; q < m; q++) {
        int64_t i = rows ? rows[q] : q;
        int32_t *I = (int32_t *)malloc((size_t)k * sizeof(int32_t));
        double *Dd = (double *)malloc((size_t)k * sizeof(double));
        int32_t cnt = 0;
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            double dx = s0 * (double)((int64_t)z[2 * i] - (int64_t)z[2 * j]);
            double dy = s1 * (double)((int64_t)z[2 * i + 1] - (int64_t)z[2 * j + 1]);
            double dd = dx * dx + dy * dy;
            int32_t p;
            if (cnt < k) p = cnt++;
            else if (knn_before(dd, (int32_t)j, Dd[k - 1], I[k - 1])) p = k - 1;
            else continue;
            while (p > 0 && knn_before(dd, (int32_t)j, Dd[p - 1], I[p - 1])) {
                Dd[p] = Dd[p - 1]; I[p] = I[p - 1]; p--;
            }
            Dd[p] = dd; I[p] = (int32_t)j;
        }
        int32_t h = 0;
        for (int32_t a = 0; a < k; a++)
            for (int32_t b = 0; b < k; b++)
                if (knn_hd[q * (int64_t)kh + b] == I[a]) { h++; break; }
        hits += h;
        if (hits_out) hits_out[q] = h;
        free(I);
        free(Dd);
    }
    return (double)hits / ((double)k * (double)m);
}

/* ------------------------------------------------------------------------ */
/* Learned warm start (not in the paper; a learned initialiser that
 * warm-starts the method): y = W3 g(W2 g(W1 x + b1) + b2) + b3 with g the exact GELU
 * g(z) = z Phi(z) = 0.5 z (1 + erf(z / sqrt 2)), dimensions d -> H -> H -> 2.
 * Weights row-major: W1[H x d], W2[H x H], W3[2 x H].  Loss over a batch of m
 * rows: L = (1/m) sum_r ||y_r - t_r||^2.  Returns L; when grad != NULL writes
 * dL/d(W1, b1, W2, b2, W3, b3) in that order (same layout as the weights), and
 * Y (m x 2) when non-NULL. */
static double gelu(double z) { return 0.5 * z * (1.0 + erf(z / sqrt(2.0))); }
static double gelu_d(double z)
{
    return 0.5 * (1.0 + erf(z / sqrt(2.0))) + z * exp(-0.5 * z * z) / sqrt(2.0 * M_PI);
}

double orc_mlp(int32_t d, int32_t H, const double *W1, const double *b1, const double *W2,
               const double *b2, const double *W3, const double *b3, const float *X,
               const float *T, int64_t m, double *Y, double *grad)
{
    double *z1 = (double *)malloc((size_t)H * sizeof(double));
    double *h1 = (double *)malloc((size_t)H * sizeof(double));
    double *z2 = (double *)malloc((size_t)H * sizeof(double));
    double *h2 = (double *)malloc((size_t)H * sizeof(double));
    double *dz2 = (double *)malloc((size_t)H * sizeof(double));
    double *dz1 = (double *)malloc((size_t)H * sizeof(double));
    double *gW1 = grad, *gb1 = grad ? grad + (size_t)H * d : NULL;
    double *gW2 = grad ? gb1 + H : NULL, *gb2 = grad ? gW2 + (size_t)H * H : NULL;
    double *gW3 = grad ? gb2 + H : NULL, *gb3 = grad ? gW3 + 2 * (size_t)H : NULL;
    if (grad) memset(grad, 0, ((size_t)H * d + H + (size_t)H * H + H + 2 * (size_t)H + 2) * sizeof(double));
    double L = 0.0;
    for (int64_t r = 0; r < m; r++) {
        const float *x = X + r * d;
        for (int32_t a = 0; a < H; a++) {
            double s = b1[a];
            for (int32_t c = 0; c < d; c++) s += W1[(size_t)a * d + c] * (double)x[c];
            z1[a] = s;
            h1[a] = gelu(s);
        }
        for (int32_t a = 0; a < H; a++) {
            double s = b2[a];
            for (int32_t c = 0; c < H; c++) s += W2[(size_t)a * H + c] * h1[c];
            z2[a] = s;
            h2[a] = gelu(s);
        }
        double dy[2];
        for (int o = 0; o < 2; o++) {
            double s = b3[o];
            for (int32_t c = 0; c < H; c++) s += W3[(size_t)o * H + c] * h2[c];
            if (Y) Y[2 * r + o] = s;
            double e = T ? s - (double)T[2 * r + o] : 0.0;
            L += e * e;
            dy[o] = 2.0 * e / (double)m;
        }
        if (!grad) continue;
        for (int o = 0; o < 2; o++) {
            gb3[o] += dy[o];
            for (int32_t c = 0; c < H; c++) gW3[(size_t)o * H + c] += dy[o] * h2[c];
        }
        for (int32_t a = 0; a < H; a++) {
            double dh = dy[0] * W3[a] + dy[1] * W3[(size_t)H + a];
            dz2[a] = dh * gelu_d(z2[a]);
        }
        for (int32_t a = 0; a < H; a++) {
            gb2[a] += dz2[a];
            for (int32_t c = 0; c < H; c++) gW2[(size_t)a * H + c] += dz2[a] * h1[c];
        }
        for (int32_t c = 0; c < H; c++) {
            double dh = 0.0;
            for (int32_t a = 0; a < H; a++) dh += dz2[a] * W2[(size_t)a * H + c];
            dz1[c] = dh * gelu_d(z1[c]);
        }
        for (int32_t a = 0; a < H; a++) {
            gb1[a] += dz1[a];
            for (int32_t c = 0; c < d; c++) gW1[(size_t)a * d + c] += dz1[a] * (double)x[c];
        }
    }
    free(z1); free(h1); free(z2); free(h2); free(dz2); free(dz1);
    return L / (double)m;
}

double orc_gelu(double z) { return gelu(z); }
double orc_gelu_d(double z) { return gelu_d(z); }

/* ------------------------------------------------------------------------ */
/* The 3-D embedding (Sec. 1's footnote: the same method on a voxel grid).
 * The screen is 2^L voxels per axis; z_d in [0, 2^32) ulps per axis and the
 * voxel is z_d >> (32 - L).  The quadtree becomes an octree: cell (l, m) of
 * level l holds the voxels whose top l bits of x, y and z give m, with the
 * bits interleaved x, y, z from the least significant (so a cell's child
 * c = 4 zbit + 2 ybit + xbit); level offsets in a flattened pyramid are
 * (8^l - 1) / 7.  Everything else is the 2-D method with a third axis. */
uint32_t orc_morton3(uint32_t px, uint32_t py, uint32_t pz)
{
    uint32_t m = 0;
    for (int b = 0; b < 10; b++) {
        m |= ((px >> b) & 1u) << (3 * b);
        m |= ((py >> b) & 1u) << (3 * b + 1);
        m |= ((pz >> b) & 1u) << (3 * b + 2);
    }
    return m;
}

int64_t orc_level_offset3(int32_t l)
{
    int64_t o = 0, p = 1;
    for (int32_t k = 0; k < l; k++) { o += p; p *= 8; }
    return o;
}

/* Sec. 4.1's tree in 3-D: counts and exact coordinate sums of every cell,
 * each point added to its cell at every level. */
void orc_pyramid3(const uint32_t *z, int64_t n, int32_t L, uint32_t *cnt, uint64_t *sx,
                  uint64_t *sy, uint64_t *sz)
{
    int64_t cells = orc_level_offset3(L + 1);
    memset(cnt, 0, (size_t)cells * sizeof(uint32_t));
    memset(sx, 0, (size_t)cells * sizeof(uint64_t));
    memset(sy, 0, (size_t)cells * sizeof(uint64_t));
    memset(sz, 0, (size_t)cells * sizeof(uint64_t));
    int F = 32 - L;
    for (int64_t i = 0; i < n; i++) {
        uint32_t m = orc_morton3(z[3 * i] >> F, z[3 * i + 1] >> F, z[3 * i + 2] >> F);
        for (int32_t l = 0; l <= L; l++) {
            int64_t c = orc_level_offset3(l) + (m >> (3 * (L - l)));
            cnt[c] += 1u;
            sx[c] += z[3 * i];
            sy[c] += z[3 * i + 1];
            sz[c] += z[3 * i + 2];
        }
    }
}

/* Eq. grad's second term with Eq. bh_criteria on the voxel-aligned octree:
 * the 2-D traversal with eight children and the cell diagonal
 * r_c^2 = W^2 (s_0^2 + s_1^2 + s_2^2); the cell holding i is opened and i is
 * taken out of its own voxel. */
void orc_bh_repulsion3(const uint32_t *z, const double *s, int64_t n, int32_t L, double theta,
                       const uint32_t *cnt, const uint64_t *sx, const uint64_t *sy,
                       const uint64_t *sz, const int64_t *rows, int64_t m, double *Frep,
                       double *Zi, int64_t *n_inter)
{
    const int F = 32 - L;
    const double th2 = theta * theta;
    const double s0 = s[0], s1 = s[1], s2 = s[2];
    (void)n;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t q = 0; q < m; q++) {
        int64_t i = rows ? rows[q] : q;
        const uint32_t zx = z[3 * i], zy = z[3 * i + 1], zz = z[3 * i + 2];
        const uint32_t mi = orc_morton3(zx >> F, zy >> F, zz >> F);
        int32_t stk_l[16 * 8];
        uint32_t stk_m[16 * 8];
        int sp = 0;
        double fx = 0.0, fy = 0.0, fz = 0.0, zsum = 0.0;
        int64_t acc = 0;
        stk_l[sp] = 0; stk_m[sp] = 0; sp++;
        while (sp > 0) {
            sp--;
            int32_t l = stk_l[sp];
            uint32_t mc = stk_m[sp];
            int64_t c = orc_level_offset3(l) + mc;
            uint64_t N = cnt[c];
            if (N == 0) continue;
            int leaf = (l == L);
            int contains = ((mi >> (3 * (L - l))) == mc);
            uint64_t Sx = sx[c], Sy = sy[c], Sz = sz[c];
            if (contains) {
                if (!leaf) {
                    for (uint32_t ch = 0; ch < 8; ch++) {
                        stk_l[sp] = l + 1; stk_m[sp] = 8 * mc + ch; sp++;
                    }
                    continue;
                }
                N -= 1;
                if (N == 0) continue;
                Sx -= zx;
                Sy -= zy;
                Sz -= zz;
            }
            double dx = s0 * com_offset(zx, Sx, N);
            double dy = s1 * com_offset(zy, Sy, N);
            double dz = s2 * com_offset(zz, Sz, N);
            double dd = dx * dx + dy * dy + dz * dz;
            if (!leaf && !contains) {
                double W = ldexp(1.0, 32 - l);
                double rc2 = (s0 * W) * (s0 * W) + (s1 * W) * (s1 * W) + (s2 * W) * (s2 * W);
                if (!(rc2 < th2 * dd)) {
                    for (uint32_t ch = 0; ch < 8; ch++) {
                        stk_l[sp] = l + 1; stk_m[sp] = 8 * mc + ch; sp++;
                    }
                    continue;
                }
            }
            double w = 1.0 / (1.0 + dd);
            double Nw = (double)N * w;
            zsum += Nw;
            fx += Nw * w * dx;
            fy += Nw * w * dy;
            fz += Nw * w * dz;
            acc++;
        }
        Frep[3 * q] = fx;
        Frep[3 * q + 1] = fy;
        Frep[3 * q + 2] = fz;
        Zi[q] = zsum;
        if (n_inter) n_inter[q] = acc;
    }
}

/* Eq. q and Eq. grad's second term without approximation, in 3-D. */
void orc_exact_repulsion3(const uint32_t *z, const double *s, int64_t n, const int64_t *rows,
                          int64_t m, double *Frep, double *Zi)
{
    const double s0 = s[0], s1 = s[1], s2 = s[2];
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t q = 0; q < m; q++) {
        int64_t i = rows ? rows[q] : q;
        double fx = 0.0, fy = 0.0, fz = 0.0, zs = 0.0;
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            double dx = s0 * (double)((int64_t)z[3 * i] - (int64_t)z[3 * j]);
            double dy = s1 * (double)((int64_t)z[3 * i + 1] - (int64_t)z[3 * j + 1]);
            double dz = s2 * (double)((int64_t)z[3 * i + 2] - (int64_t)z[3 * j + 2]);
            double w = 1.0 / (1.0 + dx * dx + dy * dy + dz * dz);
            zs += w;
            fx += w * w * dx;
            fy += w * w * dy;
            fz += w * w * dz;
        }
        Frep[3 * q] = fx;
        Frep[3 * q + 1] = fy;
        Frep[3 * q + 2] = fz;
        Zi[q] = zs;
    }
}

/* Eq. grad's first term over the sparse P, in 3-D (un-exaggerated). */
void orc_attraction3(const int64_t *row_ptr, const int32_t *col, const double *val,
                     const uint32_t *z, const double *s, const int64_t *rows, int64_t m,
                     double *Fattr)
{
    const double s0 = s[0], s1 = s[1], s2 = s[2];
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t q = 0; q < m; q++) {
        int64_t i = rows ? rows[q] : q;
        double fx = 0.0, fy = 0.0, fz = 0.0;
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; e++) {
            int64_t j = col[e];
            double dx = s0 * (double)((int64_t)z[3 * i] - (int64_t)z[3 * j]);
            double dy = s1 * (double)((int64_t)z[3 * i + 1] - (int64_t)z[3 * j + 1]);
            double dz = s2 * (double)((int64_t)z[3 * i + 2] - (int64_t)z[3 * j + 2]);
            double w = 1.0 / (1.0 + dx * dx + dy * dy + dz * dz);
            fx += val[e] * w * dx;
            fy += val[e] * w * dy;
            fz += val[e] * w * dz;
        }
        Fattr[3 * q] = fx;
        Fattr[3 * q + 1] = fy;
        Fattr[3 * q + 2] = fz;
    }
}

/* Eq. cost_func in 3-D. */
double orc_kl3(const int64_t *row_ptr, const int32_t *col, const double *val, int64_t n,
               const uint32_t *z, const double *s, double Z)
{
    const double s0 = s[0], s1 = s[1], s2 = s[2];
    double C = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : C)
    for (int64_t i = 0; i < n; i++) {
        double c = 0.0;
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; e++) {
            double p = val[e];
            if (p <= 0.0) continue;
            int64_t j = col[e];
            double dx = s0 * (double)((int64_t)z[3 * i] - (int64_t)z[3 * j]);
            double dy = s1 * (double)((int64_t)z[3 * i + 1] - (int64_t)z[3 * j + 1]);
            double dz = s2 * (double)((int64_t)z[3 * i + 2] - (int64_t)z[3 * j + 2]);
            double q = 1.0 / ((1.0 + dx * dx + dy * dy + dz * dz) * Z);
            c += p * log(p / q);
        }
        C += c;
    }
    return C;
}

/* One 3-D run: for t = t0 .. t0+iters-1 the octree, its Barnes-Hut repulsion
 * (or the exact sum), the attraction, Z, the gradient step and the screen
 * rescale of all three axes (R = 2^32).  Schedule as orc_run. */
int orc_run3(const orc_params *p, const int64_t *row_ptr, const int32_t *col, const double *val,
             int64_t n, uint32_t *z, double *s, double *u, double *gains, int32_t t0,
             int32_t iters)
{
    int64_t cells = orc_level_offset3(p->L + 1);
    uint32_t *cnt = NULL;
    uint64_t *sx = NULL, *sy = NULL, *sz = NULL;
    if (!p->exact) {
        cnt = (uint32_t *)malloc((size_t)cells * sizeof(uint32_t));
        sx = (uint64_t *)malloc((size_t)cells * sizeof(uint64_t));
        sy = (uint64_t *)malloc((size_t)cells * sizeof(uint64_t));
        sz = (uint64_t *)malloc((size_t)cells * sizeof(uint64_t));
    }
    double *Frep = (double *)malloc((size_t)n * 3 * sizeof(double));
    double *Fattr = (double *)malloc((size_t)n * 3 * sizeof(double));
    double *Zi = (double *)malloc((size_t)n * sizeof(double));
    int64_t *zhat = (int64_t *)malloc((size_t)n * 3 * sizeof(int64_t));
    if ((!p->exact && (!cnt || !sx || !sy || !sz)) || !Frep || !Fattr || !Zi || !zhat) {
        free(cnt); free(sx); free(sy); free(sz); free(Frep); free(Fattr); free(Zi); free(zhat);
        return -1;
    }
    const double R[3] = {ORC_R, ORC_R, ORC_R};
    for (int32_t t = t0; t < t0 + iters; t++) {
        if (p->exact) {
            orc_exact_repulsion3(z, s, n, NULL, n, Frep, Zi);
        } else {
            orc_pyramid3(z, n, p->L, cnt, sx, sy, sz);
            orc_bh_repulsion3(z, s, n, p->L, p->theta, cnt, sx, sy, sz, NULL, n, Frep, Zi, NULL);
        }
        double Z = 0.0;
        for (int64_t i = 0; i < n; i++) Z += Zi[i];
        orc_attraction3(row_ptr, col, val, z, s, NULL, n, Fattr);
        double alpha = t < p->exag_iters ? p->exag : 1.0;
        double mu = t < p->mom_switch ? p->mom0 : p->mom1;
        orc_update_dim(n, 3, z, s, Fattr, Frep, Z, alpha, mu, p->eta, p->min_gain, u, gains,
                       NULL, zhat);
        orc_rescale_dim(n, 3, zhat, R, z, s);
    }
    free(cnt); free(sx); free(sy); free(sz); free(Frep); free(Fattr); free(Zi); free(zhat);
    return 0;
}

/* Z of a 3-D state (Barnes-Hut with the run's theta, or exact), for the KL. */
double orc_Z3(const orc_params *p, int64_t n, const uint32_t *z, const double *s)
{
    double *Zi = (double *)malloc((size_t)n * sizeof(double));
    double *Frep = (double *)malloc((size_t)n * 3 * sizeof(double));
    double Z = -1.0;
    if (!Zi || !Frep) goto out;
    if (p->exact) {
        orc_exact_repulsion3(z, s, n, NULL, n, Frep, Zi);
    } else {
        int64_t cells = orc_level_offset3(p->L + 1);
        uint32_t *cnt = (uint32_t *)malloc((size_t)cells * sizeof(uint32_t));
        uint64_t *sx = (uint64_t *)malloc((size_t)cells * sizeof(uint64_t));
        uint64_t *sy = (uint64_t *)malloc((size_t)cells * sizeof(uint64_t));
        uint64_t *sz = (uint64_t *)malloc((size_t)cells * sizeof(uint64_t));
        if (!cnt || !sx || !sy || !sz) { free(cnt); free(sx); free(sy); free(sz); goto out; }
        orc_pyramid3(z, n, p->L, cnt, sx, sy, sz);
        orc_bh_repulsion3(z, s, n, p->L, p->theta, cnt, sx, sy, sz, NULL, n, Frep, Zi, NULL);
        free(cnt); free(sx); free(sy); free(sz);
    }
    Z = 0.0;
    for (int64_t i = 0; i < n; i++) Z += Zi[i];
out:
    free(Zi);
    free(Frep);
    return Z;
}
