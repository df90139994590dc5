// Neighbourhood precision (Eq. nei_prec): (1 / (k n)) sum_i |N_D^k(i) ∩ N_d^k(i)|,
// with N_D^k(i) the first k high-dimensional neighbours of point i and
// N_d^k(i) its k nearest neighbours in the 2-D embedding.
//
// k_nbr_precision  one thread per point (in Morton order): exact 2-D k nearest
//                  neighbours by a ring search over the pixel grid of the
//                  current tree (points of a pixel are contiguous in the
//                  counting-sort permutation); squared distances in FP64 with
//                  explicit round-to-nearest operations, ties to the lower index
#include "common.cuh"

namespace pxsne {

constexpr int kPrecMaxK = 32;

__device__ __forceinline__ double d2_fp64(uint2 a, uint2 b, double s0, double s1) {
    const double dx = __dmul_rn(s0, (double)((int64_t)a.x - (int64_t)b.x));
    const double dy = __dmul_rn(s1, (double)((int64_t)a.y - (int64_t)b.y));
    return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
}

__global__ void __launch_bounds__(128)
    k_nbr_precision(int n, int L, int K1, int k, const uint2 *__restrict__ z,
                    const uint32_t *__restrict__ perm, const float *__restrict__ leaf_n,
                    const uint32_t *__restrict__ leaf_start,
                    const uint32_t *__restrict__ blk_off, const int32_t *__restrict__ knn_hd,
                    int kh, const DevScalars *__restrict__ sc, int32_t *__restrict__ hits,
                    unsigned long long *total) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const uint32_t i = perm[t];
    const uint2 zi = z[i];
    const int F = 32 - L;
    const int R = 1 << L;
    const int px = (int)(zi.x >> F), py = (int)(zi.y >> F);
    const double s0 = sc->s[0], s1 = sc->s[1];
    // smallest pixel side in y-units
    const double w = ldexp(s0 < s1 ? s0 : s1, F);
    double bd[kPrecMaxK];
    int32_t bj[kPrecMaxK];
    for (int a = 0; a < k; a++) {
        bd[a] = INFINITY;
        bj[a] = 0x7fffffff;
    }
    int found = 0;
    for (int rho = 0; rho <= R; rho++) {
        // every pixel at Chebyshev distance >= rho holds points at distance
        // >= (rho - 1) w; stop when the k-th distance is strictly below that
        if (rho >= 1 && found >= k) {
            const double b = (double)(rho - 1) * w;
            if (bd[k - 1] < b * b * (1.0 - 1e-12)) break;
        }
        const int y0 = py - rho, y1 = py + rho, x0 = px - rho, x1 = px + rho;
        const int cells = rho == 0 ? 1 : 8 * rho;
        for (int q = 0; q < cells; q++) {
            int x, y;
            if (rho == 0) {
                x = px;
                y = py;
            } else if (q < 2 * rho + 1) {
                x = x0 + q;
                y = y0;
            } else if (q < 4 * rho + 2) {
                x = x0 + (q - (2 * rho + 1));
                y = y1;
            } else if (q < 6 * rho + 1) {
                x = x0;
                y = y0 + 1 + (q - (4 * rho + 2));
            } else {
                x = x1;
                y = y0 + 1 + (q - (6 * rho + 1));
            }
            if (x < 0 || y < 0 || x >= R || y >= R) continue;
            const uint32_t m = morton2((uint32_t)x, (uint32_t)y);
            const uint32_t c = (uint32_t)leaf_n[m];  // the pixel's count (exact float)
            if (c == 0u) continue;
            const uint32_t st = blk_off[m >> (2 * K1)] + leaf_start[m];
            for (uint32_t u = 0; u < c; u++) {
                const uint32_t j = perm[st + u];
                if (j == i) continue;
                const double dd = d2_fp64(zi, z[j], s0, s1);
                found++;
                if (!(dd < bd[k - 1] || (dd == bd[k - 1] && (int32_t)j < bj[k - 1]))) continue;
                int p = k - 1;
                while (p > 0 && (bd[p - 1] > dd || (bd[p - 1] == dd && bj[p - 1] > (int32_t)j))) {
                    bd[p] = bd[p - 1];
                    bj[p] = bj[p - 1];
                    p--;
                }
                bd[p] = dd;
                bj[p] = (int32_t)j;
            }
        }
    }
    int h = 0;
    for (int a = 0; a < k; a++)
        for (int b = 0; b < k; b++)
            if (knn_hd[(int64_t)i * kh + b] == bj[a]) {
                h++;
                break;
            }
    hits[i] = h;
    atomicAdd(total, (unsigned long long)h);
}

cudaError_t launch_nbr_precision(pxsne_ctx *c, int k, const int32_t *knn_hd, int kh,
                                 int32_t *hits, unsigned long long *total) {
    const int n = (int)c->n;
    const int K1 = c->L < kPyrK ? c->L : kPyrK;
    k_nbr_precision<<<(n + 127) / 128, 128, 0, c->stream>>>(n, c->L, K1, k, c->z, c->perm,
                                                           c->recn + rec_offset(c->L),
                                                           c->leaf_start, c->blk_off,
                                                           knn_hd, kh, c->sc, hits, total);
    return cudaGetLastError();
}

}  // namespace pxsne
