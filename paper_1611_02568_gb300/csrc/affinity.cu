// Affinity matrix P of t-SNE (Sec. 3.2) on the sparse kNN pattern of Sec. 3.3.
//
//   k_knn_tc       brute-force k nearest neighbours on the tensor cores: FP16
//                  dot-product tiles (tcgen05, FP32 accumulator in TMEM) filter
//                  candidates with a rigorous error bound; survivors are
//                  re-ranked with exact FP32 distances (the default path)
//   k_knn_tile     the same search on FP32 CUDA cores (check path): a 64 x 128 tile of
//                  approximate squared distances |q|^2 + |c|^2 - 2 q.c (FP32
//                  dot products) filters candidates against each row's current
//                  k-th distance plus an error slack; survivors get their exact
//                  FP32 sum of squared differences and enter a sorted list
//                  (ties to the lower index)
//   k_perplexity   per-row bisection on beta so that the entropy of
//                  p_{j|i} ~ exp(-beta d2) is ln(perplexity), one warp per row
//   symmetrize     p_ij = (p_{j|i} + p_{i|j}) / 2n on the union pattern, CSR
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_fp16.h>

#include "common.cuh"
#include "tc.cuh"

namespace pxsne {

static inline float __uint_as_float_host(unsigned u) {
    float f;
    memcpy(&f, &u, sizeof f);
    return f;
}

constexpr int kQR = 64;    // query rows per CTA
constexpr int kCT = 128;   // candidates per tile
constexpr int kKnnThreads = 256;

// flag |= 1 if any of the m values of X is not finite (the input check of
// P construction, on the device where X already is)
__global__ void k_nonfinite(int64_t m, const float *__restrict__ X, unsigned *flag) {
    bool bad = false;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < m;
         q += (int64_t)gridDim.x * blockDim.x)
        bad |= !isfinite(__ldcs(X + q));
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1u);
}

cudaError_t launch_nonfinite(pxsne_ctx *c, const float *X, int64_t m, unsigned *flag,
                             cudaStream_t st) {
    const int64_t need = (m + 255) / 256;
    const int cap = 8 * std::max(c->sms, 1);
    k_nonfinite<<<(unsigned)std::min<int64_t>(need, cap), 256, 0, st>>>(m, X, flag);
    return cudaGetLastError();
}

__global__ void k_row_norms(int64_t n, int D, const float *__restrict__ X, float *__restrict__ nrm) {
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    float s = 0.f;
    for (int d = lane; d < D; d += 32) {
        const float v = X[row * D + d];
        s = fmaf(v, v, s);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) nrm[row] = s;
}

// Exact FP32 squared distance between rows a and b, one warp, fixed order.
__device__ __forceinline__ float warp_exact_d2(const float *__restrict__ X, int D, int64_t a,
                                               int64_t b, int lane) {
    float s = 0.f;
    for (int d = lane; d < D; d += 32) {
        const float t = X[a * D + d] - X[b * D + d];
        s = fmaf(t, t, s);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// Insert (d, j) into the ascending list (ld, lj) of length k held in shared
// memory (entries with d = +inf are empty).  Whole warp.
__device__ __forceinline__ void warp_list_insert(float *ld, int32_t *lj, int k, float d,
                                                 int32_t j, int lane) {
    // position = number of entries ordered before (d, j)
    int pos = 0;
    for (int b = 0; b < k; b += 32) {
        const int e = b + lane;
        bool before = false;
        if (e < k) {
            const float de = ld[e];
            before = de < d || (de == d && lj[e] < j);
        }
        pos += __popc(__ballot_sync(0xffffffffu, before));
    }
    if (pos >= k) return;
    // shift [pos, k-1) up by one, highest chunk first
    for (int b = ((k - 1) / 32) * 32; b >= 0; b -= 32) {
        const int e = b + lane;
        float dv = 0.f;
        int32_t jv = 0;
        const bool mv = (e >= pos && e < k - 1);
        if (mv) {
            dv = ld[e];
            jv = lj[e];
        }
        __syncwarp();
        if (mv) {
            ld[e + 1] = dv;
            lj[e + 1] = jv;
        }
        __syncwarp();
    }
    if (lane == 0) {
        ld[pos] = d;
        lj[pos] = j;
    }
    __syncwarp();
}

// One CTA: kQR query rows against all n candidates, in tiles of kCT.
// Dynamic shared memory: qs[D][kQR], cs[D][kCT] (transposed tiles), the
// lists ld/lj[kQR][k], qn[kQR], the approximate distances ds[kQR][kCT] and
// the candidate norms of each warp's tile [8][kCT].
__global__ void __launch_bounds__(kKnnThreads)
    k_knn_tile(int64_t n, int D, int k, const float *__restrict__ X,
               const float *__restrict__ nrm, int32_t *__restrict__ out_idx,
               float *__restrict__ out_d2) {
    extern __shared__ float smem[];
    float *qs = smem;                       // D * kQR
    float *cs = qs + (size_t)D * kQR;       // D * kCT
    float *ld = cs + (size_t)D * kCT;       // kQR * k
    int32_t *lj = reinterpret_cast<int32_t *>(ld + (size_t)kQR * k);
    float *qn = reinterpret_cast<float *>(lj + (size_t)kQR * k);
    float *ds = qn + kQR;                   // kQR * kCT approximate distances
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int64_t q0 = (int64_t)blockIdx.x * kQR;
    for (int e = tid; e < kQR * k; e += kKnnThreads) {
        ld[e] = INFINITY;
        lj[e] = 0x7fffffff;
    }
    for (int e = tid; e < D * kQR; e += kKnnThreads) {
        const int d = e / kQR, q = e % kQR;
        qs[e] = (q0 + q < n) ? X[(q0 + q) * D + d] : 0.f;
    }
    if (tid < kQR) qn[tid] = (q0 + tid < n) ? nrm[q0 + tid] : 0.f;
    // approximate-distance error bound: rounding of a length-D dot product
    const float slack_rel = 4.0f * (float)(D + 4) * 5.9604645e-8f;
    for (int64_t c0 = 0; c0 < n; c0 += kCT) {
        __syncthreads();
        if ((D & 3) == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0) {
            // 16-byte loads along a row; consecutive threads take consecutive
            // rows so the transposed shared-memory writes do not conflict
            for (int e = tid; e < (D >> 2) * kCT; e += kKnnThreads) {
                const int c = e % kCT, d4 = e / kCT;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (c0 + c < n) v = *reinterpret_cast<const float4 *>(X + (c0 + c) * D + 4 * d4);
                cs[(4 * d4 + 0) * kCT + c] = v.x;
                cs[(4 * d4 + 1) * kCT + c] = v.y;
                cs[(4 * d4 + 2) * kCT + c] = v.z;
                cs[(4 * d4 + 3) * kCT + c] = v.w;
            }
        } else {
            for (int e = tid; e < D * kCT; e += kKnnThreads) {
                const int c = e % kCT, d = e / kCT;
                cs[e] = (c0 + c < n) ? X[(c0 + c) * D + d] : 0.f;
            }
        }
        __syncthreads();
        // 8 queries (warp w) x 4 candidates (4 * lane .. +3) per thread
        float acc[8][4];
#pragma unroll
        for (int a = 0; a < 8; a++)
#pragma unroll
            for (int b = 0; b < 4; b++) acc[a][b] = 0.f;
        for (int d = 0; d < D; d++) {
            const float4 qa = *reinterpret_cast<const float4 *>(qs + d * kQR + 8 * w);
            const float4 qb = *reinterpret_cast<const float4 *>(qs + d * kQR + 8 * w + 4);
            const float4 cv = *reinterpret_cast<const float4 *>(cs + d * kCT + 4 * lane);
            const float qv[8] = {qa.x, qa.y, qa.z, qa.w, qb.x, qb.y, qb.z, qb.w};
            const float cc[4] = {cv.x, cv.y, cv.z, cv.w};
#pragma unroll
            for (int a = 0; a < 8; a++)
#pragma unroll
                for (int b = 0; b < 4; b++) acc[a][b] = fmaf(qv[a], cc[b], acc[a][b]);
        }
#pragma unroll
        for (int b = 0; b < 4; b++) {
            const int64_t j = c0 + 4 * lane + b;
            const float cn = j < n ? nrm[j] : 0.f;
#pragma unroll
            for (int a = 0; a < 8; a++) {
                const int q = 8 * w + a;
                // approximate d2 and its error bound, packed for the selection
                ds[q * kCT + 4 * lane + b] = qn[q] + cn - 2.0f * acc[a][b];
            }
            ds[kQR * kCT + w * kCT + 4 * lane + b] = cn;
        }
        __syncwarp();
        // selection: the warp owns its 8 query rows, so no other warp touches
        // their lists
#pragma unroll 1
        for (int a = 0; a < 8; a++) {
            const int q = 8 * w + a;
            const int64_t qi = q0 + q;
            if (qi >= n) break;
            float *qld = ld + (size_t)q * k;
            int32_t *qlj = lj + (size_t)q * k;
            const float qnv = qn[q];
#pragma unroll 1
            for (int b = 0; b < 4; b++) {
                const int64_t j = c0 + 4 * lane + b;
                const float approx = ds[q * kCT + 4 * lane + b];
                const float cn = ds[kQR * kCT + w * kCT + 4 * lane + b];
                const float tau = qld[k - 1];
                const bool cand = (j < n) && (j != qi) &&
                                  (approx <= tau + slack_rel * (qnv + cn) || !(tau < INFINITY));
                unsigned m = __ballot_sync(0xffffffffu, cand);
                while (m) {
                    const int src = __ffs(m) - 1;
                    m &= m - 1u;
                    const int64_t jj = __shfl_sync(0xffffffffu, j, src);
                    const float dex = warp_exact_d2(X, D, qi, jj, lane);
                    const float t2 = qld[k - 1];
                    if (dex < t2 || (dex == t2 && (int32_t)jj < qlj[k - 1]))
                        warp_list_insert(qld, qlj, k, dex, (int32_t)jj, lane);
                }
            }
        }
    }
    __syncthreads();
    for (int e = tid; e < kQR * k; e += kKnnThreads) {
        const int q = e / k;
        if (q0 + q < n) {
            out_idx[(q0 + q) * k + (e % k)] = lj[e];
            out_d2[(q0 + q) * k + (e % k)] = ld[e];
        }
    }
}

// ---------------------------------------------------------------- tensor-core kNN
// The same search on the tensor cores: the dot products of a 128 x 128 tile
// come from tcgen05 MMAs on FP16 copies x~ of the rows (X scaled by 2^e),
// accumulated in FP32 in TMEM.  With the norms |x~|^2 of the rounded rows,
// |q~|^2 + |c~|^2 - 2 q~.c~ is the squared distance of the rounded rows up to
// the FP32 accumulation (kappa |q~||c~|, kappa about 2 D 2^-24) and the norms'
// own rounding (eps).  The triangle inequality gives
// |q - c| >= |q~ - c~| - |q~ - q| - |c~ - c|, and each row's rounding error
// E = |x~ - x| is known exactly, so a candidate can only belong to the k
// nearest if |q~ - c~| <= sqrt(tau) + E_q + E_c, tau the row's current k-th
// exact distance.  The band this leaves is about 2 sqrt(tau) (E_q + E_c), a
// multiple of |x| 2^-11 rather than of |x|^2 2^-11 as a bound on the dot
// product alone would be.  Only the survivors get their exact FP32 distance
// (sum of squared differences) and enter the row's sorted list.
//
// One CTA owns 128 query rows and sweeps the candidate tiles outward from its
// own in the locality order (neighbouring CTAs read the same tiles at about
// the same time, so each tile is shared through L2).  Warp roles: warp 8
// judges the candidate tiles (a tile whose rows all lie beyond the query rows'
// current k-th distances, by the triangle inequality on tile centroids and
// radii, is skipped) and streams the kept ones (pre-swizzled FP16 images, one
// bulk copy each) into a ring of shared-memory stages; warp 9 issues the MMAs
// into four TMEM accumulators; warps 0-7 filter, warps w and w + 4 on the
// same 32 query rows (TMEM lanes 32(w % 4) ..), each on 64 of a tile's 128
// columns, so that two warps per scheduler hide each other's latencies.  With h_j = (1-eps)|c~_j|^2 and g_j = |c~_j| (staged
// with the tile, with each 32-column chunk's largest E_c), a chunk is skipped
// when a bound from its min h, max g and max q.c already exceeds the
// threshold; otherwise each (row, candidate) costs two FMAs and a min: the
// chunk is skipped when
//   min_j (h_j - kappa |q~| g_j - 2 q~.c~_j) > (sqrt(tau) + E_q + max E_c)^2 - (1-eps)|q~|^2,
// and otherwise the same per-column values pick the survivors.  A warp queues the
// survivors of its 32 rows (a chain per row through the queue) over as many
// tiles as it takes to gather a batch; then the warp computes their exact
// distances, one survivor per lane, and, holding the lock its row quarter
// shares with the other warp on those rows, every lane walks its own row's
// chain inserting them, all lanes at once, against the lists' current roots.
constexpr int kTcRows = 128;     // query rows per CTA (MMA M)
constexpr int kTcCols = 128;     // candidates per tile (MMA N)
constexpr int kTcStages = 2;     // candidate-tile stages in shared memory
constexpr int kTcQueue = 384;    // survivor queue per filter warp (entries)
constexpr uint32_t kTcFlushAt = 48u;   // queued survivors that trigger a flush
constexpr int kTcAcc = 4;        // TMEM accumulators (4 x 128 columns)
constexpr int kTcFilterWarps = 8;  // two per TMEM lane quarter, 64 columns each
constexpr int kTcThreads = 32 * (kTcFilterWarps + 2);  // then the loader, then the MMA issuer
constexpr int kTcLoadWarp = kTcFilterWarps, kTcMmaWarp = kTcFilterWarps + 1;
constexpr int kTcPolls = 1 << 22;
constexpr uint32_t kTcSleepNs = 2000u;  // suspend hint of the pipeline waits
// per candidate tile: h_j (128), g_j (128), then per 32-column chunk min h and
// max g (4 + 4): 264 floats, 1056 bytes (a multiple of 16 for the bulk copy)
constexpr int kHG = 2 * kTcCols + 12;

__global__ void k_absmax(int64_t m, const float *__restrict__ X, unsigned *out) {
    unsigned v = 0u;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x)
        v = max(v, __float_as_uint(fabsf(X[i])));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, v);
}

// FP16 copy of X * scale as ready-made shared-memory images: tile t (rows
// 128t .. 128t + 127, zero rows past n and zero columns past D) in the 128-byte
// swizzled K-major layout of the MMA operands, so that one bulk copy loads it.
__global__ void k_to_half_img(int64_t n, int D, int Dp, int64_t T, float scale,
                              const float *__restrict__ X, uint8_t *__restrict__ img) {
    const int chunks = Dp >> 3;  // 16-byte chunks per row
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= T * kTcRows * chunks) return;
    const int64_t row = q / chunks;
    const int c8 = (int)(q % chunks);
    const int64_t t = row / kTcRows;
    const int r = (int)(row % kTcRows);
    __align__(16) __half h[8];
#pragma unroll
    for (int u = 0; u < 8; u++) {
        const int d = 8 * c8 + u;
        h[u] = __float2half_rn(row < n && d < D ? X[row * D + d] * scale : 0.0f);
    }
    *reinterpret_cast<uint4 *>(img + t * (int64_t)kTcRows * Dp * 2 +
                               tc::sw128_offset(r, 8 * c8, kTcRows)) =
        *reinterpret_cast<const uint4 *>(h);
}

// Per ordered row r, from the same FP16 conversion as the tile images:
// n16[r] = |x~|^2 of the rounded row x~ (in X's units) and err[r] >= |x~ - x|,
// the norm of its rounding error, rounded up, plus the largest error a
// flushed FP16 subnormal could add in each dimension.
__global__ void k_round_err(int64_t n, int D, float scale, const float *__restrict__ X,
                            float *__restrict__ n16, float *__restrict__ err) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n) return;
    const float *x = X + r * D;
    double s2 = 0.0, e2 = 0.0;
    for (int d = 0; d < D; d++) {
        const float xs = x[d] * scale;  // exact (a power of two)
        const float hs = __half2float(__float2half_rn(xs));
        const float es = hs - xs;       // exact (the two lie within a factor of two, or hs = 0)
        s2 += (double)hs * hs;
        e2 += (double)es * es;
    }
    const double inv = 1.0 / (double)scale;
    n16[r] = (float)(s2 * inv * inv);
    err[r] = (float)((sqrt(e2) * (1.0 + 1e-6) + sqrt((double)D) * 6.103515625e-05) * inv);
}

// Per candidate tile t (kHG floats from HG + kHG t): h_j = (1-eps)|c~_j|^2 of
// the rounded rows (+inf past n), then g_j = |c~_j|, then for each 32-column
// chunk the min of its h_j, the max of its g_j and the max of its rows'
// rounding errors (a warp covers one chunk).
__global__ void k_tile_norms(int64_t n, int64_t T, float eps_abs, const float *__restrict__ nrm,
                             const float *__restrict__ rerr, float *__restrict__ HG) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= T * kTcCols) return;  // whole warps (T * 128 is a multiple of 32)
    const int64_t t = i / kTcCols;
    const int j = (int)(i % kTcCols);
    const float c2 = i < n ? nrm[i] : 0.f;
    const float h = i < n ? (1.0f - eps_abs) * c2 : INFINITY, g = sqrtf(c2);
    float *hg = HG + t * kHG;
    hg[j] = h;
    hg[kTcCols + j] = g;
    float hmin = h, gmax = g, emax = i < n ? rerr[i] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        hmin = fminf(hmin, __shfl_xor_sync(0xffffffffu, hmin, o));
        gmax = fmaxf(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
        emax = fmaxf(emax, __shfl_xor_sync(0xffffffffu, emax, o));
    }
    if ((j & 31) == 0) {
        hg[2 * kTcCols + (j >> 5)] = hmin;
        hg[2 * kTcCols + 4 + (j >> 5)] = gmax;
        hg[2 * kTcCols + 8 + (j >> 5)] = emax;
    }
}

// Per tile t of the ordered rows: centroid (thread d sums dimension d over
// the tile's rows) and radius = max over its rows of |x - centroid|, raised by
// 1e-4 relative so that FP32 rounding cannot make it too small.  The
// triangle inequality then bounds every distance between two tiles from below
// by |c_a - c_b| - r_a - r_b (any centroid would do).
__global__ void __launch_bounds__(128)
    k_tile_bounds(int64_t n, int D, int Dp, const float *__restrict__ X, float *__restrict__ cent,
                  float *__restrict__ rad) {
    __shared__ float s_c[256];
    __shared__ float s_r[4];
    const int64_t t = blockIdx.x;
    const int64_t r0 = t * kTcRows;
    const int cnt = (int)(n - r0 < kTcRows ? n - r0 : kTcRows);
    const int tid = threadIdx.x;
    for (int d = tid; d < Dp; d += blockDim.x) {
        float sum = 0.f;
        if (d < D)
            for (int r = 0; r < cnt; r++) sum += X[(r0 + r) * D + d];
        const float c = d < D ? sum / (float)cnt : 0.f;
        s_c[d] = c;
        cent[t * Dp + d] = c;
    }
    __syncthreads();
    float m = 0.f;
    if (tid < cnt) {
        float acc = 0.f;
        for (int d = 0; d < D; d++) {
            const float df = X[(r0 + tid) * D + d] - s_c[d];
            acc = fmaf(df, df, acc);
        }
        m = sqrtf(acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((tid & 31) == 0) s_r[tid >> 5] = m;
    __syncthreads();
    if (tid == 0) rad[t] = fmaxf(fmaxf(s_r[0], s_r[1]), fmaxf(s_r[2], s_r[3])) * 1.0001f + 1e-30f;
}

// Exact FP32 squared distance between rows a and b by one thread, summed in
// index order (16-byte loads when rows are 16-byte aligned).
__device__ __forceinline__ float thread_exact_d2(const float *__restrict__ X, int D, int64_t a,
                                                 int64_t b, bool vec4) {
    const float *xa = X + a * D, *xb = X + b * D;
    float s = 0.f;
    if (vec4) {
        const float4 *pa = reinterpret_cast<const float4 *>(xa);
        const float4 *pb = reinterpret_cast<const float4 *>(xb);
#pragma unroll 8
        for (int d = 0; d < (D >> 2); d++) {
            const float4 u = __ldg(pa + d), v = __ldg(pb + d);
            float t = u.x - v.x;
            s = fmaf(t, t, s);
            t = u.y - v.y;
            s = fmaf(t, t, s);
            t = u.z - v.z;
            s = fmaf(t, t, s);
            t = u.w - v.w;
            s = fmaf(t, t, s);
        }
        return s;
    }
    for (int d = 0; d < D; d++) {
        const float t = xa[d] - xb[d];
        s = fmaf(t, t, s);
    }
    return s;
}

// ---- locality order for the search (rows grouped by their nearest pivot)
// dp[q] = row q n / m of X, the m pivots (m D values)
__global__ void k_pivot_rows(int64_t n, int m, int D, const float *__restrict__ X,
                             float *__restrict__ dp) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)m * D) return;
    const int64_t q = t / D, d = t % D;
    dp[t] = X[(q * n / m) * D + d];
}

// dd[q m + r] = |p_q - p_r|^2 in FP64, the dimensions added in order
__global__ void k_pivot_d2(int m, int D, const float *__restrict__ dp, double *__restrict__ dd) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)m * m) return;
    const int64_t q = t / m, r = t % m;
    double s = 0.0;
    for (int d = 0; d < D; d++) {
        const double v = (double)dp[q * D + d] - (double)dp[r * D + d];
        s += v * v;
    }
    dd[t] = s;
}

constexpr int kCells = 512;     // pivots (cells) of the locality order
constexpr int kPivChunk = 128;  // pivots staged in shared memory at a time

// cell[i] = the pivot nearest to row i (squared Euclidean, |p|^2 - 2 x.p in
// FP32), pivots staged in shared memory; DP = D rounded up to 64.
template <int DP>
__global__ void __launch_bounds__(256)
    k_assign_cells(int64_t n, int D, int m, const float *__restrict__ X,
                   const float *__restrict__ piv, const float *__restrict__ pn,
                   const float *__restrict__ nrm, uint32_t *__restrict__ cell,
                   float *__restrict__ dpiv) {
    extern __shared__ float s_piv[];  // kPivChunk x DP
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    float xr[DP];
#pragma unroll
    for (int d = 0; d < DP; d++) xr[d] = (i < n && d < D) ? X[i * D + d] : 0.f;
    float best = INFINITY;
    uint32_t bi = 0u;
    for (int p0 = 0; p0 < m; p0 += kPivChunk) {
        const int pc = min(kPivChunk, m - p0);
        __syncthreads();
        for (int q = threadIdx.x; q < pc * DP; q += blockDim.x) {
            const int pi = q / DP, d = q % DP;
            s_piv[q] = d < D ? piv[(int64_t)(p0 + pi) * D + d] : 0.f;
        }
        __syncthreads();
        for (int pi = 0; pi < pc; pi++) {
            const float4 *pr = reinterpret_cast<const float4 *>(s_piv + pi * DP);
            float dot = 0.f;
#pragma unroll
            for (int d4 = 0; d4 < DP / 4; d4++) {
                const float4 pv = pr[d4];
                dot = fmaf(xr[4 * d4], pv.x, dot);
                dot = fmaf(xr[4 * d4 + 1], pv.y, dot);
                dot = fmaf(xr[4 * d4 + 2], pv.z, dot);
                dot = fmaf(xr[4 * d4 + 3], pv.w, dot);
            }
            const float v = fmaf(-2.0f, dot, pn[p0 + pi]);
            if (v < best) {
                best = v;
                bi = (uint32_t)(p0 + pi);
            }
        }
    }
    if (i < n) {
        cell[i] = bi;
        dpiv[i] = best + nrm[i];  // squared distance to the nearest pivot
    }
}

// Sum of v[0..n) into *out (FP64, atomics per block).
__global__ void k_sum_f64(int64_t n, const float *__restrict__ v, double *out) {
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        acc += (double)v[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

// Rows far from their nearest pivot (outliers, and rows of small clusters
// that drew no pivot) go to a cell of their own after the others, so that
// they do not share tiles with a cluster's rows.
__global__ void k_far_rows(int64_t n, const float *__restrict__ dpiv, float thr, uint32_t far_cell,
                           uint32_t *__restrict__ cell) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n && dpiv[i] > thr) cell[i] = far_cell;
}

__global__ void k_cell_count(int64_t n, const uint32_t *__restrict__ cell, uint32_t *cnt) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) atomicAdd(&cnt[cell[i]], 1u);
}

// order[r]: the row at sorted position r (rows of one cell contiguous, cells
// in chain order; the order inside a cell is immaterial to the result)
// Stable counting sort of the rows by pivot cell: the rows of a cell keep
// their index order, so the locality order, its random-projection splits and
// the tiles are the same on every run.  Blocks of kCsRows rows; a row's place
// is the offset of (its cell, its block) in the cell-major scan of the
// per-block counts, plus the rows of its cell in earlier warps of the block,
// plus those in earlier lanes of its warp.  off == NULL: write the block's
// counts hist[c * nb + b]; else scatter the rows into order.
constexpr int kCsRows = 512;
__global__ void __launch_bounds__(kCsRows)
    k_cell_rank(int64_t n, int nc, const uint32_t *__restrict__ cell, uint32_t *__restrict__ hist,
                int64_t nb, const int64_t *__restrict__ off, uint32_t *__restrict__ order) {
    __shared__ uint32_t s_cnt[kCsRows / 32][kCells + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t b = blockIdx.x;
    const int64_t i = b * kCsRows + threadIdx.x;
    for (int q = threadIdx.x; q < (kCsRows / 32) * nc; q += blockDim.x) s_cnt[q / nc][q % nc] = 0u;
    __syncthreads();
    const bool valid = i < n;
    const uint32_t c = valid ? cell[i] : 0xffffffffu;
    const unsigned same = __match_any_sync(0xffffffffu, c);
    const int rw = __popc(same & ((1u << lane) - 1u));
    if (valid && rw == 0) s_cnt[warp][c] = (uint32_t)__popc(same);
    __syncthreads();
    if (off == nullptr) {
        for (int q = threadIdx.x; q < nc; q += blockDim.x) {
            uint32_t t = 0u;
            for (int w = 0; w < kCsRows / 32; w++) t += s_cnt[w][q];
            hist[(int64_t)q * nb + b] = t;
        }
        return;
    }
    if (!valid) return;
    uint32_t before = 0u;
    for (int w = 0; w < warp; w++) before += s_cnt[w][c];
    order[off[(int64_t)c * nb + b] + before + (uint32_t)rw] = (uint32_t)i;
}

// Xs[r] = X[order[r]], ns[r] = nrm[order[r]]
__global__ void k_gather_rows(int64_t n, int D, const uint32_t *__restrict__ order,
                              const float *__restrict__ X, const float *__restrict__ nrm,
                              float *__restrict__ Xs, float *__restrict__ ns) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= n * D) return;
    const int64_t r = q / D;
    const int d = (int)(q % D);
    const uint32_t i = order[r];
    Xs[q] = X[(int64_t)i * D + d];
    if (d == 0) ns[r] = nrm[i];
}

// ---- random-projection refinement of the locality order, and the
// approximate search's per-tile candidate lists.
//
// Every segment of the order (at first a pivot cell) is split in two by the
// hyperplane that bisects two of its rows, picked by a hash of the segment and
// the level (the random-projection trees of Sec. 4.3, with the bisecting
// splits of LargeVis and Annoy); the rows on the first one's side go first.
// Segments of at most kTcRows rows stay as they are, so the tiles of 128
// consecutive rows end up spatially compact, their radii small and the tile
// bound of the search tight.  The order inside a pivot cell comes from
// atomics, so the splits may differ between runs: the exact search's lists do
// not depend on them, the approximate search's may.
__device__ __forceinline__ uint32_t mix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

// seg[r] = [start, end) of the pivot cell of the row at position r
__global__ void k_seg_init(int64_t n, const uint32_t *__restrict__ order,
                           const uint32_t *__restrict__ cell, const uint32_t *__restrict__ cstart,
                           int2 *__restrict__ seg) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n) return;
    const uint32_t c = cell[order[r]];
    seg[r] = make_int2((int)cstart[c], (int)cstart[c + 1]);
}

// flag[r] = 1 if the row at position r lies on the side of its segment's
// first split row (or its segment is not split), else 0
__global__ void k_rp_side(int64_t n, int D, const float *__restrict__ X,
                          const uint32_t *__restrict__ order, const int2 *__restrict__ seg,
                          int level, uint32_t *__restrict__ flag) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int2 sg = seg[r];
    const int size = sg.y - sg.x;
    if (size <= kTcRows) {
        flag[r] = 1u;
        return;
    }
    const uint32_t h = mix32((uint32_t)sg.x * 0x9e3779b9u ^ (uint32_t)(level * 0x632be5abu));
    const int oa = (int)(h % (uint32_t)size);
    const int ob = (oa + 1 + (int)(mix32(h + 1u) % (uint32_t)(size - 1))) % size;
    const float *xa = X + (int64_t)order[sg.x + oa] * D;
    const float *xb = X + (int64_t)order[sg.x + ob] * D;
    const float *xi = X + (int64_t)order[r] * D;
    float p = 0.f;
    for (int d = 0; d < D; d++) {
        const float u = __ldg(xa + d), v = __ldg(xb + d);
        p = fmaf(__ldg(xi + d) - 0.5f * (u + v), u - v, p);
    }
    flag[r] = p >= 0.f ? 1u : 0u;
}

// Stable partition of every split segment by flag (pref = exclusive scan of
// flag over all positions): first-side rows first; each half becomes a
// segment.  A segment that every row (or none) fell on one side of is kept
// whole and split again at the next level with other rows.
__global__ void k_rp_scatter(int64_t n, const uint32_t *__restrict__ order,
                             const int2 *__restrict__ seg, const uint32_t *__restrict__ flag,
                             const int64_t *__restrict__ pref, uint32_t *__restrict__ order2,
                             int2 *__restrict__ seg2) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int2 sg = seg[r];
    const int64_t size = sg.y - sg.x;
    const int64_t ps = pref[sg.x];
    const int64_t lc = pref[sg.y] - ps;
    if (size <= kTcRows || lc == 0 || lc == size) {
        order2[r] = order[r];
        seg2[r] = sg;
        return;
    }
    const int64_t before = pref[r] - ps;  // first-side rows before r in its segment
    int64_t pos;
    int2 ns;
    if (flag[r]) {
        pos = sg.x + before;
        ns = make_int2(sg.x, sg.x + (int)lc);
    } else {
        pos = sg.x + lc + (r - sg.x - before);
        ns = make_int2(sg.x + (int)lc, sg.y);
    }
    order2[pos] = order[r];
    seg2[pos] = ns;
}

// cand[q W .. q W + W): the W tiles whose centroids are nearest to the query
// tile's, the own tile first, ascending by (distance, tile).  (Ranking by the
// triangle-inequality bound |c_q - c_t| - r_t instead would put the few tiles
// of wide radius -- outliers spread over the whole space -- ahead of the
// query's own cluster.)  One CTA per query tile keeps the best in shared memory,
// sorting (bitonic) whenever the buffer may not hold another chunk.
constexpr int kCandThreads = 256;
constexpr int kCandCap = 2048;  // buffer entries; W <= kCandCap - kCandThreads

__device__ void cand_sort(float *b, int *t, int cnt) {
    for (int i = cnt + threadIdx.x; i < kCandCap; i += kCandThreads) {
        b[i] = INFINITY;
        t[i] = 0x7fffffff;
    }
    __syncthreads();
    for (int k = 2; k <= kCandCap; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < kCandCap; i += kCandThreads) {
                const int l = i ^ j;
                if (l > i) {
                    const bool up = (i & k) == 0;
                    const bool gt = b[i] > b[l] || (b[i] == b[l] && t[i] > t[l]);
                    if (gt == up) {
                        const float fb = b[i];
                        b[i] = b[l];
                        b[l] = fb;
                        const int ft = t[i];
                        t[i] = t[l];
                        t[l] = ft;
                    }
                }
            }
            __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(kCandThreads)
    k_tile_cands(int64_t T, int Dp, const float *__restrict__ cent, int W,
                 int32_t *__restrict__ cand) {
    __shared__ float s_b[kCandCap];
    __shared__ int s_t[kCandCap];
    __shared__ float s_cq[128];
    __shared__ int s_cnt;
    __shared__ float s_thr;
    const int64_t qt = blockIdx.x;
    for (int d = threadIdx.x; d < Dp; d += kCandThreads) s_cq[d] = cent[qt * Dp + d];
    if (threadIdx.x == 0) {
        s_cnt = 0;
        s_thr = INFINITY;
    }
    __syncthreads();
    for (int64_t t0 = 0; t0 < T; t0 += kCandThreads) {
        const int64_t t = t0 + threadIdx.x;
        if (t < T) {
            float b = -INFINITY;
            if (t != qt) {
                const float4 *ct = reinterpret_cast<const float4 *>(cent + t * Dp);
                float dd = 0.f;
                for (int d4 = 0; d4 < Dp / 4; d4++) {
                    const float4 c = __ldg(ct + d4);
                    const float e0 = s_cq[4 * d4] - c.x, e1 = s_cq[4 * d4 + 1] - c.y;
                    const float e2 = s_cq[4 * d4 + 2] - c.z, e3 = s_cq[4 * d4 + 3] - c.w;
                    dd = fmaf(e0, e0, fmaf(e1, e1, fmaf(e2, e2, fmaf(e3, e3, dd))));
                }
                b = dd;
            }
            if (b < s_thr) {
                const int slot = atomicAdd(&s_cnt, 1);
                s_b[slot] = b;
                s_t[slot] = (int)t;
            }
        }
        __syncthreads();
        if (s_cnt > kCandCap - kCandThreads) {
            cand_sort(s_b, s_t, s_cnt);
            if (threadIdx.x == 0) {
                s_cnt = W;
                s_thr = s_b[W - 1];
            }
            __syncthreads();
        }
    }
    cand_sort(s_b, s_t, s_cnt);
    for (int i = threadIdx.x; i < W; i += kCandThreads) cand[qt * W + i] = s_t[i];
}

// A neighbour-list entry; (d, j) orders by distance, then by index.
struct __align__(8) KnnEntry {
    float d;
    int32_t j;
};
__device__ __forceinline__ bool knn_worse(KnnEntry a, KnnEntry b) {
    return a.d > b.d || (a.d == b.d && a.j > b.j);
}

struct KnnTcArgs {
    int64_t n, T;
    int D, Dp, k;
    float inv_s2, kappa, eps_abs;
    const float *X;       // FP32 rows (exact distances)
    const uint8_t *img;   // FP16 tile images
    const float *nrm;     // |x~|^2 of the rounded rows
    const float *rerr;    // |x~ - x|, rounded up
    const float *HG;      // per tile: h_j, |c_j|, chunk bounds (kHG floats)
    const uint32_t *order;  // sorted position -> row of X (the locality order)
    int32_t *out_idx;
    float *out_d2;
    unsigned *err;
    u64 *stats;
    const float *cent;    // per tile: centroid of its rows (Dp floats, FP32)
    const float *rad;     // per tile: an upper bound of |x - centroid| over its rows
    const int32_t *cand;  // approximate search: per query tile its W candidate tiles
    int W;                //   (own tile first); NULL: every tile (the exact search)
};

// The i-th candidate tile a CTA visits: its own, then alternately the next
// and the previous ones (mod T), so that the rows nearby in the locality order
// come first.
__device__ __forceinline__ int64_t knn_tile_at(int64_t qt, int64_t i, int64_t T) {
    const int64_t off = (i & 1) ? (i + 1) / 2 : -(i / 2);
    return ((qt + off) % T + T) % T;
}

__global__ void __launch_bounds__(kTcThreads, 1) k_knn_tc(const KnnTcArgs a) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t bar_a, bar_sf[kTcStages], bar_se[kTcStages], bar_tf[kTcAcc],
        bar_te[kTcAcc], bar_hf[kTcAcc], bar_he[kTcAcc];
    __shared__ uint32_t tslot;
    __shared__ volatile int s_abort;
    // pruning: per filter warp the largest current k-th distance of its rows
    // (only decreases), and the candidate tile of each kept slot (-1: end)
    __shared__ volatile float s_taumax[kTcFilterWarps];
    // the two filter warps of a lane quarter insert into the same rows'
    // lists, one at a time: a lock per quarter
    __shared__ int s_lock[4];
    __shared__ volatile int s_tile[8];
    __shared__ float s_cq[128];  // the query tile's centroid (loader warp)
    // 1024-byte aligned base for the swizzled operand tiles
    uint8_t *smem = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
    const int64_t n = a.n, T = a.T;
    const int k = a.k;
    const uint32_t tile_bytes = (uint32_t)kTcRows * a.Dp * 2;
    uint8_t *sA = smem;
    uint8_t *sB = smem + tile_bytes;
    // per accumulator: h_j (128) then g_j (128) of its tile
    float *hbuf = reinterpret_cast<float *>(sB + (size_t)kTcStages * tile_bytes);  // [4][kHG]
    // per row: its k best (d2, index) so far as a max-heap on (d2, index),
    // rows at an odd stride (no bank conflicts between the rows)
    const int ks = k | 1;
    KnnEntry *lst = reinterpret_cast<KnnEntry *>(hbuf + kTcAcc * kHG);
    // per filter warp: queued survivors (row lane << 24 | candidate index),
    // their exact d2 and, per entry, the previous entry of the same row
    uint32_t *qc_all = reinterpret_cast<uint32_t *>(lst + kTcRows * ks);
    float *qd_all = reinterpret_cast<float *>(qc_all + kTcFilterWarps * kTcQueue);
    uint16_t *qp_all = reinterpret_cast<uint16_t *>(qd_all + kTcFilterWarps * kTcQueue);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t qt = blockIdx.x;  // query tile
    const int64_t q0 = qt * kTcRows;

    for (int e = tid; e < kTcRows * ks; e += kTcThreads) lst[e] = KnnEntry{INFINITY, 0x7fffffff};
    if (warp == kTcMmaWarp) tc::tmem_alloc(&tslot, kTcAcc * kTcCols);
    if (tid == 0) {
        tc::mbar_init(&bar_a, 1);
        for (int s = 0; s < kTcStages; s++) {
            tc::mbar_init(&bar_sf[s], 1);
            tc::mbar_init(&bar_se[s], 1);
        }
        for (int b = 0; b < kTcAcc; b++) {
            tc::mbar_init(&bar_tf[b], 1);
            tc::mbar_init(&bar_te[b], kTcFilterWarps);
            tc::mbar_init(&bar_hf[b], 1);
            tc::mbar_init(&bar_he[b], kTcFilterWarps);
        }
        s_abort = 0;
        for (int w = 0; w < kTcFilterWarps; w++) s_taumax[w] = INFINITY;
        for (int w = 0; w < 4; w++) s_lock[w] = 0;
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tbase = tslot;

    if (warp == kTcLoadWarp) {
        // ---- producer: candidate tiles and their h values.  A tile whose
        // rows are all farther from every query row than that row's current
        // k-th distance (triangle inequality on the tiles' centroids and
        // radii, against the largest current k-th distance of the CTA) is
        // skipped.  The kept tiles form a sequence j = 0, 1, ... that the
        // MMA issuer and the filter warps follow through s_tile; the entry
        // after the last kept tile is -1 (barriers completed without data).
        // the query tile's centroid, for every lane
        for (int d = lane; d < a.Dp; d += 32) s_cq[d] = a.cent[qt * a.Dp + d];
        __syncwarp();
        const float rq = a.rad[qt];
        if (lane == 0) {
            tc::mbar_expect_tx(&bar_a, tile_bytes);
            tc::bulk_g2s(sA, a.img + qt * tile_bytes, tile_bytes, &bar_a);
        }
        int64_t j = 0;  // kept tiles so far
        u64 n_skip = 0u;
        bool fail = false;
        int64_t n_sf = 0, n_hf = 0;  // stage and h copies issued (kept tiles 0 ..)
        // the tiles are judged 32 at a time, one per lane; the kept ones are
        // then issued in order
        // candidate tiles: every tile outward from the own one, or (the
        // approximate search) the W listed for this query tile
        const int64_t NT = a.cand ? (int64_t)a.W : T;
        for (int64_t i0 = 0; i0 <= NT && !fail; i0 += 32) {
            // (one reading of the abort flag for the whole warp)
            if (__shfl_sync(0xffffffffu, s_abort, 0)) break;
            const int64_t il = i0 + lane;
            const bool in = il < NT;
            const int64_t tl =
                in ? (a.cand ? (int64_t)__ldg(a.cand + qt * a.W + il) : knn_tile_at(qt, il, T)) : 0;
            float dd = 0.f;
            if (in) {
                const float4 *ct = reinterpret_cast<const float4 *>(a.cent + tl * a.Dp);
                for (int d4 = 0; d4 < a.Dp / 4; d4++) {
                    const float4 c = __ldg(ct + d4);
                    const float e0 = s_cq[4 * d4] - c.x, e1 = s_cq[4 * d4 + 1] - c.y;
                    const float e2 = s_cq[4 * d4 + 2] - c.z, e3 = s_cq[4 * d4 + 3] - c.w;
                    dd = fmaf(e0, e0, fmaf(e1, e1, fmaf(e2, e2, fmaf(e3, e3, dd))));
                }
            }
            float taum = s_taumax[0];
#pragma unroll
            for (int w = 1; w < kTcFilterWarps; w++) taum = fmaxf(taum, s_taumax[w]);
            const float lbd = sqrtf(dd) * 0.9999f - rq - (in ? a.rad[tl] : 0.f);
            // (the approximate search takes its W tiles whole: with the bound,
            // which tiles pass would depend on how far the filter warps have
            // got, and the lists would differ between runs)
            const bool skip =
                in && il > 0 && !a.cand && lbd > 0.f && lbd * lbd > taum * 1.0001f;
            n_skip += (u64)__popc(__ballot_sync(0xffffffffu, skip));
            // kept tiles of this block, and the end mark after the last block
            unsigned keep = __ballot_sync(0xffffffffu, in && !skip);
            const bool last_block = i0 + 32 > NT;
            while (keep || last_block) {
                const bool end = keep == 0u;  // (only in the last block)
                int64_t t = -1;
                if (!end) {
                    const int src = __ffs(keep) - 1;
                    keep &= keep - 1u;
                    t = __shfl_sync(0xffffffffu, tl, src);
                }
            const int s = (int)(j % kTcStages), b = (int)(j % kTcAcc);
            // every lane waits (a converged warp is suspended and woken as
            // one); lane 0 writes the slot and issues the copies
            bool ok = j < kTcStages ||
                      tc::mbar_wait_sleep(&bar_se[s], (uint32_t)((j / kTcStages - 1) & 1), kTcPolls, kTcSleepNs);
            ok = __all_sync(0xffffffffu, ok);
            if (ok) {
                if (lane == 0) {
                    s_tile[j & 7] = (int)t;
                    if (end) {
                        tc::mbar_arrive(&bar_sf[s]);
                    } else {
                        tc::mbar_expect_tx(&bar_sf[s], tile_bytes);
                        tc::bulk_g2s(sB + (size_t)s * tile_bytes, a.img + t * tile_bytes, tile_bytes,
                                     &bar_sf[s]);
                    }
                }
                if (!end) n_sf++;
                __syncwarp();
                ok = j < kTcAcc ||
                     tc::mbar_wait_sleep(&bar_he[b], (uint32_t)((j / kTcAcc - 1) & 1), kTcPolls, kTcSleepNs);
                ok = __all_sync(0xffffffffu, ok);
                if (ok) {
                    if (lane == 0) {
                        if (end) {
                            tc::mbar_arrive(&bar_hf[b]);
                        } else {
                            tc::mbar_expect_tx(&bar_hf[b], kHG * 4);
                            tc::bulk_g2s(hbuf + b * kHG, a.HG + t * kHG, kHG * 4, &bar_hf[b]);
                        }
                    }
                    if (!end) n_hf++;
                }
            }
            if (!ok) {
                fail = true;
                if (lane == 0) {
                    s_abort = 1;
                    atomicOr(a.err, (unsigned)PXSNE_DEVERR_TIMEOUT);
                }
            }
            __syncwarp();
            if (fail) break;
            if (end) break;
            j++;
            }
        }
        if (lane == 0) {
            atomicAdd(&a.stats[2], n_skip);
            // copies still in flight complete before the CTA exits: those of
            // the last kept tiles (kept tile q used stage q % 2 and h slot
            // q % 4).  After the end mark the copies into the slots it reused
            // are known complete (their consumers released them first), and
            // waiting on them by phase parity would be ambiguous.
            const int64_t ws = fail ? kTcStages : kTcStages - 1, wh = fail ? kTcAcc : kTcAcc - 1;
            tc::mbar_wait(&bar_a, 0u, kTcPolls);
            for (int64_t q = (n_sf > ws ? n_sf - ws : 0); q < n_sf; q++)
                tc::mbar_wait(&bar_sf[q % kTcStages], (uint32_t)((q / kTcStages) & 1), kTcPolls);
            for (int64_t q = (n_hf > wh ? n_hf - wh : 0); q < n_hf; q++)
                tc::mbar_wait(&bar_hf[q % kTcAcc], (uint32_t)((q / kTcAcc) & 1), kTcPolls);
        }
    } else if (warp == kTcMmaWarp) {
        // ---- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_f16(kTcRows, kTcCols, 0);
            const uint32_t a0 = tc::smem_u32(sA);
            bool ok = tc::mbar_wait(&bar_a, 0u, kTcPolls);
            int64_t i = 0;  // kept tiles multiplied
            bool ended = false;
            for (; ok && i <= T && !s_abort; i++) {
                const int s = (int)(i % kTcStages), b = (int)(i % kTcAcc);
                ok = tc::mbar_wait_sleep(&bar_sf[s], (uint32_t)((i / kTcStages) & 1), kTcPolls, kTcSleepNs);
                if (ok && i >= kTcAcc)
                    ok = tc::mbar_wait_sleep(&bar_te[b], (uint32_t)((i / kTcAcc - 1) & 1), kTcPolls, kTcSleepNs);
                if (!ok) break;
                tc::fence_after();
                if (s_tile[i & 7] < 0) {
                    // the end: the filter warps learn it through an
                    // accumulator completed without data
                    tc::mbar_arrive(&bar_tf[b]);
                    ended = true;
                    break;
                }
                const uint32_t b0 = tc::smem_u32(sB + (size_t)s * tile_bytes);
                for (int kk = 0; kk < a.Dp / 16; kk++) {
                    const uint32_t off =
                        (uint32_t)(kk >> 2) * (kTcRows * 128) + (uint32_t)(kk & 3) * 32;
                    tc::mma_f16(tbase + (uint32_t)(b * kTcCols), tc::sdesc_sw128(a0 + off),
                                tc::sdesc_sw128(b0 + off), idesc, kk > 0 ? 1u : 0u);
                }
                tc::commit(&bar_se[s]);
                tc::commit(&bar_tf[b]);
            }
            if (!ok) {
                s_abort = 1;
                atomicOr(a.err, (unsigned)PXSNE_DEVERR_TIMEOUT);
            }
            // MMAs still in flight finish before TMEM is freed.  After the end
            // mark, the MMA into the accumulator it reused is known complete
            // (the filter warps released it first), and waiting on it by
            // phase parity would be ambiguous.
            const int64_t wa = ended ? kTcAcc - 1 : kTcAcc;
            for (int64_t j = (i > wa ? i - wa : 0); j < i; j++)
                tc::mbar_wait(&bar_tf[j % kTcAcc], (uint32_t)((j / kTcAcc) & 1), kTcPolls);
        }
    } else {
        // ---- filter: warps quarter and quarter + 4 own query rows
        // q0 + 32 quarter + lane; warp `half` filters columns 64 half .. +63
        const int quarter = warp & 3, half = warp >> 2;
        const int64_t qi = q0 + 32 * quarter + lane;
        const bool qvalid = qi < n;
        const float qn2 = qvalid ? a.nrm[qi] : 0.f, qn1 = sqrtf(qn2);
        const float Eq = qvalid ? a.rerr[qi] : 0.f;
        KnnEntry *heap = lst + (size_t)(32 * quarter + lane) * ks;
        float tau = INFINITY;
        int32_t jlast = 0x7fffffff;
        uint32_t n_exact = 0u, n_ins = 0u;
        const float Bq = a.kappa * qn1;
        const float onem = 1.0f - a.eps_abs;
        const float cneg = -2.0f * a.inv_s2;
        const bool vec4 = ((a.D & 3) == 0) && ((reinterpret_cast<uintptr_t>(a.X) & 15) == 0);
        // sqrt(tau) + |q~ - q| (+inf while the list fills); a chunk's
        // threshold adds its rows' largest rounding error
        float sqE = INFINITY;
        uint32_t *wq = qc_all + warp * kTcQueue;
        float *wd = qd_all + warp * kTcQueue;
        uint16_t *wp = qp_all + warp * kTcQueue;
        constexpr uint32_t kNil = 0xffffu;
        uint32_t qn = 0u;       // entries in the warp's queue (warp-uniform)
        uint32_t head = kNil;   // this row's last queued entry
        // exact distances of the queued survivors, one per lane, then every
        // lane walks its own row's chain and inserts
        auto flush = [&]() {
            __syncwarp();
            for (uint32_t q = lane; q < qn; q += 32) {
                const uint32_t e = wq[q];
                wd[q] = thread_exact_d2(a.X, a.D, q0 + 32 * quarter + (e >> 24), e & 0xffffffu,
                                        vec4);
            }
            __syncwarp();
            // the lists of these rows are shared with the quarter's other
            // filter warp: insert while holding the quarter's lock (bounded
            // wait; the holder waits on nothing), from the lists' current roots
            bool locked = true;
            if (lane == 0) {
                int it = 0;
                while (atomicCAS(&s_lock[quarter], 0, 1) != 0) {
                    if (++it >= kTcPolls) {
                        locked = false;
                        break;
                    }
                    __nanosleep(64);
                }
            }
            locked = __shfl_sync(0xffffffffu, locked, 0);
            __threadfence_block();
            if (!locked) {
                s_abort = 1;
                if (lane == 0) atomicOr(a.err, (unsigned)PXSNE_DEVERR_TIMEOUT);
                head = kNil;
            } else {
                const KnnEntry r0 = heap[0];
                tau = r0.d;
                jlast = r0.j;
            }
            for (uint32_t q = head; q != kNil; q = wp[q]) {
                const int32_t cand = (int32_t)__ldg(a.order + (wq[q] & 0xffffffu));
                const float d = wd[q];
                n_exact++;
                if (!(d < tau || (d == tau && cand < jlast))) continue;
                n_ins++;
                // the new entry replaces the worst (the root) and sinks
                const KnnEntry ne{d, cand};
                int p = 0;
                for (;;) {
                    int m = 2 * p + 1;
                    if (m >= k) break;
                    KnnEntry cm = heap[m];
                    if (m + 1 < k) {
                        const KnnEntry cr = heap[m + 1];
                        if (knn_worse(cr, cm)) {
                            cm = cr;
                            m++;
                        }
                    }
                    if (!knn_worse(cm, ne)) break;
                    heap[p] = cm;
                    p = m;
                }
                heap[p] = ne;
                const KnnEntry rt = heap[0];
                tau = rt.d;
                jlast = rt.j;
            }
            __syncwarp();
            __threadfence_block();
            if (locked && lane == 0) atomicExch(&s_lock[quarter], 0);
            sqE = sqrtf(tau) + Eq;
            head = kNil;
            qn = 0u;
            // the largest current k-th distance of the warp's rows, for the
            // loader's pruning (rows past n do not count)
            float tm = qvalid ? tau : -INFINITY;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) tm = fmaxf(tm, __shfl_xor_sync(0xffffffffu, tm, o));
            if (lane == 0) s_taumax[warp] = tm;
        };
        for (int64_t i = 0; i <= T; i++) {  // the kept tiles, then the end mark
            const int b = (int)(i % kTcAcc);
            const uint32_t par = (uint32_t)((i / kTcAcc) & 1);
            // warp-uniform: every lane takes the same path into the aligned
            // TMEM loads and the warp-synchronous queue below
            const bool got =
                __all_sync(0xffffffffu, tc::mbar_wait_sleep(&bar_tf[b], par, kTcPolls, kTcSleepNs) &&
                                            tc::mbar_wait_sleep(&bar_hf[b], par, kTcPolls, kTcSleepNs));
            if (!got || s_abort) {
                s_abort = 1;
                if (!got && lane == 0) atomicOr(a.err, (unsigned)PXSNE_DEVERR_TIMEOUT);
                break;
            }
            tc::fence_after();
            const int tt = s_tile[i & 7];
            if (tt < 0) break;  // no more kept tiles
            const int64_t t = tt;
            const int64_t c0 = t * kTcCols;
            const float *hb = hbuf + b * kHG;
            // the other warp of the quarter may have tightened the rows' lists
            // (a root read while it inserts is the old or the new one, both
            // at least the final k-th distance)
            {
                const float tr = reinterpret_cast<volatile const KnnEntry *>(heap)->d;
                if (tr < tau) sqE = sqrtf(tr) + Eq;
            }
            // the warp's 64 columns of its rows in one round trip; the
            // accumulator is released right after, h and g after the filter
            uint32_t raw[2][32];
#pragma unroll
            for (int cc = 0; cc < 2; cc++)
                tc::tmem_ld32_async(tbase + ((uint32_t)(32 * quarter) << 16) +
                                        (uint32_t)(b * kTcCols + 64 * half + 32 * cc),
                                    raw[cc]);
            tc::tmem_wait_ld();
            tc::fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&bar_te[b]);
#pragma unroll
            for (int cc = 0; cc < 2; cc++) {
                const int ci = 2 * half + cc;
                const int cb = 32 * ci;
                float v[32];
#pragma unroll
                for (int j = 0; j < 32; j++) v[j] = __uint_as_float(raw[cc][j]);
                // Chunk bound: e_j >= min h - kappa|q| max g - 2 max_j q.c
                // (-2 < 0, kappa|q| >= 0).  A chunk whose bound exceeds the
                // threshold by more than the FP32 roundings of both sides
                // (margin 2^-19 of the terms' sizes, eight times their bound)
                // has no survivor, and its per-candidate values are not formed.
                float mx[8];
#pragma unroll
                for (int j4 = 0; j4 < 8; j4++)
                    mx[j4] = fmaxf(fmaxf(v[4 * j4], v[4 * j4 + 1]), fmaxf(v[4 * j4 + 2], v[4 * j4 + 3]));
                const float vmax = fmaxf(fmaxf(fmaxf(mx[0], mx[1]), fmaxf(mx[2], mx[3])),
                                         fmaxf(fmaxf(mx[4], mx[5]), fmaxf(mx[6], mx[7])));
                const float hmin = hb[2 * kTcCols + ci], gmax = hb[2 * kTcCols + 4 + ci];
                // survivors: |q~ - c~| <= sqrt(tau) + |q~ - q| + |c~ - c| (the
                // true distance is at least the rounded rows' distance less
                // both rounding errors), squared with a margin of 2^-20 for
                // its own rounding; tau - (1 - eps)|q~|^2 in the form below,
                // finite while the list fills so that padding (+inf) never passes
                const float tE = sqE + hb[2 * kTcCols + 8 + ci];
                const float tauA =
                    fminf(fmaf(tE * tE, 9.5367431640625e-07f, tE * tE) - onem * qn2, 3.402823466e38f);
                const float lb = fmaf(cneg, vmax, fmaf(-Bq, gmax, hmin));
                const float margin = (fabsf(hmin) + Bq * gmax + fabsf(cneg * vmax)) * 1.9073486e-6f;
                const bool near = qvalid && !(lb > tauA + margin);
                float m = INFINITY;
                if (near) {
                    // e_j = (1-eps)|c~|^2 - kappa|q~||c~| - 2 q~.c~ (in place of v)
                    float mn[8];
#pragma unroll
                    for (int j4 = 0; j4 < 8; j4++) {
                        const float4 h4 = *reinterpret_cast<const float4 *>(hb + cb + 4 * j4);
                        const float4 g4 = *reinterpret_cast<const float4 *>(hb + kTcCols + cb + 4 * j4);
                        v[4 * j4] = fmaf(-Bq, g4.x, fmaf(cneg, v[4 * j4], h4.x));
                        v[4 * j4 + 1] = fmaf(-Bq, g4.y, fmaf(cneg, v[4 * j4 + 1], h4.y));
                        v[4 * j4 + 2] = fmaf(-Bq, g4.z, fmaf(cneg, v[4 * j4 + 2], h4.z));
                        v[4 * j4 + 3] = fmaf(-Bq, g4.w, fmaf(cneg, v[4 * j4 + 3], h4.w));
                        mn[j4] = fminf(fminf(v[4 * j4], v[4 * j4 + 1]), fminf(v[4 * j4 + 2], v[4 * j4 + 3]));
                    }
                    m = fminf(fminf(fminf(mn[0], mn[1]), fminf(mn[2], mn[3])),
                              fminf(fminf(mn[4], mn[5]), fminf(mn[6], mn[7])));
                }
                uint32_t sm = 0u;
                if (near && m <= tauA) {
                    // survivors: e_j <= (sqrt(tau) + E_q + max E_c)^2 - (1-eps)|q~|^2
#pragma unroll
                    for (int j = 0; j < 32; j++) sm |= (v[j] <= tauA) ? (1u << j) : 0u;
                    if (qi >= c0 + cb && qi < c0 + cb + 32) sm &= ~(1u << (int)(qi - c0 - cb));
                }
                if (__any_sync(0xffffffffu, sm != 0u)) {
                    // append the chunk's survivors to the queue, 8 columns at
                    // a time (at most 256 entries, which a flushed queue holds;
                    // flush first if they might not fit); one warp scan gives
                    // two groups' positions (16-bit fields)
                    uint32_t incl4[2], tot4[2];
#pragma unroll
                    for (int pr = 0; pr < 2; pr++) {
                        uint32_t x = (uint32_t)__popc(sm & (0xffu << (16 * pr))) |
                                     ((uint32_t)__popc(sm & (0xff00u << (16 * pr))) << 16);
#pragma unroll
                        for (int o = 1; o < 32; o <<= 1) {
                            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                            if (lane >= o) x += y;
                        }
                        incl4[pr] = x;
                        tot4[pr] = __shfl_sync(0xffffffffu, x, 31);
                    }
#pragma unroll
                    for (int hf = 0; hf < 4; hf++) {
                        const uint32_t hm = sm & (0xffu << (8 * hf));
                        const uint32_t cnt = (uint32_t)__popc(hm);
                        const uint32_t incl = (hf & 1) ? (incl4[hf >> 1] >> 16) : (incl4[hf >> 1] & 0xffffu);
                        const uint32_t total = (hf & 1) ? (tot4[hf >> 1] >> 16) : (tot4[hf >> 1] & 0xffffu);
                        if (total == 0u) continue;
                        if (qn + total > (uint32_t)kTcQueue) flush();
                        uint32_t mm = hm;
                        for (uint32_t q = qn + incl - cnt; mm; q++) {
                            const int j = __ffs(mm) - 1;
                            mm &= mm - 1u;
                            wq[q] = ((uint32_t)lane << 24) | (uint32_t)(c0 + cb + j);
                            wp[q] = (uint16_t)head;
                            head = q;
                        }
                        qn += total;
                        __syncwarp();
                    }
                }
            }
            // the tile's h and g are no longer needed
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&bar_he[b]);
            // the queue is flushed once it holds a batch
            if (qn >= kTcFlushAt) flush();
        }
        if (qn) flush();
        atomicAdd(&a.stats[0], (u64)n_exact);
        atomicAdd(&a.stats[1], (u64)n_ins);
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == kTcMmaWarp) tc::tmem_dealloc(tbase, kTcAcc * kTcCols);
    // heap sort of each row's list (ascending), then out
    if (tid < kTcRows) {
        KnnEntry *heap = lst + (size_t)tid * ks;
        for (int last = k - 1; last > 0; last--) {
            const KnnEntry top = heap[0], ne = heap[last];
            heap[last] = top;
            int p = 0;
            for (;;) {
                int m = 2 * p + 1;
                if (m >= last) break;
                KnnEntry cm = heap[m];
                if (m + 1 < last) {
                    const KnnEntry cr = heap[m + 1];
                    if (knn_worse(cr, cm)) {
                        cm = cr;
                        m++;
                    }
                }
                if (!knn_worse(cm, ne)) break;
                heap[p] = cm;
                p = m;
            }
            heap[p] = ne;
        }
    }
    __syncthreads();
    for (int e = tid; e < kTcRows * k; e += kTcThreads) {
        const int r = e / k, j = e % k;
        const int64_t row = q0 + r;
        if (row < n) {
            const KnnEntry v = lst[r * ks + j];
            const int64_t orow = a.order[row];
            a.out_idx[orow * k + j] = v.j;
            a.out_d2[orow * k + j] = v.d;
        }
    }
}

static size_t knn_tc_smem(int Dp, int k) {
    return (size_t)(1 + kTcStages) * kTcRows * Dp * 2 + (size_t)kTcAcc * kHG * 4 +
           (size_t)kTcRows * (k | 1) * 8 + (size_t)kTcFilterWarps * kTcQueue * (4 + 4 + 2) + 1024;
}

// The bounded wait of the pipelines above, on an mbarrier that nothing
// arrives at: it must give up after `polls` polls and flag the time-out.
__global__ void k_wait_probe(int polls, unsigned *err) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) tc::mbar_init(&bar, 1);
    __syncthreads();
    const bool got = __all_sync(0xffffffffu, tc::mbar_wait_sleep(&bar, 0u, polls, 100u));
    if (!got && threadIdx.x == 0) atomicOr(err, (unsigned)PXSNE_DEVERR_TIMEOUT);
}

void launch_wait_probe(pxsne_ctx *c, int polls) {
    k_wait_probe<<<1, 32, 0, c->stream>>>(polls, &c->sc->err);
}

// Timing events around the search kernel (created on first use).
// ---------------------------------------------------------------- neighbour exploring
// Sec. 4.3's refinement of approximate neighbour lists (LargeVis' neighbour
// exploring): a row's new list is the k nearest among its old list and the
// old lists of its first ke neighbours.  One warp per row, the rows taken in
// the search's locality order so that neighbouring warps gather neighbouring
// rows of Xs; the list lives in shared memory sorted by (d2, index) (the
// search's order and tie rule), and each candidate that beats the current
// k-th entry and is not listed yet is inserted by a warp-wide shift.  The
// distance is the search's exact FP32 one (thread_exact_d2 on the same
// rows), so an entry found by both has the same d2.  Lists are read from
// (idx_in, d2_in) and written to (idx_out, d2_out): the result does not
// depend on the order in which rows are processed.
constexpr int kExploreNbrs = 16;
constexpr int kExploreWarps = 8;
__global__ void __launch_bounds__(kExploreWarps * 32)
    k_knn_explore(int64_t n, int k, int ke, int D, int vec4, const float *__restrict__ Xs,
                  const uint32_t *__restrict__ order, const uint32_t *__restrict__ rank,
                  const int32_t *__restrict__ idx_in, const float *__restrict__ d2_in,
                  int32_t *__restrict__ idx_out, float *__restrict__ d2_out) {
    __shared__ float s_d[kExploreWarps][256];
    __shared__ int32_t s_j[kExploreWarps][256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t p = (int64_t)blockIdx.x * kExploreWarps + warp;
    if (p >= n) return;
    const int64_t i = order[p];
    // (an entry outside [0, n), which a full list never holds, is not followed)
    float *ld = s_d[warp];
    int32_t *lj = s_j[warp];
    for (int e = lane; e < k; e += 32) {
        ld[e] = d2_in[i * k + e];
        lj[e] = idx_in[i * k + e];
    }
    __syncwarp();
    float tau = ld[k - 1];
    int32_t jl = lj[k - 1];
    for (int e = 0; e < ke; e++) {
        const int64_t j = __ldg(idx_in + i * k + e);
        if (j < 0 || j >= n) continue;
        for (int f0 = 0; f0 < k; f0 += 32) {
            const int f = f0 + lane;
            int32_t l = -1;
            float d = INFINITY;
            if (f < k) {
                l = __ldg(idx_in + j * k + f);
                if (l < 0 || (int64_t)l >= n) l = -1;
                else if (l != (int32_t)i)
                    d = thread_exact_d2(Xs, D, p, (int64_t)__ldg(rank + l), vec4 != 0);
            }
            const bool pass = l >= 0 && l != (int32_t)i && (d < tau || (d == tau && l < jl));
            unsigned m = __ballot_sync(0xffffffffu, pass);
            while (m) {
                const int src = __ffs(m) - 1;
                m &= m - 1u;
                const float dc = __shfl_sync(0xffffffffu, d, src);
                const int32_t lc = __shfl_sync(0xffffffffu, l, src);
                if (!(dc < tau || (dc == tau && lc < jl))) continue;  // the list moved on
                bool dup = false;
                int before = 0;
                for (int q = lane; q < k; q += 32) {
                    dup |= lj[q] == lc;
                    before += (ld[q] < dc || (ld[q] == dc && lj[q] < lc)) ? 1 : 0;
                }
                if (__any_sync(0xffffffffu, dup)) continue;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) before += __shfl_xor_sync(0xffffffffu, before, o);
                // entries before .. k - 2 move down one place, the last drops
                float vd[8];
                int32_t vj[8];
#pragma unroll
                for (int t = 0; t < 8; t++) {
                    const int q = lane + 32 * t;
                    if (q < k && q > before) {
                        vd[t] = ld[q - 1];
                        vj[t] = lj[q - 1];
                    }
                }
                __syncwarp();
#pragma unroll
                for (int t = 0; t < 8; t++) {
                    const int q = lane + 32 * t;
                    if (q < k && q > before) {
                        ld[q] = vd[t];
                        lj[q] = vj[t];
                    } else if (q == before) {
                        ld[q] = dc;
                        lj[q] = lc;
                    }
                }
                __syncwarp();
                tau = ld[k - 1];
                jl = lj[k - 1];
            }
        }
    }
    for (int e = lane; e < k; e += 32) {
        d2_out[i * k + e] = ld[e];
        idx_out[i * k + e] = lj[e];
    }
}

__global__ void k_rank_of(int64_t n, const uint32_t *__restrict__ order, uint32_t *__restrict__ rank) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p < n) rank[order[p]] = (uint32_t)p;
}

static cudaError_t knn_mark(pxsne_ctx *c, int which, cudaStream_t st) {
    cudaError_t e;
    if (!c->knn_ev[which] && (e = cudaEventCreate(&c->knn_ev[which]))) return e;
    c->knn_timed = (which == 1);
    return cudaEventRecord(c->knn_ev[which], st);
}

cudaError_t launch_knn(pxsne_ctx *c, const float *Xdev, int64_t n, int32_t D, int32_t k,
                       int32_t *idx, float *d2) {
    cudaStream_t st = c->stream;
    cudaError_t e;
    float *nrm = nullptr;
    if ((e = cudaMallocAsync(&nrm, n * sizeof(float), st))) return e;
    k_row_norms<<<(unsigned)((n * 32 + 255) / 256), 256, 0, st>>>(n, D, Xdev, nrm);
    if ((e = cudaGetLastError())) return e;
    const int Dp = (D + 63) / 64 * 64;
    const char *force = getenv("PXSNE_KNN");
    const bool want_fp32 = force && force[0] == 'f';
    int dev = 0, smem_max = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const size_t smem_tc = knn_tc_smem(Dp, k);
    if (!want_fp32 && Dp <= 128 && smem_tc <= (size_t)smem_max) {
        c->knn_path = 1;
        unsigned *amax = nullptr;
        unsigned *err = &c->sc->err;
        if ((e = cudaMemsetAsync(&c->sc->knn_exact, 0, 3 * sizeof(u64), st))) return e;
        if ((e = cudaMallocAsync(&amax, sizeof(unsigned), st))) return e;
        if ((e = cudaMemsetAsync(amax, 0, sizeof(unsigned), st))) return e;
        k_absmax<<<1184, 256, 0, st>>>(n * D, Xdev, amax);
        unsigned hmax = 0;
        if ((e = cudaMemcpyAsync(&hmax, amax, sizeof(unsigned), cudaMemcpyDeviceToHost, st)))
            return e;
        if ((e = cudaStreamSynchronize(st))) return e;
        const float mx = __uint_as_float_host(hmax);
        // scale the largest |x| into [2^14, 2^15): FP16 stays far from overflow
        int ex = 0;
        if (mx > 0.f) ex = 14 - (int)floorf(log2f(mx));
        if (ex > 100) ex = 100;
        if (ex < -100) ex = -100;
        const float scale = ldexpf(1.0f, ex);
        const float inv_s2 = ldexpf(1.0f, -2 * ex);
        const float u = 1.0f / 2048.0f;
        // the MMA's FP32 accumulation of exact FP16 products (the FP16
        // rounding itself enters through the rows' rounding errors), and
        // 2^-19 for the filter's own arithmetic
        const float kappa = 1.25f * 2.0f * ((float)Dp * 5.9604645e-8f * 1.01f) + 1.9073486e-06f;
        (void)u;
        const float eps_abs = (float)(2 * D + 8) * 5.9604645e-8f;
        // locality order: rows grouped by their nearest of m pivots (rows
        // i n / m), the pivots chained greedily by nearest neighbour on the host
        const int m = (int)std::min<int64_t>(kCells, std::max<int64_t>(1, n / 256));
        std::vector<float> hp((size_t)m * D), hq((size_t)m * D), hn((size_t)m);
        std::vector<double> hd((size_t)m * m);
        {
            // the pivot rows and their squared distances, formed on the device
            // (a host loop over the m^2 D / 2 terms of the chain took 28 ms)
            float *dp = nullptr;
            double *dd = nullptr;
            if ((e = cudaMallocAsync(&dp, (size_t)m * D * sizeof(float), st))) return e;
            if ((e = cudaMallocAsync(&dd, (size_t)m * m * sizeof(double), st))) return e;
            k_pivot_rows<<<(unsigned)(((int64_t)m * D + 255) / 256), 256, 0, st>>>(n, m, D, Xdev,
                                                                                  dp);
            k_pivot_d2<<<(unsigned)(((int64_t)m * m + 255) / 256), 256, 0, st>>>(m, D, dp, dd);
            if ((e = cudaGetLastError())) return e;
            if ((e = cudaMemcpyAsync(hp.data(), dp, (size_t)m * D * sizeof(float),
                                     cudaMemcpyDeviceToHost, st)))
                return e;
            if ((e = cudaMemcpyAsync(hd.data(), dd, (size_t)m * m * sizeof(double),
                                     cudaMemcpyDeviceToHost, st)))
                return e;
            if ((e = cudaFreeAsync(dp, st))) return e;
            if ((e = cudaFreeAsync(dd, st))) return e;
            if ((e = cudaStreamSynchronize(st))) return e;
        }
        {
            // greedy chain: from pivot 0, always on to the nearest unused one
            std::vector<char> used((size_t)m, 0);
            int cur = 0;
            for (int q = 0; q < m; q++) {
                used[(size_t)cur] = 1;
                double pn2 = 0.0;
                for (int d = 0; d < D; d++) {
                    const float v = hp[(size_t)cur * D + d];
                    hq[(size_t)q * D + d] = v;
                    pn2 += (double)v * v;
                }
                hn[(size_t)q] = (float)pn2;
                int nxt = -1;
                double bd = 0.0;
                const double *row = hd.data() + (size_t)cur * m;
                for (int r = 0; r < m; r++) {
                    if (used[(size_t)r]) continue;
                    if (nxt < 0 || row[r] < bd) {
                        nxt = r;
                        bd = row[r];
                    }
                }
                if (nxt < 0) break;
                cur = nxt;
            }
        }
        float *piv = nullptr, *Xs = nullptr, *ns = nullptr;
        uint32_t *cell = nullptr, *order = nullptr, *ccnt = nullptr;
        if ((e = cudaMallocAsync(&piv, (size_t)m * (D + 1) * sizeof(float), st))) return e;
        if ((e = cudaMallocAsync(&cell, (size_t)n * sizeof(uint32_t), st))) return e;
        if ((e = cudaMallocAsync(&order, (size_t)n * sizeof(uint32_t), st))) return e;
        if ((e = cudaMallocAsync(&ccnt, (size_t)(m + 1) * sizeof(uint32_t), st))) return e;
        float *dpiv = nullptr;
        double *dsum = nullptr;
        if ((e = cudaMallocAsync(&dpiv, (size_t)n * sizeof(float), st))) return e;
        if ((e = cudaMallocAsync(&dsum, sizeof(double), st))) return e;
        if ((e = cudaMallocAsync(&Xs, (size_t)n * D * sizeof(float), st))) return e;
        if ((e = cudaMallocAsync(&ns, (size_t)n * sizeof(float), st))) return e;
        float *pn = piv + (size_t)m * D;
        if ((e = cudaMemcpyAsync(piv, hq.data(), (size_t)m * D * sizeof(float),
                                 cudaMemcpyHostToDevice, st)))
            return e;
        if ((e = cudaMemcpyAsync(pn, hn.data(), (size_t)m * sizeof(float), cudaMemcpyHostToDevice,
                                 st)))
            return e;
        const size_t smem_a = (size_t)std::min(m, kPivChunk) * Dp * sizeof(float);
        const unsigned ablocks = (unsigned)((n + 255) / 256);
        if (Dp == 64) {
            if ((e = cudaFuncSetAttribute(k_assign_cells<64>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_a)))
                return e;
            k_assign_cells<64><<<ablocks, 256, smem_a, st>>>(n, D, m, Xdev, piv, pn, nrm, cell, dpiv);
        } else {
            if ((e = cudaFuncSetAttribute(k_assign_cells<128>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_a)))
                return e;
            k_assign_cells<128><<<ablocks, 256, smem_a, st>>>(n, D, m, Xdev, piv, pn, nrm, cell, dpiv);
        }
        // far rows: squared distance to the nearest pivot above 3x the mean
        // (within a cluster that holds a pivot the distances concentrate near
        // the mean; an outlier or a row of a cluster without a pivot is
        // several times farther)
        if ((e = cudaMemsetAsync(dsum, 0, sizeof(double), st))) return e;
        k_sum_f64<<<ablocks < 1184 ? ablocks : 1184, 256, 0, st>>>(n, dpiv, dsum);
        double hsum = 0.0;
        if ((e = cudaMemcpyAsync(&hsum, dsum, sizeof(double), cudaMemcpyDeviceToHost, st))) return e;
        if ((e = cudaStreamSynchronize(st))) return e;
        k_far_rows<<<ablocks, 256, 0, st>>>(n, dpiv, (float)(3.0 * hsum / (double)n), (uint32_t)m,
                                            cell);
        if ((e = cudaMemsetAsync(ccnt, 0, (size_t)(m + 1) * sizeof(uint32_t), st))) return e;
        k_cell_count<<<ablocks, 256, 0, st>>>(n, cell, ccnt);
        std::vector<uint32_t> hc((size_t)m + 1);
        if ((e = cudaMemcpyAsync(hc.data(), ccnt, (size_t)(m + 1) * sizeof(uint32_t),
                                 cudaMemcpyDeviceToHost, st)))
            return e;
        if ((e = cudaStreamSynchronize(st))) return e;
        uint32_t run = 0u;
        for (int q = 0; q <= m; q++) {
            const uint32_t v = hc[(size_t)q];
            hc[(size_t)q] = run;
            run += v;
        }
        if ((e = cudaMemcpyAsync(ccnt, hc.data(), (size_t)(m + 1) * sizeof(uint32_t),
                                 cudaMemcpyHostToDevice, st)))
            return e;
        {
            const int nc = m + 1;  // the pivots' cells and the far rows' one
            const int64_t nb = (n + kCsRows - 1) / kCsRows;
            uint32_t *hist = nullptr;
            int64_t *off = nullptr;
            if ((e = cudaMallocAsync(&hist, (size_t)(nc * nb) * sizeof(uint32_t), st))) return e;
            if ((e = cudaMallocAsync(&off, (size_t)(nc * nb + 1) * sizeof(int64_t), st))) return e;
            k_cell_rank<<<(unsigned)nb, kCsRows, 0, st>>>(n, nc, cell, hist, nb, nullptr, nullptr);
            if ((e = cudaGetLastError())) return e;
            if ((e = scan_u32_to_i64(hist, (int64_t)nc * nb, off, st))) return e;
            k_cell_rank<<<(unsigned)nb, kCsRows, 0, st>>>(n, nc, cell, hist, nb, off, order);
            if ((e = cudaGetLastError())) return e;
            cudaFreeAsync(hist, st);
            cudaFreeAsync(off, st);
        }
        const int probe = c->p.knn_probe;
        {
            // split every cell by random projections until segments hold at
            // most one tile's rows: compact tiles, tighter tile bounds (and,
            // for the approximate search, a meaningful nearest-tile order)
            uint32_t biggest = 0u;
            for (int q = 0; q <= m; q++) {
                const uint32_t end = q < m ? hc[(size_t)q + 1] : (uint32_t)n;
                biggest = std::max(biggest, end - hc[(size_t)q]);
            }
            int levels = 4;
            while (((uint64_t)kTcRows << (levels - 4)) < biggest) levels++;
            uint32_t *cst = nullptr, *order2 = nullptr, *flag = nullptr;
            int2 *seg = nullptr, *seg2 = nullptr;
            int64_t *pref = nullptr;
            if ((e = cudaMallocAsync(&cst, (size_t)(m + 2) * sizeof(uint32_t), st))) return e;
            if ((e = cudaMallocAsync(&order2, (size_t)n * sizeof(uint32_t), st))) return e;
            if ((e = cudaMallocAsync(&flag, (size_t)n * sizeof(uint32_t), st))) return e;
            if ((e = cudaMallocAsync(&seg, (size_t)n * sizeof(int2), st))) return e;
            if ((e = cudaMallocAsync(&seg2, (size_t)n * sizeof(int2), st))) return e;
            if ((e = cudaMallocAsync(&pref, (size_t)(n + 1) * sizeof(int64_t), st))) return e;
            std::vector<uint32_t> hs((size_t)m + 2);
            for (int q = 0; q <= m; q++) hs[(size_t)q] = hc[(size_t)q];
            hs[(size_t)m + 1] = (uint32_t)n;
            if ((e = cudaMemcpyAsync(cst, hs.data(), hs.size() * sizeof(uint32_t),
                                     cudaMemcpyHostToDevice, st)))
                return e;
            k_seg_init<<<ablocks, 256, 0, st>>>(n, order, cell, cst, seg);
            for (int lv = 0; lv < levels; lv++) {
                k_rp_side<<<ablocks, 256, 0, st>>>(n, D, Xdev, order, seg, lv, flag);
                if ((e = cudaGetLastError())) return e;
                if ((e = scan_u32_to_i64(flag, n, pref, st))) return e;
                k_rp_scatter<<<ablocks, 256, 0, st>>>(n, order, seg, flag, pref, order2, seg2);
                if ((e = cudaGetLastError())) return e;
                std::swap(order, order2);
                std::swap(seg, seg2);
            }
            cudaFreeAsync(cst, st);
            cudaFreeAsync(order2, st);
            cudaFreeAsync(flag, st);
            cudaFreeAsync(seg, st);
            cudaFreeAsync(seg2, st);
            cudaFreeAsync(pref, st);
        }
        k_gather_rows<<<(unsigned)((n * D + 255) / 256), 256, 0, st>>>(n, D, order, Xdev, nrm, Xs,
                                                                       ns);
        if ((e = cudaGetLastError())) return e;
        // the search runs on the ordered rows
        const float *Xo = Xs;
        const int64_t T = (n + kTcCols - 1) / kTcCols;
        const size_t img_bytes = (size_t)T * kTcRows * Dp * 2;
        uint8_t *img = nullptr;
        float *HG = nullptr;
        if ((e = cudaMallocAsync(&img, img_bytes, st))) return e;
        if ((e = cudaMallocAsync(&HG, (size_t)T * kHG * sizeof(float), st))) return e;
        const int64_t nchunks = T * kTcRows * (Dp / 8);
        k_to_half_img<<<(unsigned)((nchunks + 255) / 256), 256, 0, st>>>(n, D, Dp, T, scale, Xo,
                                                                          img);
        float *n16 = nullptr, *rerr = nullptr;
        if ((e = cudaMallocAsync(&n16, (size_t)n * sizeof(float), st))) return e;
        if ((e = cudaMallocAsync(&rerr, (size_t)n * sizeof(float), st))) return e;
        k_round_err<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, D, scale, Xo, n16, rerr);
        k_tile_norms<<<(unsigned)((T * kTcCols + 255) / 256), 256, 0, st>>>(n, T, eps_abs, n16,
                                                                           rerr, HG);
        if ((e = cudaGetLastError())) return e;
        // tile centroids and radii (the loader's pruning bound)
        float *cent = nullptr, *rad = nullptr;
        if ((e = cudaMallocAsync(&cent, (size_t)T * Dp * sizeof(float), st))) return e;
        if ((e = cudaMallocAsync(&rad, (size_t)T * sizeof(float), st))) return e;
        k_tile_bounds<<<(unsigned)T, 128, 0, st>>>(n, D, Dp, Xo, cent, rad);
        if ((e = cudaGetLastError())) return e;
        c->knn_tiles = T;
        if ((e = cudaFuncSetAttribute(k_knn_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem_tc)))
            return e;
        KnnTcArgs ka;
        ka.n = n;
        ka.T = T;
        ka.D = D;
        ka.Dp = Dp;
        ka.k = k;
        ka.inv_s2 = inv_s2;
        ka.kappa = kappa;
        ka.eps_abs = eps_abs;
        ka.X = Xo;
        ka.img = img;
        ka.nrm = n16;
        ka.rerr = rerr;
        ka.HG = HG;
        ka.order = order;
        ka.out_idx = idx;
        ka.out_d2 = d2;
        ka.err = err;
        ka.stats = &c->sc->knn_exact;
        ka.cent = cent;
        ka.rad = rad;
        ka.cand = nullptr;
        ka.W = 0;
        // (the search's time includes its candidate lists)
        if ((e = knn_mark(c, 0, st))) return e;
        int32_t *cand = nullptr;
        if (probe > 0) {
            const int W = (int)std::min<int64_t>(probe, T);
            if ((e = cudaMallocAsync(&cand, (size_t)T * W * sizeof(int32_t), st))) return e;
            k_tile_cands<<<(unsigned)T, kCandThreads, 0, st>>>(T, Dp, cent, W, cand);
            if ((e = cudaGetLastError())) return e;
            ka.cand = cand;
            ka.W = W;
        }
        k_knn_tc<<<(unsigned)T, kTcThreads, smem_tc, st>>>(ka);
        if ((e = cudaGetLastError())) return e;
        if (probe > 0 && c->p.knn_explore > 0) {
            // rounds of neighbour exploring, ping-ponging with a second pair
            // of lists; the last round writes into idx / d2
            uint32_t *rank = nullptr;
            int32_t *idx2 = nullptr;
            float *d22 = nullptr;
            if ((e = cudaMallocAsync(&rank, (size_t)n * sizeof(uint32_t), st))) return e;
            if ((e = cudaMallocAsync(&idx2, (size_t)n * k * sizeof(int32_t), st))) return e;
            if ((e = cudaMallocAsync(&d22, (size_t)n * k * sizeof(float), st))) return e;
            k_rank_of<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, order, rank);
            const int R = c->p.knn_explore;
            const int ke = std::min(k, kExploreNbrs);
            const int v4 = ((D & 3) == 0) && ((reinterpret_cast<uintptr_t>(Xo) & 15) == 0);
            const unsigned eb = (unsigned)((n + kExploreWarps - 1) / kExploreWarps);
            // with R odd the first round reads a copy of the search's lists
            if ((R & 1) &&
                (e = cudaMemcpyAsync(idx2, idx, (size_t)n * k * sizeof(int32_t),
                                     cudaMemcpyDeviceToDevice, st)))
                return e;
            if ((R & 1) && (e = cudaMemcpyAsync(d22, d2, (size_t)n * k * sizeof(float),
                                                cudaMemcpyDeviceToDevice, st)))
                return e;
            for (int r = 0; r < R; r++) {
                // round r writes the pair that the last round must end in
                const bool into_main = ((R - 1 - r) & 1) == 0;
                const int32_t *ii = into_main ? idx2 : idx;
                const float *di = into_main ? d22 : d2;
                int32_t *io = into_main ? idx : idx2;
                float *dout = into_main ? d2 : d22;
                k_knn_explore<<<eb, kExploreWarps * 32, 0, st>>>(n, k, ke, D, v4, Xo, order, rank,
                                                                ii, di, io, dout);
                if ((e = cudaGetLastError())) return e;
            }
            cudaFreeAsync(rank, st);
            cudaFreeAsync(idx2, st);
            cudaFreeAsync(d22, st);
        }
        if ((e = knn_mark(c, 1, st))) return e;
        if (cand) cudaFreeAsync(cand, st);
        cudaFreeAsync(img, st);
        cudaFreeAsync(HG, st);
        cudaFreeAsync(n16, st);
        cudaFreeAsync(rerr, st);
        cudaFreeAsync(cent, st);
        cudaFreeAsync(rad, st);
        cudaFreeAsync(amax, st);
        cudaFreeAsync(piv, st);
        cudaFreeAsync(cell, st);
        cudaFreeAsync(order, st);
        cudaFreeAsync(ccnt, st);
        cudaFreeAsync(dpiv, st);
        cudaFreeAsync(dsum, st);
        cudaFreeAsync(Xs, st);
        cudaFreeAsync(ns, st);
        return cudaFreeAsync(nrm, st);
    }
    c->knn_path = 0;
    const size_t smem = (size_t)D * (kQR + kCT) * 4 + (size_t)kQR * k * 8 + kQR * 4 +
                        (size_t)(kQR + kKnnThreads / 32) * kCT * 4;
    if ((e = cudaFuncSetAttribute(k_knn_tile, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)))
        return e;
    if ((e = knn_mark(c, 0, st))) return e;
    k_knn_tile<<<(unsigned)((n + kQR - 1) / kQR), kKnnThreads, smem, st>>>(n, D, k, Xdev, nrm,
                                                                          idx, d2);
    if ((e = cudaGetLastError())) return e;
    if ((e = knn_mark(c, 1, st))) return e;
    return cudaFreeAsync(nrm, st);
}

// ---------------------------------------------------------------- perplexity
// Sec. 3.2: bisection on beta_i (start 1; double or halve until bracketed,
// then halve the bracket) until |H_i - ln u| < 1e-5 or 200 steps, with the
// exponents shifted by the row's smallest distance.
__global__ void __launch_bounds__(256)
    k_perplexity(int64_t n, int k, float target, const float *__restrict__ d2,
                 float *__restrict__ pcond, float *__restrict__ beta_out, DevScalars *sc) {
    constexpr int VPL = 8;  // values per lane, k <= 256
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    float d[VPL];
    float dmin = INFINITY;
#pragma unroll
    for (int v = 0; v < VPL; v++) {
        const int e = lane + 32 * v;
        d[v] = e < k ? d2[row * k + e] : INFINITY;
        dmin = fminf(dmin, d[v]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dmin = fminf(dmin, __shfl_xor_sync(0xffffffffu, dmin, o));
#pragma unroll
    for (int v = 0; v < VPL; v++) d[v] = (lane + 32 * v < k) ? d[v] - dmin : 0.f;
    float beta = 1.f, lo = 0.f, hi = 0.f;
    bool has_lo = false, has_hi = false, ok = false;
    float sum = 0.f, hs = 0.f;
    for (int it = 0; it < 200; it++) {
        sum = 0.f;
        hs = 0.f;
#pragma unroll
        for (int v = 0; v < VPL; v++) {
            if (lane + 32 * v < k) {
                const float ev = expf(-beta * d[v]);
                sum += ev;
                hs = fmaf(d[v], ev, hs);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sum += __shfl_xor_sync(0xffffffffu, sum, o);
            hs += __shfl_xor_sync(0xffffffffu, hs, o);
        }
        const float H = logf(sum) + beta * hs / sum;
        if (fabsf(H - target) < 1e-5f) {
            ok = true;
            break;
        }
        if (H > target) {
            lo = beta;
            has_lo = true;
            // capped below FP32 overflow: a row whose target is out of reach
            // (all distances tied) keeps finite, uniform weights
            beta = has_hi ? 0.5f * (beta + hi) : fminf(2.f * beta, 1.7014118e38f);
        } else {
            hi = beta;
            has_hi = true;
            beta = has_lo ? 0.5f * (beta + lo) : 0.5f * beta;
        }
    }
    sum = 0.f;
    float ev[VPL];
#pragma unroll
    for (int v = 0; v < VPL; v++) {
        ev[v] = (lane + 32 * v < k) ? expf(-beta * d[v]) : 0.f;
        sum += ev[v];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    const float inv = 1.f / sum;
#pragma unroll
    for (int v = 0; v < VPL; v++) {
        const int e = lane + 32 * v;
        if (e < k) pcond[row * k + e] = ev[v] * inv;
    }
    if (lane == 0) {
        beta_out[row] = beta;
        if (!ok) atomicOr(&sc->err, (unsigned)PXSNE_DEVERR_BISECT);
    }
}

cudaError_t launch_perplexity(pxsne_ctx *c, const float *d2, int64_t n, int32_t k,
                              float perplexity, float *pcond, float *beta) {
    k_perplexity<<<(unsigned)((n * 32 + 255) / 256), 256, 0, c->stream>>>(
        n, k, logf(perplexity), d2, pcond, beta, c->sc);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- symmetrize
__global__ void k_indeg(int64_t nk, const int32_t *__restrict__ idx, uint32_t *deg) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < nk) atomicAdd(&deg[idx[e]], 1u);
}

// Exclusive scan of 32-bit counts into int64 offsets: per-block scan, then a
// single-block scan of the block totals, then the add.
constexpr int kScanB = 1024;
__global__ void __launch_bounds__(kScanB)
    k_scan_blocks(int64_t m, const uint32_t *__restrict__ in, int64_t *__restrict__ out,
                  int64_t *__restrict__ bsum) {
    __shared__ int64_t s[kScanB];
    const int64_t i = blockIdx.x * (int64_t)kScanB + threadIdx.x;
    const int64_t v = i < m ? (int64_t)in[i] : 0;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < kScanB; o <<= 1) {
        const int64_t t = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
        __syncthreads();
        s[threadIdx.x] += t;
        __syncthreads();
    }
    if (i < m) out[i] = s[threadIdx.x] - v;
    if (threadIdx.x == kScanB - 1) bsum[blockIdx.x] = s[threadIdx.x];
}

__global__ void __launch_bounds__(kScanB) k_scan_bsum(int64_t nb, int64_t *bsum, int64_t *total) {
    __shared__ int64_t s[kScanB];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < nb; base += kScanB) {
        const int64_t i = base + threadIdx.x;
        const int64_t v = i < nb ? bsum[i] : 0;
        s[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < kScanB; o <<= 1) {
            const int64_t t = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
            __syncthreads();
            s[threadIdx.x] += t;
            __syncthreads();
        }
        const int64_t cy = carry;
        if (i < nb) bsum[i] = cy + s[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == kScanB - 1) carry = cy + s[threadIdx.x];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void k_scan_add(int64_t m, int64_t *out, const int64_t *__restrict__ bsum,
                           const int64_t *__restrict__ total) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < m) out[i] += bsum[i / kScanB];
    if (i == m) out[m] = *total;
}

// out[0..m] = exclusive scan of in[0..m) with out[m] = total (int64).
cudaError_t scan_u32_to_i64(const uint32_t *in, int64_t m, int64_t *out, cudaStream_t st) {
    const int64_t nb = (m + kScanB - 1) / kScanB;
    int64_t *bsum = nullptr;
    cudaError_t e;
    if ((e = cudaMallocAsync(&bsum, (nb + 1) * sizeof(int64_t), st))) return e;
    k_scan_blocks<<<(unsigned)(nb > 0 ? nb : 1), kScanB, 0, st>>>(m, in, out, bsum);
    k_scan_bsum<<<1, kScanB, 0, st>>>(nb, bsum, bsum + nb);
    k_scan_add<<<(unsigned)((m + 1 + 255) / 256), 256, 0, st>>>(m, out, bsum, bsum + nb);
    if ((e = cudaGetLastError())) return e;
    return cudaFreeAsync(bsum, st);
}

// Row i of the union pattern: its own k entries (j, p_{j|i}) first, then the
// incoming ones (j, p_{i|j}) for every j that lists i.
__global__ void k_fill(int64_t n, int k, const int32_t *__restrict__ idx,
                       const float *__restrict__ pcond, const int64_t *__restrict__ tptr,
                       uint32_t *__restrict__ cursor, int32_t *__restrict__ tcol,
                       float *__restrict__ tval) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * k) return;
    const int64_t i = e / k;
    const int a = (int)(e % k);
    const int32_t j = idx[e];
    const float p = pcond[e];
    tcol[tptr[i] + a] = j;
    tval[tptr[i] + a] = p;
    const uint32_t slot = (uint32_t)k + atomicAdd(&cursor[j], 1u);
    tcol[tptr[j] + slot] = (int32_t)i;
    tval[tptr[j] + slot] = p;
}

// Sort each temporary row by (col, position) (rank sort, one warp per row,
// the row's columns staged in shared memory when it has at most kSmRow
// entries), then merge equal columns (a column appears at most twice: once
// from the row's own list, once from the other row's); count = number of
// distinct columns.  With write == 1 the merged row goes to (col, val / 2n) at
// rp[i], padded with (i, 0) to rp[i + 1].
constexpr int kSmRow = 1024;
__global__ void __launch_bounds__(256)
    k_sort_merge(int64_t n, int write, const int64_t *__restrict__ tptr,
                 const int32_t *__restrict__ tcol, const float *__restrict__ tval,
                 int32_t *__restrict__ scol, float *__restrict__ sval,
                 uint32_t *__restrict__ cnt, const int64_t *__restrict__ rp,
                 int32_t *__restrict__ col, float *__restrict__ val) {
    __shared__ int32_t s_c[8][kSmRow];
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31, w = (threadIdx.x >> 5) & 7;
    if (row >= n) return;
    const int64_t a = tptr[row], b = tptr[row + 1];
    const int len = (int)(b - a);
    if (!write) {
        if (len <= kSmRow) {
            // columns in shared memory, padded to a multiple of 4 with a value
            // above every column; each pass ranks up to 8 elements per lane
            // against all columns, read 16 bytes at a time
            int32_t *sc = s_c[w];
            const int len4 = (len + 3) & ~3;
            for (int e = lane; e < len4; e += 32) sc[e] = e < len ? tcol[a + e] : 0x7fffffff;
            __syncwarp();
            const int4 *sc4 = reinterpret_cast<const int4 *>(sc);
            for (int e0 = 0; e0 < len; e0 += 256) {
                int32_t ce[8];
                int r[8];
#pragma unroll
                for (int m = 0; m < 8; m++) {
                    const int e = e0 + 32 * m + lane;
                    ce[m] = e < len ? sc[e] : 0x7fffffff;
                    r[m] = 0;
                }
                for (int f4 = 0; f4 < (len4 >> 2); f4++) {
                    const int4 c4 = sc4[f4];
                    const int f = 4 * f4;
#pragma unroll
                    for (int m = 0; m < 8; m++) {
                        const int e = e0 + 32 * m + lane;
                        r[m] += (c4.x < ce[m]) || (c4.x == ce[m] && f < e);
                        r[m] += (c4.y < ce[m]) || (c4.y == ce[m] && f + 1 < e);
                        r[m] += (c4.z < ce[m]) || (c4.z == ce[m] && f + 2 < e);
                        r[m] += (c4.w < ce[m]) || (c4.w == ce[m] && f + 3 < e);
                    }
                }
#pragma unroll
                for (int m = 0; m < 8; m++) {
                    const int e = e0 + 32 * m + lane;
                    if (e < len) {
                        scol[a + r[m]] = ce[m];
                        sval[a + r[m]] = tval[a + e];
                    }
                }
            }
        } else {
            return;  // a long row: k_sort_long
        }
        __syncwarp();
        uint32_t u = 0;
        for (int e0 = 0; e0 < len; e0 += 32) {
            const int e = e0 + lane;
            const bool head = e < len && (e == 0 || scol[a + e] != scol[a + e - 1]);
            u += (uint32_t)__popc(__ballot_sync(0xffffffffu, head));
        }
        if (lane == 0) cnt[row] = u;
    } else {
        const float inv2n = (float)(0.5 / (double)n);
        const int64_t o0 = rp[row];
        uint32_t done = 0;  // distinct columns written so far
        for (int e0 = 0; e0 < len; e0 += 32) {
            const int e = e0 + lane;
            int32_t ce = 0;
            bool head = false;
            if (e < len) {
                ce = scol[a + e];
                head = (e == 0 || ce != scol[a + e - 1]);
            }
            const unsigned hm = __ballot_sync(0xffffffffu, head);
            if (head) {
                float v = sval[a + e];
                if (e + 1 < len && scol[a + e + 1] == ce) v += sval[a + e + 1];
                const int64_t o = o0 + done + __popc(hm & ((1u << lane) - 1u));
                col[o] = ce;
                val[o] = v * inv2n;
            }
            done += (uint32_t)__popc(hm);
        }
        for (int64_t q = o0 + done + lane; q < rp[row + 1]; q += 32) {  // padding
            col[q] = (int32_t)row;
            val[q] = 0.f;
        }
    }
}

// Rows longer than kSmRow (the hubs of the kNN graph, with thousands of
// incoming entries): one CTA per row sorts the keys (col << 32 | position) by a
// bitonic network in global scratch padded to a power of two, then writes the
// sorted row and its count of distinct columns.
__global__ void k_long_rows(int64_t n, const int64_t *__restrict__ tptr, uint32_t *list,
                            uint32_t *nlong, uint32_t *plen) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t len = tptr[i + 1] - tptr[i];
    if (len > kSmRow) {
        const uint32_t q = atomicAdd(nlong, 1u);
        uint32_t p2 = 1u;
        while (p2 < (uint64_t)len) p2 <<= 1;
        list[q] = (uint32_t)i;
        plen[q] = p2;
    }
}

__global__ void __launch_bounds__(1024)
    k_sort_long(const uint32_t *__restrict__ list, const uint32_t *__restrict__ plen,
                const int64_t *__restrict__ soff, const int64_t *__restrict__ tptr,
                const int32_t *__restrict__ tcol, const float *__restrict__ tval,
                unsigned long long *scratch, int32_t *__restrict__ scol,
                float *__restrict__ sval, uint32_t *__restrict__ cnt) {
    __shared__ uint32_t s_w[32];
    const uint32_t row = list[blockIdx.x];
    const int64_t a = tptr[row];
    const int len = (int)(tptr[row + 1] - a);
    const int P = (int)plen[blockIdx.x];
    unsigned long long *key = scratch + soff[blockIdx.x];
    const int tid = threadIdx.x;
    for (int i = tid; i < P; i += blockDim.x)
        key[i] = i < len ? (((unsigned long long)(uint32_t)tcol[a + i]) << 32) | (uint32_t)i
                         : ~0ull;
    __syncthreads();
    for (int k2 = 2; k2 <= P; k2 <<= 1) {
        for (int j = k2 >> 1; j > 0; j >>= 1) {
            for (int i = tid; i < P; i += blockDim.x) {
                const int l = i ^ j;
                if (l > i) {
                    const unsigned long long x = key[i], y = key[l];
                    const bool asc = (i & k2) == 0;
                    if ((x > y) == asc) {
                        key[i] = y;
                        key[l] = x;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = tid; i < len; i += blockDim.x) {
        const unsigned long long u = key[i];
        scol[a + i] = (int32_t)(u >> 32);
        sval[a + i] = tval[a + (uint32_t)(u & 0xffffffffull)];
    }
    __syncthreads();
    uint32_t u = 0u;
    for (int i = tid; i < len; i += blockDim.x)
        u += (i == 0 || scol[a + i] != scol[a + i - 1]) ? 1u : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
    if ((tid & 31) == 0) s_w[tid >> 5] = u;
    __syncthreads();
    if (tid == 0) {
        uint32_t t = 0u;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += s_w[w];
        cnt[row] = t;
    }
}

__global__ void k_round4(int64_t n, const uint32_t *in, uint32_t *out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = (in[i] + 3u) & ~3u;
}

__global__ void k_add_const(int64_t n, const uint32_t *in, uint32_t *out, uint32_t a) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = in[i] + a;
}

cudaError_t build_symmetric_csr(pxsne_ctx *c, const int32_t *idx, const float *pcond,
                                int64_t n, int32_t k, std::string &err) {
    cudaStream_t st = c->stream;
    cudaError_t e;
    const int64_t nk = n * k;
    uint32_t *deg = nullptr, *cursor = nullptr;
    int64_t *tptr = nullptr;
    int32_t *tcol = nullptr, *scol = nullptr;
    float *tval = nullptr, *sval = nullptr;
#define TRY(x)                 \
    do {                       \
        if ((e = (x))) {       \
            err = #x;          \
            return e;          \
        }                      \
    } while (0)
    TRY(cudaMallocAsync(&deg, n * sizeof(uint32_t), st));
    TRY(cudaMallocAsync(&cursor, n * sizeof(uint32_t), st));
    TRY(cudaMallocAsync(&tptr, (n + 1) * sizeof(int64_t), st));
    TRY(cudaMemsetAsync(deg, 0, n * sizeof(uint32_t), st));
    TRY(cudaMemsetAsync(cursor, 0, n * sizeof(uint32_t), st));
    k_indeg<<<(unsigned)((nk + 255) / 256), 256, 0, st>>>(nk, idx, deg);
    TRY(cudaGetLastError());
    // temporary rows of length k + indeg(i); 2 n k entries in total
    uint32_t *len = cursor;
    k_add_const<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, deg, len, (uint32_t)k);
    TRY(cudaGetLastError());
    TRY(scan_u32_to_i64(len, n, tptr, st));
    TRY(cudaMemsetAsync(cursor, 0, n * sizeof(uint32_t), st));
    TRY(cudaMallocAsync(&tcol, 2 * nk * sizeof(int32_t), st));
    TRY(cudaMallocAsync(&tval, 2 * nk * sizeof(float), st));
    TRY(cudaMallocAsync(&scol, 2 * nk * sizeof(int32_t), st));
    TRY(cudaMallocAsync(&sval, 2 * nk * sizeof(float), st));
    k_fill<<<(unsigned)((nk + 255) / 256), 256, 0, st>>>(n, k, idx, pcond, tptr, cursor, tcol,
                                                        tval);
    TRY(cudaGetLastError());
    uint32_t *ucnt = deg;  // reuse
    k_sort_merge<<<(unsigned)((n * 32 + 255) / 256), 256, 0, st>>>(
        n, 0, tptr, tcol, tval, scol, sval, ucnt, nullptr, nullptr, nullptr);
    TRY(cudaGetLastError());
    {
        // long rows
        uint32_t *list = nullptr, *nlong = nullptr, *plen = nullptr;
        TRY(cudaMallocAsync(&list, (size_t)n * sizeof(uint32_t), st));
        TRY(cudaMallocAsync(&plen, (size_t)n * sizeof(uint32_t), st));
        TRY(cudaMallocAsync(&nlong, sizeof(uint32_t), st));
        TRY(cudaMemsetAsync(nlong, 0, sizeof(uint32_t), st));
        k_long_rows<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, tptr, list, nlong, plen);
        TRY(cudaGetLastError());
        uint32_t hl = 0;
        TRY(cudaMemcpyAsync(&hl, nlong, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
        TRY(cudaStreamSynchronize(st));
        if (hl > 0) {
            std::vector<uint32_t> hp(hl);
            TRY(cudaMemcpyAsync(hp.data(), plen, hl * sizeof(uint32_t), cudaMemcpyDeviceToHost,
                                st));
            TRY(cudaStreamSynchronize(st));
            std::vector<int64_t> ho(hl);
            int64_t tot = 0;
            for (uint32_t q = 0; q < hl; q++) {
                ho[q] = tot;
                tot += hp[q];
            }
            int64_t *soff = nullptr;
            unsigned long long *scr = nullptr;
            TRY(cudaMallocAsync(&soff, hl * sizeof(int64_t), st));
            TRY(cudaMallocAsync(&scr, (size_t)tot * sizeof(unsigned long long), st));
            TRY(cudaMemcpyAsync(soff, ho.data(), hl * sizeof(int64_t), cudaMemcpyHostToDevice, st));
            k_sort_long<<<hl, 1024, 0, st>>>(list, plen, soff, tptr, tcol, tval, scr, scol, sval,
                                             ucnt);
            TRY(cudaGetLastError());
            cudaFreeAsync(soff, st);
            cudaFreeAsync(scr, st);
        }
        cudaFreeAsync(list, st);
        cudaFreeAsync(plen, st);
        cudaFreeAsync(nlong, st);
    }
    if (c->rp) { cudaFreeAsync(c->rp, st); c->rp = nullptr; }
    if (c->col) { cudaFreeAsync(c->col, st); c->col = nullptr; }
    if (c->val) { cudaFreeAsync(c->val, st); c->val = nullptr; }
    if (c->rowlen) { cudaFreeAsync(c->rowlen, st); c->rowlen = nullptr; }
    // true row lengths and nnz
    TRY(cudaMallocAsync(&c->rowlen, n * sizeof(int32_t), st));
    TRY(cudaMemcpyAsync(c->rowlen, ucnt, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    int64_t *uscan = nullptr;
    TRY(cudaMallocAsync(&uscan, (n + 1) * sizeof(int64_t), st));
    TRY(scan_u32_to_i64(ucnt, n, uscan, st));
    int64_t nnz = 0, nnz_pad = 0;
    TRY(cudaMemcpyAsync(&nnz, uscan + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    // padded offsets
    k_round4<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, ucnt, cursor);
    TRY(cudaGetLastError());
    TRY(cudaMallocAsync(&c->rp, (n + 1) * sizeof(int64_t), st));
    TRY(scan_u32_to_i64(cursor, n, c->rp, st));
    TRY(cudaMemcpyAsync(&nnz_pad, c->rp + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    TRY(cudaStreamSynchronize(st));
    TRY(cudaMallocAsync(&c->col, (nnz_pad > 0 ? nnz_pad : 4) * sizeof(int32_t), st));
    TRY(cudaMallocAsync(&c->val, (nnz_pad > 0 ? nnz_pad : 4) * sizeof(float), st));
    k_sort_merge<<<(unsigned)((n * 32 + 255) / 256), 256, 0, st>>>(
        n, 1, tptr, tcol, tval, scol, sval, ucnt, c->rp, c->col, c->val);
    TRY(cudaGetLastError());
    c->nnz_pad = nnz_pad;
    c->nnz = nnz;
    cudaFreeAsync(deg, st);
    cudaFreeAsync(cursor, st);
    cudaFreeAsync(tptr, st);
    cudaFreeAsync(uscan, st);
    cudaFreeAsync(tcol, st);
    cudaFreeAsync(tval, st);
    cudaFreeAsync(scol, st);
    cudaFreeAsync(sval, st);
#undef TRY
    return cudaGetLastError();
}

}  // namespace pxsne
