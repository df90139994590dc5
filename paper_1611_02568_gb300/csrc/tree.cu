// Pixel-aligned quadtree of PixelSNE (Sec. 4.1) and the screen-driven rescale
// (Sec. 4.2), built every iteration as a dense Morton-ordered pyramid.
//
//   k_snap_hist   rescale zhat -> z (exact integer, Sec. 4.2), pixel snap
//                 (Eq. z1), leaf histogram of counts and exact coordinate sums
//   k_pyr_pass    bottom-up reduction, 5 levels per CTA pass, writing the
//                 16-byte cell records the traversal reads
//   k_scan1 / k_perm_scatter   counting sort of the points by pixel Morton key
//                 (the traversal order of the next kernels)
#include <cmath>
#include <cstdio>

#include "common.cuh"

namespace pxsne {

__global__ void k_snap_hist(int n, int L, int rescale, float theta, u64 Rx, u64 Ry,
                            const longlong2 *__restrict__ zhat, uint2 *__restrict__ z,
                            const uint32_t *__restrict__ perm, uint32_t *__restrict__ rank,
                            uint32_t *__restrict__ cnt, u64 *__restrict__ sx,
                            u64 *__restrict__ sy, DevScalars *sc,
                            const uint32_t *__restrict__ ainv, uint2 *__restrict__ zp) {
    const int F = 32 - L;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int par = sc->t & 1;
    i64 mnx = 0, mny = 0;
    u64 gx = 1, gy = 1;
    double qx = 0.0, qy = 0.0;
    __shared__ double s_q[2];
    if (rescale) {
        mnx = sc->mm[par][0];
        mny = sc->mm[par][1];
        gx = (u64)(sc->mm[par][2] - mnx) + 1ull;
        gy = (u64)(sc->mm[par][3] - mny) + 1ull;
        // R_d / gamma_d is the same for every point: one FP64 division per
        // CTA (FP64 issues at a small fraction of the FP32 rate)
        if (threadIdx.x == 0) {
            s_q[0] = (double)Rx / (double)gx;
            s_q[1] = (double)Ry / (double)gy;
        }
        __syncthreads();
        qx = s_q[0];
        qy = s_q[1];
        if (tid == 0) {
            sc->n_accept = 0ull;
            sc->n_test = 0ull;
            sc->n_steps = 0ull;
            sc->n_nodes = 0ull;
            // Eq. beta_scaling carried as s_d <- (s_d * gamma_d) / R_d
            sc->s[0] = (sc->s[0] * (double)gx) / (double)Rx;
            sc->s[1] = (sc->s[1] * (double)gy) / (double)Ry;
            derive_scalars(sc, theta, L);
            sc->mm[par ^ 1][0] = 0x7fffffffffffffffll;
            sc->mm[par ^ 1][1] = 0x7fffffffffffffffll;
            sc->mm[par ^ 1][2] = (i64)0x8000000000000000ull;
            sc->mm[par ^ 1][3] = (i64)0x8000000000000000ull;
        }
    }
    if (!rescale && tid == 0) {
        sc->n_accept = 0ull;
        sc->n_test = 0ull;
        sc->n_steps = 0ull;
        sc->n_nodes = 0ull;
    }
    // Points arrive in the Morton order of a recent state, so lanes with equal
    // leaf keys mostly form runs: each run adds its count and sums with one
    // set of atomics (segmented shuffle scan), and each lane's rank inside its
    // pixel is the run's base plus its position in the run.
    const bool valid = tid < n;
    const int lane = threadIdx.x & 31;
    uint32_t i = 0u, zx = 0u, zy = 0u, m = 0xffffffffu;
    if (valid) {
        i = perm[tid];
        if (rescale) {
            const longlong2 h = zhat[i];
            zx = rescale_exact((u64)(h.x - mnx), gx, qx, Rx);
            zy = rescale_exact((u64)(h.y - mny), gy, qy, Ry);
            z[i] = make_uint2(zx, zy);
            zp[ainv[i]] = make_uint2(zx, zy);  // the attraction's copy
        } else {
            const uint2 v = z[i];
            zx = v.x;
            zy = v.y;
        }
        m = morton2(zx >> F, zy >> F);
    }
    const uint32_t prev = __shfl_up_sync(0xffffffffu, m, 1);
    const bool head = (lane == 0) || (prev != m);
    const unsigned heads = __ballot_sync(0xffffffffu, head);
    const unsigned upto = (lane == 31) ? 0xffffffffu : ((2u << lane) - 1u);
    const int start = 31 - __clz(heads & upto);
    const unsigned later = heads & ~upto;
    const int end = later ? __ffs(later) - 2 : 31;
    // the coordinate sums are kept for centres of mass only (sx == NULL: a
    // count-only tree for geometric centres)
    const bool sums = sx != nullptr;
    u64 vx = zx, vy = zy;
    if (sums) {
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const u64 tx = __shfl_up_sync(0xffffffffu, vx, o);
            const u64 ty = __shfl_up_sync(0xffffffffu, vy, o);
            if (lane - o >= start) {
                vx += tx;
                vy += ty;
            }
        }
    }
    uint32_t base = 0u;
    if (lane == end && valid) {
        base = atomicAdd(&cnt[m], (uint32_t)(end - start + 1));
        if (sums) {
            atomicAdd(&sx[m], vx);
            atomicAdd(&sy[m], vy);
        }
    }
    base = __shfl_sync(0xffffffffu, base, end);
    if (valid) rank[i] = base + (uint32_t)(lane - start);
}

// Centre-of-mass record of cell m of level l (layout in common.cuh).
__device__ __forceinline__ float4 make_record(uint32_t N, u64 Sx, u64 Sy, int l, uint32_t m) {
    if (N == 0) return make_float4(0.f, 0.f, 0.f, 0.f);
    const int sh = 32 - l;
    const uint32_t bx = l > 0 ? gather_bits16(m) << sh : 0u;
    const uint32_t by = l > 0 ? gather_bits16(m >> 1) << sh : 0u;
    float4 r;
    record_axis(N, Sx, bx, sh, r.x, r.y);
    record_axis(N, Sy, by, sh, r.z, r.w);
    return r;
}

// Block-wide exclusive scan of one value per thread (nt threads, nt <= 1024).
__device__ uint32_t block_excl_scan(uint32_t v, int nt, uint32_t *s_warp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned mask = nt >= 32 ? 0xffffffffu : ((1u << nt) - 1u);
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(mask, x, o);
        if (lane >= o) x += y;
    }
    if (nt <= 32) return x - v;
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const int nw = nt >> 5;
        uint32_t w = lane < nw ? s_warp[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) s_warp[lane] = w;
    }
    __syncthreads();
    const uint32_t before = warp > 0 ? s_warp[warp - 1] : 0u;
    __syncthreads();
    return before + x - v;
}

// The leaf histogram is consumed by the first pass of the pyramid, which sets
// the groups of four leaves it read back to zero where any was occupied, so
// the next iteration's histogram starts from zero without a memset of every
// leaf (sx == NULL: counts only).
__device__ __forceinline__ void clear_leaves(uint32_t cell0, uint4 c4, uint32_t *cnt, u64 *sx,
                                             u64 *sy) {
    if ((c4.x | c4.y | c4.z | c4.w) == 0u) return;
    reinterpret_cast<uint4 *>(cnt)[cell0 >> 2] = make_uint4(0u, 0u, 0u, 0u);
    if (sx == nullptr) return;
    const ulonglong2 z2{0ull, 0ull};
    reinterpret_cast<ulonglong2 *>(sx)[cell0 >> 1] = z2;
    reinterpret_cast<ulonglong2 *>(sx)[(cell0 >> 1) + 1] = z2;
    reinterpret_cast<ulonglong2 *>(sy)[cell0 >> 1] = z2;
    reinterpret_cast<ulonglong2 *>(sy)[(cell0 >> 1) + 1] = z2;
}

// One bottom-up pass: reads the sums of level h for 4^K consecutive cells per
// CTA (an aligned 2^K x 2^K block), writes the records of levels h .. h-K+1
// (and of level h-K when `top`), and the sums of level h-K (one cell per CTA).
// With leaf_start != NULL it also writes the exclusive scan of the counts of
// level h within each CTA (the local start of each pixel in Morton order).
template <int K>
__global__ void __launch_bounds__(1 << (2 * (K - 1)))
    k_pyr_pass(int h, int top, const uint32_t *__restrict__ in_cnt,
               const u64 *__restrict__ in_sx, const u64 *__restrict__ in_sy,
               float4 *__restrict__ rec, float *__restrict__ recn,
               uint32_t *__restrict__ out_cnt,
               u64 *__restrict__ out_sx, u64 *__restrict__ out_sy,
               uint32_t *__restrict__ leaf_start, DevScalars *sc, int bump_t, int clear) {
    constexpr int NT = 1 << (2 * (K - 1));
    __shared__ uint32_t s_c[NT];
    __shared__ u64 s_x[NT], s_y[NT];
    __shared__ uint32_t s_warp[32];
    const int tid = threadIdx.x;
    const int64_t b = blockIdx.x;
    const int64_t cell0 = b * (NT * 4) + 4 * tid;
    const bool sums = in_sx != nullptr;  // count-only tree otherwise
    const uint4 c4 = reinterpret_cast<const uint4 *>(in_cnt)[cell0 >> 2];
    ulonglong2 x01{0, 0}, x23{0, 0}, y01{0, 0}, y23{0, 0};
    if (sums) {
        x01 = reinterpret_cast<const ulonglong2 *>(in_sx)[cell0 >> 1];
        x23 = reinterpret_cast<const ulonglong2 *>(in_sx)[(cell0 >> 1) + 1];
        y01 = reinterpret_cast<const ulonglong2 *>(in_sy)[cell0 >> 1];
        y23 = reinterpret_cast<const ulonglong2 *>(in_sy)[(cell0 >> 1) + 1];
        float4 *rl = rec + rec_offset(h) + cell0;
        rl[0] = make_record(c4.x, x01.x, y01.x, h, (uint32_t)cell0);
        rl[1] = make_record(c4.y, x01.y, y01.y, h, (uint32_t)cell0 + 1u);
        rl[2] = make_record(c4.z, x23.x, y23.x, h, (uint32_t)cell0 + 2u);
        rl[3] = make_record(c4.w, x23.y, y23.y, h, (uint32_t)cell0 + 3u);
    }
    reinterpret_cast<float4 *>(recn + rec_offset(h))[cell0 >> 2] =
        make_float4((float)c4.x, (float)c4.y, (float)c4.z, (float)c4.w);
    if (clear) clear_leaves(cell0, c4, const_cast<uint32_t *>(in_cnt), const_cast<u64 *>(in_sx),
                            const_cast<u64 *>(in_sy));
    uint32_t N = c4.x + c4.y + c4.z + c4.w;
    u64 X = x01.x + x01.y + x23.x + x23.y;
    u64 Y = y01.x + y01.y + y23.x + y23.y;
    if (leaf_start != nullptr) {
        const uint32_t e = block_excl_scan(N, NT, s_warp);
        uint4 st;
        st.x = e;
        st.y = e + c4.x;
        st.z = st.y + c4.y;
        st.w = st.z + c4.z;
        reinterpret_cast<uint4 *>(leaf_start)[cell0 >> 2] = st;
    }
    int lvl = h - 1;
    int64_t idx = b * NT + tid;
#pragma unroll
    for (int j = K - 1; j >= 0; j--) {
        const int cells = 1 << (2 * j);
        if (tid < cells) {
            if (j > 0 || top) {
                if (sums) rec[rec_offset(lvl) + idx] = make_record(N, X, Y, lvl, (uint32_t)idx);
                recn[rec_offset(lvl) + idx] = (float)N;
            }
            if (j == 0) {
                out_cnt[b] = N;
                if (sums) {
                    out_sx[b] = X;
                    out_sy[b] = Y;
                }
            }
        }
        if (j == 0) break;
        __syncthreads();
        if (tid < cells) {
            s_c[tid] = N;
            s_x[tid] = X;
            s_y[tid] = Y;
        }
        __syncthreads();
        if (tid < (cells >> 2)) {
            const int a = 4 * tid;
            N = s_c[a] + s_c[a + 1] + s_c[a + 2] + s_c[a + 3];
            X = s_x[a] + s_x[a + 1] + s_x[a + 2] + s_x[a + 3];
            Y = s_y[a] + s_y[a + 1] + s_y[a + 2] + s_y[a + 3];
        }
        lvl--;
        idx = b * (cells >> 2) + tid;
    }
    if (bump_t && b == 0 && tid == 0) sc->t += 1;
}

// The first pass with K = 5 levels over the leaves, by warp shuffles: a
// thread owns 4 leaves (one level-(h-1) cell); lanes 4k..4k+3 make a level-(h-2)
// cell, 16 lanes a level-(h-3) cell, two warps a level-(h-4) cell and the CTA
// one level-(h-5) cell.  It writes the records of levels h .. h-4, the sums of
// level h-5 and, per CTA, the exclusive scan of the leaf counts (local start of
// each pixel in Morton order).  With fuse_top the last CTA to finish also does
// the rest of the pyramid (pyr_top).
__device__ __forceinline__ u64 shfl_xor_u64(u64 v, int o) {
    return __shfl_xor_sync(0xffffffffu, v, o);
}

__device__ __forceinline__ void put_record(float4 *rec, float *recn, int l, uint32_t m,
                                           uint32_t N, u64 X, u64 Y) {
    // NULL: counts only; an empty cell's record is never read, so not written
    if (rec != nullptr && N != 0u) rec[rec_offset(l) + m] = make_record(N, X, Y, l, m);
    recn[rec_offset(l) + m] = (float)N;
}

// Levels h0-1 .. 0 from the sums of level h0 (4^h0 cells in c0/x0/y0, whose
// records are written), by one CTA of 256 threads, ping-ponging through
// c1/x1/y1; also blk_off = the exclusive scan of the level-h0 counts (each the
// pixel total of one first-pass CTA).
__device__ void pyr_top(int h0, uint32_t *c0, u64 *x0, u64 *y0, uint32_t *c1, u64 *x1, u64 *y1,
                        float4 *rec, float *recn, uint32_t *blk_off, uint32_t *s_warp) {
    const int tid = threadIdx.x;
    const int nb = 1 << (2 * h0);
    // blk_off: each thread scans a contiguous segment (16-byte loads when the
    // segments are multiples of four)
    const int seg = (nb + 255) / 256;
    const int a = tid * seg, e = min(nb, a + seg);
    uint32_t v = 0u;
    if ((seg & 3) == 0) {
        for (int i = a; i < e; i += 4) {
            const uint4 q = __ldcg(reinterpret_cast<const uint4 *>(c0 + i));
            v += q.x + q.y + q.z + q.w;
        }
    } else {
        for (int i = a; i < e; i++) v += __ldcg(c0 + i);
    }
    uint32_t run = block_excl_scan(v, 256, s_warp);
    if ((seg & 3) == 0) {
        for (int i = a; i < e; i += 4) {
            const uint4 q = __ldcg(reinterpret_cast<const uint4 *>(c0 + i));
            uint4 o;
            o.x = run;
            o.y = o.x + q.x;
            o.z = o.y + q.y;
            o.w = o.z + q.z;
            run = o.w + q.w;
            *reinterpret_cast<uint4 *>(blk_off + i) = o;
        }
    } else {
        for (int i = a; i < e; i++) {
            const uint32_t ci = __ldcg(c0 + i);
            blk_off[i] = run;
            run += ci;
        }
    }
    uint32_t *cc = c0, *cn = c1;
    u64 *xc = x0, *xn = x1, *yc = y0, *yn = y1;
    const bool sums = rec != nullptr;
    for (int l = h0;; l--) {
        const int cells = 1 << (2 * l);
        if (l < h0)
            for (int c = tid; c < cells; c += 256)
                put_record(rec, recn, l, (uint32_t)c, __ldcg(cc + c), sums ? __ldcg(xc + c) : 0ull,
                           sums ? __ldcg(yc + c) : 0ull);
        if (l == 0) break;
        for (int p = tid; p < (cells >> 2); p += 256) {
            const uint4 q4 = __ldcg(reinterpret_cast<const uint4 *>(cc) + p);
            cn[p] = q4.x + q4.y + q4.z + q4.w;
            if (sums) {
                const ulonglong2 xa = __ldcg(reinterpret_cast<const ulonglong2 *>(xc) + 2 * p);
                const ulonglong2 xb = __ldcg(reinterpret_cast<const ulonglong2 *>(xc) + 2 * p + 1);
                const ulonglong2 ya = __ldcg(reinterpret_cast<const ulonglong2 *>(yc) + 2 * p);
                const ulonglong2 yb = __ldcg(reinterpret_cast<const ulonglong2 *>(yc) + 2 * p + 1);
                xn[p] = xa.x + xa.y + xb.x + xb.y;
                yn[p] = ya.x + ya.y + yb.x + yb.y;
            }
        }
        __threadfence_block();
        __syncthreads();
        uint32_t *tc = cc;
        cc = cn;
        cn = tc;
        u64 *tx = xc;
        xc = xn;
        xn = tx;
        u64 *ty = yc;
        yc = yn;
        yn = ty;
    }
}

__global__ void __launch_bounds__(256)
    k_pyr_bottom(int h, uint32_t *__restrict__ in_cnt, u64 *__restrict__ in_sx,
                 u64 *__restrict__ in_sy, float4 *__restrict__ rec, float *__restrict__ recn,
                 uint32_t *out_cnt, u64 *out_sx, u64 *out_sy, uint32_t *scr_cnt, u64 *scr_sx,
                 u64 *scr_sy, uint32_t *__restrict__ leaf_start, uint32_t *blk_off,
                 DevScalars *sc, int bump_t) {
    __shared__ uint32_t s_n[8];
    __shared__ u64 s_x[8], s_y[8];
    __shared__ uint32_t s_warp[32];
    __shared__ bool s_last;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t b = blockIdx.x;
    const uint32_t cell0 = b * 1024u + 4u * (uint32_t)tid;
    // rec == NULL: a count-only tree (geometric centres), no sums read or kept
    const bool sums = rec != nullptr;
    const uint4 c4 = reinterpret_cast<const uint4 *>(in_cnt)[cell0 >> 2];
    ulonglong2 x01{0, 0}, x23{0, 0}, y01{0, 0}, y23{0, 0};
    if (sums) {
        x01 = reinterpret_cast<const ulonglong2 *>(in_sx)[cell0 >> 1];
        x23 = reinterpret_cast<const ulonglong2 *>(in_sx)[(cell0 >> 1) + 1];
        y01 = reinterpret_cast<const ulonglong2 *>(in_sy)[cell0 >> 1];
        y23 = reinterpret_cast<const ulonglong2 *>(in_sy)[(cell0 >> 1) + 1];
        float4 *rl = rec + rec_offset(h) + cell0;
        // (an empty cell's record is never read: not written)
        if (c4.x) rl[0] = make_record(c4.x, x01.x, y01.x, h, cell0);
        if (c4.y) rl[1] = make_record(c4.y, x01.y, y01.y, h, cell0 + 1u);
        if (c4.z) rl[2] = make_record(c4.z, x23.x, y23.x, h, cell0 + 2u);
        if (c4.w) rl[3] = make_record(c4.w, x23.y, y23.y, h, cell0 + 3u);
    }
    reinterpret_cast<float4 *>(recn + rec_offset(h))[cell0 >> 2] =
        make_float4((float)c4.x, (float)c4.y, (float)c4.z, (float)c4.w);
    clear_leaves(cell0, c4, in_cnt, in_sx, in_sy);
    uint32_t N = c4.x + c4.y + c4.z + c4.w;
    u64 X = x01.x + x01.y + x23.x + x23.y;
    u64 Y = y01.x + y01.y + y23.x + y23.y;
    // inclusive warp scan of the level-(h-1) counts (for the pixel starts)
    uint32_t inc = N;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    put_record(rec, recn, h - 1, b * 256u + (uint32_t)tid, N, X, Y);
    // levels h-2 (4 lanes) and h-3 (16 lanes)
#pragma unroll
    for (int o = 1; o <= 2; o <<= 1) {
        N += __shfl_xor_sync(0xffffffffu, N, o);
        if (sums) {
            X += shfl_xor_u64(X, o);
            Y += shfl_xor_u64(Y, o);
        }
    }
    if ((lane & 3) == 0) put_record(rec, recn, h - 2, b * 64u + (uint32_t)(tid >> 2), N, X, Y);
#pragma unroll
    for (int o = 4; o <= 8; o <<= 1) {
        N += __shfl_xor_sync(0xffffffffu, N, o);
        if (sums) {
            X += shfl_xor_u64(X, o);
            Y += shfl_xor_u64(Y, o);
        }
    }
    if ((lane & 15) == 0) put_record(rec, recn, h - 3, b * 16u + (uint32_t)(tid >> 4), N, X, Y);
    N += __shfl_xor_sync(0xffffffffu, N, 16);
    if (sums) {
        X += shfl_xor_u64(X, 16);
        Y += shfl_xor_u64(Y, 16);
    }
    if (lane == 0) {
        s_n[warp] = N;
        s_x[warp] = X;
        s_y[warp] = Y;
    }
    __syncthreads();
    // pixel starts within the CTA
    uint32_t before = 0u;
    for (int w = 0; w < warp; w++) before += s_n[w];
    const uint32_t e0 = before + inc - (c4.x + c4.y + c4.z + c4.w);
    uint4 st;
    st.x = e0;
    st.y = e0 + c4.x;
    st.z = st.y + c4.y;
    st.w = st.z + c4.z;
    reinterpret_cast<uint4 *>(leaf_start)[cell0 >> 2] = st;
    // level h-4: pairs of warps; level h-5: the CTA
    if (tid < 4)
        put_record(rec, recn, h - 4, b * 4u + (uint32_t)tid, s_n[2 * tid] + s_n[2 * tid + 1],
                   s_x[2 * tid] + s_x[2 * tid + 1], s_y[2 * tid] + s_y[2 * tid + 1]);
    if (tid == 0) {
        uint32_t n5 = 0u;
        u64 x5 = 0ull, y5 = 0ull;
        for (int w = 0; w < 8; w++) {
            n5 += s_n[w];
            x5 += s_x[w];
            y5 += s_y[w];
        }
        out_cnt[b] = n5;
        if (sums) {
            out_sx[b] = x5;
            out_sy[b] = y5;
        }
        put_record(rec, recn, h - 5, b, n5, x5, y5);
        // the last CTA to finish builds the top of the pyramid
        __threadfence();
        const unsigned tk = atomicAdd(&sc->pyr_ticket, 1u);
        s_last = (tk == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    pyr_top(h - 5, out_cnt, out_sx, out_sy, scr_cnt, scr_sx, scr_sy, rec, recn, blk_off, s_warp);
    if (tid == 0) {
        sc->pyr_ticket = 0u;
        if (bump_t) sc->t += 1;
    }
}

// Exclusive scan of m values in one CTA of 1024 threads.
__global__ void __launch_bounds__(1024) k_scan1(const uint32_t *__restrict__ in,
                                                uint32_t *__restrict__ out, int64_t m) {
    __shared__ uint32_t s_warp[32];
    __shared__ uint32_t s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < m; base += 1024) {
        const int64_t i = base + threadIdx.x;
        const uint32_t v = i < m ? in[i] : 0u;
        const uint32_t e = block_excl_scan(v, 1024, s_warp);
        const uint32_t carry = s_carry;
        if (i < m) out[i] = carry + e;
        __syncthreads();
        if (threadIdx.x == 1023) s_carry = carry + e + v;
        __syncthreads();
    }
}

__global__ void k_perm_scatter(int n, int L, int K1, const uint2 *__restrict__ z,
                               const uint32_t *__restrict__ rank,
                               const uint32_t *__restrict__ leaf_start,
                               const uint32_t *__restrict__ blk_off,
                               uint32_t *__restrict__ perm, DevScalars *sc) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int F = 32 - L;
    const uint2 v = z[i];
    const uint32_t m = morton2(v.x >> F, v.y >> F);
    const uint32_t pos = blk_off[m >> (2 * K1)] + leaf_start[m] + rank[i];
    if (pos < (uint32_t)n) perm[pos] = (uint32_t)i;
    else atomicOr(&sc->err, (unsigned)PXSNE_DEVERR_STACK);
}

static cudaError_t pyr_pass(int K, int64_t blocks, cudaStream_t st, int h, int top,
                            const uint32_t *ic, const u64 *ix, const u64 *iy, float4 *rec,
                            float *recn,
                            uint32_t *oc, u64 *ox, u64 *oy, uint32_t *ls, DevScalars *sc,
                            int bump, int clear) {
    const dim3 g((unsigned)blocks);
    switch (K) {
    case 1: k_pyr_pass<1><<<g, 1, 0, st>>>(h, top, ic, ix, iy, rec, recn, oc, ox, oy, ls, sc, bump, clear); break;
    case 2: k_pyr_pass<2><<<g, 4, 0, st>>>(h, top, ic, ix, iy, rec, recn, oc, ox, oy, ls, sc, bump, clear); break;
    case 3: k_pyr_pass<3><<<g, 16, 0, st>>>(h, top, ic, ix, iy, rec, recn, oc, ox, oy, ls, sc, bump, clear); break;
    case 4: k_pyr_pass<4><<<g, 64, 0, st>>>(h, top, ic, ix, iy, rec, recn, oc, ox, oy, ls, sc, bump, clear); break;
    default: k_pyr_pass<5><<<g, 256, 0, st>>>(h, top, ic, ix, iy, rec, recn, oc, ox, oy, ls, sc, bump, clear); break;
    }
    return cudaGetLastError();
}

// Tree of the current state.  rescale != 0: zhat -> z first (an iteration);
// otherwise z is taken as it is (initial state).  Also rebuilds the traversal
// order and, for an iteration, advances the iteration counter.
cudaError_t launch_snap(pxsne_ctx *c, bool rescale, cudaEvent_t *marks) {
    cudaStream_t st = c->stream;
    const int L = c->L;
    cudaError_t e;
    if (marks && (e = cudaEventRecord(marks[KG_SNAP], st))) return e;
    // geometric centres (Sec. 4.1's approximation) need the counts only; the
    // leaves are zero here (set at allocation, cleared by the pyramid's first
    // pass after each histogram)
    const bool sums = c->p.centre_mode == 0;
    const int n = (int)c->n;
    k_snap_hist<<<(n + 255) / 256, 256, 0, st>>>(n, L, rescale ? 1 : 0, c->p.theta,
                                                 screen_extent(c->p.screen_x, L),
                                                 screen_extent(c->p.screen_y, L), c->zhat,
                                                 c->z, c->perm, c->rank, c->leaf_cnt,
                                                 sums ? c->leaf_sx : nullptr,
                                                 sums ? c->leaf_sy : nullptr, c->sc, c->ainv,
                                                 c->zp);
    return cudaGetLastError();
}

cudaError_t launch_pyramid(pxsne_ctx *c, bool rescale, cudaEvent_t *marks) {
    cudaStream_t st = c->stream;
    const int L = c->L;
    const int64_t leaves = int64_t(1) << (2 * L);
    const int n = (int)c->n;
    cudaError_t e;
    if (marks && (e = cudaEventRecord(marks[KG_PYRAMID], st))) return e;
    const int K1 = L < kPyrK ? L : kPyrK;
    const bool sums = c->p.centre_mode == 0;  // count-only tree for geometric centres
    if (L >= kPyrK && L - kPyrK <= 7) {
        // one pass: shuffle-reduced bottom levels, the top by the last CTA
        k_pyr_bottom<<<(unsigned)(leaves >> 10), 256, 0, st>>>(
            L, c->leaf_cnt, sums ? c->leaf_sx : nullptr, sums ? c->leaf_sy : nullptr,
            sums ? c->rec : nullptr, c->recn, c->lvl_cnt[0],
            c->lvl_sx[0], c->lvl_sy[0], c->lvl_cnt[1], c->lvl_sx[1], c->lvl_sy[1],
            c->leaf_start, c->blk_off, c->sc, rescale ? 1 : 0);
        if ((e = cudaGetLastError())) return e;
    } else {
        // bottom-up passes
        int h = L;
        int cur = 0;
        {
            const int64_t blocks = leaves >> (2 * K1);
            const int top = (h - K1 == 0);
            if ((e = pyr_pass(K1, blocks, st, h, top, c->leaf_cnt, sums ? c->leaf_sx : nullptr,
                              c->leaf_sy,
                              c->rec, c->recn, c->lvl_cnt[0], c->lvl_sx[0], c->lvl_sy[0],
                              c->leaf_start, c->sc, (rescale && top) ? 1 : 0, 1)))
                return e;
            h -= K1;
        }
        // traversal order: scan of the per-CTA pixel totals of the first pass
        k_scan1<<<1, 1024, 0, st>>>(c->lvl_cnt[0], c->blk_off, int64_t(1) << (2 * h));
        if ((e = cudaGetLastError())) return e;
        while (h > 0) {
            const int K = h < kPyrK ? h : kPyrK;
            const int64_t blocks = (int64_t(1) << (2 * h)) >> (2 * K);
            const int top = (h - K == 0);
            if ((e = pyr_pass(K, blocks, st, h, top, c->lvl_cnt[cur],
                              sums ? c->lvl_sx[cur] : nullptr, c->lvl_sy[cur], c->rec, c->recn,
                              c->lvl_cnt[cur ^ 1],
                              c->lvl_sx[cur ^ 1], c->lvl_sy[cur ^ 1], nullptr, c->sc,
                              (rescale && top) ? 1 : 0, 0)))
                return e;
            cur ^= 1;
            h -= K;
        }
    }
    if (marks && (e = cudaEventRecord(marks[KG_PERM], st))) return e;
    k_perm_scatter<<<(n + 255) / 256, 256, 0, st>>>(n, L, K1, c->z, c->rank, c->leaf_start,
                                                    c->blk_off, c->perm, c->sc);
    return cudaGetLastError();
}

// Tree of the current state.  rescale != 0: zhat -> z first (an iteration);
// otherwise z is taken as it is (initial state).  Also rebuilds the traversal
// order and, for an iteration, advances the iteration counter.
cudaError_t launch_tree(pxsne_ctx *c, bool rescale, cudaEvent_t *marks) {
    cudaError_t e = launch_snap(c, rescale, marks);
    if (e) return e;
    return launch_pyramid(c, rescale, marks);
}

// ---------------------------------------------------------------- init / output
__device__ __forceinline__ uint32_t f2key(float f) {
    uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float key2f(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

__global__ void k_minmax_y0(int n, const float2 *__restrict__ Y, uint32_t *mm,
                            DevScalars *sc) {
    uint32_t mnx = 0xffffffffu, mny = 0xffffffffu, mxx = 0u, mxy = 0u;
    bool bad = false;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float2 y = Y[i];
        bad |= !isfinite(y.x) || !isfinite(y.y);
        const uint32_t kx = f2key(y.x), ky = f2key(y.y);
        mnx = min(mnx, kx); mxx = max(mxx, kx);
        mny = min(mny, ky); mxy = max(mxy, ky);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mnx = min(mnx, __shfl_xor_sync(0xffffffffu, mnx, o));
        mny = min(mny, __shfl_xor_sync(0xffffffffu, mny, o));
        mxx = max(mxx, __shfl_xor_sync(0xffffffffu, mxx, o));
        mxy = max(mxy, __shfl_xor_sync(0xffffffffu, mxy, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&mm[0], mnx); atomicMin(&mm[1], mny);
        atomicMax(&mm[2], mxx); atomicMax(&mm[3], mxy);
    }
    if (bad) atomicOr(&sc->err, (unsigned)PXSNE_DEVERR_NONFINITE);
}

// Eq. z1/z2 mapping of the initial embedding onto the fixed-point screen (FP64).
__global__ void k_map_y0(int n, int L, float theta, double Rx, double Ry,
                         const float2 *__restrict__ Y,
                         const uint32_t *__restrict__ mm, uint2 *__restrict__ z,
                         float2 *__restrict__ u, float2 *__restrict__ gains, DevScalars *sc) {
    const double mnx = (double)key2f(mm[0]), mny = (double)key2f(mm[1]);
    const double rx = (double)key2f(mm[2]) - mnx, ry = (double)key2f(mm[3]) - mny;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        sc->s[0] = rx > 0.0 ? rx / Rx : 1.0 / Rx;
        sc->s[1] = ry > 0.0 ? ry / Ry : 1.0 / Ry;
        derive_scalars(sc, theta, L);
        sc->t = 0;
        sc->Z = 0.0;
        for (int p = 0; p < 2; p++) {
            sc->mm[p][0] = 0x7fffffffffffffffll;
            sc->mm[p][1] = 0x7fffffffffffffffll;
            sc->mm[p][2] = (i64)0x8000000000000000ull;
            sc->mm[p][3] = (i64)0x8000000000000000ull;
        }
    }
    if (i >= n) return;
    const float2 y = Y[i];
    uint32_t zx = 0u, zy = 0u;
    if (rx > 0.0) {
        const double q = floor(((double)y.x - mnx) * Rx / rx);
        zx = q >= Rx - 1.0 ? (uint32_t)(Rx - 1.0) : (uint32_t)q;
    }
    if (ry > 0.0) {
        const double q = floor(((double)y.y - mny) * Ry / ry);
        zy = q >= Ry - 1.0 ? (uint32_t)(Ry - 1.0) : (uint32_t)q;
    }
    z[i] = make_uint2(zx, zy);
    u[i] = make_float2(0.f, 0.f);
    gains[i] = make_float2(1.f, 1.f);
}

cudaError_t launch_init_map(pxsne_ctx *c, const float *Y0dev, uint32_t *mm_scratch) {
    cudaStream_t st = c->stream;
    const int n = (int)c->n;
    const uint32_t init[4] = {0xffffffffu, 0xffffffffu, 0u, 0u};
    cudaError_t e;
    if ((e = cudaMemcpyAsync(mm_scratch, init, sizeof(init), cudaMemcpyHostToDevice, st)))
        return e;
    const int blocks = (n + 255) / 256 < 1184 ? (n + 255) / 256 : 1184;
    k_minmax_y0<<<blocks > 0 ? blocks : 1, 256, 0, st>>>(
        n, reinterpret_cast<const float2 *>(Y0dev), mm_scratch, c->sc);
    if ((e = cudaGetLastError())) return e;
    k_map_y0<<<(n + 255) / 256, 256, 0, st>>>(n, c->L, c->p.theta,
                                              (double)screen_extent(c->p.screen_x, c->L),
                                              (double)screen_extent(c->p.screen_y, c->L),
                                              reinterpret_cast<const float2 *>(Y0dev),
                                              mm_scratch, c->z, c->u, c->gains, c->sc);
    return cudaGetLastError();
}

__global__ void k_sum_z(int n, const uint2 *__restrict__ z, u64 *sums) {
    u64 ax = 0, ay = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint2 v = z[i];
        ax += v.x;
        ay += v.y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ax += __shfl_xor_sync(0xffffffffu, ax, o);
        ay += __shfl_xor_sync(0xffffffffu, ay, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&sums[0], ax);
        atomicAdd(&sums[1], ay);
    }
}

__global__ void k_write_y(int n, int L, const uint2 *__restrict__ z, const u64 *__restrict__ sums,
                          const DevScalars *__restrict__ sc, float2 *__restrict__ Y,
                          int2 *__restrict__ pix) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint2 v = z[i];
    if (Y) {
        const double mx = (double)sums[0] / (double)n, my = (double)sums[1] / (double)n;
        Y[i] = make_float2((float)(sc->s[0] * ((double)v.x - mx)),
                           (float)(sc->s[1] * ((double)v.y - my)));
    }
    if (pix) pix[i] = make_int2((int)(v.x >> (32 - L)), (int)(v.y >> (32 - L)));
}

cudaError_t launch_centre_y(pxsne_ctx *c, float *Ydev, int32_t *pixdev, float *scratch) {
    cudaStream_t st = c->stream;
    const int n = (int)c->n;
    u64 *sums = reinterpret_cast<u64 *>(scratch);
    cudaError_t e;
    if (Ydev) {  // the mean, for centred coordinates (pixels alone need none)
        if ((e = cudaMemsetAsync(sums, 0, 2 * sizeof(u64), st))) return e;
        const int blocks = (n + 255) / 256 < 1184 ? (n + 255) / 256 : 1184;
        k_sum_z<<<blocks > 0 ? blocks : 1, 256, 0, st>>>(n, c->z, sums);
        if ((e = cudaGetLastError())) return e;
    }
    k_write_y<<<(n + 255) / 256, 256, 0, st>>>(n, c->L, c->z, sums, c->sc,
                                               reinterpret_cast<float2 *>(Ydev),
                                               reinterpret_cast<int2 *>(pixdev));
    return cudaGetLastError();
}

__global__ void k_level_counts(int64_t cells, const float *__restrict__ recn, uint32_t *cnt) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < cells) cnt[i] = (uint32_t)recn[i];
}

cudaError_t launch_level_counts(pxsne_ctx *c, int level, uint32_t *cnt) {
    const int64_t cells = int64_t(1) << (2 * level);
    k_level_counts<<<(unsigned)((cells + 255) / 256), 256, 0, c->stream>>>(
        cells, c->recn + rec_offset(level), cnt);
    return cudaGetLastError();
}

// The leaf histogram of the current state, for inspection (the iteration's
// own is cleared by the pyramid once read): counts and exact coordinate sums.
__global__ void k_leaf_hist(int n, int L, const uint2 *__restrict__ z, uint32_t *cnt, u64 *sx,
                            u64 *sy) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint2 v = z[i];
    const uint32_t m = morton2(v.x >> (32 - L), v.y >> (32 - L));
    if (cnt) atomicAdd(&cnt[m], 1u);
    if (sx) atomicAdd(&sx[m], (u64)v.x);
    if (sy) atomicAdd(&sy[m], (u64)v.y);
}

cudaError_t launch_leaf_hist(pxsne_ctx *c, uint32_t *cnt, u64 *sx, u64 *sy) {
    const int n = (int)c->n;
    const size_t leaves = size_t(1) << (2 * c->L);
    cudaError_t e;
    if (cnt && (e = cudaMemsetAsync(cnt, 0, leaves * 4, c->stream))) return e;
    if (sx && (e = cudaMemsetAsync(sx, 0, leaves * 8, c->stream))) return e;
    if (sy && (e = cudaMemsetAsync(sy, 0, leaves * 8, c->stream))) return e;
    k_leaf_hist<<<(n + 255) / 256, 256, 0, c->stream>>>(n, c->L, c->z, cnt, sx, sy);
    return cudaGetLastError();
}

__global__ void k_morton_keys(int n, int L, const uint2 *__restrict__ z, uint32_t *keys) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint2 v = z[i];
    keys[i] = morton2(v.x >> (32 - L), v.y >> (32 - L));
}

cudaError_t launch_morton_keys(pxsne_ctx *c, uint32_t *keys) {
    const int n = (int)c->n;
    k_morton_keys<<<(n + 255) / 256, 256, 0, c->stream>>>(n, c->L, c->z, keys);
    return cudaGetLastError();
}

}  // namespace pxsne
