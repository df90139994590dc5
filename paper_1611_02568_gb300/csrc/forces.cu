// Forces of the PixelSNE gradient (Eq. grad) on the pixel-aligned tree.
//
//   k_bh_traverse  repulsion by Barnes-Hut (Sec. 3.3, Eq. bh_criteria) on the
//                  dense pyramid, one warp per 64 points of the Morton order
//                  (two per lane, as packed FP32 pairs); each point keeps its
//                  own accept/open decisions (lane masks per stack entry), so
//                  it sees exactly the cells its own depth-first search would
//   k_attract      attraction over the CSR of P, one warp per row
//   k_zsum         Z = sum_i Z_i in FP64, fixed summation order
//   k_kl           Eq. cost_func in FP64 accumulation
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace pxsne {

// One warp = 64 points consecutive in Morton order, two per lane (lane l holds
// points l and l + 32); the two are held and computed as packed FP32 pairs
// (each component rounded to nearest exactly as the scalar operation).  Each
// stack entry is a node whose four children are to be tested, with one mask per
// half of the warp's points marking the points that opened it, so every point
// sees exactly the cells its own depth-first search would.  A child's record is
// loaded once for all the warp's points.  The per-child step is branch-free
// within a level: every lane computes its points' offsets, distances and kernel
// values, and the accept/open decisions only gate the accumulation and the
// push.  Children at the leaf level are always accepted (bounded depth, Sec.
// 4.1) except for a point's own pixel, which is used without the point itself;
// children above it follow Eq. bh_criteria, and the cell holding a point's own
// pixel is opened.  A point accumulates its cells in the fixed depth-first order
// of the tree, so its result does not depend on the warp it shares.
// CENTRE = 0: centre of mass; 1: geometric cell centre.  COUNT = 1 also
// counts tested and accepted (point, cell) pairs.
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    return __ffma2_rn(a, b, c);
}
__device__ __forceinline__ float2 bc2(float v) { return make_float2(v, v); }
// The kernel value 1 / (1 + d^2) (argument >= 1): the hardware's approximate
// reciprocal (PTX rcp.approx, relative error within 2^-23), one instruction.
__device__ __forceinline__ float rcp1(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Offset z - c of a lane's two points from the cell's centre: of mass (the
// split record r), or (CENTRE = 1) the geometric centre, passed in r.x / r.z
// as exact floats (multiples of 2^16 below level 16), so that z - c =
// (z_hi - c) + z_lo with one rounding, as for a centre of mass.
template <int CENTRE>
__device__ __forceinline__ void cell_offset2(float4 r, float2 zhx, float2 zlx, float2 zhy,
                                             float2 zly, float2 &dx, float2 &dy) {
    if (CENTRE == 0) {
        dx = add2(add2(zhx, bc2(-r.x)), add2(zlx, bc2(-r.y)));
        dy = add2(add2(zhy, bc2(-r.z)), add2(zly, bc2(-r.w)));
    } else {
        dx = add2(add2(zhx, bc2(-r.x)), zlx);
        dy = add2(add2(zhy, bc2(-r.z)), zly);
    }
}

// COUNT: one warp step's (tested, accepted) pairs and the step itself, added
// to the CTA's counters of the child's level by lane 0.
__device__ __forceinline__ void count_level(u64 *lv, bool me0, bool me1, bool acc0, bool acc1,
                                            int lane) {
    const unsigned t = __popc(__ballot_sync(0xffffffffu, me0)) +
                       __popc(__ballot_sync(0xffffffffu, me1));
    const unsigned a = __popc(__ballot_sync(0xffffffffu, acc0)) +
                       __popc(__ballot_sync(0xffffffffu, acc1));
    if (lane == 0) {
        atomicAdd(&lv[0], (u64)t);
        atomicAdd(&lv[1], (u64)a);
        atomicAdd(&lv[2], 1ull);
    }
}

// A coordinate's two 16-bit halves as floats, each offset by a power of two
// that leaves the half's bits as the mantissa: hi_bits(v) = 2^39 + (v >> 16)
// 2^16 (ulp 2^16 at 2^39) and lo_bits(v) = 2^23 + (v & 0xffff) (ulp 1 at
// 2^23), both exact and built by bit operations instead of integer-to-float
// conversions.  The difference of two such values cancels the offset
// exactly, so (hi_bits(a) - hi_bits(b)) + (lo_bits(a) - lo_bits(b)) is the
// exact difference of the halves with one final rounding, as when the halves
// are converted and subtracted directly.
__device__ __forceinline__ float hi_bits(uint32_t v) {
    return __uint_as_float(0x53000000u | (v >> 16));
}
__device__ __forceinline__ float lo_bits(uint32_t v) {
    return __uint_as_float(0x4B000000u | (v & 0xffffu));
}

// Eq. grad, first term: Fattr_i = sum_j p_ij w_ij (y_i - y_j), one warp per
// row (row lengths vary with the in-degree of the kNN graph; a warp per row
// keeps long rows from stalling short ones).  It runs over the relabelled copy
// of P (rows and columns in the Morton order of a recent state), so a row's
// gathered positions zp[j] lie close together in memory, and writes each row's
// force back under the point's own index.  Each lane keeps four entries in
// flight; P is streamed with evict-first loads so that the positions stay in
// L2.  z_i - z_j is formed exactly in float from the 16-bit halves of the
// fixed-point coordinates (both differences are exact; one final rounding).
// Entry order within a row is that of P, so the sums equal those over P.
struct AttractArgs {
    const int64_t *rp;
    const int32_t *col;
    const float *val;
    const uint2 *z;         // positions under the relabelled labels
    const uint32_t *aperm;  // relabelled row -> point
    float2 *Fattr;
};

__device__ __forceinline__ void attract_row(int row, int lane, const AttractArgs &a, float sf0,
                                            float sf1) {
    constexpr int U = 4;
    const int64_t *__restrict__ rp = a.rp;
    const int32_t *__restrict__ col = a.col;
    const float *__restrict__ val = a.val;
    const uint2 *__restrict__ z = a.z;
    const uint2 zi = z[row];
    // the row's halves offset by the same constants as hi_bits / lo_bits
    const float xh = hi_bits(zi.x), xl = lo_bits(zi.x);
    const float yh = hi_bits(zi.y), yl = lo_bits(zi.y);
    const int64_t e0 = rp[row], e1 = rp[row + 1];
    float fx = 0.f, fy = 0.f;
    // software pipeline: the next batch of P is requested while the current
    // batch's positions are being gathered
    int32_t jn[U];
    float pn[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
        const int64_t q = e0 + lane + 32 * u;
        jn[u] = q < e1 ? __ldcs(col + q) : row;
        pn[u] = q < e1 ? __ldcs(val + q) : 0.f;
    }
    for (int64_t e = e0 + lane; e < e1; e += 32 * U) {
        int32_t j[U];
        float p[U];
        uint2 zj[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            j[u] = jn[u];
            p[u] = pn[u];
            zj[u] = z[j[u]];
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int64_t q = e + 32 * (U + u);
            jn[u] = q < e1 ? __ldcs(col + q) : row;
            pn[u] = q < e1 ? __ldcs(val + q) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            const float dx = ((xh - hi_bits(zj[u].x)) + (xl - lo_bits(zj[u].x))) * sf0;
            const float dy = ((yh - hi_bits(zj[u].y)) + (yl - lo_bits(zj[u].y))) * sf1;
            const float w = __fdividef(1.0f, 1.0f + fmaf(dx, dx, dy * dy));
            const float pw = p[u] * w;
            fx = fmaf(pw, dx, fx);
            fy = fmaf(pw, dy, fy);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        fx += __shfl_xor_sync(0xffffffffu, fx, o);
        fy += __shfl_xor_sync(0xffffffffu, fy, o);
    }
    if (lane == 0) a.Fattr[a.aperm[row]] = make_float2(fx, fy);
}

struct __align__(16) TravEntry {
    uint32_t node, m0, m1, pad;
};

template <int CENTRE, int COUNT, bool OWN>
__global__ void __launch_bounds__(kTravWarps * 32, 4)
    k_bh_traverse(int n, int L, const uint2 *__restrict__ z, const uint32_t *__restrict__ perm,
                  const float4 *__restrict__ rec, const float *__restrict__ recn,
                  DevScalars *sc, float2 *__restrict__ Frep, float *__restrict__ Zi) {
    // stack entry: (level << 28) | Morton index of a node, and for each half of
    // the warp's points the mask of the lanes whose point opens it
    __shared__ TravEntry s_stk[kTravWarps][kTravStack];
    __shared__ float s_T[kMaxL + 2];
    __shared__ int s_off[kMaxL + 2];
    const int stk_lim = sc->stack_limit > 0 ? min(max(sc->stack_limit, 4), kTravStack) : kTravStack;
    // COUNT: (tested, accepted, warp steps) by level of the child
    __shared__ u64 s_lv[COUNT ? kMaxL + 2 : 1][3];
    if (threadIdx.x < kMaxL + 2) {
        s_T[threadIdx.x] = sc->T[threadIdx.x];
        s_off[threadIdx.x] = threadIdx.x <= L ? (int)rec_offset(threadIdx.x) : 0;
        if (COUNT) s_lv[threadIdx.x][0] = s_lv[threadIdx.x][1] = s_lv[threadIdx.x][2] = 0ull;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int F = 32 - L;
    const float2 sf0 = bc2(sc->sf[0]), sf1 = bc2(sc->sf[1]);
    uint32_t n_acc = 0u, n_tst = 0u, n_stp = 0u, n_nod = 0u;
    TravEntry *stk = s_stk[w];
    // Each warp takes the next 64 points of the Morton order until none are
    // left: a warp whose points are cheap moves on instead of idling until
    // the slowest warp of its CTA is done.
    for (;;) {
        unsigned chunk = 0u;
        if (lane == 0) chunk = atomicAdd(&sc->trav_next, 1u);
        chunk = __shfl_sync(0xffffffffu, chunk, 0);
        if ((int64_t)chunk * 64 >= n) break;
        const int base = (int)chunk * 64;
        const int idx0 = base + lane, idx1 = base + 32 + lane;
        const bool valid0 = idx0 < n, valid1 = idx1 < n;
        const unsigned act0 = __ballot_sync(0xffffffffu, valid0);
        const unsigned act1 = __ballot_sync(0xffffffffu, valid1);
        const uint32_t i0 = valid0 ? perm[idx0] : 0u, i1 = valid1 ? perm[idx1] : 0u;
        const uint2 z0 = z[i0], z1 = z[i1];
        const uint32_t mi0 = morton2(z0.x >> F, z0.y >> F), mi1 = morton2(z1.x >> F, z1.y >> F);
        // z split at bit 16, both halves exact in float (see rec in common.cuh)
        const float2 zhx = make_float2((float)(z0.x & 0xffff0000u), (float)(z1.x & 0xffff0000u));
        const float2 zlx = make_float2((float)(z0.x & 0xffffu), (float)(z1.x & 0xffffu));
        const float2 zhy = make_float2((float)(z0.y & 0xffff0000u), (float)(z1.y & 0xffff0000u));
        const float2 zly = make_float2((float)(z0.y & 0xffffu), (float)(z1.y & 0xffffu));
        float2 fx = bc2(0.f), fy = bc2(0.f), zs = bc2(0.f);

        // The root contains every point: start with its four children.
        if (lane == 0) stk[0] = TravEntry{0u, act0, act1, 0u};  // (level 0 << 28) | morton 0
        int sp = 1;
        __syncwarp();
        bool overflow = false;
        while (sp > 0) {
            sp--;
            TravEntry top = stk[sp];
            __syncwarp();
            // the entry is the same for every lane: taken from lane 0, so that
            // the node, its level and addresses are known to be warp-uniform
            top.node = __shfl_sync(0xffffffffu, top.node, 0);
            top.m0 = __shfl_sync(0xffffffffu, top.m0, 0);
            top.m1 = __shfl_sync(0xffffffffu, top.m1, 0);
            const uint32_t node = top.node;
            const int lc = (int)(node >> 28) + 1;  // level of the children
            const uint32_t m0 = (node & 0x0fffffffu) << 2;
            const int at = s_off[lc] + (int)m0;
            const float4 nv = __ldg(reinterpret_cast<const float4 *>(recn + at));
            // the four children's records are requested together with their
            // counts (one latency per node instead of two)
            float4 rr[4];
            if (CENTRE == 0) {
#pragma unroll
                for (int ch = 0; ch < 4; ch++) rr[ch] = __ldg(rec + at + ch);
            } else {
                // geometric centres: the node's corner (exact floats) and width
                // 2^(33 - lc); child ch's centre is a quarter or three quarters
                // across on each axis
                const uint32_t pm = node & 0x0fffffffu;
                const float wp = __int_as_float((127 + 33 - lc) << 23);
                const float px = (float)gather_bits16(pm) * wp, py = (float)gather_bits16(pm >> 1) * wp;
#pragma unroll
                for (int ch = 0; ch < 4; ch++)
                    rr[ch] = make_float4(fmaf(wp, (ch & 1) ? 0.75f : 0.25f, px), 0.f,
                                         fmaf(wp, (ch & 2) ? 0.75f : 0.25f, py), 0.f);
            }
            const bool me0 = (top.m0 >> lane) & 1u, me1 = (top.m1 >> lane) & 1u;
            const float Nc[4] = {nv.x, nv.y, nv.z, nv.w};
            if (COUNT) {
                n_nod++;
                n_stp += (nv.x != 0.f) + (nv.y != 0.f) + (nv.z != 0.f) + (nv.w != 0.f);
            }
            if (lc == L) {
                const uint32_t mine0 = mi0, mine1 = mi1;  // own pixels
#pragma unroll
                for (int ch = 0; ch < 4; ch++) {
                    const float N = Nc[ch];
                    if (N == 0.f) continue;
                    const uint32_t mc = m0 + ch;
                    const float4 r = rr[ch];
                    float2 dx, dy;
                    cell_offset2<CENTRE>(r, zhx, zlx, zhy, zly, dx, dy);
                    const bool own0 = me0 && (mine0 == mc), own1 = me1 && (mine1 == mc);
                    float2 Nf = bc2(N);
                    if (__any_sync(0xffffffffu, own0 || own1)) {  // own pixel: take the point out
                        if (own0) {
                            Nf.x = N - 1.0f;
                            if (CENTRE == 0 && N > 1.0f) {
                                const float k = N / Nf.x;
                                dx.x *= k;
                                dy.x *= k;
                            }
                        }
                        if (own1) {
                            Nf.y = N - 1.0f;
                            if (CENTRE == 0 && N > 1.0f) {
                                const float k = N / Nf.y;
                                dx.y *= k;
                                dy.y *= k;
                            }
                        }
                    }
                    dx = mul2(dx, sf0);
                    dy = mul2(dy, sf1);
                    const float2 d2 = fma2(dx, dx, mul2(dy, dy));
                    const bool acc0 = me0 && (Nf.x > 0.f), acc1 = me1 && (Nf.y > 0.f);
                    if (COUNT) {
                        n_tst += (me0 ? 1u : 0u) + (me1 ? 1u : 0u);
                        n_acc += (acc0 ? 1u : 0u) + (acc1 ? 1u : 0u);
                        count_level(s_lv[lc], me0, me1, acc0, acc1, lane);
                    }
                    const float2 w1 = add2(bc2(1.0f), d2);
                    const float2 q = make_float2(rcp1(w1.x), rcp1(w1.y));
                    const float2 Nq = mul2(make_float2(acc0 ? Nf.x : 0.0f, acc1 ? Nf.y : 0.0f), q);
                    zs = add2(zs, Nq);
                    const float2 Nq2 = mul2(Nq, q);
                    fx = fma2(Nq2, dx, fx);
                    fy = fma2(Nq2, dy, fy);
                }
            } else {
                const float Tl = s_T[lc];
                // a point's own cell: opened by the criterion itself when theta < 1
                // (the point and the centre of mass lie in the cell, so d <= r_c <
                // r_c / theta); tested explicitly otherwise
                const int sh = 2 * (L - lc);
                const uint32_t mine0 = OWN ? mi0 >> sh : 0xffffffffu, mine1 = OWN ? mi1 >> sh : 0xffffffffu;
                // room for the (at most four) entries this node may push
                if (sp + 4 > stk_lim) {
                    overflow = true;
                    break;
                }
#pragma unroll
                for (int ch = 0; ch < 4; ch++) {
                    const float N = Nc[ch];
                    if (N == 0.f) continue;
                    const uint32_t mc = m0 + ch;
                    const float4 r = rr[ch];
                    float2 dx, dy;
                    cell_offset2<CENTRE>(r, zhx, zlx, zhy, zly, dx, dy);
                    dx = mul2(dx, sf0);
                    dy = mul2(dy, sf1);
                    const float2 d2 = fma2(dx, dx, mul2(dy, dy));
                    const bool far0 = (d2.x > Tl) && (!OWN || mine0 != mc);
                    const bool far1 = (d2.y > Tl) && (!OWN || mine1 != mc);
                    const bool acc0 = me0 && far0, acc1 = me1 && far1;
                    if (COUNT) {
                        n_tst += (me0 ? 1u : 0u) + (me1 ? 1u : 0u);
                        n_acc += (acc0 ? 1u : 0u) + (acc1 ? 1u : 0u);
                        count_level(s_lv[lc], me0, me1, acc0, acc1, lane);
                    }
                    const float2 w1 = add2(bc2(1.0f), d2);
                    const float2 q = make_float2(rcp1(w1.x), rcp1(w1.y));
                    const float2 Nq = mul2(make_float2(acc0 ? N : 0.0f, acc1 ? N : 0.0f), q);
                    zs = add2(zs, Nq);
                    const float2 Nq2 = mul2(Nq, q);
                    fx = fma2(Nq2, dx, fx);
                    fy = fma2(Nq2, dy, fy);
                    const unsigned ob0 = __ballot_sync(0xffffffffu, me0 && !far0);
                    const unsigned ob1 = __ballot_sync(0xffffffffu, me1 && !far1);
                    // written in any case above the top; kept if some point opens it
                    if (lane == 0) stk[sp] = TravEntry{((uint32_t)lc << 28) | mc, ob0, ob1, 0u};
                    sp += (ob0 | ob1) != 0u;
                }
            }
            __syncwarp();
            if (overflow) break;
        }
        if (valid0) {
            Frep[i0] = make_float2(fx.x, fy.x);
            Zi[i0] = zs.x;
        }
        if (valid1) {
            Frep[i1] = make_float2(fx.y, fy.y);
            Zi[i1] = zs.y;
        }
        if (overflow && lane == 0) atomicOr(&sc->err, (unsigned)PXSNE_DEVERR_STACK);
        __syncwarp();
    }
    // every warp has taken its last chunk: the last one out resets the counter
    // for the next launch
    if (lane == 0 && atomicAdd(&sc->trav_done, 1u) == gridDim.x * kTravWarps - 1u) {
        sc->trav_next = 0u;
        sc->trav_done = 0u;
    }
    if (COUNT) {
        __syncthreads();
        if (threadIdx.x < (L + 1) * 3) {
            const int l = threadIdx.x / 3, q = threadIdx.x % 3;
            if (s_lv[l][q]) atomicAdd(&sc->lvl[l][q], s_lv[l][q]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            n_acc += __shfl_xor_sync(0xffffffffu, n_acc, o);
            n_tst += __shfl_xor_sync(0xffffffffu, n_tst, o);
        }
        if (lane == 0) {
            atomicAdd(&sc->n_accept, (u64)n_acc);
            atomicAdd(&sc->n_test, (u64)n_tst);
            atomicAdd(&sc->n_steps, (u64)n_stp);
            atomicAdd(&sc->n_nodes, (u64)n_nod);
        }
    }
}

// The attraction as its own kernel: one warp per row, the warps of a small
// persistent grid taking the rows kAttRows at a time until none are left, so
// that it runs beside the traversal on the SMs' spare registers.
constexpr int kAttRows = 4;
__global__ void __launch_bounds__(256)
    k_attract(int n, AttractArgs a, DevScalars *sc) {
    const int lane = threadIdx.x & 31;
    const float sf0 = sc->sf[0], sf1 = sc->sf[1];
    for (;;) {
        unsigned chunk = 0u;
        if (lane == 0) chunk = atomicAdd(&sc->att_next, 1u);
        chunk = __shfl_sync(0xffffffffu, chunk, 0);
        if ((int64_t)chunk * kAttRows >= n) break;
        const int r0 = (int)chunk * kAttRows, r1 = min(n, r0 + kAttRows);
        for (int row = r0; row < r1; row++) attract_row(row, lane, a, sf0, sf1);
    }
    if (lane == 0 && atomicAdd(&sc->att_done, 1u) == gridDim.x * (blockDim.x >> 5) - 1u) {
        sc->att_next = 0u;
        sc->att_done = 0u;
    }
}

// Relabelling: new label r is the point perm[r] (Morton order of the last
// tree).  Maps, padded row lengths under the new labels, and the positions.
__global__ void k_relabel_maps(int n, const uint32_t *__restrict__ perm,
                               const int64_t *__restrict__ rp, const uint2 *__restrict__ z,
                               uint32_t *__restrict__ aperm, uint32_t *__restrict__ ainv,
                               uint32_t *__restrict__ len2, uint2 *__restrict__ zp) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const uint32_t i = perm[r];
    aperm[r] = i;
    ainv[i] = (uint32_t)r;
    len2[r] = (uint32_t)(rp[i + 1] - rp[i]);
    zp[r] = z[i];
}

// Row r of the relabelled P is row aperm[r] of P with every column j replaced
// by ainv[j], entries in the same order; one warp per row, 16-byte quads (rows
// are padded to multiples of four on both sides).
__global__ void __launch_bounds__(256)
    k_relabel_rows(int n, const uint32_t *__restrict__ aperm, const uint32_t *__restrict__ ainv,
                   const int64_t *__restrict__ rp, const int4 *__restrict__ col4,
                   const float4 *__restrict__ val4, const int64_t *__restrict__ rp2,
                   int4 *__restrict__ col2, float4 *__restrict__ val2) {
    const int lane = threadIdx.x & 31;
    const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (r >= n) return;
    const uint32_t i = aperm[r];
    const int64_t q0 = rp[i] >> 2, q1 = rp[i + 1] >> 2, d0 = rp2[r] >> 2;
    for (int64_t q = q0 + lane; q < q1; q += 32) {
        const int4 c = __ldcs(col4 + q);
        const float4 v = __ldcs(val4 + q);
        col2[d0 + (q - q0)] = make_int4((int)ainv[c.x], (int)ainv[c.y], (int)ainv[c.z],
                                        (int)ainv[c.w]);
        val2[d0 + (q - q0)] = v;
    }
}

// Deterministic FP64 block sum (fixed tree order) of blockDim.x values.
__device__ double block_sum_f64(double v, double *s_red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) s_red[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0) {
        const int nw = blockDim.x >> 5;
        for (int k = 0; k < nw; k++) t += s_red[k];
    }
    __syncthreads();
    return t;
}

// Z = sum_i Z_i: each block sums a fixed contiguous chunk, the last block to
// finish adds the partials in index order.
__global__ void __launch_bounds__(512)
    k_zsum(int n, const float *__restrict__ Zi, double *__restrict__ part, DevScalars *sc) {
    __shared__ double s_red[16];
    __shared__ bool s_last;
    const int chunk = (n + gridDim.x - 1) / gridDim.x;
    const int a = blockIdx.x * chunk, b = min(n, a + chunk);
    double v = 0.0;
    for (int k = a + threadIdx.x; k < b; k += blockDim.x) v += (double)Zi[k];
    const double t = block_sum_f64(v, s_red);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = t;
        __threadfence();
        const unsigned tk = atomicAdd(&sc->ticket, 1u);
        s_last = (tk == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double w = 0.0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x)
        w += reinterpret_cast<volatile double *>(part)[k];
    const double Z = block_sum_f64(w, s_red);
    if (threadIdx.x == 0) {
        sc->Z = Z;
        sc->ticket = 0u;
    }
}

static AttractArgs attract_args(const pxsne_ctx *c) {
    return AttractArgs{c->rp2, c->col2, c->val2, c->zp, c->aperm, c->Fattr};
}

// One wave of kTravCtasPerSm CTAs per SM (at most the four the launch bounds
// allow), fewer when the points fill fewer.
template <int CENTRE, int COUNT, bool OWN>
static void traverse_as(pxsne_ctx *c, cudaStream_t st) {
    const int n = (int)c->n;
    const int per_block = kTravWarps * 64;
    const int blocks = std::min((n + per_block - 1) / per_block, kTravCtasPerSm * std::max(c->sms, 1));
    k_bh_traverse<CENTRE, COUNT, OWN><<<blocks, kTravWarps * 32, 0, st>>>(
        n, c->L, c->z, c->perm, c->rec, c->recn, c->sc, c->Frep, c->Zi);
}

static cudaError_t traverse(pxsne_ctx *c, cudaStream_t st, bool count) {
    // the own-cell test is redundant below theta = 1 (with a margin for the
    // rounding of d^2)
    const bool own = c->p.theta >= 0.999f;
    if (c->p.centre_mode == 0) {
        if (count) own ? traverse_as<0, 1, true>(c, st) : traverse_as<0, 1, false>(c, st);
        else own ? traverse_as<0, 0, true>(c, st) : traverse_as<0, 0, false>(c, st);
    } else {
        if (count) own ? traverse_as<1, 1, true>(c, st) : traverse_as<1, 1, false>(c, st);
        else own ? traverse_as<1, 0, true>(c, st) : traverse_as<1, 0, false>(c, st);
    }
    return cudaGetLastError();
}

cudaError_t launch_attract(pxsne_ctx *c, cudaStream_t st) {
    const int n = (int)c->n;
    const int need = (int)((int64_t(n) + 8 * kAttRows - 1) / (8 * kAttRows));
    const int blocks = std::min(need, kAttCtasPerSm * std::max(c->sms, 1));
    k_attract<<<blocks, 256, 0, st>>>(n, attract_args(c), c->sc);
    return cudaGetLastError();
}

static cudaError_t zsum(pxsne_ctx *c, cudaStream_t st) {
    k_zsum<<<c->zblocks, 512, 0, st>>>((int)c->n, c->Zi, c->zpart, c->sc);
    return cudaGetLastError();
}

cudaError_t launch_zsum(pxsne_ctx *c) { return zsum(c, c->stream); }

cudaError_t launch_relabel(pxsne_ctx *c, cudaStream_t st) {
    const int n = (int)c->n;
    k_relabel_maps<<<(n + 255) / 256, 256, 0, st>>>(n, c->perm, c->rp, c->z, c->aperm, c->ainv,
                                                     c->rl2, c->zp);
    cudaError_t e = cudaGetLastError();
    if (e) return e;
    if ((e = scan_u32_to_i64(c->rl2, n, c->rp2, st))) return e;
    const unsigned blocks = (unsigned)(((int64_t)n * 32 + 255) / 256);
    k_relabel_rows<<<blocks, 256, 0, st>>>(n, c->aperm, c->ainv, c->rp,
                                           reinterpret_cast<const int4 *>(c->col),
                                           reinterpret_cast<const float4 *>(c->val), c->rp2,
                                           reinterpret_cast<int4 *>(c->col2),
                                           reinterpret_cast<float4 *>(c->val2));
    return cudaGetLastError();
}

// The traversal of the current tree again, with the work counters (the
// tree's snap kernel reset them); Frep and Zi are rewritten with the same
// values.
cudaError_t launch_count_traversal(pxsne_ctx *c) { return traverse(c, c->stream, true); }

__global__ void k_accumulate_counters(DevScalars *sc) {
    sc->tot[0] += sc->n_accept;
    sc->tot[1] += sc->n_test;
    sc->tot[2] += sc->n_steps;
    sc->tot[3] += sc->n_nodes;
}

cudaError_t launch_accumulate_counters(pxsne_ctx *c) {
    k_accumulate_counters<<<1, 1, 0, c->stream>>>(c->sc);
    return cudaGetLastError();
}

cudaError_t launch_traverse_zsum(pxsne_ctx *c) {
    cudaError_t e = traverse(c, c->stream, false);
    if (e) return e;
    return zsum(c, c->stream);
}

// Sequential forces (traversal, attraction, Z) with optional timing marks.
cudaError_t launch_forces(pxsne_ctx *c, cudaEvent_t *marks) {
    cudaStream_t st = c->stream;
    cudaError_t e;
    if (marks && (e = cudaEventRecord(marks[KG_TRAVERSE], st))) return e;
    // the initial state's traversal keeps the work counters (the level
    // counters restart with it); a timed one is the kernel of the iteration
    // itself
    if (!marks && (e = cudaMemsetAsync(c->sc->lvl, 0, sizeof(c->sc->lvl), st))) return e;
    if ((e = traverse(c, st, marks == nullptr))) return e;
    if (marks && (e = cudaEventRecord(marks[KG_ATTRACT], st))) return e;
    if ((e = launch_attract(c, st))) return e;
    if (marks && (e = cudaEventRecord(marks[KG_ZSUM], st))) return e;
    if ((e = zsum(c, st))) return e;
    if (marks && (e = cudaEventRecord(marks[KG_COUNT], st))) return e;
    return cudaSuccess;
}

// Eq. cost_func: C = sum_ij p_ij ln(p_ij Z / w_ij)
//                  = sum p (ln p - ln w) + (sum p) ln Z,
// one warp per row, FP32 terms accumulated in FP64, fixed order.
__global__ void __launch_bounds__(256)
    k_kl(int n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
         const float *__restrict__ val, const uint2 *__restrict__ z, DevScalars *sc,
         double *__restrict__ part, double *out) {
    __shared__ double s_red[8];
    __shared__ bool s_last;
    const int lane = threadIdx.x & 31;
    const int warps_total = gridDim.x * (blockDim.x >> 5);
    const float sf0 = sc->sf[0], sf1 = sc->sf[1];
    double acc = 0.0, psum = 0.0;
    for (int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < n;
         row += warps_total) {
        const uint2 zi = z[row];
        for (int64_t e = rp[row] + lane; e < rp[row + 1]; e += 32) {
            const float p = val[e];
            if (!(p > 0.f)) continue;
            const uint2 zj = z[col[e]];
            const float dx = (float)((int64_t)zi.x - (int64_t)zj.x) * sf0;
            const float dy = (float)((int64_t)zi.y - (int64_t)zj.y) * sf1;
            acc += (double)(p * (logf(p) + log1pf(fmaf(dx, dx, dy * dy))));
            psum += (double)p;
        }
    }
    const double a = block_sum_f64(acc, s_red);
    const double ps = block_sum_f64(psum, s_red);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = ps;
        __threadfence();
        const unsigned tk = atomicAdd(&sc->ticket2, 1u);
        s_last = (tk == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (threadIdx.x == 0) {
        double A = 0.0, S = 0.0;
        volatile double *vp = part;
        for (int k = 0; k < (int)gridDim.x; k++) {
            A += vp[2 * k];
            S += vp[2 * k + 1];
        }
        *out = A + S * log(sc->Z);
        sc->ticket2 = 0u;
    }
}

cudaError_t launch_kl(pxsne_ctx *c, double *out_dev) {
    k_kl<<<c->klblocks, 256, 0, c->stream>>>((int)c->n, c->rp, c->col, c->val, c->z, c->sc,
                                             c->klpart, out_dev);
    return cudaGetLastError();
}

}  // namespace pxsne
