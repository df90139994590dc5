// The 3-D embedding (dim = 3): PixelSNE on a voxel grid, the extension the
// paper's introduction names beside the 2-D screen.  Each point's position is
// u32 fixed point on three axes (voxel = z >> (32 - L), 2^L voxels per axis),
// the pixel quadtree becomes a voxel octree (eight children per cell, Morton
// bits x, y, z from the least significant), and every other step is the 2-D
// method with a third coordinate:
//
//   k3_minmax, k3_map   Eq. z1/z2 per axis (FP64), the state's start
//   k3_update           Eq. grad and the gains/momentum step per coordinate
//   k3_snap             the exact-integer rescale of Sec. 4.2 per axis, the
//                       voxel snap and the leaf histogram (counts, exact sums)
//   k3_perm, k3_reduce  the counting sort of the points by voxel; the
//                       octree's upper levels with their cells' records
//   k3_traverse         Barnes-Hut (Eq. bh_criteria) on the octree, one point
//                       per lane, 32 points of consecutive voxels per warp
//   k3_attract          Eq. grad's first term over P, one warp per row
//   k3_kl, k3_centre_y  Eq. cost_func; the embedding's output
//
// The kernels follow the 2-D ones' arithmetic: exact offsets from the split
// centre of mass, FP32 forces, FP64 Z and KL.
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace pxsne {

namespace {

constexpr double kR3 = 4294967296.0;  // 2^32 ulps per axis
constexpr int kT3Warps = 8;           // warps per traversal CTA
constexpr int kT3Stack = 72;          // entries per warp; depth <= 7 L + 1 <= 64

__host__ __device__ inline int64_t off3(int l) { return ((int64_t(1) << (3 * l)) - 1) / 7; }

// Morton key of voxel (px, py, pz): bit b of x at 3b, of y at 3b + 1, of z at 3b + 2.
__device__ __forceinline__ uint32_t morton3(uint32_t px, uint32_t py, uint32_t pz) {
    uint32_t m = 0u;
#pragma unroll
    for (int b = 0; b < 10; b++)
        m |= (((px >> b) & 1u) << (3 * b)) | (((py >> b) & 1u) << (3 * b + 1)) |
             (((pz >> b) & 1u) << (3 * b + 2));
    return m;
}

// Coordinate `axis` (0, 1, 2) of a cell from its Morton index.
__device__ __forceinline__ uint32_t demorton3(uint32_t m, int axis) {
    uint32_t v = 0u;
#pragma unroll
    for (int b = 0; b < 10; b++) v |= ((m >> (3 * b + axis)) & 1u) << b;
    return v;
}

__device__ __forceinline__ float rcp3(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Ordered u32 key of a float (for the integer min/max atomics), and back.
__device__ __forceinline__ uint32_t key3(float f) {
    const uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float unkey3(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// Per-iteration scalars of the 3-D state from s (one thread).
__device__ void derive3(DevScalars *sc, float theta, int L) {
    for (int d = 0; d < 3; d++) {
        sc->inv_s3[d] = 1.0 / sc->s3[d];
        sc->sf3[d] = (float)sc->s3[d];
    }
    const double th2 = (double)theta * (double)theta;
    const double ss = sc->s3[0] * sc->s3[0] + sc->s3[1] * sc->s3[1] + sc->s3[2] * sc->s3[2];
    for (int l = 0; l <= kMaxL + 1; l++) {
        if (l > L) {
            sc->T3[l] = INFINITY;
            continue;
        }
        // the cell diagonal squared, W^2 (s0^2 + s1^2 + s2^2), W = 2^(32-l) ulps;
        // Eq. bh_criteria accepts when r_c^2 < theta^2 d^2
        const double rc2 = ldexp(1.0, 64 - 2 * l) * ss;
        sc->T3[l] = th2 > 0.0 ? (float)(rc2 / th2) : INFINITY;
    }
}

__device__ void reset_mm3(DevScalars *sc, int par) {
    for (int d = 0; d < 3; d++) {
        sc->mm3[par][d] = 0x7fffffffffffffffll;
        sc->mm3[par][3 + d] = (i64)0x8000000000000000ull;
    }
}

__global__ void k3_set_scalars(DevScalars *sc, double s0, double s1, double s2, int t, float theta,
                               int L) {
    sc->s3[0] = s0;
    sc->s3[1] = s1;
    sc->s3[2] = s2;
    sc->t = t;
    sc->Z = 0.0;
    derive3(sc, theta, L);
    reset_mm3(sc, 0);
    reset_mm3(sc, 1);
}

// ---- the start (Eq. z1/z2 per axis)
__global__ void k3_minmax(int n, const float *__restrict__ Y, uint32_t *mm, DevScalars *sc) {
    uint32_t lo[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, hi[3] = {0u, 0u, 0u};
    bool bad = false;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        for (int d = 0; d < 3; d++) {
            const float y = Y[3 * (int64_t)i + d];
            bad |= !isfinite(y);
            const uint32_t k = key3(y);
            lo[d] = min(lo[d], k);
            hi[d] = max(hi[d], k);
        }
    for (int d = 0; d < 3; d++) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo[d] = min(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
            hi[d] = max(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
        }
    }
    if ((threadIdx.x & 31) == 0)
        for (int d = 0; d < 3; d++) {
            atomicMin(&mm[d], lo[d]);
            atomicMax(&mm[3 + d], hi[d]);
        }
    if (bad) atomicOr(&sc->err, (unsigned)PXSNE_DEVERR_NONFINITE);
}

__global__ void k3_map(int n, int L, float theta, const float *__restrict__ Y,
                       const uint32_t *__restrict__ mm, uint4 *__restrict__ z,
                       float4 *__restrict__ u, float4 *__restrict__ gains, DevScalars *sc) {
    double mn[3], rg[3];
    for (int d = 0; d < 3; d++) {
        mn[d] = (double)unkey3(mm[d]);
        rg[d] = (double)unkey3(mm[3 + d]) - mn[d];
    }
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        for (int d = 0; d < 3; d++) sc->s3[d] = rg[d] > 0.0 ? rg[d] / kR3 : 1.0 / kR3;
        derive3(sc, theta, L);
        sc->t = 0;
        sc->Z = 0.0;
        reset_mm3(sc, 0);
        reset_mm3(sc, 1);
    }
    if (i >= n) return;
    uint32_t q3[3] = {0u, 0u, 0u};
    for (int d = 0; d < 3; d++) {
        if (!(rg[d] > 0.0)) continue;
        const double q = floor(((double)Y[3 * (int64_t)i + d] - mn[d]) * kR3 / rg[d]);
        q3[d] = q >= kR3 - 1.0 ? 0xffffffffu : (uint32_t)q;
    }
    z[i] = make_uint4(q3[0], q3[1], q3[2], 0u);
    u[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    gains[i] = make_float4(1.f, 1.f, 1.f, 0.f);
}

// ---- the gradient step per coordinate, and the extremes of zhat per axis
__global__ void __launch_bounds__(256)
    k3_update(int n, UpdateParams p, const uint4 *__restrict__ z, const float4 *__restrict__ Frep,
              const float4 *__restrict__ Fattr, float4 *__restrict__ u, float4 *__restrict__ gains,
              long long *__restrict__ zhat, DevScalars *sc) {
    __shared__ i64 s_mm[6][8];
    const int t = sc->t;
    const float alpha = t < p.exag_iters ? p.exag : 1.0f;
    const float mu = t < p.mom_switch ? p.mom0 : p.mom1;
    // 1 / Z once per CTA (an FP64 division)
    __shared__ float s_invZ;
    if (threadIdx.x == 0) {
        const double Z = sc->Z;
        s_invZ = Z > 0.0 ? (float)(1.0 / Z) : 0.0f;
    }
    __syncthreads();
    const float invZ = s_invZ;
    const double is0 = sc->inv_s3[0], is1 = sc->inv_s3[1], is2 = sc->inv_s3[2];
    i64 lo[3], hi[3];
    for (int d = 0; d < 3; d++) {
        lo[d] = 0x7fffffffffffffffll;
        hi[d] = (i64)0x8000000000000000ull;
    }
    unsigned err = 0u;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float4 fr = Frep[i], fa = Fattr[i];
        float4 uu = u[i], gg = gains[i];
        const uint4 zz = z[i];
        i64 zh[3];
        zh[0] = step1(fa.x, fr.x, alpha, invZ, mu, p, uu.x, gg.x, zz.x, is0, err);
        zh[1] = step1(fa.y, fr.y, alpha, invZ, mu, p, uu.y, gg.y, zz.y, is1, err);
        zh[2] = step1(fa.z, fr.z, alpha, invZ, mu, p, uu.z, gg.z, zz.z, is2, err);
        u[i] = uu;
        gains[i] = gg;
        for (int d = 0; d < 3; d++) {
            zhat[3 * (int64_t)i + d] = zh[d];
            lo[d] = min(lo[d], zh[d]);
            hi[d] = max(hi[d], zh[d]);
        }
    }
    for (int d = 0; d < 3; d++) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo[d] = min(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
            hi[d] = max(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
        }
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0)
        for (int d = 0; d < 3; d++) {
            s_mm[d][w] = lo[d];
            s_mm[3 + d][w] = hi[d];
        }
    if (err) atomicOr(&sc->err, err);
    __syncthreads();
    if (threadIdx.x < 6) {
        const int k = threadIdx.x;
        const int nw = blockDim.x >> 5;
        i64 v = s_mm[k][0];
        for (int q = 1; q < nw; q++) v = k < 3 ? min(v, s_mm[k][q]) : max(v, s_mm[k][q]);
        long long *dst = reinterpret_cast<long long *>(&sc->mm3[t & 1][k]);
        if (k < 3) atomicMin(dst, (long long)v);
        else atomicMax(dst, (long long)v);
    }
}

// ---- the rescale (Sec. 4.2, exact integers, R = 2^32 per axis), the voxel
// snap and the leaf histogram; the rank of each point inside its voxel is the
// count before it (the order inside a voxel enters no result)
__global__ void k3_snap(int n, int L, int rescale, float theta, const long long *__restrict__ zhat,
                        uint4 *__restrict__ z, uint32_t *__restrict__ rank,
                        uint32_t *__restrict__ cnt, u64 *__restrict__ sx, u64 *__restrict__ sy,
                        u64 *__restrict__ sz, DevScalars *sc) {
    const int F = 32 - L;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t zv[3];
    if (rescale) {
        const int par = sc->t & 1;
        i64 mn[3];
        u64 g[3];
        double q[3];
        __shared__ double s_q[3];
        for (int d = 0; d < 3; d++) {
            mn[d] = sc->mm3[par][d];
            g[d] = (u64)(sc->mm3[par][3 + d] - mn[d]) + 1ull;
        }
        // one FP64 division per axis and CTA (the same for every point)
        if (threadIdx.x < 3) s_q[threadIdx.x] = kR3 / (double)g[threadIdx.x];
        __syncthreads();
        for (int d = 0; d < 3; d++) q[d] = s_q[d];
        if (i == 0) {
            // Eq. beta_scaling carried as s_d <- (s_d * gamma_d) / 2^32
            for (int d = 0; d < 3; d++) sc->s3[d] = (sc->s3[d] * (double)g[d]) / kR3;
            derive3(sc, theta, L);
            reset_mm3(sc, par ^ 1);
        }
        if (i >= n) return;
        for (int d = 0; d < 3; d++)
            zv[d] = rescale_exact((u64)(zhat[3 * (int64_t)i + d] - mn[d]), g[d], q[d],
                                  u64(1) << 32);
        z[i] = make_uint4(zv[0], zv[1], zv[2], 0u);
    } else {
        if (i >= n) return;
        const uint4 v = z[i];
        zv[0] = v.x;
        zv[1] = v.y;
        zv[2] = v.z;
    }
    const uint32_t m = morton3(zv[0] >> F, zv[1] >> F, zv[2] >> F);
    rank[i] = atomicAdd(&cnt[m], 1u);
    atomicAdd(&sx[m], (u64)zv[0]);
    atomicAdd(&sy[m], (u64)zv[1]);
    atomicAdd(&sz[m], (u64)zv[2]);
}

// Record of cell at (level l, Morton c): {c_hi x, y, z, N} and {c_lo x, y,
// z, 0}, the centre of mass split at bit 16 as in 2-D (record_axis); zeros
// for an empty cell.
__device__ __forceinline__ void put_record3(int l, int64_t c, int64_t at, uint32_t N, u64 X, u64 Y,
                                            u64 Zs, float4 *__restrict__ ra,
                                            float4 *__restrict__ rb) {
    if (N == 0u) {
        ra[at] = make_float4(0.f, 0.f, 0.f, 0.f);
        rb[at] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    const int sh = 32 - l;
    float hx, lx, hy, ly, hz, lz;
    const uint32_t bx = l > 0 ? demorton3((uint32_t)c, 0) << sh : 0u;
    const uint32_t by = l > 0 ? demorton3((uint32_t)c, 1) << sh : 0u;
    const uint32_t bz = l > 0 ? demorton3((uint32_t)c, 2) << sh : 0u;
    record_axis(N, X, bx, sh, hx, lx);
    record_axis(N, Y, by, sh, hy, ly);
    record_axis(N, Zs, bz, sh, hz, lz);
    ra[at] = make_float4(hx, hy, hz, (float)N);
    rb[at] = make_float4(lx, ly, lz, 0.f);
}

// Cells of level l from their eight children at level l + 1: one thread per
// child (coalesced), which writes the child's record (and, clear = the
// children are the leaves, sets an occupied leaf back to zero once read, so
// the next histogram starts from zeros without a memset of every leaf); the
// eight threads of a parent add up by shuffles.  At l = 0 the root's own
// record is written too.
__global__ void k3_reduce(int l, int clear, uint32_t *cnt, u64 *sx, u64 *sy, u64 *sz,
                          float4 *__restrict__ ra, float4 *__restrict__ rb) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;  // child at level l + 1
    const bool in = k < (int64_t(1) << (3 * (l + 1)));
    const int64_t at = off3(l + 1) + k;
    uint32_t N = 0u;
    u64 X = 0ull, Y = 0ull, Zs = 0ull;
    if (in) {
        N = cnt[at];
        X = sx[at];
        Y = sy[at];
        Zs = sz[at];
        put_record3(l + 1, k, at, N, X, Y, Zs, ra, rb);
        if (clear && N != 0u) {
            cnt[at] = 0u;
            sx[at] = 0ull;
            sy[at] = 0ull;
            sz[at] = 0ull;
        }
    }
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
        N += __shfl_xor_sync(0xffffffffu, N, o);
        X += __shfl_xor_sync(0xffffffffu, X, o);
        Y += __shfl_xor_sync(0xffffffffu, Y, o);
        Zs += __shfl_xor_sync(0xffffffffu, Zs, o);
    }
    if (in && (k & 7) == 0) {
        const int64_t c = k >> 3, me = off3(l) + c;
        cnt[me] = N;
        sx[me] = X;
        sy[me] = Y;
        sz[me] = Zs;
        if (l == 0) put_record3(0, 0, me, N, X, Y, Zs, ra, rb);
    }
}

// the counting sort by voxel: perm[start of the voxel + rank] = i; the
// iteration counter advances here for an iteration
__global__ void k3_perm(int n, int L, const uint4 *__restrict__ z, const uint32_t *__restrict__ rank,
                        const int64_t *__restrict__ vstart, uint32_t *__restrict__ perm,
                        DevScalars *sc, int bump_t) {
    const int F = 32 - L;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (bump_t && i == 0) sc->t += 1;
    if (i >= n) return;
    const uint4 v = z[i];
    const uint32_t m = morton3(v.x >> F, v.y >> F, v.z >> F);
    const int64_t pos = vstart[m] + rank[i];
    if (pos >= 0 && pos < n) perm[pos] = (uint32_t)i;
    else atomicOr(&sc->err, (unsigned)PXSNE_DEVERR_STACK);
}

// ---- Barnes-Hut on the octree.  A warp takes 32 points consecutive in voxel
// order, one per lane, and walks the octree depth-first; each stack entry is a
// node with the mask of the lanes whose point opens it, so every point sees
// exactly the cells its own depth-first search would, in the tree's order.
// Children at the voxel level are always accepted (bounded depth) except a
// point's own voxel, used without the point itself; above it Eq. bh_criteria
// decides and the cell holding a point is opened.
struct __align__(8) T3Entry {
    uint32_t node, mask;  // (level << 27) | Morton index; lanes that opened it
};

__global__ void __launch_bounds__(kT3Warps * 32)
    k3_traverse(int n, int L, const uint4 *__restrict__ z, const uint32_t *__restrict__ perm,
                const float4 *__restrict__ ra, const float4 *__restrict__ rb, DevScalars *sc,
                float4 *__restrict__ Frep, float *__restrict__ Zi) {
    __shared__ T3Entry s_stk[kT3Warps][kT3Stack];
    __shared__ float s_T[kMaxL + 2];
    __shared__ int64_t s_off[kMaxL + 2];
    if (threadIdx.x < kMaxL + 2) {
        s_T[threadIdx.x] = sc->T3[threadIdx.x];
        s_off[threadIdx.x] = threadIdx.x <= L ? off3(threadIdx.x) : 0;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int idx = (blockIdx.x * kT3Warps + w) * 32 + lane;
    const bool valid = idx < n;
    const unsigned act = __ballot_sync(0xffffffffu, valid);
    if (act == 0u) return;
    const int F = 32 - L;
    const uint32_t i = valid ? perm[idx] : 0u;
    const uint4 zi = z[i];
    const uint32_t mi = morton3(zi.x >> F, zi.y >> F, zi.z >> F);
    const float hx = (float)(zi.x & 0xffff0000u), lx = (float)(zi.x & 0xffffu);
    const float hy = (float)(zi.y & 0xffff0000u), ly = (float)(zi.y & 0xffffu);
    const float hz = (float)(zi.z & 0xffff0000u), lz = (float)(zi.z & 0xffffu);
    const float s0 = sc->sf3[0], s1 = sc->sf3[1], s2 = sc->sf3[2];
    float fx = 0.f, fy = 0.f, fz = 0.f, zs = 0.f;
    T3Entry *stk = s_stk[w];
    if (lane == 0) stk[0] = T3Entry{0u, act};
    int sp = 1;
    __syncwarp();
    bool overflow = false;
    while (sp > 0) {
        sp--;
        T3Entry top = stk[sp];
        __syncwarp();
        top.node = __shfl_sync(0xffffffffu, top.node, 0);
        top.mask = __shfl_sync(0xffffffffu, top.mask, 0);
        const int lc = (int)(top.node >> 27) + 1;
        const uint32_t m0 = (top.node & 0x07ffffffu) << 3;
        const int64_t at = s_off[lc] + m0;
        const bool me = (top.mask >> lane) & 1u;
        // the eight children's first record halves (with the counts) are
        // requested together, one latency per node; the second halves are
        // read per child (an empty cell's is read and not used)
        float4 rpre[8];
#pragma unroll
        for (int ch = 0; ch < 8; ch++) rpre[ch] = __ldg(ra + at + ch);
        if (lc == L) {
#pragma unroll
            for (int ch = 0; ch < 8; ch++) {
                const float4 r = rpre[ch];
                const float4 q4 = __ldg(rb + at + ch);
                const float N = r.w;
                if (N == 0.f) continue;
                float dx = (hx - r.x) + (lx - q4.x);
                float dy = (hy - r.y) + (ly - q4.y);
                float dz = (hz - r.z) + (lz - q4.z);
                const bool own = me && (mi == m0 + (uint32_t)ch);
                float Nf = N;
                if (own) {  // own voxel: take the point out
                    Nf = N - 1.0f;
                    if (N > 1.0f) {
                        const float k = N / Nf;
                        dx *= k;
                        dy *= k;
                        dz *= k;
                    }
                }
                dx *= s0;
                dy *= s1;
                dz *= s2;
                const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                const bool acc = me && (Nf > 0.f);
                const float q = rcp3(1.0f + d2);
                const float Nq = (acc ? Nf : 0.0f) * q;
                zs += Nq;
                const float Nq2 = Nq * q;
                fx = fmaf(Nq2, dx, fx);
                fy = fmaf(Nq2, dy, fy);
                fz = fmaf(Nq2, dz, fz);
            }
        } else {
            const float Tl = s_T[lc];
            const uint32_t mine = mi >> (3 * (L - lc));  // the point's own cell at this level
            if (sp + 8 > kT3Stack) {
                overflow = true;
                break;
            }
#pragma unroll
            for (int ch = 0; ch < 8; ch++) {
                const float4 r = rpre[ch];
                const float4 q4 = __ldg(rb + at + ch);
                const float N = r.w;
                if (N == 0.f) continue;
                const uint32_t mc = m0 + (uint32_t)ch;
                const float dx = ((hx - r.x) + (lx - q4.x)) * s0;
                const float dy = ((hy - r.y) + (ly - q4.y)) * s1;
                const float dz = ((hz - r.z) + (lz - q4.z)) * s2;
                const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                const bool far = (d2 > Tl) && (mine != mc);
                const bool acc = me && far;
                const float q = rcp3(1.0f + d2);
                const float Nq = (acc ? N : 0.0f) * q;
                zs += Nq;
                const float Nq2 = Nq * q;
                fx = fmaf(Nq2, dx, fx);
                fy = fmaf(Nq2, dy, fy);
                fz = fmaf(Nq2, dz, fz);
                const unsigned ob = __ballot_sync(0xffffffffu, me && !far);
                if (lane == 0) stk[sp] = T3Entry{((uint32_t)lc << 27) | mc, ob};
                sp += ob != 0u;
            }
        }
        __syncwarp();
        if (overflow) break;
    }
    if (valid) {
        Frep[i] = make_float4(fx, fy, fz, 0.f);
        Zi[i] = zs;
    }
    if (overflow && lane == 0) atomicOr(&sc->err, (unsigned)PXSNE_DEVERR_STACK);
}

// ---- Eq. grad's first term, one warp per row of P (rows padded with zero
// entries that point at the row itself); z_i - z_j exact in float from the
// 16-bit halves, one rounding
__global__ void __launch_bounds__(256)
    k3_attract(int n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
               const float *__restrict__ val, const uint4 *__restrict__ z,
               const DevScalars *__restrict__ sc, float4 *__restrict__ Fattr) {
    const int lane = threadIdx.x & 31;
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (row >= n) return;
    const float s0 = sc->sf3[0], s1 = sc->sf3[1], s2 = sc->sf3[2];
    const uint4 zi = z[row];
    const float xh = (float)(zi.x & 0xffff0000u), xl = (float)(zi.x & 0xffffu);
    const float yh = (float)(zi.y & 0xffff0000u), yl = (float)(zi.y & 0xffffu);
    const float zh = (float)(zi.z & 0xffff0000u), zl = (float)(zi.z & 0xffffu);
    float fx = 0.f, fy = 0.f, fz = 0.f;
    for (int64_t e = rp[row] + lane; e < rp[row + 1]; e += 32) {
        const int32_t j = __ldcs(col + e);
        const float p = __ldcs(val + e);
        const uint4 zj = z[j];
        const float dx =
            ((xh - (float)(zj.x & 0xffff0000u)) + (xl - (float)(zj.x & 0xffffu))) * s0;
        const float dy =
            ((yh - (float)(zj.y & 0xffff0000u)) + (yl - (float)(zj.y & 0xffffu))) * s1;
        const float dz =
            ((zh - (float)(zj.z & 0xffff0000u)) + (zl - (float)(zj.z & 0xffffu))) * s2;
        const float wgt = __fdividef(1.0f, 1.0f + fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
        const float pw = p * wgt;
        fx = fmaf(pw, dx, fx);
        fy = fmaf(pw, dy, fy);
        fz = fmaf(pw, dz, fz);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        fx += __shfl_xor_sync(0xffffffffu, fx, o);
        fy += __shfl_xor_sync(0xffffffffu, fy, o);
        fz += __shfl_xor_sync(0xffffffffu, fz, o);
    }
    if (lane == 0) Fattr[row] = make_float4(fx, fy, fz, 0.f);
}

// ---- Eq. cost_func: sum p (ln p + ln(1 + d^2)) + (sum p) ln Z, FP32 terms
// accumulated in FP64 in a fixed order, the last block adding the partials
__device__ double block_sum3(double v, double *s_red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) s_red[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) t += s_red[k];
    __syncthreads();
    return t;
}

__global__ void __launch_bounds__(256)
    k3_kl(int n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
          const float *__restrict__ val, const uint4 *__restrict__ z, DevScalars *sc,
          double *__restrict__ part, double *out) {
    __shared__ double s_red[8];
    __shared__ bool s_last;
    const int lane = threadIdx.x & 31;
    const int warps_total = gridDim.x * (blockDim.x >> 5);
    const float s0 = sc->sf3[0], s1 = sc->sf3[1], s2 = sc->sf3[2];
    double acc = 0.0, psum = 0.0;
    for (int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < n;
         row += warps_total) {
        const uint4 zi = z[row];
        for (int64_t e = rp[row] + lane; e < rp[row + 1]; e += 32) {
            const float p = val[e];
            if (!(p > 0.f)) continue;
            const uint4 zj = z[col[e]];
            const float dx = (float)((int64_t)zi.x - (int64_t)zj.x) * s0;
            const float dy = (float)((int64_t)zi.y - (int64_t)zj.y) * s1;
            const float dz = (float)((int64_t)zi.z - (int64_t)zj.z) * s2;
            acc += (double)(p * (logf(p) + log1pf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)))));
            psum += (double)p;
        }
    }
    const double a = block_sum3(acc, s_red);
    const double ps = block_sum3(psum, s_red);
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

// ---- output: y = s z minus the per-axis mean (FP64 sums), voxels z >> F
__global__ void k3_sum_y(int n, const uint4 *__restrict__ z, const DevScalars *sc, double *sums) {
    double a[3] = {0.0, 0.0, 0.0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint4 v = z[i];
        a[0] += (double)v.x * sc->s3[0];
        a[1] += (double)v.y * sc->s3[1];
        a[2] += (double)v.z * sc->s3[2];
    }
    for (int d = 0; d < 3; d++) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a[d] += __shfl_xor_sync(0xffffffffu, a[d], o);
        if ((threadIdx.x & 31) == 0) atomicAdd(&sums[d], a[d]);
    }
}

__global__ void k3_write_y(int n, int L, const uint4 *__restrict__ z, const DevScalars *sc,
                           const double *sums, float *Y, int32_t *pix) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 v = z[i];
    const uint32_t zz[3] = {v.x, v.y, v.z};
    for (int d = 0; d < 3; d++) {
        if (Y) Y[3 * (int64_t)i + d] = (float)((double)zz[d] * sc->s3[d] - sums[d] / (double)n);
        if (pix) pix[3 * (int64_t)i + d] = (int32_t)(zz[d] >> (32 - L));
    }
}

// The leaf histogram of the current state, for inspection (the iteration's
// own is cleared by the first reduction once read).
__global__ void k3_leaf_hist(int n, int L, const uint4 *__restrict__ z, uint32_t *cnt, u64 *sx,
                             u64 *sy, u64 *sz) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int F = 32 - L;
    const uint4 v = z[i];
    const uint32_t m = morton3(v.x >> F, v.y >> F, v.z >> F);
    atomicAdd(&cnt[m], 1u);
    atomicAdd(&sx[m], (u64)v.x);
    atomicAdd(&sy[m], (u64)v.y);
    atomicAdd(&sz[m], (u64)v.z);
}

__global__ void k3_morton(int n, int L, const uint4 *__restrict__ z, uint32_t *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 v = z[i];
    out[i] = morton3(v.x >> (32 - L), v.y >> (32 - L), v.z >> (32 - L));
}

__global__ void k3_fill(int n, float4 *p, float4 v) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

}  // namespace

cudaError_t launch_fill3(pxsne_ctx *c, float4 *p, float x, float y, float z) {
    const int n = (int)c->n;
    k3_fill<<<(n + 255) / 256, 256, 0, c->stream>>>(n, p, make_float4(x, y, z, 0.f));
    return cudaGetLastError();
}

int64_t cells3(int L) { return off3(L + 1); }
int64_t level_offset3(int l) { return off3(l); }

cudaError_t launch_leaf_hist3(pxsne_ctx *c, uint32_t *cnt, u64 *sums) {
    const int n = (int)c->n;
    const size_t leaves = size_t(1) << (3 * c->L);
    cudaError_t e;
    if ((e = cudaMemsetAsync(cnt, 0, leaves * 4, c->stream))) return e;
    if ((e = cudaMemsetAsync(sums, 0, 3 * leaves * 8, c->stream))) return e;
    k3_leaf_hist<<<(n + 255) / 256, 256, 0, c->stream>>>(n, c->L, c->z3, cnt, sums, sums + leaves,
                                                         sums + 2 * leaves);
    return cudaGetLastError();
}

cudaError_t launch_morton3(pxsne_ctx *c, uint32_t *out) {
    const int n = (int)c->n;
    k3_morton<<<(n + 255) / 256, 256, 0, c->stream>>>(n, c->L, c->z3, out);
    return cudaGetLastError();
}

template <class T>
static cudaError_t alloc_n(T **p, size_t count) {
    if (*p) {
        cudaFree(*p);
        *p = nullptr;
    }
    return cudaMalloc(reinterpret_cast<void **>(p), (count ? count : 1) * sizeof(T));
}

template <class T>
static void free_p(T *&p) {
    if (p) cudaFree(p);
    p = nullptr;
}

cudaError_t alloc3(pxsne_ctx *c) {
    const size_t n = (size_t)c->n;
    const int64_t cells = cells3(c->L);
    cudaError_t e;
    if ((e = alloc_n(&c->z3, n))) return e;
    if ((e = alloc_n(&c->zhat3, 3 * n))) return e;
    if ((e = alloc_n(&c->u3, n))) return e;
    if ((e = alloc_n(&c->gains3, n))) return e;
    if ((e = alloc_n(&c->Frep3, n))) return e;
    if ((e = alloc_n(&c->Fattr3, n))) return e;
    if ((e = alloc_n(&c->cnt3, (size_t)cells))) return e;
    if ((e = alloc_n(&c->sum3, 3 * (size_t)cells))) return e;
    if ((e = alloc_n(&c->rec3a, (size_t)cells))) return e;
    if ((e = alloc_n(&c->rec3b, (size_t)cells))) return e;
    if ((e = alloc_n(&c->vstart3, (size_t)(int64_t(1) << (3 * c->L)) + 1))) return e;
    // the leaf histogram starts from zeros; the first reduction clears what it read
    if ((e = cudaMemsetAsync(c->cnt3, 0, (size_t)cells * sizeof(uint32_t), c->stream))) return e;
    if ((e = cudaMemsetAsync(c->sum3, 0, 3 * (size_t)cells * sizeof(u64), c->stream))) return e;
    c->dev_bytes += (int64_t)n * (16 + 24 + 16 * 4) + cells * (4 + 24 + 32) +
                    ((int64_t(1) << (3 * c->L)) + 1) * 8;
    return cudaSuccess;
}

void free3(pxsne_ctx *c) {
    free_p(c->z3);
    free_p(c->zhat3);
    free_p(c->u3);
    free_p(c->gains3);
    free_p(c->Frep3);
    free_p(c->Fattr3);
    free_p(c->cnt3);
    free_p(c->sum3);
    free_p(c->rec3a);
    free_p(c->rec3b);
    free_p(c->vstart3);
}

cudaError_t launch_set_scalars3(pxsne_ctx *c, const double *s, int t) {
    k3_set_scalars<<<1, 1, 0, c->stream>>>(c->sc, s[0], s[1], s[2], t, c->p.theta, c->L);
    return cudaGetLastError();
}

cudaError_t launch_init3(pxsne_ctx *c, const float *Y0dev, double *scratch) {
    cudaStream_t st = c->stream;
    const int n = (int)c->n;
    uint32_t *mm = reinterpret_cast<uint32_t *>(scratch);
    const uint32_t init[6] = {0xffffffffu, 0xffffffffu, 0xffffffffu, 0u, 0u, 0u};
    cudaError_t e;
    if ((e = cudaMemcpyAsync(mm, init, sizeof(init), cudaMemcpyHostToDevice, st))) return e;
    const int blocks = std::min((n + 255) / 256, 1184);
    k3_minmax<<<blocks > 0 ? blocks : 1, 256, 0, st>>>(n, Y0dev, mm, c->sc);
    k3_map<<<(n + 255) / 256, 256, 0, st>>>(n, c->L, c->p.theta, Y0dev, mm, c->z3, c->u3,
                                             c->gains3, c->sc);
    return cudaGetLastError();
}

// the tree of the current state (rescale: zhat -> z first, an iteration)
static cudaError_t tree3(pxsne_ctx *c, bool rescale) {
    cudaStream_t st = c->stream;
    const int L = c->L, n = (int)c->n;
    const int64_t cells = cells3(L), leaves = int64_t(1) << (3 * L);
    const int64_t lo = off3(L);
    uint32_t *cnt = c->cnt3;
    u64 *sx = c->sum3, *sy = c->sum3 + cells, *sz = c->sum3 + 2 * cells;
    cudaError_t e;
    // the leaves are zero here (set at allocation, cleared by the first
    // reduction after each histogram)
    k3_snap<<<(n + 255) / 256, 256, 0, st>>>(n, L, rescale ? 1 : 0, c->p.theta, c->zhat3, c->z3,
                                              c->rank, cnt + lo, sx + lo, sy + lo, sz + lo, c->sc);
    if ((e = cudaGetLastError())) return e;
    // the voxel order (before the leaves are cleared)
    if ((e = scan_u32_to_i64(cnt + lo, leaves, c->vstart3, st))) return e;
    k3_perm<<<(n + 255) / 256, 256, 0, st>>>(n, L, c->z3, c->rank, c->vstart3, c->perm, c->sc,
                                              rescale ? 1 : 0);
    if ((e = cudaGetLastError())) return e;
    for (int l = L - 1; l >= 0; l--) {
        const int64_t m = int64_t(1) << (3 * (l + 1));  // the children
        k3_reduce<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(l, l == L - 1 ? 1 : 0, cnt, sx, sy,
                                                               sz, c->rec3a, c->rec3b);
    }
    return cudaGetLastError();
}

static cudaError_t forces3(pxsne_ctx *c) {
    cudaStream_t st = c->stream;
    const int n = (int)c->n;
    const int per_block = kT3Warps * 32;
    k3_traverse<<<(n + per_block - 1) / per_block, per_block, 0, st>>>(
        n, c->L, c->z3, c->perm, c->rec3a, c->rec3b, c->sc, c->Frep3, c->Zi);
    cudaError_t e = cudaGetLastError();
    if (e) return e;
    k3_attract<<<(unsigned)(((int64_t)n * 32 + 255) / 256), 256, 0, st>>>(
        n, c->rp, c->col, c->val, c->z3, c->sc, c->Fattr3);
    if ((e = cudaGetLastError())) return e;
    return launch_zsum(c);
}

cudaError_t launch_prime3(pxsne_ctx *c, bool rescale) {
    cudaError_t e = tree3(c, rescale);
    if (e) return e;
    return forces3(c);
}

cudaError_t launch_iteration3(pxsne_ctx *c) {
    UpdateParams p;
    p.eta = c->p.eta;
    p.exag = c->p.exaggeration;
    p.mom0 = c->p.momentum0;
    p.mom1 = c->p.momentum1;
    p.min_gain = c->p.min_gain;
    p.exag_iters = c->p.exag_iters;
    p.mom_switch = c->p.momentum_switch;
    const int n = (int)c->n;
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = std::max(1, std::min((n + 255) / 256, 4 * (sms > 0 ? sms : 1)));
    k3_update<<<blocks, 256, 0, c->stream>>>(n, p, c->z3, c->Frep3, c->Fattr3, c->u3, c->gains3,
                                              c->zhat3, c->sc);
    cudaError_t e = cudaGetLastError();
    if (e) return e;
    return launch_prime3(c, true);
}

cudaError_t launch_kl3(pxsne_ctx *c, double *out_dev) {
    k3_kl<<<c->klblocks, 256, 0, c->stream>>>((int)c->n, c->rp, c->col, c->val, c->z3, c->sc,
                                              c->klpart, out_dev);
    return cudaGetLastError();
}

cudaError_t launch_centre_y3(pxsne_ctx *c, float *Ydev, int32_t *pixdev, double *scratch) {
    cudaStream_t st = c->stream;
    const int n = (int)c->n;
    cudaError_t e;
    if ((e = cudaMemsetAsync(scratch, 0, 3 * sizeof(double), st))) return e;
    k3_sum_y<<<std::min((n + 255) / 256, 1184), 256, 0, st>>>(n, c->z3, c->sc, scratch);
    k3_write_y<<<(n + 255) / 256, 256, 0, st>>>(n, c->L, c->z3, c->sc, scratch, Ydev, pixdev);
    return cudaGetLastError();
}

}  // namespace pxsne
