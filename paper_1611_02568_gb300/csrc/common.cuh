// Internal declarations shared by the CUDA translation units of the PixelSNE
// library (sm_103a).  Nothing here is part of the public ABI (include/pxsne.h).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <string>

#include "pxsne.h"

namespace pxsne {

typedef unsigned long long u64;
typedef long long i64;

constexpr int kMaxL = 14;           // screen up to 2^14 x 2^14 (Morton keys < 2^28)
constexpr int64_t kMaxN = 1 << 24;  // cell counts are exact floats below 2^24
constexpr int kTravWarps = 8;       // warps per CTA in the traversal
constexpr int kTravStack = 48;      // entries per warp; depth <= 3L - 2 <= 40
// Persistent grids of the forces: CTAs per SM of the traversal and of the
// attraction that runs beside it on the side stream.  The traversal alone is
// fastest at four CTAs (all of the SM's registers); at two it leaves room
// for three of the attraction's CTAs from the start, and the whole
// 1000-iteration schedule at n = 1M runs 6.6 % faster than with four.
constexpr int kTravCtasPerSm = 2;
constexpr int kAttCtasPerSm = 4;
constexpr int kPyrK = 5;            // pyramid levels reduced per CTA pass

// Scalars of the iteration that live on the device so that a captured graph
// can replay iterations without host involvement.
struct DevScalars {
    double s[2];         // y-units per ulp (s_d^2 = beta_d of Eq. beta_scaling)
    double inv_s[2];     // 1 / s_d
    float sf[2];         // s_d rounded to float
    float T[kMaxL + 2];  // BH acceptance: accept cell of level l iff d^2 > T[l]
    i64 mm[2][4];        // [t & 1] = {min_x, min_y, max_x, max_y} of zhat
    double Z;            // sum_i Z_i of the current state
    double kl_acc[2];    // KL partial results {sum p ln(p/w), sum p}
    int t;               // iteration counter
    unsigned err;        // PXSNE_DEVERR_* flags
    unsigned ticket;     // last-block-done counter of the Z reduction
    unsigned ticket2;    // same for the KL reduction
    unsigned pyr_ticket; // last-block-done counter of the pyramid's first pass
    int stack_limit;     // entries of a traversal warp's stack in use (0: all
                         // kTravStack; lowered only by pxsne_test_stack_limit)
    unsigned trav_next;  // next 64-point chunk of the traversal (0 between launches)
    unsigned trav_done;  // traversal warps finished (the last one resets both)
    unsigned att_next;   // the same two counters for the attraction's row chunks
    unsigned att_done;
    u64 n_accept;        // accepted (point, cell) pairs of the last traversal
    u64 n_test;          // (point, cell) pairs tested by the last traversal
    u64 n_steps;         // warp-level (node, non-empty child) steps of the last traversal
    u64 n_nodes;         // stack entries popped by the last traversal
    u64 tot[4];          // sums of the four counters above over a profiled run
    u64 lvl[kMaxL + 2][3];  // (tested, accepted, warp steps) by child level, summed
                            // over the counting traversals since the last reset
    u64 knn_exact;       // exact distances computed by the last neighbour search
    u64 knn_insert;      // list insertions of the last neighbour search
    u64 knn_skip;        // (query tile, candidate tile) pairs it skipped by the tile bound
    // the 3-D embedding (dim = 3): the same scalars for three axes
    double s3[3], inv_s3[3];
    float sf3[3];
    float T3[kMaxL + 2];
    i64 mm3[2][6];       // [t & 1] = {min_x, min_y, min_z, max_x, max_y, max_z} of zhat
};

// The pyramid of cell records.  Cell (l, m) (level l, Morton index m) is at
// rec_offset(l) + m of two arrays:
//   rec  float4 {c_hi_x, c_lo_x, c_hi_y, c_lo_y}: the centre of mass S_c / N_c in
//        ulps, split at bit 16 (c_hi = floor(com) with the low 16 bits cleared,
//        exact in float; c_lo = the rest, in [0, 65536]; the centre's offset in
//        its cell is one FP32 quotient, good to about 2^-23 of the cell width),
//        so that a point's offset z - com is (z_hi - c_hi) + (z_lo - c_lo)
//        with one rounding;
//   recn float N_c (exact below 2^24).
// The record of an empty cell (N_c = 0) is not written each iteration; it
// keeps an earlier value and is never read.
// rec_offset pads level 0 to four slots so that every group of four siblings
// starts on a 16-byte boundary.
__host__ __device__ inline int64_t rec_offset(int l) {
    return l == 0 ? 0 : ((int64_t(1) << (2 * l)) + 8) / 3;
}

__host__ __device__ inline int64_t level_offset(int l) {
    return ((int64_t(1) << (2 * l)) - 1) / 3;
}

__device__ __forceinline__ uint32_t spread_bits16(uint32_t x) {
    x &= 0x0000ffffu;
    x = (x | (x << 8)) & 0x00ff00ffu;
    x = (x | (x << 4)) & 0x0f0f0f0fu;
    x = (x | (x << 2)) & 0x33333333u;
    x = (x | (x << 1)) & 0x55555555u;
    return x;
}

__device__ __forceinline__ uint32_t gather_bits16(uint32_t x) {
    x &= 0x55555555u;
    x = (x | (x >> 1)) & 0x33333333u;
    x = (x | (x >> 2)) & 0x0f0f0f0fu;
    x = (x | (x >> 4)) & 0x00ff00ffu;
    x = (x | (x >> 8)) & 0x0000ffffu;
    return x;
}

// Morton key of pixel (px, py): x bits at even positions, y bits at odd ones.
__device__ __forceinline__ uint32_t morton2(uint32_t px, uint32_t py) {
    return spread_bits16(px) | (spread_bits16(py) << 1);
}

// floor(a * R / gamma) for 0 <= a < gamma < 2^61 and R <= 2^32, exactly: a
// double estimate (q = R / gamma) within one of the quotient, then a
// remainder correction in wrapping 64-bit arithmetic (the true remainder is
// within +-3 gamma).
__device__ __forceinline__ uint32_t rescale_exact(u64 a, u64 gamma, double q, u64 R) {
    u64 q0 = (u64)((double)a * q);
    if (q0 > R - 1ull) q0 = R - 1ull;
    i64 r = (i64)(a * R - q0 * gamma);
#pragma unroll 1
    for (int k = 0; k < 4 && r < 0; k++) { q0--; r += (i64)gamma; }
#pragma unroll 1
    for (int k = 0; k < 4 && (u64)r >= gamma; k++) { q0++; r -= (i64)gamma; }
    return (uint32_t)q0;
}

// One axis of a centre-of-mass record: the centre base + S_off / N of a cell
// whose lower corner is `base` (S_off = S - N base, the sum of the points'
// offsets in the cell, exact), split at bit 16 as the layout in common.cuh
// asks.  The offset is one FP32 quotient (relative error about 2^-23 of the
// cell width, a fraction of an ulp at the leaves).
__device__ __forceinline__ void record_axis(uint32_t N, u64 S, uint32_t base, int sh,
                                            float &hi, float &lo) {
    const u64 soff = S - (u64)N * base;
    float c = (float)soff / (float)N;  // in [0, 2^sh]
    c = fminf(c, 4294967040.0f);
    uint32_t q = (uint32_t)c;
    float fr = c - (float)q;
    const uint32_t wmax = sh >= 32 ? 0xffffffffu : ((1u << sh) - 1u);
    if (q > wmax) {  // rounding at the cell's far edge
        q = wmax;
        fr = 1.0f;
    }
    hi = (float)(base + (q & 0xffff0000u));
    lo = (float)(q & 0xffffu) + fr;
}

// Optimiser parameters of the update kernels (Eq. grad and BH-SNE's gains and
// momentum).
struct UpdateParams {
    float eta, exag, mom0, mom1, min_gain;
    int exag_iters, mom_switch;
};

__device__ __forceinline__ int sgnf(float x) { return (x > 0.f) - (x < 0.f); }

// Step of one coordinate; returns zhat.
__device__ __forceinline__ i64 step1(float fa, float fr, float alpha, float invZ, float mu,
                                     const UpdateParams &p, float &u, float &gain,
                                     uint32_t z, double inv_s, unsigned &err) {
    const float g = 4.0f * (alpha * fa - fr * invZ);
    float gn = (sgnf(g) != sgnf(u)) ? gain + 0.2f : gain * 0.8f;
    gn = fmaxf(gn, p.min_gain);
    gain = gn;
    u = mu * u - p.eta * gn * g;
    double st = (double)u * inv_s;
    const double lim = 288230376151711744.0;  // 2^58 ulps
    if (!(fabs(st) <= lim)) {
        err |= isfinite(st) ? (unsigned)PXSNE_DEVERR_RANGE : (unsigned)PXSNE_DEVERR_NONFINITE;
        st = isfinite(st) ? copysign(lim, st) : 0.0;
        if (!isfinite(u)) u = 0.f;
    }
    return (i64)z + __double2ll_rn(st);
}

// Extent R_d of screen axis d in ulps: r_d 2^(32 - L) (2^32 when r_d = 0,
// the square 2^L screen).
__host__ __device__ inline u64 screen_extent(int32_t r, int L) {
    return r > 0 ? (u64)r << (32 - L) : (u64(1) << 32);
}

// Derived per-iteration scalars from s (called by one thread).
__device__ inline void derive_scalars(DevScalars *sc, float theta, int L) {
    const double s0 = sc->s[0], s1 = sc->s[1];
    sc->inv_s[0] = 1.0 / s0;
    sc->inv_s[1] = 1.0 / s1;
    sc->sf[0] = (float)s0;
    sc->sf[1] = (float)s1;
    const double th2 = (double)theta * (double)theta;
    for (int l = 0; l <= kMaxL + 1; l++) {
        if (l > L) { sc->T[l] = INFINITY; continue; }
        // diagonal of a level-l cell in y-units, squared: W^2 (s0^2 + s1^2),
        // W = 2^(32-l) ulps; Eq. bh_criteria accepts when r_c^2 < theta^2 d^2
        double W2 = ldexp(1.0, 64 - 2 * l);
        double rc2 = W2 * (s0 * s0 + s1 * s1);
        sc->T[l] = th2 > 0.0 ? (float)(rc2 / th2) : INFINITY;
    }
}


}  // namespace pxsne

// Host-side context.
struct pxsne_ctx {
    pxsne_params p;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t side = nullptr;          // stream of the attraction (overlaps the traversal)
    int sms = 0;                          // streaming multiprocessors of the device
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int device = 0;
    std::string err;

    int64_t n = 0;
    int32_t D = 0;
    int64_t nnz = 0;

    // P as CSR
    // P as CSR with every row padded to a multiple of 4 entries (padding:
    // column = the row itself, value 0); rp holds the padded offsets and
    // rowlen the true row lengths
    int64_t *rp = nullptr;
    int32_t *col = nullptr;
    float *val = nullptr;
    int32_t *rowlen = nullptr;
    int64_t nnz_pad = 0;

    // neighbour lists of the last affinities call
    int32_t *knn_idx = nullptr;
    float *knn_d2 = nullptr;
    float *beta = nullptr;
    int32_t knn_k = 0;
    int knn_path = -1;  // 1: tensor-core kNN, 0: FP32 CUDA-core kNN
    int64_t knn_tiles = 0;  // row tiles of the last tensor-core search
    cudaEvent_t knn_ev[2] = {nullptr, nullptr};  // around the last search kernel
    bool knn_timed = false;

    // embedding state (data order)
    uint2 *z = nullptr;
    longlong2 *zhat = nullptr;
    float2 *u = nullptr;
    float2 *gains = nullptr;
    float2 *Frep = nullptr;
    float *Zi = nullptr;
    float2 *Fattr = nullptr;
    uint32_t *perm = nullptr;  // traversal order (Morton order of a recent state)
    uint32_t *rank = nullptr;  // rank of each point inside its pixel

    // P relabelled for the attraction: rows and columns renumbered in the
    // Morton order of a recent state (aperm: new label -> point, ainv: point
    // -> new label), refreshed every kRelabelEvery iterations; zp holds the
    // positions under the new labels (written by the snap kernel)
    int64_t *rp2 = nullptr;
    int32_t *col2 = nullptr;
    float *val2 = nullptr;
    uint32_t *aperm = nullptr, *ainv = nullptr, *rl2 = nullptr;
    uint2 *zp = nullptr;
    int since_relabel = 0;

    // tree
    int L = 0;
    uint32_t *leaf_cnt = nullptr;
    unsigned long long *leaf_sx = nullptr, *leaf_sy = nullptr;
    float4 *rec = nullptr;
    float *recn = nullptr;
    uint32_t *lvl_cnt[2] = {nullptr, nullptr};
    unsigned long long *lvl_sx[2] = {nullptr, nullptr}, *lvl_sy[2] = {nullptr, nullptr};
    uint32_t *leaf_start = nullptr;
    uint32_t *blk_off = nullptr;

    double *zpart = nullptr;
    int zblocks = 0;
    double *klpart = nullptr;
    int klblocks = 0;

    // the 3-D embedding (dim = 3): positions, velocities, gains and forces
    // per point as 4-wide vectors (the fourth lane unused), zhat as three
    // int64 per point, and the octree's per-level counts and exact sums, its
    // records {c_hi x, y, z, N} and {c_lo x, y, z, 0} per cell
    int dim = 2;
    uint4 *z3 = nullptr;
    long long *zhat3 = nullptr;
    float4 *u3 = nullptr, *gains3 = nullptr, *Frep3 = nullptr, *Fattr3 = nullptr;
    uint32_t *cnt3 = nullptr;
    unsigned long long *sum3 = nullptr;  // [3][cells]
    float4 *rec3a = nullptr, *rec3b = nullptr;
    int64_t *vstart3 = nullptr;          // exclusive scan of the voxel counts

    pxsne::DevScalars *sc = nullptr;
    bool state_ready = false;
    cudaGraphExec_t graph = nullptr;
    int64_t dev_bytes = 0;
};

// Launchers implemented in the .cu files (all enqueue on ctx->stream).
namespace pxsne {
cudaError_t launch_init_map(pxsne_ctx *c, const float *Y0dev, uint32_t *mm_scratch);
// Kernel groups of one iteration, in launch order (timing marks).
enum KernelGroup {
    KG_RELABEL = 0,  // k_relabel_maps + scan + k_relabel_rows (every kRelabelEvery iterations)
    KG_UPDATE,       // k_update
    KG_SNAP,         // leaf memsets + k_snap_hist
    KG_PYRAMID,      // k_pyr_pass x passes + k_scan1
    KG_PERM,         // k_perm_scatter
    KG_TRAVERSE,     // k_bh_traverse
    KG_ATTRACT,      // k_attract
    KG_ZSUM,         // k_zsum
    KG_COUNT
};
// marks (optional): an event is recorded on the stream before each group g
// (marks[g]) and after the last one (marks[KG_COUNT]).
cudaError_t launch_tree(pxsne_ctx *c, bool rescale, cudaEvent_t *marks = nullptr);
cudaError_t launch_forces(pxsne_ctx *c, cudaEvent_t *marks = nullptr);
// The two halves of launch_tree and of launch_forces, for the overlapped
// schedule: snap (memsets + histogram) then pyramid (passes, scan, scatter);
// attraction alone on stream `st`, then traversal + Z.
cudaError_t launch_snap(pxsne_ctx *c, bool rescale, cudaEvent_t *marks = nullptr);
cudaError_t launch_pyramid(pxsne_ctx *c, bool rescale, cudaEvent_t *marks = nullptr);
cudaError_t launch_attract(pxsne_ctx *c, cudaStream_t st);
cudaError_t launch_count_traversal(pxsne_ctx *c);
// tot[] += the counters of the last counting traversal (one thread)
cudaError_t launch_accumulate_counters(pxsne_ctx *c);
// Renumber P's rows and columns in the Morton order of the last tree (perm)
// into rp2/col2/val2 and refresh aperm, ainv and zp.
constexpr int kRelabelEvery = 100;
cudaError_t launch_relabel(pxsne_ctx *c, cudaStream_t st);
// out[0..m] = exclusive scan of in[0..m) with out[m] = the total
cudaError_t scan_u32_to_i64(const uint32_t *in, int64_t m, int64_t *out, cudaStream_t st);
cudaError_t launch_traverse_zsum(pxsne_ctx *c);
cudaError_t launch_update(pxsne_ctx *c, cudaEvent_t *marks = nullptr);
cudaError_t launch_kl(pxsne_ctx *c, double *out_dev);
cudaError_t launch_centre_y(pxsne_ctx *c, float *Ydev, int32_t *pixdev, float *scratch);
cudaError_t launch_philox_y0(pxsne_ctx *c, float *Y0dev, uint64_t seed, float sigma);
cudaError_t launch_nonfinite(pxsne_ctx *c, const float *X, int64_t m, unsigned *flag,
                             cudaStream_t st);
cudaError_t launch_knn(pxsne_ctx *c, const float *Xdev, int64_t n, int32_t D, int32_t k,
                       int32_t *idx, float *d2);
cudaError_t launch_perplexity(pxsne_ctx *c, const float *d2, int64_t n, int32_t k,
                              float perplexity, float *pcond, float *beta);
cudaError_t build_symmetric_csr(pxsne_ctx *c, const int32_t *idx, const float *pcond,
                                int64_t n, int32_t k, std::string &err);
cudaError_t launch_level_counts(pxsne_ctx *c, int level, uint32_t *cnt);
// counts and exact coordinate sums of the leaves of the current state (any may be NULL)
cudaError_t launch_leaf_hist(pxsne_ctx *c, uint32_t *cnt, u64 *sx, u64 *sy);
cudaError_t launch_morton_keys(pxsne_ctx *c, uint32_t *keys);
// One CTA waiting on an mbarrier that nothing arrives at (bounded; sets
// PXSNE_DEVERR_TIMEOUT when the polls run out).
void launch_wait_probe(pxsne_ctx *c, int polls);
cudaError_t launch_nbr_precision(pxsne_ctx *c, int k, const int32_t *knn_hd, int kh,
                                 int32_t *hits, unsigned long long *total);
// Z = sum_i Z_i (FP64, fixed order) on the main stream.
cudaError_t launch_zsum(pxsne_ctx *c);
// The 3-D embedding (dim3.cu): buffers, the start, one iteration, the tree
// and forces of the current state, KL, and the state's output.
constexpr int kMaxL3 = 9;   // voxel screen up to 2^9 per axis (Morton keys < 2^27)
int64_t cells3(int L);      // (8^(L+1) - 1) / 7
int64_t level_offset3(int l);  // (8^l - 1) / 7
// counts and exact coordinate sums (three arrays of 8^L) of the current voxels
cudaError_t launch_leaf_hist3(pxsne_ctx *c, uint32_t *cnt, u64 *sums);
cudaError_t launch_morton3(pxsne_ctx *c, uint32_t *out);
cudaError_t launch_fill3(pxsne_ctx *c, float4 *p, float x, float y, float z);
cudaError_t alloc3(pxsne_ctx *c);
void free3(pxsne_ctx *c);
cudaError_t launch_init3(pxsne_ctx *c, const float *Y0dev, double *scratch);
cudaError_t launch_iteration3(pxsne_ctx *c);
cudaError_t launch_prime3(pxsne_ctx *c, bool rescale);
cudaError_t launch_kl3(pxsne_ctx *c, double *out_dev);
cudaError_t launch_centre_y3(pxsne_ctx *c, float *Ydev, int32_t *pixdev, double *scratch);
cudaError_t launch_set_scalars3(pxsne_ctx *c, const double *s, int t);
}  // namespace pxsne
