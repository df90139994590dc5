// Learned warm start: a d -> 256 -> 256 -> 2 MLP with exact GELU, BF16 weights
// and activations as tensor-core operands, FP32 accumulation, trained with MSE
// and Adam by the kernels below.  It maps a data row x to an initial 2-D
// position, from which the plain method refines.
//
//   k_gemm<NT, EPI>  C = A B^T on the tensor cores (tcgen05, accumulator in
//                    TMEM), A [M x K] and B [N x K] BF16 row-major; fused
//                    epilogues: bias + GELU (forward), GELU' (backward), FP32
//                    atomic accumulation (weight gradients, split over K)
//   k_out_layer      y = W3 h2 + b3; with targets also the loss, dL/dy,
//                    dL/dW3, dL/db3 and dz2 = (W3^T dy) * GELU'(z2)
//   k_colsum         bias gradients
//   k_adam           Adam on the FP32 master weights, BF16 copies refreshed
#include <cuda_bf16.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <algorithm>
#include <random>
#include <string>
#include <vector>

#include "common.cuh"
#include "tc.cuh"

namespace pxsne {
namespace {

constexpr int kH = 256;          // hidden width
constexpr int kMaxBatch = 8192;  // rows per training step
constexpr int kGemmThreads = 128;
constexpr int kGemmPolls = 1 << 24;
constexpr int kSplitK = 512;     // batch rows per CTA in the weight-gradient GEMMs

typedef __nv_bfloat16 bf16;

__device__ __forceinline__ float gelu_f(float z) {
    return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f));
}
__device__ __forceinline__ float gelu_df(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) +
           z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

enum { EPI_Z_GELU = 0, EPI_DGELU = 1, EPI_ATOMIC = 2 };

struct Epi {
    int ld;              // leading dimension of the row-major outputs (= N)
    int ldT;             // leading dimension of the transposed outputs (= rows)
    int rows;            // valid rows (stores beyond are skipped)
    const float *bias;   // EPI_Z_GELU
    float *Z;            // EPI_Z_GELU: pre-activation out; EPI_DGELU: pre-activation in
    bf16 *H;             // activation / gradient out, row-major (may be null)
    bf16 *HT;            // same, transposed (may be null)
    float *acc;          // EPI_ATOMIC target
    unsigned *err;
};

// C[m0:m0+128, n0:n0+NT] = sum over this CTA's K range of A B^T.
template <int NT, int EPI>
__global__ void __launch_bounds__(kGemmThreads)
    k_gemm(int M, int N, int K, int k_split, const bf16 *__restrict__ A, int lda,
           const bf16 *__restrict__ B, int ldb, Epi ep) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t mbar[2];
    __shared__ uint32_t tslot;
    __shared__ int s_abort;
    uint8_t *smem = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
    constexpr uint32_t A_BYTES = 128 * 128, B_BYTES = NT * 128;
    uint8_t *sA[2] = {smem, smem + A_BYTES + B_BYTES};
    uint8_t *sB[2] = {smem + A_BYTES, smem + 2 * A_BYTES + B_BYTES};
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * 128, n0 = blockIdx.y * NT;
    const int kb0 = blockIdx.z * k_split;
    const int kb1 = min(K, kb0 + k_split);
    const int chunks = (kb1 - kb0) / 64;
    if (warp == 0) tc::tmem_alloc(&tslot, NT < 32 ? 32 : NT);
    if (tid == 0) {
        tc::mbar_init(&mbar[0], 1);
        tc::mbar_init(&mbar[1], 1);
        s_abort = 0;
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tbase = tslot;
    const uint32_t idesc = tc::idesc_f16(128, NT, 1);
    for (int i = 0; i < chunks; i++) {
        const int s = i & 1;
        if (i >= 2 && !tc::mbar_wait(&mbar[s], (uint32_t)(((i - 2) >> 1) & 1), kGemmPolls))
            s_abort = 1;
        __syncthreads();
        if (s_abort) break;
        const int kc = kb0 + 64 * i;
        for (int q = tid; q < 128 * 8; q += kGemmThreads) {
            const int r = q >> 3, c8 = q & 7;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (m0 + r < M) v = *reinterpret_cast<const uint4 *>(A + (size_t)(m0 + r) * lda + kc + 8 * c8);
            *reinterpret_cast<uint4 *>(sA[s] + tc::sw128_offset(r, 8 * c8, 128)) = v;
        }
        for (int q = tid; q < NT * 8; q += kGemmThreads) {
            const int r = q >> 3, c8 = q & 7;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (n0 + r < N) v = *reinterpret_cast<const uint4 *>(B + (size_t)(n0 + r) * ldb + kc + 8 * c8);
            *reinterpret_cast<uint4 *>(sB[s] + tc::sw128_offset(r, 8 * c8, NT)) = v;
        }
        tc::fence_proxy_async();
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        if (tid == 0) {
            const uint32_t a0 = tc::smem_u32(sA[s]), b0 = tc::smem_u32(sB[s]);
            for (int kk = 0; kk < 4; kk++)
                tc::mma_f16(tbase, tc::sdesc_sw128(a0 + 32 * kk), tc::sdesc_sw128(b0 + 32 * kk),
                            idesc, (i > 0 || kk > 0) ? 1u : 0u);
            tc::commit(&mbar[s]);
        }
    }
    bool ok = !s_abort && chunks > 0;
    if (ok) {
        const int last = chunks - 1;
        ok = __all_sync(0xffffffffu,
                        tc::mbar_wait(&mbar[last & 1], (uint32_t)((last >> 1) & 1), kGemmPolls));
    }
    if (!ok && lane == 0 && chunks > 0) atomicOr(ep.err, (unsigned)PXSNE_DEVERR_TIMEOUT);
    if (!ok && lane == 0) s_abort = 1;
    tc::fence_after();
    // Epilogue, 32 columns at a time: each thread holds one row of the block
    // (TMEM lane = row); values pass through shared memory (the operand
    // stages are free now) so that row-major stores, loads and atomics are
    // made by a warp along a row, coalesced.  Transposed stores go straight
    // from the row's thread (consecutive rows, coalesced as well).
    __syncthreads();
    ok = !s_abort;  // the same in every warp (the barriers below need it)
    if (ok) {
        constexpr int SP = 33;  // padded row pitch: conflict-free both ways
        float *sZ = reinterpret_cast<float *>(smem);
        float *sH = sZ + 128 * SP;
        const int rl = 32 * warp + lane, row = m0 + rl;
        const bool rv = row < ep.rows;
#pragma unroll 1
        for (int cb = 0; cb < NT; cb += 32) {
            const int colb = n0 + cb;
            if (EPI == EPI_DGELU) {
                // the pre-activations of this block, loaded along rows
                for (int r = warp; r < 128; r += kGemmThreads / 32) {
                    const int gr = m0 + r, gc = colb + lane;
                    sZ[r * SP + lane] = (gr < ep.rows && gc < N) ? ep.Z[(size_t)gr * ep.ld + gc] : 0.f;
                }
                __syncthreads();
            }
            float v[32];
            tc::tmem_ld32(tbase + ((uint32_t)(32 * warp) << 16) + (uint32_t)cb, v);
#pragma unroll
            for (int j = 0; j < 32; j++) {
                const int col = colb + j;
                if (EPI == EPI_Z_GELU) {
                    const float z = v[j] + (col < N ? ep.bias[col] : 0.f);
                    const float h = gelu_f(z);
                    sZ[rl * SP + j] = z;
                    sH[rl * SP + j] = h;
                    if (ep.HT && rv && col < N) ep.HT[(size_t)col * ep.ldT + row] = __float2bfloat16_rn(h);
                } else if (EPI == EPI_DGELU) {
                    const float g = v[j] * gelu_df(sZ[rl * SP + j]);
                    sH[rl * SP + j] = g;
                    if (ep.HT && rv && col < N) ep.HT[(size_t)col * ep.ldT + row] = __float2bfloat16_rn(g);
                } else {
                    sZ[rl * SP + j] = v[j];
                }
            }
            __syncthreads();
            for (int r = warp; r < 128; r += kGemmThreads / 32) {
                const int gr = m0 + r, gc = colb + lane;
                if (gr >= ep.rows || gc >= N) continue;
                const size_t o = (size_t)gr * ep.ld + gc;
                if (EPI == EPI_Z_GELU) {
                    ep.Z[o] = sZ[r * SP + lane];
                    if (ep.H) ep.H[o] = __float2bfloat16_rn(sH[r * SP + lane]);
                } else if (EPI == EPI_DGELU) {
                    if (ep.H) ep.H[o] = __float2bfloat16_rn(sH[r * SP + lane]);
                } else {
                    atomicAdd(ep.acc + o, sZ[r * SP + lane]);
                }
            }
            __syncthreads();
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, NT < 32 ? 32 : NT);
}

template <int NT, int EPI>
cudaError_t gemm(cudaStream_t st, int M, int N, int K, int k_split, const bf16 *A, int lda,
                 const bf16 *B, int ldb, const Epi &ep) {
    const size_t smem = 2 * (128 * 128 + NT * 128) + 1024;
    cudaError_t e = cudaFuncSetAttribute(k_gemm<NT, EPI>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e) return e;
    const dim3 g((M + 127) / 128, (N + NT - 1) / NT, (K + k_split - 1) / k_split);
    k_gemm<NT, EPI><<<g, kGemmThreads, smem, st>>>(M, N, K, k_split, A, lda, B, ldb, ep);
    return cudaGetLastError();
}

// Output layer: a CTA takes 32 consecutive rows of the batch, a warp 4 of
// them, a lane 8 of the 256 hidden units of a row (16-byte loads and stores).
// With targets: loss (sum of squared errors / m), dy = 2 (y - t) / m,
// dz2 = (W3^T dy) * GELU'(z2), row-major and transposed (the transposed copy
// is staged in shared memory and written 8 rows per 16-byte store), and
// dL/dW3, dL/db3 accumulated per warp and added atomically.
constexpr int kOutRows = 32;
__global__ void __launch_bounds__(256)
    k_out_layer(int m, int rows_pad, const bf16 *__restrict__ H2, const float *__restrict__ Z2,
                const bf16 *__restrict__ W3, const float *__restrict__ b3,
                const float *__restrict__ T, float *__restrict__ Y, bf16 *__restrict__ dZ2,
                bf16 *__restrict__ dZ2T, float *__restrict__ gW3, float *__restrict__ gb3,
                double *__restrict__ loss) {
    constexpr int SP = kH + 8;  // row pitch of the staged gradient (bf16)
    __shared__ __align__(16) bf16 sG[kOutRows * SP];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r0 = blockIdx.x * kOutRows;
    float aW3[2][8];
#pragma unroll
    for (int o = 0; o < 2; o++)
#pragma unroll
        for (int u = 0; u < 8; u++) aW3[o][u] = 0.f;
    float ab3[2] = {0.f, 0.f};
    double aloss = 0.0;
    float w3[2][8];
#pragma unroll
    for (int u = 0; u < 8; u++) {
        w3[0][u] = __bfloat162float(W3[lane * 8 + u]);
        w3[1][u] = __bfloat162float(W3[kH + lane * 8 + u]);
    }
    for (int i = 0; i < kOutRows / 8; i++) {
        const int rl = warp * (kOutRows / 8) + i, r = r0 + rl;
        uint4 gq = make_uint4(0u, 0u, 0u, 0u);  // the row's 8 gradients (bf16), 0 if padding
        if (r < m) {
            const uint4 hq = *reinterpret_cast<const uint4 *>(H2 + (size_t)r * kH + lane * 8);
            const bf16 *hb = reinterpret_cast<const bf16 *>(&hq);
            float h[8];
#pragma unroll
            for (int u = 0; u < 8; u++) h[u] = __bfloat162float(hb[u]);
            float y0 = 0.f, y1 = 0.f;
#pragma unroll
            for (int u = 0; u < 8; u++) {
                y0 = fmaf(w3[0][u], h[u], y0);
                y1 = fmaf(w3[1][u], h[u], y1);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                y0 += __shfl_xor_sync(0xffffffffu, y0, o);
                y1 += __shfl_xor_sync(0xffffffffu, y1, o);
            }
            y0 += b3[0];
            y1 += b3[1];
            if (lane == 0 && Y) {
                Y[2 * r] = y0;
                Y[2 * r + 1] = y1;
            }
            if (T) {
                const float e0 = y0 - T[2 * r], e1 = y1 - T[2 * r + 1];
                if (lane == 0) aloss += (double)e0 * e0 + (double)e1 * e1;
                const float d0 = 2.0f * e0 / (float)m, d1 = 2.0f * e1 / (float)m;
                ab3[0] += d0;
                ab3[1] += d1;
                const float4 za = *reinterpret_cast<const float4 *>(Z2 + (size_t)r * kH + lane * 8);
                const float4 zb = *reinterpret_cast<const float4 *>(Z2 + (size_t)r * kH + lane * 8 + 4);
                const float z[8] = {za.x, za.y, za.z, za.w, zb.x, zb.y, zb.z, zb.w};
                bf16 *gb = reinterpret_cast<bf16 *>(&gq);
#pragma unroll
                for (int u = 0; u < 8; u++) {
                    aW3[0][u] = fmaf(d0, h[u], aW3[0][u]);
                    aW3[1][u] = fmaf(d1, h[u], aW3[1][u]);
                    gb[u] = __float2bfloat16_rn((d0 * w3[0][u] + d1 * w3[1][u]) * gelu_df(z[u]));
                }
            }
        }
        if (T && r < rows_pad) {
            *reinterpret_cast<uint4 *>(dZ2 + (size_t)r * kH + lane * 8) = gq;
            *reinterpret_cast<uint4 *>(sG + rl * SP + lane * 8) = gq;
        }
    }
    if (!T) return;
    __syncthreads();
    // transposed copy: thread c writes unit c of the CTA's 32 rows, 8 rows per
    // 16-byte store
    {
        const int c = threadIdx.x;
#pragma unroll
        for (int q = 0; q < kOutRows; q += 8) {
            if (r0 + q >= rows_pad) break;
            uint4 v;
            bf16 *vb = reinterpret_cast<bf16 *>(&v);
#pragma unroll
            for (int k = 0; k < 8; k++) vb[k] = sG[(q + k) * SP + c];
            *reinterpret_cast<uint4 *>(dZ2T + (size_t)c * rows_pad + r0 + q) = v;
        }
    }
#pragma unroll
    for (int o = 0; o < 2; o++)
#pragma unroll
        for (int u = 0; u < 8; u++) atomicAdd(&gW3[o * kH + lane * 8 + u], aW3[o][u]);
    if (lane == 0) {
        atomicAdd(&gb3[0], ab3[0]);
        atomicAdd(&gb3[1], ab3[1]);
        atomicAdd(loss, aloss / (double)m);
    }
}

// gb[c] += sum over rows of G[r][c] (G BF16 [m x 256]).
__global__ void __launch_bounds__(256) k_colsum(int m, const bf16 *__restrict__ G, float *gb) {
    const int c = threadIdx.x;
    float s = 0.f;
    for (int r = blockIdx.x; r < m; r += gridDim.x) s += __bfloat162float(G[(size_t)r * kH + c]);
    atomicAdd(&gb[c], s);
}

// Batch rows X[perm[r]] -> BF16 row-major [rows_pad x dp] and transposed
// [dp x rows_pad] (zero padding), targets T[perm[r]].
__global__ void k_gather(int m, int rows_pad, int d, int dp, const float *__restrict__ X,
                         const float *__restrict__ T, const int64_t *__restrict__ perm,
                         int64_t base, bf16 *__restrict__ Xb, bf16 *__restrict__ XT,
                         float *__restrict__ Tb) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= (int64_t)rows_pad * dp) return;
    const int r = (int)(i / dp), c = (int)(i % dp);
    float v = 0.f;
    int64_t src = -1;
    if (r < m) {
        src = perm ? perm[base + r] : base + r;
        if (c < d) v = X[src * d + c];
    }
    const bf16 b = __float2bfloat16_rn(v);
    Xb[(size_t)r * dp + c] = b;
    if (XT) XT[(size_t)c * rows_pad + r] = b;
    if (Tb && c < 2) Tb[2 * r + c] = (r < m && T) ? T[src * 2 + c] : 0.f;
}

struct AdamCfg {
    float lr, b1, b2, eps, c1, c2;  // c1 = 1/(1-b1^t), c2 = 1/(1-b2^t)
};

// Adam on the flat FP32 parameters, then BF16 copies of W1 [256 x dp], W2,
// W2^T and W3 (biases stay FP32).
__global__ void k_adam(int64_t np, int d, int dp, AdamCfg a, float *__restrict__ w,
                       const float *__restrict__ g, float *__restrict__ mo,
                       float *__restrict__ ve, bf16 *__restrict__ W1b, bf16 *__restrict__ W2b,
                       bf16 *__restrict__ W2Tb, bf16 *__restrict__ W3b) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= np) return;
    const float gi = g[i];
    const float m1 = a.b1 * mo[i] + (1.0f - a.b1) * gi;
    const float v1 = a.b2 * ve[i] + (1.0f - a.b2) * gi * gi;
    mo[i] = m1;
    ve[i] = v1;
    const float wi = w[i] - a.lr * (m1 * a.c1) / (sqrtf(v1 * a.c2) + a.eps);
    w[i] = wi;
    const int64_t o1 = (int64_t)kH * d, o2 = o1 + kH, o3 = o2 + (int64_t)kH * kH,
                  o4 = o3 + kH, o5 = o4 + 2 * kH;
    const bf16 b = __float2bfloat16_rn(wi);
    if (i < o1) {
        W1b[(i / d) * dp + (i % d)] = b;
    } else if (i >= o2 && i < o3) {
        const int64_t q = i - o2, r = q / kH, c = q % kH;
        W2b[r * kH + c] = b;
        W2Tb[c * kH + r] = b;
    } else if (i >= o4 && i < o5) {
        W3b[i - o4] = b;
    }
}

// BF16 copies of the weights after set_params.
__global__ void k_refresh(int64_t np, int d, int dp, const float *__restrict__ w, bf16 *W1b,
                          bf16 *W2b, bf16 *W2Tb, bf16 *W3b) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= np) return;
    const int64_t o1 = (int64_t)kH * d, o2 = o1 + kH, o3 = o2 + (int64_t)kH * kH,
                  o4 = o3 + kH, o5 = o4 + 2 * kH;
    const bf16 b = __float2bfloat16_rn(w[i]);
    if (i < o1) {
        W1b[(i / d) * dp + (i % d)] = b;
    } else if (i >= o2 && i < o3) {
        const int64_t q = i - o2, r = q / kH, c = q % kH;
        W2b[r * kH + c] = b;
        W2Tb[c * kH + r] = b;
    } else if (i >= o4 && i < o5) {
        W3b[i - o4] = b;
    }
}

}  // namespace
}  // namespace pxsne

using namespace pxsne;

struct pxsne_mlp {
    int d = 0, dp = 0;
    int64_t np = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
    unsigned *derr = nullptr;
    // FP32 master parameters, gradients, Adam moments (flat)
    float *w = nullptr, *g = nullptr, *mo = nullptr, *ve = nullptr;
    int64_t steps = 0;
    // BF16 operand copies
    bf16 *W1b = nullptr, *W2b = nullptr, *W2Tb = nullptr, *W3b = nullptr;
    // batch buffers (kMaxBatch rows)
    bf16 *Xb = nullptr, *XT = nullptr, *H1 = nullptr, *H1T = nullptr, *H2 = nullptr;
    bf16 *dZ2 = nullptr, *dZ2T = nullptr, *dZ1 = nullptr, *dZ1T = nullptr;
    float *Z1 = nullptr, *Z2 = nullptr, *Tb = nullptr, *Yb = nullptr;
    double *loss = nullptr;
    // resident data for training / prediction
    float *Xd = nullptr, *Td = nullptr;
    int64_t *perm = nullptr;
    int64_t data_n = 0, data_cap = 0;
};

namespace {

int mfail(pxsne_mlp *m, int code, const char *msg, cudaError_t e = cudaSuccess) {
    if (e != cudaSuccess) cudaGetLastError();
    if (m) {
        m->err = msg;
        if (e != cudaSuccess) {
            m->err += ": ";
            m->err += cudaGetErrorString(e);
        }
    }
    return code;
}

#define MCK(m, x)                                                                   \
    do {                                                                            \
        cudaError_t e_ = (x);                                                       \
        if (e_ != cudaSuccess)                                                      \
            return mfail((m), e_ == cudaErrorMemoryAllocation ? PXSNE_E_OOM : PXSNE_E_CUDA, \
                         #x, e_);                                                   \
    } while (0)

template <class T>
cudaError_t mal(T **p, size_t count) {
    return cudaMalloc(reinterpret_cast<void **>(p), (count ? count : 1) * sizeof(T));
}

// Pointers into the flat parameter / gradient vectors.
struct Layout {
    int64_t W1, b1, W2, b2, W3, b3;
};
Layout layout(int d) {
    Layout L;
    L.W1 = 0;
    L.b1 = (int64_t)kH * d;
    L.W2 = L.b1 + kH;
    L.b2 = L.W2 + (int64_t)kH * kH;
    L.W3 = L.b2 + kH;
    L.b3 = L.W3 + 2 * kH;
    return L;
}

// Forward on rows [0, m) of the staged batch (Xb); with `train` also the
// backward pass into m->g (which must be zeroed) and the loss into m->loss.
int forward_backward(pxsne_mlp *M, int m, bool train) {
    cudaStream_t st = M->stream;
    const int rp = (m + 127) / 128 * 128;  // rows of the batch buffers in use (x128)
    const Layout L = layout(M->d);
    Epi e{};
    e.err = M->derr;
    // layer 1: Z1 = X W1^T + b1, H1 = GELU(Z1) (+ H1^T for dW2)
    e.ld = kH;
    e.ldT = rp;
    e.rows = m;
    e.bias = M->w + L.b1;
    e.Z = M->Z1;
    e.H = M->H1;
    e.HT = train ? M->H1T : nullptr;
    MCK(M, (gemm<64, EPI_Z_GELU>(st, rp, kH, M->dp, M->dp, M->Xb, M->dp, M->W1b, M->dp, e)));
    // layer 2
    e.bias = M->w + L.b2;
    e.Z = M->Z2;
    e.H = M->H2;
    e.HT = nullptr;
    MCK(M, (gemm<64, EPI_Z_GELU>(st, rp, kH, kH, kH, M->H1, kH, M->W2b, kH, e)));
    // output layer (+ loss, dW3, db3, dZ2)
    const int ob = (rp + kOutRows - 1) / kOutRows;
    k_out_layer<<<ob, 256, 0, st>>>(m, rp, M->H2, M->Z2, M->W3b, M->w + L.b3,
                                    train ? M->Tb : nullptr, M->Yb, M->dZ2, M->dZ2T,
                                    M->g + L.W3, M->g + L.b3, M->loss);
    MCK(M, cudaGetLastError());
    if (!train) return PXSNE_OK;
    // dW2 = dZ2^T H1 (K = batch rows, split in 1024-row slices)
    Epi a{};
    a.err = M->derr;
    a.ld = kH;
    a.rows = kH;
    a.acc = M->g + L.W2;
    MCK(M, (gemm<64, EPI_ATOMIC>(st, kH, kH, rp, kSplitK, M->dZ2T, rp, M->H1T, rp, a)));
    k_colsum<<<128, kH, 0, st>>>(m, M->dZ2, M->g + L.b2);
    MCK(M, cudaGetLastError());
    // dZ1 = (dZ2 W2) * GELU'(Z1)
    Epi b{};
    b.err = M->derr;
    b.ld = kH;
    b.ldT = rp;
    b.rows = rp;  // padded rows: dZ2 = 0 there, so dZ1 = 0
    b.Z = M->Z1;
    b.H = M->dZ1;
    b.HT = M->dZ1T;
    MCK(M, (gemm<64, EPI_DGELU>(st, rp, kH, kH, kH, M->dZ2, kH, M->W2Tb, kH, b)));
    // dW1 = dZ1^T X
    a.ld = M->d;
    a.acc = M->g + L.W1;
    MCK(M, (gemm<64, EPI_ATOMIC>(st, kH, M->d, rp, kSplitK, M->dZ1T, rp, M->XT, rp, a)));
    k_colsum<<<128, kH, 0, st>>>(m, M->dZ1, M->g + L.b1);
    MCK(M, cudaGetLastError());
    return PXSNE_OK;
}

int stage_data(pxsne_mlp *M, const float *X, const float *T, int64_t n, int on_device) {
    cudaStream_t st = M->stream;
    if (n > M->data_cap) {
        cudaFree(M->Xd);
        cudaFree(M->Td);
        cudaFree(M->perm);
        M->Xd = nullptr;
        M->Td = nullptr;
        M->perm = nullptr;
        MCK(M, mal(&M->Xd, (size_t)n * M->d));
        MCK(M, mal(&M->Td, (size_t)n * 2));
        MCK(M, mal(&M->perm, (size_t)n));
        M->data_cap = n;
    }
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    MCK(M, cudaMemcpyAsync(M->Xd, X, (size_t)n * M->d * 4, kind, st));
    if (T) MCK(M, cudaMemcpyAsync(M->Td, T, (size_t)n * 8, kind, st));
    M->data_n = n;
    return PXSNE_OK;
}

int check_dev(pxsne_mlp *M) {
    MCK(M, cudaStreamSynchronize(M->stream));
    unsigned e = 0;
    MCK(M, cudaMemcpy(&e, M->derr, 4, cudaMemcpyDeviceToHost));
    if (e) {
        cudaMemset(M->derr, 0, 4);
        return mfail(M, PXSNE_E_DEVICE, "tensor-core wait timed out");
    }
    return PXSNE_OK;
}

}  // namespace

extern "C" {

int pxsne_mlp_create(pxsne_mlp **out, int32_t d_in, uint64_t seed, void *stream) {
    if (!out) return PXSNE_E_ARG;
    *out = nullptr;
    if (d_in < 1 || d_in > 1024) return PXSNE_E_ARG;
    pxsne_mlp *M = new (std::nothrow) pxsne_mlp();
    if (!M) return PXSNE_E_OOM;
    M->d = d_in;
    M->dp = (d_in + 63) / 64 * 64;
    M->np = layout(d_in).b3 + 2;
    cudaError_t e = cudaSuccess;
    if (stream) {
        M->stream = (cudaStream_t)stream;
    } else {
        e = cudaStreamCreateWithFlags(&M->stream, cudaStreamNonBlocking);
        M->own_stream = (e == cudaSuccess);
    }
    const size_t B = kMaxBatch;
    if (!e) e = mal(&M->derr, 1);
    if (!e) e = cudaMemset(M->derr, 0, 4);
    if (!e) e = mal(&M->w, M->np);
    if (!e) e = mal(&M->g, M->np);
    if (!e) e = mal(&M->mo, M->np);
    if (!e) e = mal(&M->ve, M->np);
    if (!e) e = mal(&M->W1b, (size_t)kH * M->dp);
    if (!e) e = mal(&M->W2b, (size_t)kH * kH);
    if (!e) e = mal(&M->W2Tb, (size_t)kH * kH);
    if (!e) e = mal(&M->W3b, (size_t)2 * kH);
    if (!e) e = mal(&M->Xb, B * M->dp);
    if (!e) e = mal(&M->XT, B * M->dp);
    if (!e) e = mal(&M->H1, B * kH);
    if (!e) e = mal(&M->H1T, B * kH);
    if (!e) e = mal(&M->H2, B * kH);
    if (!e) e = mal(&M->dZ2, B * kH);
    if (!e) e = mal(&M->dZ2T, B * kH);
    if (!e) e = mal(&M->dZ1, B * kH);
    if (!e) e = mal(&M->dZ1T, B * kH);
    if (!e) e = mal(&M->Z1, B * kH);
    if (!e) e = mal(&M->Z2, B * kH);
    if (!e) e = mal(&M->Tb, B * 2);
    if (!e) e = mal(&M->Yb, B * 2);
    if (!e) e = mal(&M->loss, 1);
    // every buffer starts at zero (padding rows and columns are read as zeros)
    if (!e) e = cudaMemset(M->W1b, 0, (size_t)kH * M->dp * 2);
    {
        struct Z { void *p; size_t bytes; } zs[] = {
            {M->g, (size_t)M->np * 4}, {M->Xb, B * M->dp * 2}, {M->XT, B * M->dp * 2},
            {M->H1, B * kH * 2}, {M->H1T, B * kH * 2}, {M->H2, B * kH * 2},
            {M->dZ2, B * kH * 2}, {M->dZ2T, B * kH * 2}, {M->dZ1, B * kH * 2},
            {M->dZ1T, B * kH * 2}, {M->Z1, B * kH * 4}, {M->Z2, B * kH * 4},
            {M->Tb, B * 8}, {M->Yb, B * 8}, {M->loss, 8}};
        for (auto &z : zs)
            if (!e) e = cudaMemset(z.p, 0, z.bytes);
    }
    if (e) {
        cudaGetLastError();
        pxsne_mlp_destroy(M);
        return e == cudaErrorMemoryAllocation ? PXSNE_E_OOM : PXSNE_E_CUDA;
    }
    // He-style initialisation from the seed: W ~ N(0, 2 / fan_in), b = 0
    std::vector<float> w((size_t)M->np, 0.f);
    std::mt19937_64 rng(seed);
    const Layout L = layout(d_in);
    auto fill = [&](int64_t off, int64_t count, double fan_in, double gain) {
        std::normal_distribution<double> nd(0.0, gain / std::sqrt(fan_in));
        for (int64_t q = 0; q < count; q++) w[(size_t)(off + q)] = (float)nd(rng);
    };
    fill(L.W1, (int64_t)kH * d_in, d_in, std::sqrt(2.0));
    fill(L.W2, (int64_t)kH * kH, kH, std::sqrt(2.0));
    fill(L.W3, 2 * kH, kH, 1.0);
    int rc = pxsne_mlp_set_params(M, w.data());
    if (rc) {
        pxsne_mlp_destroy(M);
        return rc;
    }
    *out = M;
    return PXSNE_OK;
}

void pxsne_mlp_destroy(pxsne_mlp *M) {
    if (!M) return;
    if (M->stream) cudaStreamSynchronize(M->stream);
    void *ptrs[] = {M->derr, M->w,   M->g,   M->mo,  M->ve,  M->W1b,  M->W2b, M->W2Tb, M->W3b,
                    M->Xb,   M->XT,  M->H1,  M->H1T, M->H2,  M->dZ2,  M->dZ2T, M->dZ1, M->dZ1T,
                    M->Z1,   M->Z2,  M->Tb,  M->Yb,  M->loss, M->Xd,  M->Td,  M->perm};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (M->own_stream) cudaStreamDestroy(M->stream);
    delete M;
}

const char *pxsne_mlp_last_error(const pxsne_mlp *M) { return M ? M->err.c_str() : ""; }

int64_t pxsne_mlp_num_params(const pxsne_mlp *M) { return M ? M->np : 0; }

int pxsne_mlp_set_params(pxsne_mlp *M, const float *params) {
    if (!M || !params) return PXSNE_E_ARG;
    for (int64_t i = 0; i < M->np; i++)
        if (!std::isfinite(params[i])) return mfail(M, PXSNE_E_ARG, "non-finite parameter");
    cudaStream_t st = M->stream;
    MCK(M, cudaMemcpyAsync(M->w, params, (size_t)M->np * 4, cudaMemcpyHostToDevice, st));
    MCK(M, cudaMemsetAsync(M->mo, 0, (size_t)M->np * 4, st));
    MCK(M, cudaMemsetAsync(M->ve, 0, (size_t)M->np * 4, st));
    M->steps = 0;
    k_refresh<<<(unsigned)((M->np + 255) / 256), 256, 0, st>>>(M->np, M->d, M->dp, M->w, M->W1b,
                                                               M->W2b, M->W2Tb, M->W3b);
    MCK(M, cudaGetLastError());
    return check_dev(M);
}

int pxsne_mlp_get_params(pxsne_mlp *M, float *params) {
    if (!M || !params) return PXSNE_E_ARG;
    MCK(M, cudaMemcpyAsync(params, M->w, (size_t)M->np * 4, cudaMemcpyDeviceToHost, M->stream));
    return check_dev(M);
}

int pxsne_mlp_loss_grad(pxsne_mlp *M, const float *X, const float *T, int64_t n, float *grad,
                        double *loss, int on_device) {
    if (!M || !X || !T || n < 1 || n > kMaxBatch) return mfail(M, PXSNE_E_ARG, "1 <= n <= 8192");
    int rc = stage_data(M, X, T, n, on_device);
    if (rc) return rc;
    cudaStream_t st = M->stream;
    const int m = (int)n, rp = (m + 127) / 128 * 128;
    k_gather<<<(unsigned)(((int64_t)rp * M->dp + 255) / 256), 256, 0, st>>>(
        m, rp, M->d, M->dp, M->Xd, M->Td, nullptr, 0, M->Xb, M->XT, M->Tb);
    MCK(M, cudaGetLastError());
    MCK(M, cudaMemsetAsync(M->g, 0, (size_t)M->np * 4, st));
    MCK(M, cudaMemsetAsync(M->loss, 0, 8, st));
    rc = forward_backward(M, m, true);
    if (rc) return rc;
    if (grad) MCK(M, cudaMemcpyAsync(grad, M->g, (size_t)M->np * 4, cudaMemcpyDeviceToHost, st));
    if (loss) MCK(M, cudaMemcpyAsync(loss, M->loss, 8, cudaMemcpyDeviceToHost, st));
    return check_dev(M);
}

int pxsne_mlp_train(pxsne_mlp *M, const float *X, const float *T, int64_t n, int32_t epochs,
                    int32_t batch, float lr, uint64_t shuffle_seed, double *final_loss,
                    int on_device) {
    if (!M || !X || !T || n < 1 || epochs < 0 || batch < 1 || batch > kMaxBatch || !(lr > 0.f))
        return mfail(M, PXSNE_E_ARG, "bad training arguments");
    int rc = stage_data(M, X, T, n, on_device);
    if (rc) return rc;
    cudaStream_t st = M->stream;
    std::vector<int64_t> perm((size_t)n);
    for (int64_t i = 0; i < n; i++) perm[(size_t)i] = i;
    std::mt19937_64 rng(shuffle_seed);
    double last = 0.0;
    for (int32_t ep = 0; ep < epochs; ep++) {
        for (int64_t i = n - 1; i > 0; i--) {
            std::uniform_int_distribution<int64_t> u(0, i);
            std::swap(perm[(size_t)i], perm[(size_t)u(rng)]);
        }
        MCK(M, cudaMemcpyAsync(M->perm, perm.data(), (size_t)n * 8, cudaMemcpyHostToDevice, st));
        MCK(M, cudaMemsetAsync(M->loss, 0, 8, st));
        int64_t nb = 0;
        for (int64_t base = 0; base < n; base += batch, nb++) {
            const int m = (int)std::min<int64_t>(batch, n - base);
            const int rp = (m + 127) / 128 * 128;
            k_gather<<<(unsigned)(((int64_t)rp * M->dp + 255) / 256), 256, 0, st>>>(
                m, rp, M->d, M->dp, M->Xd, M->Td, M->perm, base, M->Xb, M->XT, M->Tb);
            MCK(M, cudaGetLastError());
            MCK(M, cudaMemsetAsync(M->g, 0, (size_t)M->np * 4, st));
            rc = forward_backward(M, m, true);
            if (rc) return rc;
            M->steps++;
            AdamCfg a;
            a.lr = lr;
            a.b1 = 0.9f;
            a.b2 = 0.999f;
            a.eps = 1e-8f;
            a.c1 = (float)(1.0 / (1.0 - std::pow(0.9, (double)M->steps)));
            a.c2 = (float)(1.0 / (1.0 - std::pow(0.999, (double)M->steps)));
            k_adam<<<(unsigned)((M->np + 255) / 256), 256, 0, st>>>(
                M->np, M->d, M->dp, a, M->w, M->g, M->mo, M->ve, M->W1b, M->W2b, M->W2Tb, M->W3b);
            MCK(M, cudaGetLastError());
        }
        double s = 0.0;
        MCK(M, cudaMemcpyAsync(&s, M->loss, 8, cudaMemcpyDeviceToHost, st));
        rc = check_dev(M);
        if (rc) return rc;
        last = s / (double)(nb > 0 ? nb : 1);
    }
    if (final_loss) *final_loss = last;
    return check_dev(M);
}

int pxsne_mlp_predict(pxsne_mlp *M, const float *X, int64_t n, float *Y, int on_device) {
    if (!M || !X || !Y || n < 1) return mfail(M, PXSNE_E_ARG, "bad arguments");
    int rc = stage_data(M, X, nullptr, n, on_device);
    if (rc) return rc;
    cudaStream_t st = M->stream;
    float *Yd = Y;
    if (!on_device) MCK(M, mal(&Yd, (size_t)n * 2));
    for (int64_t base = 0; base < n; base += kMaxBatch) {
        const int m = (int)std::min<int64_t>(kMaxBatch, n - base);
        const int rp = (m + 127) / 128 * 128;
        k_gather<<<(unsigned)(((int64_t)rp * M->dp + 255) / 256), 256, 0, st>>>(
            m, rp, M->d, M->dp, M->Xd, nullptr, nullptr, base, M->Xb, nullptr, nullptr);
        MCK(M, cudaGetLastError());
        rc = forward_backward(M, m, false);
        if (rc) return rc;
        MCK(M, cudaMemcpyAsync(Yd + 2 * base, M->Yb, (size_t)m * 8, cudaMemcpyDeviceToDevice, st));
    }
    if (!on_device) {
        MCK(M, cudaMemcpyAsync(Y, Yd, (size_t)n * 8, cudaMemcpyDeviceToHost, st));
        rc = check_dev(M);
        cudaFree(Yd);
        return rc;
    }
    return check_dev(M);
}

}  // extern "C"

// ---------------------------------------------------------------- target alignment
namespace pxsne {
namespace {
// sums[0..1] = sum y, [2] = sum |y - mean|^2, [3..6] = sum (y - mean)^T (r - rmean)
__global__ void k_align_sums(int64_t n, const float2 *__restrict__ Y,
                             const float2 *__restrict__ R, const double *__restrict__ mean,
                             int pass, double *sums) {
    double a[5] = {0, 0, 0, 0, 0};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float2 y = Y[i];
        if (pass == 0) {
            a[0] += y.x;
            a[1] += y.y;
            if (R) {
                const float2 r = R[i];
                a[2] += r.x;
                a[3] += r.y;
            }
        } else {
            const double yx = y.x - mean[0], yy = y.y - mean[1];
            a[0] += yx * yx + yy * yy;
            if (R) {
                const float2 r = R[i];
                const double rx = r.x - mean[2], ry = r.y - mean[3];
                a[1] += yx * rx;
                a[2] += yx * ry;
                a[3] += yy * rx;
                a[4] += yy * ry;
            }
        }
    }
    for (int q = 0; q < 5; q++) {
        double v = a[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(&sums[q], v);
    }
}

__global__ void k_align_apply(int64_t n, const float2 *__restrict__ Y, double mx, double my,
                              double scale, double r00, double r01, double r10, double r11,
                              float2 *__restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float2 y = Y[i];
    const double a = (y.x - mx) * scale, b = (y.y - my) * scale;
    out[i] = make_float2((float)(a * r00 + b * r10), (float)(a * r01 + b * r11));
}
}  // namespace
}  // namespace pxsne

extern "C" int pxsne_embed_align(const float *Y, const float *Yref, int64_t n, float *Yout,
                                 int on_device) {
    using namespace pxsne;
    if (!Y || !Yout || n < 2) return PXSNE_E_ARG;
    cudaStream_t st = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e) return PXSNE_E_CUDA;
    float *dY = nullptr, *dR = nullptr, *dO = nullptr;
    double *dsum = nullptr, *dmean = nullptr;
    int rc = PXSNE_OK;
    auto ck = [&](cudaError_t x) {
        if (x != cudaSuccess && rc == PXSNE_OK) rc = PXSNE_E_CUDA;
        return x == cudaSuccess;
    };
    const size_t bytes = (size_t)n * 8;
    if (on_device) {
        dY = const_cast<float *>(Y);
        dR = const_cast<float *>(Yref);
        dO = Yout;
    } else {
        ck(cudaMallocAsync(&dY, bytes, st));
        ck(cudaMallocAsync(&dO, bytes, st));
        if (Yref) ck(cudaMallocAsync(&dR, bytes, st));
        if (rc == PXSNE_OK) {
            ck(cudaMemcpyAsync(dY, Y, bytes, cudaMemcpyHostToDevice, st));
            if (Yref) ck(cudaMemcpyAsync(dR, Yref, bytes, cudaMemcpyHostToDevice, st));
        }
    }
    ck(cudaMallocAsync(&dsum, 5 * 8, st));
    ck(cudaMallocAsync(&dmean, 4 * 8, st));
    double h[5], mean[4] = {0, 0, 0, 0};
    const int blocks = 296;
    if (rc == PXSNE_OK) {
        ck(cudaMemsetAsync(dsum, 0, 5 * 8, st));
        k_align_sums<<<blocks, 256, 0, st>>>(n, reinterpret_cast<const float2 *>(dY),
                                             reinterpret_cast<const float2 *>(dR), dmean, 0, dsum);
        ck(cudaGetLastError());
        ck(cudaMemcpyAsync(h, dsum, 5 * 8, cudaMemcpyDeviceToHost, st));
        ck(cudaStreamSynchronize(st));
    }
    if (rc == PXSNE_OK) {
        for (int q = 0; q < 4; q++) mean[q] = h[q] / (double)n;
        ck(cudaMemcpyAsync(dmean, mean, 4 * 8, cudaMemcpyHostToDevice, st));
        ck(cudaMemsetAsync(dsum, 0, 5 * 8, st));
        k_align_sums<<<blocks, 256, 0, st>>>(n, reinterpret_cast<const float2 *>(dY),
                                             reinterpret_cast<const float2 *>(dR), dmean, 1, dsum);
        ck(cudaGetLastError());
        ck(cudaMemcpyAsync(h, dsum, 5 * 8, cudaMemcpyDeviceToHost, st));
        ck(cudaStreamSynchronize(st));
    }
    if (rc == PXSNE_OK) {
        // unit RMS per coordinate: sum |y|^2 / (2 n) = 1
        const double rms = std::sqrt(h[0] / (2.0 * (double)n));
        const double scale = rms > 0.0 ? 1.0 / rms : 1.0;
        // orthogonal R maximising tr(R^T M), M = Y^T Ref (2 x 2), closed form:
        // rotations give hypot(M00 + M11, M10 - M01), reflections
        // hypot(M00 - M11, M10 + M01)
        double r00 = 1, r01 = 0, r10 = 0, r11 = 1;
        if (Yref) {
            const double M00 = h[1], M01 = h[2], M10 = h[3], M11 = h[4];
            const double rot = std::hypot(M00 + M11, M10 - M01);
            const double ref = std::hypot(M00 - M11, M10 + M01);
            if (rot >= ref) {
                const double phi = std::atan2(M10 - M01, M00 + M11);
                const double c = std::cos(phi), s = std::sin(phi);
                r00 = c; r01 = -s; r10 = s; r11 = c;
            } else {
                const double phi = std::atan2(M10 + M01, M00 - M11);
                const double c = std::cos(phi), s = std::sin(phi);
                r00 = c; r01 = s; r10 = s; r11 = -c;
            }
        }
        k_align_apply<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
            n, reinterpret_cast<const float2 *>(dY), mean[0], mean[1], scale, r00, r01, r10, r11,
            reinterpret_cast<float2 *>(dO));
        ck(cudaGetLastError());
        if (!on_device) ck(cudaMemcpyAsync(Yout, dO, bytes, cudaMemcpyDeviceToHost, st));
        ck(cudaStreamSynchronize(st));
    }
    if (!on_device) {
        if (dY) cudaFreeAsync(dY, st);
        if (dO) cudaFreeAsync(dO, st);
        if (dR) cudaFreeAsync(dR, st);
    }
    if (dsum) cudaFreeAsync(dsum, st);
    if (dmean) cudaFreeAsync(dmean, st);
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    return rc;
}
