// Gradient step of PixelSNE (Eq. grad with the BH-SNE optimiser the paper
// keeps) and the random initial embedding.
//
//   k_update   g = 4 (alpha Fattr - Frep / Z); per-coordinate gains and
//              momentum; zhat = z + rint(u / s) in int64 ulps; per-axis
//              min/max of zhat for the screen rescale of Sec. 4.2
//   k_philox_y0  Y0 ~ N(0, sigma^2 I) from Philox4x32-10 + Box-Muller
#include <cmath>

#include "common.cuh"

namespace pxsne {

__global__ void __launch_bounds__(256)
    k_update(int n, UpdateParams p, const uint2 *__restrict__ z,
             const float2 *__restrict__ Frep, const float2 *__restrict__ Fattr,
             float2 *__restrict__ u, float2 *__restrict__ gains, longlong2 *__restrict__ zhat,
             DevScalars *sc) {
    __shared__ i64 s_mm[4][8];
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
    const double is0 = sc->inv_s[0], is1 = sc->inv_s[1];
    i64 mnx = 0x7fffffffffffffffll, mny = 0x7fffffffffffffffll;
    i64 mxx = (i64)0x8000000000000000ull, mxy = (i64)0x8000000000000000ull;
    unsigned err = 0u;
    // a fixed grid strides over the points, so that few CTAs meet in the
    // min/max atomics below
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float2 fr = Frep[i], fa = Fattr[i];
        float2 uu = u[i], gg = gains[i];
        const uint2 zz = z[i];
        longlong2 zh;
        zh.x = step1(fa.x, fr.x, alpha, invZ, mu, p, uu.x, gg.x, zz.x, is0, err);
        zh.y = step1(fa.y, fr.y, alpha, invZ, mu, p, uu.y, gg.y, zz.y, is1, err);
        u[i] = uu;
        gains[i] = gg;
        zhat[i] = zh;
        mnx = min(mnx, zh.x);
        mxx = max(mxx, zh.x);
        mny = min(mny, zh.y);
        mxy = max(mxy, zh.y);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mnx = min(mnx, __shfl_xor_sync(0xffffffffu, mnx, o));
        mny = min(mny, __shfl_xor_sync(0xffffffffu, mny, o));
        mxx = max(mxx, __shfl_xor_sync(0xffffffffu, mxx, o));
        mxy = max(mxy, __shfl_xor_sync(0xffffffffu, mxy, o));
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        s_mm[0][w] = mnx; s_mm[1][w] = mny; s_mm[2][w] = mxx; s_mm[3][w] = mxy;
    }
    if (err) atomicOr(&sc->err, err);
    __syncthreads();
    if (threadIdx.x < 4) {
        const int k = threadIdx.x;
        const int nw = blockDim.x >> 5;
        i64 v = s_mm[k][0];
        for (int q = 1; q < nw; q++) v = k < 2 ? min(v, s_mm[k][q]) : max(v, s_mm[k][q]);
        i64 *dst = &sc->mm[t & 1][k];
        if (k < 2) atomicMin(reinterpret_cast<long long *>(dst), (long long)v);
        else atomicMax(reinterpret_cast<long long *>(dst), (long long)v);
    }
}

cudaError_t launch_update(pxsne_ctx *c, cudaEvent_t *marks) {
    UpdateParams p;
    p.eta = c->p.eta;
    p.exag = c->p.exaggeration;
    p.mom0 = c->p.momentum0;
    p.mom1 = c->p.momentum1;
    p.min_gain = c->p.min_gain;
    p.exag_iters = c->p.exag_iters;
    p.mom_switch = c->p.momentum_switch;
    const int n = (int)c->n;
    if (marks) {
        cudaError_t e = cudaEventRecord(marks[KG_UPDATE], c->stream);
        if (e) return e;
    }
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int need = (n + 255) / 256, cap = 8 * (sms > 0 ? sms : 152);
    k_update<<<need < cap ? need : cap, 256, 0, c->stream>>>(n, p, c->z, c->Frep, c->Fattr, c->u,
                                                             c->gains, c->zhat, c->sc);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- Philox4x32-10
// Counter-based generator of Salmon, Moraes, Dror and Shaw (SC'11), 10 rounds.
__device__ __forceinline__ void philox_round(uint32_t c[4], const uint32_t k[2]) {
    const uint32_t m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
    const uint32_t lo0 = m0 * c[0], hi0 = __umulhi(m0, c[0]);
    const uint32_t lo1 = m1 * c[2], hi1 = __umulhi(m1, c[2]);
    const uint32_t n0 = hi1 ^ c[1] ^ k[0], n2 = hi0 ^ c[3] ^ k[1];
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
}

__device__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
    uint32_t k[2] = {k0, k1};
#pragma unroll
    for (int r = 0; r < 10; r++) {
        if (r > 0) {
            k[0] += 0x9E3779B9u;
            k[1] += 0xBB67AE85u;
        }
        philox_round(c, k);
    }
}

// Point i uses counter (i, 0, 0, 0) and key (seed low, seed high); the first
// two words give two uniforms u = (r + 0.5) 2^-32 and Box-Muller two normals.
__global__ void k_philox_y0(int n, uint64_t seed, float sigma, float2 *__restrict__ Y) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t c[4] = {(uint32_t)i, 0u, 0u, 0u};
    philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    const double u1 = ((double)c[0] + 0.5) * (1.0 / 4294967296.0);
    const double u2 = ((double)c[1] + 0.5) * (1.0 / 4294967296.0);
    const double rad = sqrt(-2.0 * log(u1));
    const double ang = 6.283185307179586 * u2;
    Y[i] = make_float2((float)(sigma * rad * cos(ang)), (float)(sigma * rad * sin(ang)));
}

cudaError_t launch_philox_y0(pxsne_ctx *c, float *Y0dev, uint64_t seed, float sigma) {
    const int n = (int)c->n;
    k_philox_y0<<<(n + 255) / 256, 256, 0, c->stream>>>(n, seed, sigma,
                                                        reinterpret_cast<float2 *>(Y0dev));
    return cudaGetLastError();
}

}  // namespace pxsne
