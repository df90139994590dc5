// KL evaluation that allocates no memory (pxsne_kl_noalloc).
//
// Some callers cannot call cudaMalloc: code that runs while another
// component owns the device memory pool (a framework's caching allocator
// holding a fixed arena, or a process under a hard memory cap), and loops
// that must not pay the implicit device-wide synchronisation of cudaMalloc /
// cudaFree (a live view that evaluates the cost next to a running
// optimisation).  This entry point takes every input and the output from the
// caller and keeps its only scratch, the per-block partial sums of the
// reduction, in a fixed file-scope device array.
#include <cmath>
#include <mutex>

#include "common.cuh"

namespace {

using pxsne::u64;

constexpr int kNoallocThreads = 256;
constexpr int kNoallocRowsPerBlock = 2048;
constexpr int kNoallocMaxBlocks = 8192;
// Largest n accepted: one block per 2048 rows, at most 8192 blocks.
constexpr int64_t kNoallocMaxRows = (int64_t)kNoallocRowsPerBlock * kNoallocMaxBlocks;

// Shared by every call on a device (kept until the process exits):
// [0, 2 * kNoallocMaxBlocks) doubles of block partials {sum p ln(p w^-1), sum p},
// then the ticket of the last-block-done reduction and the count of entries
// whose column lay outside [0, n) (both cleared by every call).
struct NoallocScratch {
    double part[2 * kNoallocMaxBlocks];
    unsigned ticket;
    unsigned bad;
};
static __device__ __align__(256) NoallocScratch g_kl_scratch;

std::mutex g_mu;
NoallocScratch *g_addr[64] = {nullptr};

// Address of the scratch array on the current device (looked up once per
// device with that device current, then kept: a cudaDeviceReset of that
// device makes the kept address stale).
cudaError_t scratch_on_current_device(NoallocScratch **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_kl_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = static_cast<NoallocScratch *>(p);
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

// Eq. cost_func over the rows [b * 2048, (b + 1) * 2048) of block b, one warp
// per row; FP32 terms, FP64 accumulation, partials combined in block order by
// the last block to finish.  An entry whose column is outside [0, n) is
// skipped and counted; the result is then NaN.
__global__ void __launch_bounds__(kNoallocThreads)
    k_kl_noalloc(int64_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                 const float *__restrict__ val, const uint2 *__restrict__ z, float sf0, float sf1,
                 double lnZ, NoallocScratch *scr, double *__restrict__ out) {
    __shared__ double s_red[2][kNoallocThreads / 32];
    __shared__ unsigned s_bad[kNoallocThreads / 32];
    __shared__ bool s_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t r0 = (int64_t)blockIdx.x * kNoallocRowsPerBlock;
    const int64_t r1 = r0 + kNoallocRowsPerBlock < n ? r0 + kNoallocRowsPerBlock : n;
    double acc = 0.0, psum = 0.0;
    unsigned nbad = 0u;
    for (int64_t row = r0 + warp; row < r1; row += kNoallocThreads / 32) {
        const uint2 zi = z[row];
        for (int64_t e = rp[row] + lane; e < rp[row + 1]; e += 32) {
            const float p = val[e];
            if (!(p > 0.f)) continue;
            const int32_t j = col[e];
            if ((uint64_t)(uint32_t)j >= (uint64_t)n) {
                nbad++;
                continue;
            }
            const uint2 zj = z[j];
            const float dx = (float)((int64_t)zi.x - (int64_t)zj.x) * sf0;
            const float dy = (float)((int64_t)zi.y - (int64_t)zj.y) * sf1;
            acc += (double)(p * (logf(p) + log1pf(fmaf(dx, dx, dy * dy))));
            psum += (double)p;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc += __shfl_xor_sync(0xffffffffu, acc, o);
        psum += __shfl_xor_sync(0xffffffffu, psum, o);
        nbad += __shfl_xor_sync(0xffffffffu, nbad, o);
    }
    if (lane == 0) {
        s_red[0][warp] = acc;
        s_red[1][warp] = psum;
        s_bad[warp] = nbad;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, p = 0.0;
        unsigned b = 0u;
        for (int w = 0; w < kNoallocThreads / 32; w++) {
            a += s_red[0][w];
            p += s_red[1][w];
            b += s_bad[w];
        }
        scr->part[2 * blockIdx.x] = a;
        scr->part[2 * blockIdx.x + 1] = p;
        if (b) atomicAdd(&scr->bad, b);
        __threadfence();
        const unsigned tk = atomicAdd(&scr->ticket, 1u);
        s_last = (tk == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last || threadIdx.x != 0) return;
    __threadfence();
    const volatile double *vp = scr->part;
    double A = 0.0, S = 0.0;
    for (unsigned b = 0; b < gridDim.x; b++) {
        A += vp[2 * b];
        S += vp[2 * b + 1];
    }
    const unsigned bad = *reinterpret_cast<volatile unsigned *>(&scr->bad);
    *out = bad == 0u ? A + S * lnZ : __longlong_as_double(0x7ff8000000000000ll);
    scr->ticket = 0u;
}

}  // namespace

extern "C" int pxsne_kl_noalloc(const int64_t *row_ptr, const int32_t *col, const float *val,
                                int64_t n, const uint32_t *z, double s0, double s1, double Z,
                                double *out, void *stream) {
    if (!row_ptr || !col || !val || !z || !out || n < 1) return PXSNE_E_ARG;
    if (n > kNoallocMaxRows) return PXSNE_E_ARG;
    if (!(std::isfinite(s0) && s0 > 0.0) || !(std::isfinite(s1) && s1 > 0.0) ||
        !(std::isfinite(Z) && Z > 0.0))
        return PXSNE_E_ARG;
    NoallocScratch *scr = nullptr;
    cudaError_t e = scratch_on_current_device(&scr);
    if (e != cudaSuccess) return PXSNE_E_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the ticket and the bad-column count must start at zero; the partials
    // are all overwritten
    e = cudaMemsetAsync(&scr->ticket, 0, 2 * sizeof(unsigned), st);
    if (e != cudaSuccess) return PXSNE_E_CUDA;
    const unsigned blocks = (unsigned)((n + kNoallocRowsPerBlock - 1) / kNoallocRowsPerBlock);
    k_kl_noalloc<<<blocks, kNoallocThreads, 0, st>>>(n, row_ptr, col, val,
                                                      reinterpret_cast<const uint2 *>(z),
                                                      (float)s0, (float)s1, log(Z), scr, out);
    e = cudaGetLastError();
    return e == cudaSuccess ? PXSNE_OK : PXSNE_E_CUDA;
}

extern "C" int64_t pxsne_kl_noalloc_max_rows(void) { return kNoallocMaxRows; }
