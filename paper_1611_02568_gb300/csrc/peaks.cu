// Peaks of the GPU the library runs on, measured by plain kernels, as the
// denominators of the iteration's rooflines (no counterpart in the paper):
//
//   k_l2_read     streams a buffer that fits in L2 (16-byte loads that skip
//                 L1, every CTA over the whole buffer, many passes) -> the L2
//                 read bandwidth the traversal's cell records are fetched at
//   k_ffma        independent chains of FP32 fused multiply-adds, scalar and
//                 as packed pairs -> the FP32 issue rate the traversal's
//                 arithmetic runs at
//
// Each runs on the caller's stream and is timed with CUDA events there.
#include <cuda_runtime.h>

#include "common.cuh"

namespace {

// total 16-byte reads over a buffer of mask + 1 elements (a power of two),
// grid-stride so that a warp reads 512 contiguous bytes per load
__global__ void __launch_bounds__(512)
    k_l2_read(const uint4 *__restrict__ buf, uint32_t mask, int64_t total,
              uint32_t *__restrict__ sink) {
    uint32_t acc = 0u;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += 4 * stride) {
        uint4 v[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const uint32_t j = (uint32_t)(k + u * stride) & mask;
            asm volatile("ld.global.cg.v4.u32 {%0, %1, %2, %3}, [%4];"
                         : "=r"(v[u].x), "=r"(v[u].y), "=r"(v[u].z), "=r"(v[u].w)
                         : "l"(buf + j));
        }
#pragma unroll
        for (int u = 0; u < 4; u++) acc ^= v[u].x ^ v[u].y ^ v[u].z ^ v[u].w;
    }
    if (acc == 0x9e3779b9u) sink[0] = acc;  // keeps the loads
}

template <bool PACKED>
__global__ void __launch_bounds__(256) k_ffma(int iters, float seed, float *__restrict__ sink) {
    constexpr int C = 8;  // independent chains per thread
    float2 a[C];
#pragma unroll
    for (int c = 0; c < C; c++)
        a[c] = make_float2(seed + threadIdx.x * 1e-7f + c, seed - c * 1e-7f);
    const float2 m = make_float2(0.999999f, 0.999998f), b = make_float2(1e-7f, 2e-7f);
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int c = 0; c < C; c++) {
            if (PACKED) {
                a[c] = __ffma2_rn(a[c], m, b);
            } else {
                a[c].x = fmaf(a[c].x, m.x, b.x);
                a[c].y = fmaf(a[c].y, m.y, b.y);
            }
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < C; c++) s += a[c].x + a[c].y;
    if (s == 1234.5f) sink[0] = s;  // keeps the chains
}

template <typename F>
cudaError_t time_ms(cudaStream_t st, F launch, int reps, double *best) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (!e) e = cudaEventCreate(&e1);
    double b = 1e30;
    for (int r = 0; r < reps && !e; r++) {
        e = cudaEventRecord(e0, st);
        if (!e) launch();
        if (!e) e = cudaGetLastError();
        if (!e) e = cudaEventRecord(e1, st);
        if (!e) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (!e) e = cudaEventElapsedTime(&ms, e0, e1);
        if (!e && ms < b) b = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    *best = b;
    return e;
}

}  // namespace

extern "C" int pxsne_measure_peaks(void *stream, double *l2_read_gbs, double *fp32_tflops,
                                   double *fp32_packed_tflops, int32_t *sm_count,
                                   int64_t *l2_bytes) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) || cudaGetDeviceProperties(&prop, dev)) return PXSNE_E_CUDA;
    if (sm_count) *sm_count = prop.multiProcessorCount;
    if (l2_bytes) *l2_bytes = prop.l2CacheSize;
    const int sms = prop.multiProcessorCount;
    uint32_t *sink = nullptr;
    if (cudaMalloc(&sink, 64)) return PXSNE_E_OOM;
    int rc = PXSNE_OK;
    if (l2_read_gbs) {
        // buffers of 1/16, 1/8 and 1/4 of L2 (powers of two, resident after the
        // first pass), 2, 4 or 8 CTAs of 512 threads per SM: the best of all
        // on three allocations held at once (the rate depends on where in the
        // two dies' L2 halves a buffer's lines fall)
        int64_t top = 1 << 20;
        while (top * 2 <= (int64_t)prop.l2CacheSize / 4) top *= 2;
        uint4 *bufs[3] = {nullptr, nullptr, nullptr};
        double best = 0.0;
        for (int a = 0; a < 3 && rc == PXSNE_OK; a++) {
            if (cudaMalloc(&bufs[a], top)) {
                rc = PXSNE_E_OOM;
                break;
            }
            uint4 *buf = bufs[a];
            cudaMemsetAsync(buf, 1, top, st);
            for (int64_t bytes = top / 4; bytes <= top && rc == PXSNE_OK; bytes *= 2) {
                const int64_t n16 = bytes / 16;
                const int64_t total = (top / 16) * 64;  // 64 passes over the largest buffer
                for (int per_sm = 2; per_sm <= 8 && rc == PXSNE_OK; per_sm *= 2) {
                    double ms = 0.0;
                    auto go = [&] {
                        k_l2_read<<<sms * per_sm, 512, 0, st>>>(buf, (uint32_t)(n16 - 1), total,
                                                                sink);
                    };
                    if (time_ms(st, go, 1, &ms) || time_ms(st, go, 5, &ms)) rc = PXSNE_E_CUDA;
                    else best = fmax(best, (double)total * 16.0 / (ms * 1e-3) / 1e9);
                }
            }
        }
        for (uint4 *b : bufs)
            if (b) cudaFree(b);
        if (rc == PXSNE_OK) *l2_read_gbs = best;
    }
    const int iters = 4096;
    // flops per launch: threads x iterations x 8 chains x 2 lanes x 2 (FMA);
    // 4, 8 or 16 CTAs of 256 threads per SM, the best
    if (rc == PXSNE_OK && fp32_tflops) {
        double best = 0.0;
        for (int per_sm = 4; per_sm <= 16 && rc == PXSNE_OK; per_sm *= 2) {
            const int blocks = sms * per_sm;
            const double flops = (double)blocks * 256 * iters * 8 * 2 * 2;
            double ms = 0.0;
            auto go = [&] { k_ffma<false><<<blocks, 256, 0, st>>>(iters, 1.0f, (float *)sink); };
            if (time_ms(st, go, 1, &ms) || time_ms(st, go, 5, &ms)) rc = PXSNE_E_CUDA;
            else best = fmax(best, flops / (ms * 1e-3) / 1e12);
        }
        if (rc == PXSNE_OK) *fp32_tflops = best;
    }
    if (rc == PXSNE_OK && fp32_packed_tflops) {
        double best = 0.0;
        for (int per_sm = 4; per_sm <= 16 && rc == PXSNE_OK; per_sm *= 2) {
            const int blocks = sms * per_sm;
            const double flops = (double)blocks * 256 * iters * 8 * 2 * 2;
            double ms = 0.0;
            auto go = [&] { k_ffma<true><<<blocks, 256, 0, st>>>(iters, 1.0f, (float *)sink); };
            if (time_ms(st, go, 1, &ms) || time_ms(st, go, 5, &ms)) rc = PXSNE_E_CUDA;
            else best = fmax(best, flops / (ms * 1e-3) / 1e12);
        }
        if (rc == PXSNE_OK) *fp32_packed_tflops = best;
    }
    cudaFree(sink);
    return rc;
}
