// PCA to d_out dimensions, the standard pre-processing the paper applies to all
// datasets before P is built (Sec. 5.1.1).
//
//   k_colsum_f64   column means (FP64 accumulation)
//   k_cov          covariance (X - mu)^T (X - mu) / (n - 1): 64 x 64 output
//                  tiles per CTA over a slice of rows in FP32, slices added in
//                  FP64
//   k_project      (X - mu) V for the leading eigenvectors V
// The eigenvectors come from block subspace iteration with a Rayleigh-Ritz
// step on the host in FP64 (cyclic Jacobi on the small projected matrix).
#include <algorithm>
#include <cmath>
#include <random>
#include <vector>

#include "common.cuh"

namespace pxsne {
namespace {

__global__ void k_colsum_f64(int64_t n, int D, const float *__restrict__ X, double *sum) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= D) return;
    double s = 0.0;
    for (int64_t r = blockIdx.y; r < n; r += gridDim.y) s += X[r * D + c];
    atomicAdd(&sum[c], s);
}

constexpr int kCT = 64;    // covariance tile
constexpr int kCR = 32;    // rows per smem stage
constexpr int kCRows = 4096;  // rows per slice (grid z)

__global__ void __launch_bounds__(256)
    k_cov(int64_t n, int D, const float *__restrict__ X, const double *__restrict__ sum,
          double *cov) {
    __shared__ float sa[kCR][kCT + 1], sb[kCR][kCT + 1];
    const int a0 = blockIdx.x * kCT, b0 = blockIdx.y * kCT;
    if (b0 < a0) return;  // lower triangle mirrored at the end
    const int64_t r0 = (int64_t)blockIdx.z * kCRows;
    const int64_t r1 = r0 + kCRows < n ? r0 + kCRows : n;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    float acc[4][4] = {};
    for (int64_t rb = r0; rb < r1; rb += kCR) {
        for (int q = tid; q < kCR * kCT; q += 256) {
            const int rr = q / kCT, cc = q % kCT;
            const int64_t r = rb + rr;
            float va = 0.f, vb = 0.f;
            if (r < r1) {
                if (a0 + cc < D) va = X[r * D + a0 + cc] - (float)(sum[a0 + cc] / (double)n);
                if (b0 + cc < D) vb = X[r * D + b0 + cc] - (float)(sum[b0 + cc] / (double)n);
            }
            sa[rr][cc] = va;
            sb[rr][cc] = vb;
        }
        __syncthreads();
        for (int rr = 0; rr < kCR; rr++) {
            float xa[4], xb[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                xa[u] = sa[rr][ty + 16 * u];
                xb[u] = sb[rr][tx + 16 * u];
            }
#pragma unroll
            for (int u = 0; u < 4; u++)
#pragma unroll
                for (int v = 0; v < 4; v++) acc[u][v] = fmaf(xa[u], xb[v], acc[u][v]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; u++)
#pragma unroll
        for (int v = 0; v < 4; v++) {
            const int a = a0 + ty + 16 * u, b = b0 + tx + 16 * v;
            if (a < D && b < D && b >= a) atomicAdd(&cov[(int64_t)a * D + b], (double)acc[u][v]);
        }
}

__global__ void k_project(int64_t n, int D, int dout, const float *__restrict__ X,
                          const double *__restrict__ sum, const float *__restrict__ V,
                          float *__restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n * dout) return;
    const int64_t r = i / dout;
    const int c = (int)(i % dout);
    float s = 0.f;
    for (int a = 0; a < D; a++) s = fmaf(X[r * D + a] - (float)(sum[a] / (double)n), V[(int64_t)a * dout + c], s);
    out[i] = s;
}

// Symmetric eigendecomposition of a small b x b matrix (cyclic Jacobi, FP64):
// on return A's diagonal holds the eigenvalues and U (row-major) the
// eigenvectors as columns.
void jacobi_eig(int b, std::vector<double> &A, std::vector<double> &U) {
    U.assign((size_t)b * b, 0.0);
    for (int i = 0; i < b; i++) U[(size_t)i * b + i] = 1.0;
    for (int sweep = 0; sweep < 60; sweep++) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < b; i++)
            for (int j = 0; j < b; j++) {
                const double v = A[(size_t)i * b + j] * A[(size_t)i * b + j];
                tot += v;
                if (i != j) off += v;
            }
        if (off <= 1e-30 * tot || off == 0.0) break;
        for (int p = 0; p < b; p++)
            for (int q = p + 1; q < b; q++) {
                const double apq = A[(size_t)p * b + q];
                if (std::fabs(apq) < 1e-300) continue;
                const double app = A[(size_t)p * b + p], aqq = A[(size_t)q * b + q];
                // rotation angle zeroing A[p][q]: tan(2 phi) = 2 apq / (aqq - app)
                const double tau = (aqq - app) / (2.0 * apq);
                const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
                const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
                for (int k = 0; k < b; k++) {  // columns p, q
                    const double akp = A[(size_t)k * b + p], akq = A[(size_t)k * b + q];
                    A[(size_t)k * b + p] = c * akp - s * akq;
                    A[(size_t)k * b + q] = s * akp + c * akq;
                }
                for (int k = 0; k < b; k++) {  // rows p, q
                    const double apk = A[(size_t)p * b + k], aqk = A[(size_t)q * b + k];
                    A[(size_t)p * b + k] = c * apk - s * aqk;
                    A[(size_t)q * b + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < b; k++) {
                    const double ukp = U[(size_t)k * b + p], ukq = U[(size_t)k * b + q];
                    U[(size_t)k * b + p] = c * ukp - s * ukq;
                    U[(size_t)k * b + q] = s * ukp + c * ukq;
                }
            }
    }
}

// Modified Gram-Schmidt on the b columns of Q (D x b, row-major).
void orthonormalize(int D, int b, std::vector<double> &Q) {
    for (int j = 0; j < b; j++) {
        for (int i = 0; i < j; i++) {
            double d = 0.0;
            for (int a = 0; a < D; a++) d += Q[(size_t)a * b + i] * Q[(size_t)a * b + j];
            for (int a = 0; a < D; a++) Q[(size_t)a * b + j] -= d * Q[(size_t)a * b + i];
        }
        double nn = 0.0;
        for (int a = 0; a < D; a++) nn += Q[(size_t)a * b + j] * Q[(size_t)a * b + j];
        nn = std::sqrt(nn);
        for (int a = 0; a < D; a++) Q[(size_t)a * b + j] = nn > 0 ? Q[(size_t)a * b + j] / nn : 0.0;
    }
}

}  // namespace
}  // namespace pxsne

using namespace pxsne;

extern "C" int pxsne_pca(const float *X, int64_t n, int32_t D, int32_t dout, float *Xout,
                         float *components, float *eigenvalues, int on_device, uint64_t seed) {
    if (!X || !Xout || n < 2 || D < 1 || dout < 1 || dout > D) return PXSNE_E_ARG;
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) return PXSNE_E_CUDA;
    int rc = PXSNE_OK;
    auto ck = [&](cudaError_t e) {
        if (e != cudaSuccess && rc == PXSNE_OK) {
            cudaGetLastError();
            rc = e == cudaErrorMemoryAllocation ? PXSNE_E_OOM : PXSNE_E_CUDA;
        }
        return rc == PXSNE_OK;
    };
    float *dX = nullptr, *dO = nullptr, *dV = nullptr;
    double *dsum = nullptr, *dcov = nullptr;
    const float *Xs = X;
    if (!on_device) {
        ck(cudaMallocAsync(&dX, (size_t)n * D * 4, st));
        if (rc == PXSNE_OK) ck(cudaMemcpyAsync(dX, X, (size_t)n * D * 4, cudaMemcpyHostToDevice, st));
        Xs = dX;
    }
    ck(cudaMallocAsync(&dsum, (size_t)D * 8, st));
    ck(cudaMallocAsync(&dcov, (size_t)D * D * 8, st));
    std::vector<double> C((size_t)D * D), mean(D);
    if (rc == PXSNE_OK) {
        ck(cudaMemsetAsync(dsum, 0, (size_t)D * 8, st));
        ck(cudaMemsetAsync(dcov, 0, (size_t)D * D * 8, st));
        const dim3 gs((D + 127) / 128, 256);
        k_colsum_f64<<<gs, 128, 0, st>>>(n, D, Xs, dsum);
        const dim3 gc((D + kCT - 1) / kCT, (D + kCT - 1) / kCT, (unsigned)((n + kCRows - 1) / kCRows));
        k_cov<<<gc, 256, 0, st>>>(n, D, Xs, dsum, dcov);
        ck(cudaGetLastError());
        ck(cudaMemcpyAsync(C.data(), dcov, (size_t)D * D * 8, cudaMemcpyDeviceToHost, st));
        ck(cudaStreamSynchronize(st));
    }
    std::vector<double> lam(dout);
    std::vector<float> Vf((size_t)D * dout);
    if (rc == PXSNE_OK) {
        for (int a = 0; a < D; a++)
            for (int b = a; b < D; b++) {
                const double v = C[(size_t)a * D + b] / (double)(n - 1);
                C[(size_t)a * D + b] = v;
                C[(size_t)b * D + a] = v;
            }
        // block subspace iteration on C, then Rayleigh-Ritz
        const int b = std::min<int>(D, dout + 16);
        std::vector<double> Q((size_t)D * b), Y((size_t)D * b);
        std::mt19937_64 rng(seed);
        std::normal_distribution<double> nd(0.0, 1.0);
        for (auto &q : Q) q = nd(rng);
        orthonormalize(D, b, Q);
        const int iters = (b == D) ? 1 : 40;
        for (int it = 0; it < iters; it++) {
            std::fill(Y.begin(), Y.end(), 0.0);
            for (int a = 0; a < D; a++)
                for (int c = 0; c < D; c++) {
                    const double cac = C[(size_t)a * D + c];
                    const double *qc = &Q[(size_t)c * b];
                    double *ya = &Y[(size_t)a * b];
                    for (int j = 0; j < b; j++) ya[j] += cac * qc[j];
                }
            Q.swap(Y);
            orthonormalize(D, b, Q);
        }
        // T = Q^T C Q
        std::vector<double> CQ((size_t)D * b, 0.0), T((size_t)b * b, 0.0), U;
        for (int a = 0; a < D; a++)
            for (int c = 0; c < D; c++) {
                const double cac = C[(size_t)a * D + c];
                for (int j = 0; j < b; j++) CQ[(size_t)a * b + j] += cac * Q[(size_t)c * b + j];
            }
        for (int i = 0; i < b; i++)
            for (int j = 0; j < b; j++) {
                double s = 0.0;
                for (int a = 0; a < D; a++) s += Q[(size_t)a * b + i] * CQ[(size_t)a * b + j];
                T[(size_t)i * b + j] = s;
            }
        for (int i = 0; i < b; i++)
            for (int j = i + 1; j < b; j++) {
                const double v = 0.5 * (T[(size_t)i * b + j] + T[(size_t)j * b + i]);
                T[(size_t)i * b + j] = T[(size_t)j * b + i] = v;
            }
        jacobi_eig(b, T, U);
        std::vector<int> order(b);
        for (int i = 0; i < b; i++) order[i] = i;
        std::sort(order.begin(), order.end(),
                  [&](int x, int y) { return T[(size_t)x * b + x] > T[(size_t)y * b + y]; });
        for (int c = 0; c < dout; c++) {
            const int o = order[c];
            lam[c] = T[(size_t)o * b + o];
            // v = Q u_o, sign fixed so that the largest |component| is positive
            double best = 0.0;
            int ba = 0;
            std::vector<double> v(D, 0.0);
            for (int a = 0; a < D; a++) {
                double s = 0.0;
                for (int j = 0; j < b; j++) s += Q[(size_t)a * b + j] * U[(size_t)j * b + o];
                v[a] = s;
                if (std::fabs(s) > best) {
                    best = std::fabs(s);
                    ba = a;
                }
            }
            const double sg = v[ba] < 0 ? -1.0 : 1.0;
            for (int a = 0; a < D; a++) Vf[(size_t)a * dout + c] = (float)(sg * v[a]);
        }
        if (components) std::copy(Vf.begin(), Vf.end(), components);
        if (eigenvalues)
            for (int c = 0; c < dout; c++) eigenvalues[c] = (float)lam[c];
        ck(cudaMallocAsync(&dV, (size_t)D * dout * 4, st));
        float *out = Xout;
        if (!on_device) ck(cudaMallocAsync(&dO, (size_t)n * dout * 4, st)), out = dO;
        if (rc == PXSNE_OK) {
            ck(cudaMemcpyAsync(dV, Vf.data(), (size_t)D * dout * 4, cudaMemcpyHostToDevice, st));
            k_project<<<(unsigned)((n * dout + 255) / 256), 256, 0, st>>>(n, D, dout, Xs, dsum, dV, out);
            ck(cudaGetLastError());
            if (!on_device)
                ck(cudaMemcpyAsync(Xout, dO, (size_t)n * dout * 4, cudaMemcpyDeviceToHost, st));
            ck(cudaStreamSynchronize(st));
        }
    }
    if (dX) cudaFreeAsync(dX, st);
    if (dO) cudaFreeAsync(dO, st);
    if (dV) cudaFreeAsync(dV, st);
    if (dsum) cudaFreeAsync(dsum, st);
    if (dcov) cudaFreeAsync(dcov, st);
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    return rc;
}
