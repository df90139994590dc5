// C ABI of the PixelSNE library (include/pxsne.h): context, buffers, the
// per-iteration schedule (captured once as a CUDA graph) and the inspection
// hooks.  All compute is in the kernels of tree.cu, forces.cu, update.cu and
// affinity.cu.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"

using namespace pxsne;

namespace {

thread_local std::string g_create_err;

int fail(pxsne_ctx *c, int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    else g_create_err = buf;
    return code;
}

int cuda_fail(pxsne_ctx *c, cudaError_t e, const char *what) {
    cudaGetLastError();
    return fail(c, e == cudaErrorMemoryAllocation ? PXSNE_E_OOM : PXSNE_E_CUDA, "%s: %s (%s)",
                what, cudaGetErrorName(e), cudaGetErrorString(e));
}

#define CK(c, x)                                              \
    do {                                                      \
        cudaError_t e_ = (x);                                 \
        if (e_ != cudaSuccess) return cuda_fail((c), e_, #x); \
    } while (0)

template <class T>
cudaError_t dalloc(pxsne_ctx *c, T **p, size_t count) {
    if (*p) {
        cudaFree(*p);
        *p = nullptr;
    }
    size_t bytes = count * sizeof(T);
    if (bytes == 0) bytes = 16;
    (void)c;
    return cudaMalloc(reinterpret_cast<void **>(p), bytes);
}

template <class T>
void dfree(T *&p) {
    if (p) cudaFree(p);
    p = nullptr;
}

void drop_graph(pxsne_ctx *c) {
    if (c->graph) {
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
}

void free_state(pxsne_ctx *c) {
    drop_graph(c);
    dfree(c->z); dfree(c->zhat); dfree(c->u); dfree(c->gains);
    dfree(c->Frep); dfree(c->Zi); dfree(c->Fattr); dfree(c->perm); dfree(c->rank);
    dfree(c->leaf_cnt); dfree(c->leaf_sx); dfree(c->leaf_sy); dfree(c->rec); dfree(c->recn);
    for (int k = 0; k < 2; k++) { dfree(c->lvl_cnt[k]); dfree(c->lvl_sx[k]); dfree(c->lvl_sy[k]); }
    dfree(c->leaf_start); dfree(c->blk_off); dfree(c->zpart); dfree(c->klpart);
    dfree(c->rp2); dfree(c->col2); dfree(c->val2);
    dfree(c->aperm); dfree(c->ainv); dfree(c->rl2); dfree(c->zp);
    free3(c);
    c->state_ready = false;
}

int check_params(const pxsne_params *p) {
    if (!p) return fail(nullptr, PXSNE_E_ARG, "params is NULL");
    if (p->log2_r < 1 || p->log2_r > kMaxL)
        return fail(nullptr, PXSNE_E_ARG, "log2_r = %d outside [1, %d]", p->log2_r, kMaxL);
    if (!(p->theta >= 0.f)) return fail(nullptr, PXSNE_E_ARG, "theta must be >= 0");
    if (!(p->eta > 0.f)) return fail(nullptr, PXSNE_E_ARG, "eta must be > 0");
    if (!(p->exaggeration > 0.f)) return fail(nullptr, PXSNE_E_ARG, "exaggeration must be > 0");
    if (!(p->momentum0 >= 0.f) || !(p->momentum1 >= 0.f) || p->momentum0 >= 1.f ||
        p->momentum1 >= 1.f)
        return fail(nullptr, PXSNE_E_ARG, "momentum must be in [0, 1)");
    if (!(p->min_gain > 0.f)) return fail(nullptr, PXSNE_E_ARG, "min_gain must be > 0");
    if (p->k < 1 || p->k > 256) return fail(nullptr, PXSNE_E_ARG, "k = %d outside [1, 256]", p->k);
    if (!(p->perplexity > 0.f) || p->perplexity > (float)p->k)
        return fail(nullptr, PXSNE_E_ARG, "perplexity must be in (0, k]");
    if (!(p->init_sigma > 0.f)) return fail(nullptr, PXSNE_E_ARG, "init_sigma must be > 0");
    if (p->centre_mode != 0 && p->centre_mode != 1)
        return fail(nullptr, PXSNE_E_ARG, "centre_mode must be 0 or 1");
    const int32_t side = 1 << p->log2_r;
    if (p->screen_x < 0 || p->screen_x > side || p->screen_y < 0 || p->screen_y > side)
        return fail(nullptr, PXSNE_E_ARG, "screen %d x %d outside [1, %d] (0: %d)", p->screen_x,
                    p->screen_y, side, side);
    if (p->knn_probe < 0 || p->knn_probe > 1792)
        return fail(nullptr, PXSNE_E_ARG, "knn_probe = %d outside [0, 1792]", p->knn_probe);
    if (p->knn_probe > 0 && p->knn_probe < (p->k + 127) / 128 + 1)
        return fail(nullptr, PXSNE_E_ARG,
                    "knn_probe = %d: at least ceil(k / 128) + 1 = %d tiles hold k other rows",
                    p->knn_probe, (p->k + 127) / 128 + 1);
    if (p->knn_explore < 0 || p->knn_explore > 8)
        return fail(nullptr, PXSNE_E_ARG, "knn_explore = %d outside [0, 8]", p->knn_explore);
    if (p->knn_explore > 0 && p->knn_probe == 0)
        return fail(nullptr, PXSNE_E_ARG, "knn_explore refines an approximate search (knn_probe > 0)");
    if (p->dim != 0 && p->dim != 2 && p->dim != 3)
        return fail(nullptr, PXSNE_E_ARG, "dim = %d: 2 or 3", p->dim);
    if (p->dim == 3 && (p->log2_r > kMaxL3 || p->screen_x || p->screen_y || p->centre_mode))
        return fail(nullptr, PXSNE_E_ARG,
                    "dim 3: log2_r <= %d, a cube of 2^L voxels, centres of mass", kMaxL3);
    return PXSNE_OK;
}

bool is3(const pxsne_ctx *c) { return c->p.dim == 3; }

int unsupported3(pxsne_ctx *c, const char *what) {
    return fail(c, PXSNE_E_UNSUPPORTED, "%s: 2-D embeddings only", what);
}

// Allocate the per-point and tree buffers for the current n and L.
int ensure_state(pxsne_ctx *c) {
    if ((c->z || c->z3) && c->L == c->p.log2_r) return PXSNE_OK;
    free_state(c);
    const int64_t n = c->n;
    c->L = c->p.log2_r;
    if (is3(c)) {
        // the 3-D state: the shared per-point buffers and the octree's
        CK(c, dalloc(c, &c->Zi, n));
        CK(c, dalloc(c, &c->perm, n));
        CK(c, dalloc(c, &c->rank, n));
        CK(c, alloc3(c));
        c->zblocks = (int)std::min<int64_t>(1024, std::max<int64_t>(1, (n + 4095) / 4096));
        CK(c, dalloc(c, &c->zpart, c->zblocks));
        c->klblocks = 304;
        CK(c, dalloc(c, &c->klpart, 2 * c->klblocks));
        return PXSNE_OK;
    }
    const int L = c->L;
    const int64_t leaves = int64_t(1) << (2 * L);
    const int64_t cells = rec_offset(L + 1);
    const int K1 = L < kPyrK ? L : kPyrK;
    const int64_t lvl = int64_t(1) << (2 * (L - K1));
    CK(c, dalloc(c, &c->z, n));
    CK(c, dalloc(c, &c->zhat, n));
    CK(c, dalloc(c, &c->u, n));
    CK(c, dalloc(c, &c->gains, n));
    CK(c, dalloc(c, &c->Frep, n));
    CK(c, dalloc(c, &c->Zi, n));
    CK(c, dalloc(c, &c->Fattr, n));
    CK(c, dalloc(c, &c->perm, n));
    CK(c, dalloc(c, &c->rank, n));
    CK(c, dalloc(c, &c->rp2, n + 1));
    CK(c, dalloc(c, &c->col2, (size_t)(c->nnz_pad > 0 ? c->nnz_pad : 4)));
    CK(c, dalloc(c, &c->val2, (size_t)(c->nnz_pad > 0 ? c->nnz_pad : 4)));
    CK(c, dalloc(c, &c->aperm, n));
    CK(c, dalloc(c, &c->ainv, n));
    CK(c, dalloc(c, &c->rl2, n));
    CK(c, dalloc(c, &c->zp, n));
    CK(c, dalloc(c, &c->leaf_cnt, leaves));
    CK(c, dalloc(c, &c->leaf_sx, leaves));
    CK(c, dalloc(c, &c->leaf_sy, leaves));
    // the leaf histogram starts from zeros; the pyramid clears what it read
    CK(c, cudaMemsetAsync(c->leaf_cnt, 0, (size_t)leaves * sizeof(uint32_t), c->stream));
    CK(c, cudaMemsetAsync(c->leaf_sx, 0, (size_t)leaves * sizeof(u64), c->stream));
    CK(c, cudaMemsetAsync(c->leaf_sy, 0, (size_t)leaves * sizeof(u64), c->stream));
    CK(c, dalloc(c, &c->rec, cells));
    CK(c, dalloc(c, &c->recn, cells));
    // records of empty cells are never written by the pyramid (nor read by
    // the traversal): they start as zeros
    CK(c, cudaMemsetAsync(c->rec, 0, (size_t)cells * sizeof(float4), c->stream));
    CK(c, dalloc(c, &c->leaf_start, leaves));
    CK(c, dalloc(c, &c->blk_off, lvl));
    for (int k = 0; k < 2; k++) {
        CK(c, dalloc(c, &c->lvl_cnt[k], lvl + 4));
        CK(c, dalloc(c, &c->lvl_sx[k], lvl + 4));
        CK(c, dalloc(c, &c->lvl_sy[k], lvl + 4));
    }
    c->zblocks = (int)((n + 4095) / 4096);
    if (c->zblocks > 1024) c->zblocks = 1024;
    if (c->zblocks < 1) c->zblocks = 1;
    CK(c, dalloc(c, &c->zpart, c->zblocks));
    c->klblocks = 304;
    CK(c, dalloc(c, &c->klpart, 2 * c->klblocks));
    return PXSNE_OK;
}

__global__ void k_iota(int n, uint32_t *p) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = (uint32_t)i;
}

__global__ void k_set_scalars(DevScalars *sc, double s0, double s1, int t, float theta, int L) {
    sc->s[0] = s0;
    sc->s[1] = s1;
    sc->t = t;
    sc->Z = 0.0;
    for (int p = 0; p < 2; p++) {
        sc->mm[p][0] = 0x7fffffffffffffffll;
        sc->mm[p][1] = 0x7fffffffffffffffll;
        sc->mm[p][2] = (long long)0x8000000000000000ull;
        sc->mm[p][3] = (long long)0x8000000000000000ull;
    }
    derive_scalars(sc, theta, L);
}

__global__ void k_fill_f2(int n, float2 *p, float v) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = make_float2(v, v);
}

// Tree and forces of the state just written (no rescale).
int prime(pxsne_ctx *c) {
    const int n = (int)c->n;
    if (is3(c)) {
        CK(c, launch_prime3(c, false));
        c->state_ready = true;
        return PXSNE_OK;
    }
    k_iota<<<(n + 255) / 256, 256, 0, c->stream>>>(n, c->perm);
    CK(c, cudaGetLastError());
    CK(c, launch_tree(c, false));
    // a state set from outside: P relabelled for its Morton order before the
    // first attraction
    CK(c, launch_relabel(c, c->stream));
    c->since_relabel = 0;
    CK(c, launch_forces(c));
    c->state_ready = true;
    return PXSNE_OK;
}

// The attraction's relabelled copy of P follows the Morton order of the last
// tree; it is refreshed every kRelabelEvery iterations (before the update).
cudaError_t relabel_if_due(pxsne_ctx *c) {
    if (is3(c) || c->since_relabel < kRelabelEvery) return cudaSuccess;
    c->since_relabel = 0;
    return launch_relabel(c, c->stream);
}

// One iteration.  With timing marks every kernel runs in order on the main
// stream.  Without, the attraction (which needs only the rescaled positions
// and P) runs on the side stream concurrently with the traversal: both are
// persistent grids sized to share the SMs (kTravCtasPerSm, kAttCtasPerSm),
// the traversal enqueued first.  The two join before the next update.
int one_iteration(pxsne_ctx *c, cudaEvent_t *marks = nullptr) {
    if (is3(c)) {
        CK(c, launch_iteration3(c));
        return PXSNE_OK;
    }
    CK(c, launch_update(c, marks));
    if (marks || !c->side) {
        CK(c, launch_tree(c, true, marks));
        CK(c, launch_forces(c, marks));
        return PXSNE_OK;
    }
    CK(c, launch_tree(c, true));
    CK(c, cudaEventRecord(c->ev_fork, c->stream));
    CK(c, launch_traverse_zsum(c));
    CK(c, cudaStreamWaitEvent(c->side, c->ev_fork, 0));
    CK(c, launch_attract(c, c->side));
    CK(c, cudaEventRecord(c->ev_join, c->side));
    CK(c, cudaStreamWaitEvent(c->stream, c->ev_join, 0));
    return PXSNE_OK;
}

const char *kGroupNames[KG_COUNT] = {"k_relabel", "k_update", "k_snap_hist", "k_pyr_pass",
                                     "k_perm_scatter", "k_bh_traverse", "k_attract",
                                     "k_zsum"};

int check_device(pxsne_ctx *c, uint32_t *flags_out) {
    CK(c, cudaStreamSynchronize(c->stream));
    unsigned err = 0;
    CK(c, cudaMemcpy(&err, &c->sc->err, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (flags_out) *flags_out = err;
    if (err) {
        const unsigned zero = 0;
        CK(c, cudaMemcpy(&c->sc->err, &zero, sizeof(unsigned), cudaMemcpyHostToDevice));
        return fail(c, PXSNE_E_DEVICE, "device error flags 0x%x%s%s%s%s%s", err,
                    (err & PXSNE_DEVERR_NONFINITE) ? " non-finite" : "",
                    (err & PXSNE_DEVERR_STACK) ? " stack-overflow" : "",
                    (err & PXSNE_DEVERR_BISECT) ? " bisection" : "",
                    (err & PXSNE_DEVERR_RANGE) ? " step-range" : "",
                    (err & PXSNE_DEVERR_TIMEOUT) ? " tensor-core-timeout" : "");
    }
    return PXSNE_OK;
}

int need_state(pxsne_ctx *c) {
    if (!c) return PXSNE_E_ARG;
    if (!c->state_ready) return fail(c, PXSNE_E_STATE, "no embedding state (call pxsne_init)");
    return PXSNE_OK;
}

}  // namespace

extern "C" {

void pxsne_default_params(pxsne_params *p) {
    if (!p) return;
    p->log2_r = 11;
    p->theta = 0.5f;
    p->eta = 200.f;
    p->exaggeration = 12.f;
    p->exag_iters = 250;
    p->momentum0 = 0.5f;
    p->momentum1 = 0.8f;
    p->momentum_switch = 250;
    p->min_gain = 0.01f;
    p->k = 90;
    p->perplexity = 30.f;
    p->init_sigma = 1e-4f;
    p->centre_mode = 0;
    p->screen_x = 0;
    p->screen_y = 0;
    p->knn_probe = 0;
    p->dim = 2;
    p->knn_explore = 0;
}

int pxsne_create(pxsne_ctx **out, const pxsne_params *p, void *stream) {
    if (!out) return fail(nullptr, PXSNE_E_ARG, "out is NULL");
    *out = nullptr;
    int rc = check_params(p);
    if (rc) return rc;
    pxsne_ctx *c = new (std::nothrow) pxsne_ctx();
    if (!c) return fail(nullptr, PXSNE_E_OOM, "host allocation");
    c->p = *p;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e == cudaSuccess) {
        if (stream) {
            c->stream = (cudaStream_t)stream;
        } else {
            e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
            c->own_stream = (e == cudaSuccess);
        }
    }
    if (e == cudaSuccess) {
        // the attraction's stream at the least priority: the traversal's
        // blocks, enqueued before it, are dispatched first
        int lo = 0, hi = 0;
        e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, lo);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = dalloc(c, &c->sc, 1);
    if (e == cudaSuccess) e = cudaMemset(c->sc, 0, sizeof(DevScalars));
    if (e != cudaSuccess) {
        cudaGetLastError();
        fail(nullptr, e == cudaErrorMemoryAllocation ? PXSNE_E_OOM : PXSNE_E_CUDA,
             "pxsne_create: %s", cudaGetErrorString(e));
        if (c->sc) cudaFree(c->sc);
        if (c->ev_join) cudaEventDestroy(c->ev_join);
        if (c->ev_fork) cudaEventDestroy(c->ev_fork);
        if (c->side) cudaStreamDestroy(c->side);
        if (c->own_stream) cudaStreamDestroy(c->stream);
        delete c;
        return e == cudaErrorMemoryAllocation ? PXSNE_E_OOM : PXSNE_E_CUDA;
    }
    *out = c;
    return PXSNE_OK;
}

void pxsne_destroy(pxsne_ctx *c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    free_state(c);
    dfree(c->rp); dfree(c->col); dfree(c->val); dfree(c->rowlen);
    dfree(c->knn_idx); dfree(c->knn_d2); dfree(c->beta);
    dfree(c->sc);
    for (auto &ev : c->knn_ev)
        if (ev) cudaEventDestroy(ev);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->side) cudaStreamDestroy(c->side);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
}

const char *pxsne_last_error(const pxsne_ctx *c) {
    return c ? c->err.c_str() : g_create_err.c_str();
}

int pxsne_affinities(pxsne_ctx *c, const float *X, int64_t n, int32_t D, float perplexity,
                     int x_on_device) {
    if (!c) return PXSNE_E_ARG;
    if (!X) return fail(c, PXSNE_E_ARG, "X is NULL");
    const int k = c->p.k;
    if (n < 2 || n > kMaxN) return fail(c, PXSNE_E_ARG, "n = %lld outside [2, 2^24]", (long long)n);
    if ((int64_t)k >= n) return fail(c, PXSNE_E_ARG, "k = %d must be < n = %lld", k, (long long)n);
    if (D < 1 || D > 256) return fail(c, PXSNE_E_UNSUPPORTED, "D = %d outside [1, 256]", D);
    if (perplexity <= 0.f) perplexity = c->p.perplexity;
    if (perplexity > (float)k) return fail(c, PXSNE_E_ARG, "perplexity > k");
    cudaStream_t st = c->stream;
    float *Xd = nullptr;
    const float *Xuse = X;
    if (!x_on_device) {
        CK(c, cudaMallocAsync(&Xd, (size_t)n * D * sizeof(float), st));
        CK(c, cudaMemcpyAsync(Xd, X, (size_t)n * D * sizeof(float), cudaMemcpyHostToDevice, st));
        Xuse = Xd;
    }
    {
        // X is checked for non-finite entries on the device, before any
        // state is replaced (a host loop over the n D values cost more than
        // the copy)
        unsigned *flag = nullptr, bad = 0u;
        CK(c, cudaMallocAsync(&flag, sizeof(unsigned), st));
        CK(c, cudaMemsetAsync(flag, 0, sizeof(unsigned), st));
        CK(c, launch_nonfinite(c, Xuse, n * D, flag, st));
        CK(c, cudaMemcpyAsync(&bad, flag, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
        CK(c, cudaFreeAsync(flag, st));
        CK(c, cudaStreamSynchronize(st));
        if (bad) {
            if (Xd) CK(c, cudaFreeAsync(Xd, st));
            return fail(c, PXSNE_E_ARG, "X has a non-finite entry");
        }
    }
    free_state(c);
    dfree(c->rp); dfree(c->col); dfree(c->val); dfree(c->rowlen);
    dfree(c->knn_idx); dfree(c->knn_d2); dfree(c->beta);
    c->n = n;
    c->D = D;
    c->nnz = 0;
    CK(c, dalloc(c, &c->knn_idx, (size_t)n * k));
    CK(c, dalloc(c, &c->knn_d2, (size_t)n * k));
    CK(c, dalloc(c, &c->beta, (size_t)n));
    c->knn_k = k;
    CK(c, launch_knn(c, Xuse, n, D, k, c->knn_idx, c->knn_d2));
    if (Xd) CK(c, cudaFreeAsync(Xd, st));
    float *pcond = nullptr;
    CK(c, cudaMallocAsync(&pcond, (size_t)n * k * sizeof(float), st));
    CK(c, launch_perplexity(c, c->knn_d2, n, k, perplexity, pcond, c->beta));
    std::string where;
    cudaError_t e = build_symmetric_csr(c, c->knn_idx, pcond, n, k, where);
    if (e != cudaSuccess) return cuda_fail(c, e, where.c_str());
    CK(c, cudaFreeAsync(pcond, st));
    return check_device(c, nullptr);
}

int pxsne_set_P(pxsne_ctx *c, int64_t n, const int64_t *row_ptr, const int32_t *col,
                const float *val) {
    if (!c) return PXSNE_E_ARG;
    if (n < 2 || n > kMaxN || !row_ptr) return fail(c, PXSNE_E_ARG, "bad n or row_ptr");
    if (row_ptr[0] != 0) return fail(c, PXSNE_E_ARG, "row_ptr[0] != 0");
    for (int64_t i = 0; i < n; i++)
        if (row_ptr[i + 1] < row_ptr[i]) return fail(c, PXSNE_E_ARG, "row_ptr not monotone");
    const int64_t nnz = row_ptr[n];
    if (nnz > 0 && (!col || !val)) return fail(c, PXSNE_E_ARG, "col/val NULL");
    for (int64_t i = 0; i < n; i++)
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; e++) {
            if (col[e] < 0 || col[e] >= n || col[e] == i)
                return fail(c, PXSNE_E_ARG, "bad column %d in row %lld", col[e], (long long)i);
            if (!(val[e] >= 0.f) || !std::isfinite(val[e]))
                return fail(c, PXSNE_E_ARG, "bad value in row %lld", (long long)i);
        }
    // rows padded to multiples of 4 (padding: column = row, value 0)
    std::vector<int64_t> rp(n + 1);
    std::vector<int32_t> len(n);
    rp[0] = 0;
    for (int64_t i = 0; i < n; i++) {
        len[i] = (int32_t)(row_ptr[i + 1] - row_ptr[i]);
        rp[i + 1] = rp[i] + ((len[i] + 3) & ~3);
    }
    const int64_t nnz_pad = rp[n];
    std::vector<int32_t> pc(nnz_pad > 0 ? nnz_pad : 4);
    std::vector<float> pv(nnz_pad > 0 ? nnz_pad : 4);
    for (int64_t i = 0; i < n; i++) {
        int64_t o = rp[i];
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; e++, o++) {
            pc[o] = col[e];
            pv[o] = val[e];
        }
        for (; o < rp[i + 1]; o++) {
            pc[o] = (int32_t)i;
            pv[o] = 0.f;
        }
    }
    free_state(c);
    dfree(c->rp); dfree(c->col); dfree(c->val); dfree(c->rowlen);
    dfree(c->knn_idx); dfree(c->knn_d2); dfree(c->beta);
    c->knn_k = 0;
    c->n = n;
    c->nnz = nnz;
    c->nnz_pad = nnz_pad;
    CK(c, dalloc(c, &c->rp, n + 1));
    CK(c, dalloc(c, &c->rowlen, n));
    CK(c, dalloc(c, &c->col, pc.size()));
    CK(c, dalloc(c, &c->val, pv.size()));
    CK(c, cudaMemcpyAsync(c->rp, rp.data(), (n + 1) * 8, cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaMemcpyAsync(c->rowlen, len.data(), n * 4, cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaMemcpyAsync(c->col, pc.data(), pc.size() * 4, cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaMemcpyAsync(c->val, pv.data(), pv.size() * 4, cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return PXSNE_OK;
}

int pxsne_init(pxsne_ctx *c, const float *Y0, int y_on_device, uint64_t seed) {
    if (!c) return PXSNE_E_ARG;
    if (c->n < 2 || !c->rp) return fail(c, PXSNE_E_STATE, "no affinities (call pxsne_affinities)");
    int rc = ensure_state(c);
    if (rc) return rc;
    cudaStream_t st = c->stream;
    const int64_t n = c->n;
    if (is3(c)) {
        if (!Y0) return fail(c, PXSNE_E_UNSUPPORTED, "dim 3: the start Y0 must be given");
        float *Yd3 = nullptr;
        double *scr = nullptr;
        CK(c, cudaMallocAsync(&scr, 8 * sizeof(double), st));
        const float *Y3 = Y0;
        if (!y_on_device) {
            CK(c, cudaMallocAsync(&Yd3, (size_t)n * 12, st));
            CK(c, cudaMemcpyAsync(Yd3, Y0, (size_t)n * 12, cudaMemcpyHostToDevice, st));
            Y3 = Yd3;
        }
        const unsigned zero3 = 0;
        CK(c, cudaMemcpyAsync(&c->sc->err, &zero3, sizeof(unsigned), cudaMemcpyHostToDevice, st));
        CK(c, launch_init3(c, Y3, scr));
        rc = prime(c);
        if (rc) return rc;
        if (Yd3) CK(c, cudaFreeAsync(Yd3, st));
        CK(c, cudaFreeAsync(scr, st));
        rc = check_device(c, nullptr);
        if (rc) c->state_ready = false;
        return rc;
    }
    float *Yd = nullptr;
    uint32_t *mm = nullptr;
    CK(c, cudaMallocAsync(&mm, 4 * sizeof(uint32_t), st));
    const float *Yuse = Y0;
    if (!Y0 || !y_on_device) {
        CK(c, cudaMallocAsync(&Yd, (size_t)n * 2 * sizeof(float), st));
        if (Y0) {
            CK(c, cudaMemcpyAsync(Yd, Y0, (size_t)n * 8, cudaMemcpyHostToDevice, st));
        } else {
            CK(c, launch_philox_y0(c, Yd, seed, c->p.init_sigma));
        }
        Yuse = Yd;
    }
    const unsigned zero = 0;
    CK(c, cudaMemcpyAsync(&c->sc->err, &zero, sizeof(unsigned), cudaMemcpyHostToDevice, st));
    CK(c, launch_init_map(c, Yuse, mm));
    rc = prime(c);
    if (rc) return rc;
    if (Yd) CK(c, cudaFreeAsync(Yd, st));
    CK(c, cudaFreeAsync(mm, st));
    rc = check_device(c, nullptr);
    if (rc) {
        c->state_ready = false;
        return rc;
    }
    return PXSNE_OK;
}

int pxsne_set_state(pxsne_ctx *c, const uint32_t *z, const double *s, const float *u,
                    const float *gains, int32_t t) {
    if (!c) return PXSNE_E_ARG;
    if (c->n < 2 || !c->rp) return fail(c, PXSNE_E_STATE, "no affinities");
    if (!z || !s || !(s[0] > 0.0) || !(s[1] > 0.0) || t < 0)
        return fail(c, PXSNE_E_ARG, "bad z, s or t");
    int rc = ensure_state(c);
    if (rc) return rc;
    const int n = (int)c->n;
    cudaStream_t st = c->stream;
    if (is3(c)) {
        if (!(s[2] > 0.0)) return fail(c, PXSNE_E_ARG, "bad s");
        // host rows of three values into the 4-wide device vectors
        CK(c, cudaMemcpy2DAsync(c->z3, 16, z, 12, 12, (size_t)n, cudaMemcpyHostToDevice, st));
        CK(c, launch_fill3(c, c->u3, 0.f, 0.f, 0.f));
        CK(c, launch_fill3(c, c->gains3, 1.f, 1.f, 1.f));
        if (u) CK(c, cudaMemcpy2DAsync(c->u3, 16, u, 12, 12, (size_t)n, cudaMemcpyHostToDevice, st));
        if (gains)
            CK(c, cudaMemcpy2DAsync(c->gains3, 16, gains, 12, 12, (size_t)n,
                                    cudaMemcpyHostToDevice, st));
        CK(c, launch_set_scalars3(c, s, t));
        rc = prime(c);
        if (rc) return rc;
        return check_device(c, nullptr);
    }
    CK(c, cudaMemcpyAsync(c->z, z, (size_t)n * 8, cudaMemcpyHostToDevice, st));
    if (u) CK(c, cudaMemcpyAsync(c->u, u, (size_t)n * 8, cudaMemcpyHostToDevice, st));
    else k_fill_f2<<<(n + 255) / 256, 256, 0, st>>>(n, c->u, 0.f);
    if (gains) CK(c, cudaMemcpyAsync(c->gains, gains, (size_t)n * 8, cudaMemcpyHostToDevice, st));
    else k_fill_f2<<<(n + 255) / 256, 256, 0, st>>>(n, c->gains, 1.f);
    k_set_scalars<<<1, 1, 0, st>>>(c->sc, s[0], s[1], t, c->p.theta, c->L);
    CK(c, cudaGetLastError());
    rc = prime(c);
    if (rc) return rc;
    return check_device(c, nullptr);
}

int pxsne_step(pxsne_ctx *c, int32_t iters) {
    int rc = need_state(c);
    if (rc) return rc;
    if (iters < 0) return fail(c, PXSNE_E_ARG, "iters < 0");
    if (iters == 0) return PXSNE_OK;
    if (!c->graph && c->stream != nullptr && c->stream != cudaStreamLegacy &&
        c->stream != cudaStreamPerThread) {
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            int r = one_iteration(c);
            cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
            if (r == PXSNE_OK && e2 == cudaSuccess && g) {
                if (cudaGraphInstantiate(&c->graph, g, 0) != cudaSuccess) c->graph = nullptr;
            }
            if (g) cudaGraphDestroy(g);
        }
        cudaGetLastError();
    }
    for (int32_t k = 0; k < iters; k++) {
        CK(c, relabel_if_due(c));
        if (c->graph) {
            CK(c, cudaGraphLaunch(c->graph, c->stream));
        } else {
            rc = one_iteration(c);
            if (rc) return rc;
        }
        c->since_relabel++;
    }
    return PXSNE_OK;
}

int pxsne_step_profiled(pxsne_ctx *c, int32_t iters, double *group_ms, int32_t n_groups,
                        double *total_ms) {
    int rc = need_state(c);
    if (rc) return rc;
    if (is3(c)) return unsupported3(c, "pxsne_step_profiled");
    if (iters < 1 || !group_ms || n_groups < KG_COUNT)
        return fail(c, PXSNE_E_ARG, "need iters >= 1 and %d group slots", (int)KG_COUNT);
    // destroyed on every return path, the early ones included
    struct Events {
        std::vector<cudaEvent_t> v;
        ~Events() {
            for (auto e : v)
                if (e) cudaEventDestroy(e);
        }
    } evs;
    evs.v.assign((size_t)iters * (KG_COUNT + 1) + 2, nullptr);
    std::vector<cudaEvent_t> &ev = evs.v;
    for (auto &e : ev) CK(c, cudaEventCreate(&e));
    cudaEvent_t *t0 = &ev[ev.size() - 2], *t1 = &ev[ev.size() - 1];
    CK(c, cudaMemsetAsync(c->sc->tot, 0, sizeof(c->sc->tot), c->stream));
    CK(c, cudaMemsetAsync(c->sc->lvl, 0, sizeof(c->sc->lvl), c->stream));
    CK(c, cudaEventRecord(*t0, c->stream));
    for (int32_t k = 0; k < iters; k++) {
        cudaEvent_t *m = &ev[(size_t)k * (KG_COUNT + 1)];
        CK(c, cudaEventRecord(m[KG_RELABEL], c->stream));
        CK(c, relabel_if_due(c));
        rc = one_iteration(c, m);
        if (rc) break;
        c->since_relabel++;
        // work counters of this iteration's state: one more traversal after
        // the iteration's last mark, outside the timed groups
        CK(c, launch_count_traversal(c));
        CK(c, launch_accumulate_counters(c));
    }
    if (!rc) {
        CK(c, cudaEventRecord(*t1, c->stream));
        // the sums over the run replace the last state's counters
        CK(c, cudaMemcpyAsync(&c->sc->n_accept, c->sc->tot, sizeof(c->sc->tot),
                              cudaMemcpyDeviceToDevice, c->stream));
        CK(c, cudaEventSynchronize(*t1));
        for (int g = 0; g < KG_COUNT; g++) group_ms[g] = 0.0;
        for (int32_t k = 0; k < iters; k++) {
            cudaEvent_t *m = &ev[(size_t)k * (KG_COUNT + 1)];
            for (int g = 0; g < KG_COUNT; g++) {
                float ms = 0.f;
                CK(c, cudaEventElapsedTime(&ms, m[g], m[g + 1]));
                group_ms[g] += ms;
            }
        }
        if (total_ms) {
            float ms = 0.f;
            CK(c, cudaEventElapsedTime(&ms, *t0, *t1));
            *total_ms = ms;
        }
    }
    if (rc) return rc;
    return check_device(c, nullptr);
}

const char *pxsne_kernel_group_name(int32_t g) {
    return (g >= 0 && g < KG_COUNT) ? kGroupNames[g] : nullptr;
}

int pxsne_set_schedule(pxsne_ctx *c, const pxsne_params *p) {
    if (!c || !p) return PXSNE_E_ARG;
    pxsne_params q = c->p;
    q.eta = p->eta;
    q.exaggeration = p->exaggeration;
    q.exag_iters = p->exag_iters;
    q.momentum0 = p->momentum0;
    q.momentum1 = p->momentum1;
    q.momentum_switch = p->momentum_switch;
    q.min_gain = p->min_gain;
    int rc = check_params(&q);
    if (rc) return fail(c, rc, "%s", g_create_err.c_str());
    c->p = q;
    drop_graph(c);  // the update kernel's arguments are part of the graph
    return PXSNE_OK;
}

int pxsne_kl(pxsne_ctx *c, double *out) {
    int rc = need_state(c);
    if (rc) return rc;
    if (!out) return fail(c, PXSNE_E_ARG, "out is NULL");
    double *d = nullptr;
    CK(c, cudaMallocAsync(&d, sizeof(double), c->stream));
    if (is3(c)) CK(c, launch_kl3(c, d));
    else CK(c, launch_kl(c, d));
    CK(c, cudaMemcpyAsync(out, d, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaFreeAsync(d, c->stream));
    return check_device(c, nullptr);
}

int pxsne_get_Y(pxsne_ctx *c, float *Y, int32_t *pix, int on_device) {
    int rc = need_state(c);
    if (rc) return rc;
    if (on_device < 0 || on_device > 2) return fail(c, PXSNE_E_ARG, "on_device = %d", on_device);
    const bool async = on_device == 2;
    cudaStream_t st = c->stream;
    const int64_t n = c->n;
    const size_t row = is3(c) ? 12 : 8;  // bytes of one point's values
    float *scratch = nullptr;
    CK(c, cudaMallocAsync(&scratch, 32, st));
    float *Yd = Y;
    int32_t *Pd = pix;
    if (!on_device) {
        Yd = nullptr;
        Pd = nullptr;
        if (Y) CK(c, cudaMallocAsync(&Yd, (size_t)n * row, st));
        if (pix) CK(c, cudaMallocAsync(&Pd, (size_t)n * row, st));
    }
    if (is3(c)) CK(c, launch_centre_y3(c, Yd, Pd, reinterpret_cast<double *>(scratch)));
    else CK(c, launch_centre_y(c, Yd, Pd, scratch));
    if (!on_device) {
        if (Y) {
            CK(c, cudaMemcpyAsync(Y, Yd, (size_t)n * row, cudaMemcpyDeviceToHost, st));
            CK(c, cudaFreeAsync(Yd, st));
        }
        if (pix) {
            CK(c, cudaMemcpyAsync(pix, Pd, (size_t)n * row, cudaMemcpyDeviceToHost, st));
            CK(c, cudaFreeAsync(Pd, st));
        }
    }
    CK(c, cudaFreeAsync(scratch, st));
    if (async) {
        CK(c, cudaGetLastError());
        return PXSNE_OK;
    }
    return check_device(c, nullptr);
}

int pxsne_nbr_precision(pxsne_ctx *c, int32_t k, const int32_t *knn_hd, int32_t kh,
                        int on_device, double *precision, int32_t *hits) {
    int rc = need_state(c);
    if (rc) return rc;
    if (is3(c)) return unsupported3(c, "pxsne_nbr_precision");
    if (!knn_hd) {
        if (!c->knn_idx) return fail(c, PXSNE_E_STATE, "no neighbour lists: pass knn_hd");
        knn_hd = c->knn_idx;
        kh = c->knn_k;
        on_device = 1;
    }
    if (k < 1 || k > 32 || k > kh || (int64_t)k >= c->n)
        return fail(c, PXSNE_E_ARG, "need 1 <= k <= min(32, kh) and k < n");
    cudaStream_t st = c->stream;
    const int64_t n = c->n;
    int32_t *dh = nullptr, *dk = nullptr;
    unsigned long long *dt = nullptr;
    CK(c, cudaMallocAsync(&dh, (size_t)n * 4, st));
    CK(c, cudaMallocAsync(&dt, 8, st));
    CK(c, cudaMemsetAsync(dt, 0, 8, st));
    const int32_t *kd = knn_hd;
    if (!on_device) {
        CK(c, cudaMallocAsync(&dk, (size_t)n * kh * 4, st));
        CK(c, cudaMemcpyAsync(dk, knn_hd, (size_t)n * kh * 4, cudaMemcpyHostToDevice, st));
        kd = dk;
    }
    CK(c, launch_nbr_precision(c, k, kd, kh, dh, dt));
    unsigned long long tot = 0;
    CK(c, cudaMemcpyAsync(&tot, dt, 8, cudaMemcpyDeviceToHost, st));
    if (hits) CK(c, cudaMemcpyAsync(hits, dh, (size_t)n * 4, cudaMemcpyDeviceToHost, st));
    CK(c, cudaFreeAsync(dh, st));
    CK(c, cudaFreeAsync(dt, st));
    if (dk) CK(c, cudaFreeAsync(dk, st));
    rc = check_device(c, nullptr);
    if (rc) return rc;
    if (precision) *precision = (double)tot / ((double)k * (double)n);
    return PXSNE_OK;
}

int pxsne_sync(pxsne_ctx *c, uint32_t *dev_errors) {
    if (!c) return PXSNE_E_ARG;
    return check_device(c, dev_errors);
}

int pxsne_get_sizes(pxsne_ctx *c, int64_t *n, int64_t *nnz) {
    if (!c) return PXSNE_E_ARG;
    if (n) *n = c->n;
    if (nnz) *nnz = c->nnz;
    return PXSNE_OK;
}

int pxsne_get_P(pxsne_ctx *c, int64_t *row_ptr, int32_t *col, float *val) {
    if (!c) return PXSNE_E_ARG;
    if (!c->rp) return fail(c, PXSNE_E_STATE, "no affinities");
    cudaStream_t st = c->stream;
    const int64_t n = c->n;
    std::vector<int64_t> rp(n + 1);
    std::vector<int32_t> len(n);
    CK(c, cudaMemcpyAsync(rp.data(), c->rp, (n + 1) * 8, cudaMemcpyDeviceToHost, st));
    CK(c, cudaMemcpyAsync(len.data(), c->rowlen, n * 4, cudaMemcpyDeviceToHost, st));
    std::vector<int32_t> pc;
    std::vector<float> pv;
    if (col) pc.resize(c->nnz_pad);
    if (val) pv.resize(c->nnz_pad);
    if (col && c->nnz_pad)
        CK(c, cudaMemcpyAsync(pc.data(), c->col, c->nnz_pad * 4, cudaMemcpyDeviceToHost, st));
    if (val && c->nnz_pad)
        CK(c, cudaMemcpyAsync(pv.data(), c->val, c->nnz_pad * 4, cudaMemcpyDeviceToHost, st));
    int rc = check_device(c, nullptr);
    if (rc) return rc;
    int64_t o = 0;
    if (row_ptr) row_ptr[0] = 0;
    for (int64_t i = 0; i < n; i++) {
        for (int32_t a = 0; a < len[i]; a++, o++) {
            if (col) col[o] = pc[rp[i] + a];
            if (val) val[o] = pv[rp[i] + a];
        }
        if (row_ptr) row_ptr[i + 1] = o;
    }
    return PXSNE_OK;
}

int pxsne_get_knn(pxsne_ctx *c, int32_t *idx, float *d2, float *beta) {
    if (!c) return PXSNE_E_ARG;
    if (!c->knn_idx) return fail(c, PXSNE_E_STATE, "no neighbour lists (P was injected?)");
    cudaStream_t st = c->stream;
    const size_t nk = (size_t)c->n * c->knn_k;
    if (idx) CK(c, cudaMemcpyAsync(idx, c->knn_idx, nk * 4, cudaMemcpyDeviceToHost, st));
    if (d2) CK(c, cudaMemcpyAsync(d2, c->knn_d2, nk * 4, cudaMemcpyDeviceToHost, st));
    if (beta) CK(c, cudaMemcpyAsync(beta, c->beta, c->n * 4, cudaMemcpyDeviceToHost, st));
    return check_device(c, nullptr);
}

int pxsne_get_state(pxsne_ctx *c, uint32_t *z, double *s, float *u, float *gains, int32_t *t) {
    int rc = need_state(c);
    if (rc) return rc;
    cudaStream_t st = c->stream;
    const size_t n = (size_t)c->n;
    if (is3(c)) {
        if (z) CK(c, cudaMemcpy2DAsync(z, 12, c->z3, 16, 12, n, cudaMemcpyDeviceToHost, st));
        if (u) CK(c, cudaMemcpy2DAsync(u, 12, c->u3, 16, 12, n, cudaMemcpyDeviceToHost, st));
        if (gains)
            CK(c, cudaMemcpy2DAsync(gains, 12, c->gains3, 16, 12, n, cudaMemcpyDeviceToHost, st));
    } else {
        if (z) CK(c, cudaMemcpyAsync(z, c->z, n * 8, cudaMemcpyDeviceToHost, st));
        if (u) CK(c, cudaMemcpyAsync(u, c->u, n * 8, cudaMemcpyDeviceToHost, st));
        if (gains) CK(c, cudaMemcpyAsync(gains, c->gains, n * 8, cudaMemcpyDeviceToHost, st));
    }
    DevScalars h;
    CK(c, cudaMemcpyAsync(&h, c->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, st));
    rc = check_device(c, nullptr);
    if (rc) return rc;
    if (s) {
        if (is3(c)) {
            for (int d = 0; d < 3; d++) s[d] = h.s3[d];
        } else {
            s[0] = h.s[0];
            s[1] = h.s[1];
        }
    }
    if (t) *t = h.t;
    return PXSNE_OK;
}

int pxsne_get_tree(pxsne_ctx *c, int32_t level, uint32_t *cnt, uint64_t *sx, uint64_t *sy,
                   uint32_t *morton) {
    int rc = need_state(c);
    if (rc) return rc;
    if (is3(c)) return unsupported3(c, "pxsne_get_tree (use pxsne_get_tree3)");
    if (level < 0 || level > c->L) return fail(c, PXSNE_E_ARG, "level out of range");
    if (level == c->L && (sx || sy) && c->p.centre_mode != 0)
        return fail(c, PXSNE_E_UNSUPPORTED, "the geometric-centre tree keeps no coordinate sums");
    cudaStream_t st = c->stream;
    const size_t cells = size_t(1) << (2 * level);
    if (cnt) {
        uint32_t *d = nullptr;
        CK(c, cudaMallocAsync(&d, cells * 4, st));
        CK(c, launch_level_counts(c, level, d));
        CK(c, cudaMemcpyAsync(cnt, d, cells * 4, cudaMemcpyDeviceToHost, st));
        CK(c, cudaFreeAsync(d, st));
    }
    if (level == c->L && (sx || sy)) {
        u64 *d = nullptr;
        CK(c, cudaMallocAsync(&d, cells * 16, st));
        CK(c, launch_leaf_hist(c, nullptr, d, d + cells));
        if (sx) CK(c, cudaMemcpyAsync(sx, d, cells * 8, cudaMemcpyDeviceToHost, st));
        if (sy) CK(c, cudaMemcpyAsync(sy, d + cells, cells * 8, cudaMemcpyDeviceToHost, st));
        CK(c, cudaFreeAsync(d, st));
    }
    if (morton) {
        uint32_t *d = nullptr;
        CK(c, cudaMallocAsync(&d, (size_t)c->n * 4, st));
        CK(c, launch_morton_keys(c, d));
        CK(c, cudaMemcpyAsync(morton, d, (size_t)c->n * 4, cudaMemcpyDeviceToHost, st));
        CK(c, cudaFreeAsync(d, st));
    }
    return check_device(c, nullptr);
}

int pxsne_get_forces(pxsne_ctx *c, float *Frep, float *Zi, float *Fattr, double *Z) {
    int rc = need_state(c);
    if (rc) return rc;
    cudaStream_t st = c->stream;
    const size_t n = (size_t)c->n;
    if (is3(c)) {
        if (Frep)
            CK(c, cudaMemcpy2DAsync(Frep, 12, c->Frep3, 16, 12, n, cudaMemcpyDeviceToHost, st));
        if (Fattr)
            CK(c, cudaMemcpy2DAsync(Fattr, 12, c->Fattr3, 16, 12, n, cudaMemcpyDeviceToHost, st));
    } else {
        if (Frep) CK(c, cudaMemcpyAsync(Frep, c->Frep, n * 8, cudaMemcpyDeviceToHost, st));
        if (Fattr) CK(c, cudaMemcpyAsync(Fattr, c->Fattr, n * 8, cudaMemcpyDeviceToHost, st));
    }
    if (Zi) CK(c, cudaMemcpyAsync(Zi, c->Zi, n * 4, cudaMemcpyDeviceToHost, st));
    if (Z) CK(c, cudaMemcpyAsync(Z, &c->sc->Z, sizeof(double), cudaMemcpyDeviceToHost, st));
    return check_device(c, nullptr);
}

int pxsne_get_counters(pxsne_ctx *c, uint64_t *n_accept, uint64_t *n_test,
                       uint64_t *n_warp_steps, uint64_t *n_nodes) {
    int rc = need_state(c);
    if (rc) return rc;
    if (is3(c)) return unsupported3(c, "pxsne_get_counters");
    DevScalars h;
    CK(c, cudaMemcpyAsync(&h, c->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, c->stream));
    rc = check_device(c, nullptr);
    if (rc) return rc;
    if (n_accept) *n_accept = h.n_accept;
    if (n_test) *n_test = h.n_test;
    if (n_warp_steps) *n_warp_steps = h.n_steps;
    if (n_nodes) *n_nodes = h.n_nodes;
    return PXSNE_OK;
}

int pxsne_get_level_counters(pxsne_ctx *c, uint64_t *counts, int32_t levels) {
    int rc = need_state(c);
    if (rc) return rc;
    if (is3(c)) return unsupported3(c, "pxsne_get_level_counters");
    if (!counts || levels < c->L + 1)
        return fail(c, PXSNE_E_ARG, "need room for %d levels", c->L + 1);
    DevScalars h;
    CK(c, cudaMemcpyAsync(&h, c->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, c->stream));
    rc = check_device(c, nullptr);
    if (rc) return rc;
    for (int l = 0; l < levels; l++)
        for (int q = 0; q < 3; q++) counts[3 * l + q] = l <= c->L ? h.lvl[l][q] : 0ull;
    return PXSNE_OK;
}

int pxsne_get_knn_pruning(pxsne_ctx *c, uint64_t *skipped_pairs, uint64_t *pairs) {
    if (!c) return PXSNE_E_ARG;
    DevScalars h;
    CK(c, cudaMemcpyAsync(&h, c->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, c->stream));
    int rc = check_device(c, nullptr);
    if (rc) return rc;
    const bool tc_path = c->knn_path == 1;
    if (skipped_pairs) *skipped_pairs = tc_path ? h.knn_skip : 0u;
    if (pairs) *pairs = tc_path ? (uint64_t)c->knn_tiles * (uint64_t)c->knn_tiles : 0u;
    return PXSNE_OK;
}

int pxsne_get_knn_counters(pxsne_ctx *c, uint64_t *exact, uint64_t *inserted, int32_t *path) {
    if (!c) return PXSNE_E_ARG;
    DevScalars h;
    CK(c, cudaMemcpyAsync(&h, c->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, c->stream));
    int rc = check_device(c, nullptr);
    if (rc) return rc;
    if (exact) *exact = h.knn_exact;
    if (inserted) *inserted = h.knn_insert;
    if (path) *path = c->knn_path;
    return PXSNE_OK;
}

int pxsne_test_bounded_wait(pxsne_ctx *c, int32_t polls, uint32_t *flags) {
    if (!c || polls < 1 || polls > 65536) return fail(c, PXSNE_E_ARG, "polls outside [1, 65536]");
    launch_wait_probe(c, polls);
    CK(c, cudaGetLastError());
    return check_device(c, flags);
}

int pxsne_get_knn_time(pxsne_ctx *c, double *search_ms) {
    if (!c || !search_ms) return PXSNE_E_ARG;
    if (!c->knn_timed) return fail(c, PXSNE_E_STATE, "no neighbour search has run");
    CK(c, cudaEventSynchronize(c->knn_ev[1]));
    float ms = 0.f;
    CK(c, cudaEventElapsedTime(&ms, c->knn_ev[0], c->knn_ev[1]));
    *search_ms = ms;
    return PXSNE_OK;
}

int64_t pxsne_device_bytes(const pxsne_ctx *c) {
    if (!c) return 0;
    int64_t b = sizeof(DevScalars);
    const int64_t n = c->n;
    if (c->rp) b += (n + 1) * 8 + n * 4 + c->nnz_pad * 8;
    if (c->knn_idx) b += n * c->knn_k * 8 + n * 4;
    if (c->z) {
        const int L = c->L;
        const int64_t leaves = int64_t(1) << (2 * L);
        const int K1 = L < kPyrK ? L : kPyrK;
        const int64_t lvl = int64_t(1) << (2 * (L - K1));
        b += n * (8 + 16 + 8 + 8 + 8 + 4 + 8 + 4 + 4);
        b += leaves * (4 + 8 + 8 + 4) + rec_offset(L + 1) * 20 + lvl * 4 + 2 * (lvl + 4) * 20;
        b += (int64_t)c->zblocks * 8 + (int64_t)c->klblocks * 16;
        b += (n + 1) * 8 + c->nnz_pad * 8 + n * (4 + 4 + 4 + 8);  // relabelled P, maps, zp
    }
    return b;
}

}  // extern "C"

// ---------------------------------------------------------------- checkpoints
// A checkpoint is one flat file: a 144-byte header, then the payload
//   row_ptr[n+1] int64, col[nnz] int32, val[nnz] float32   (P as CSR)
//   z[2n] uint32, u[2n] float32, gains[2n] float32           (the state)
// in the byte order of the machine that wrote it (little-endian on every
// supported host).  The header's checksum is FNV-1a (64-bit offset basis and
// prime) applied to the payload taken as consecutive little-endian 64-bit
// words, the last one zero-padded.
namespace {

struct CheckpointHeader {
    char magic[8];          // "PXSNECK" + NUL
    uint32_t version;       // 1
    uint32_t header_bytes;  // sizeof(CheckpointHeader)
    pxsne_params params;    // the context's parameters and schedule
    int64_t n, nnz;
    int32_t t, pad1;
    double s[2];
    uint64_t payload_bytes;
    uint64_t checksum;
};
static_assert(sizeof(pxsne_params) == 72, "pxsne_params layout");
static_assert(sizeof(CheckpointHeader) == 144, "checkpoint header layout");
constexpr char kMagic[8] = {'P', 'X', 'S', 'N', 'E', 'C', 'K', 0};

struct Fnv64Words {
    uint64_t h = 14695981039346656037ull;
    unsigned char carry[8];
    int nc = 0;
    void word(uint64_t w) {
        h ^= w;
        h *= 1099511628211ull;
    }
    void add(const void *p, size_t bytes) {
        const unsigned char *b = static_cast<const unsigned char *>(p);
        while (bytes && nc) {
            carry[nc++] = *b++;
            bytes--;
            if (nc == 8) {
                uint64_t w;
                memcpy(&w, carry, 8);
                word(w);
                nc = 0;
            }
        }
        for (; bytes >= 8; b += 8, bytes -= 8) {
            uint64_t w;
            memcpy(&w, b, 8);
            word(w);
        }
        while (bytes--) carry[nc++] = *b++;
    }
    uint64_t done() {
        if (nc) {
            memset(carry + nc, 0, 8 - nc);
            uint64_t w;
            memcpy(&w, carry, 8);
            word(w);
            nc = 0;
        }
        return h;
    }
};

uint64_t payload_bytes_of(int64_t n, int64_t nnz) {
    return 8ull * (uint64_t)(n + 1) + 8ull * (uint64_t)nnz + 24ull * (uint64_t)n;
}

}  // namespace

int pxsne_save(pxsne_ctx *c, const char *path) {
    int rc = need_state(c);
    if (rc) return rc;
    if (is3(c)) return unsupported3(c, "pxsne_save");
    if (!path) return fail(c, PXSNE_E_ARG, "path is NULL");
    const int64_t n = c->n, nnz = c->nnz;
    std::vector<int64_t> rp(n + 1);
    std::vector<int32_t> col(nnz > 0 ? nnz : 1);
    std::vector<float> val(nnz > 0 ? nnz : 1);
    if ((rc = pxsne_get_P(c, rp.data(), col.data(), val.data()))) return rc;
    std::vector<uint32_t> z(2 * n);
    std::vector<float> u(2 * n), g(2 * n);
    CheckpointHeader h;
    memset(&h, 0, sizeof(h));
    if ((rc = pxsne_get_state(c, z.data(), h.s, u.data(), g.data(), &h.t))) return rc;
    memcpy(h.magic, kMagic, 8);
    h.version = 1;
    h.header_bytes = sizeof(CheckpointHeader);
    h.params = c->p;
    h.n = n;
    h.nnz = nnz;
    h.payload_bytes = payload_bytes_of(n, nnz);
    Fnv64Words f;
    f.add(rp.data(), 8 * (size_t)(n + 1));
    f.add(col.data(), 4 * (size_t)nnz);
    f.add(val.data(), 4 * (size_t)nnz);
    f.add(z.data(), 8 * (size_t)n);
    f.add(u.data(), 8 * (size_t)n);
    f.add(g.data(), 8 * (size_t)n);
    h.checksum = f.done();
    // written to a temporary name, then renamed over the target
    const std::string tmp = std::string(path) + ".tmp";
    FILE *fp = fopen(tmp.c_str(), "wb");
    if (!fp) return fail(c, PXSNE_E_ARG, "cannot open %s for writing", tmp.c_str());
    bool ok = fwrite(&h, sizeof(h), 1, fp) == 1;
    ok = ok && fwrite(rp.data(), 8, (size_t)(n + 1), fp) == (size_t)(n + 1);
    ok = ok && (nnz == 0 || fwrite(col.data(), 4, (size_t)nnz, fp) == (size_t)nnz);
    ok = ok && (nnz == 0 || fwrite(val.data(), 4, (size_t)nnz, fp) == (size_t)nnz);
    ok = ok && fwrite(z.data(), 8, (size_t)n, fp) == (size_t)n;
    ok = ok && fwrite(u.data(), 8, (size_t)n, fp) == (size_t)n;
    ok = ok && fwrite(g.data(), 8, (size_t)n, fp) == (size_t)n;
    ok = (fclose(fp) == 0) && ok;
    if (!ok || rename(tmp.c_str(), path) != 0) {
        remove(tmp.c_str());
        return fail(c, PXSNE_E_ARG, "writing %s failed", path);
    }
    return PXSNE_OK;
}

int pxsne_load(pxsne_ctx **out, const char *path, void *stream) {
    if (!out) return fail(nullptr, PXSNE_E_ARG, "out is NULL");
    *out = nullptr;
    if (!path) return fail(nullptr, PXSNE_E_ARG, "path is NULL");
    FILE *fp = fopen(path, "rb");
    if (!fp) return fail(nullptr, PXSNE_E_ARG, "cannot open %s", path);
    struct Closer {
        FILE *f;
        ~Closer() { fclose(f); }
    } closer{fp};
    CheckpointHeader h;
    if (fread(&h, sizeof(h), 1, fp) != 1) return fail(nullptr, PXSNE_E_ARG, "%s: short header", path);
    if (memcmp(h.magic, kMagic, 8) != 0) return fail(nullptr, PXSNE_E_ARG, "%s: not a checkpoint", path);
    if (h.version != 1 || h.header_bytes != sizeof(CheckpointHeader))
        return fail(nullptr, PXSNE_E_UNSUPPORTED, "%s: version %u", path, h.version);
    if (h.n < 2 || h.n > kMaxN || h.nnz < 0 || h.nnz > (int64_t(1) << 40) || h.t < 0 ||
        !(std::isfinite(h.s[0]) && h.s[0] > 0.0) || !(std::isfinite(h.s[1]) && h.s[1] > 0.0) ||
        h.payload_bytes != payload_bytes_of(h.n, h.nnz))
        return fail(nullptr, PXSNE_E_ARG, "%s: bad sizes in the header", path);
    int rc = check_params(&h.params);
    if (rc) return rc;
    const int64_t n = h.n, nnz = h.nnz;
    std::vector<int64_t> rp(n + 1);
    std::vector<int32_t> col(nnz > 0 ? nnz : 1);
    std::vector<float> val(nnz > 0 ? nnz : 1);
    std::vector<uint32_t> z(2 * n);
    std::vector<float> u(2 * n), g(2 * n);
    bool ok = fread(rp.data(), 8, (size_t)(n + 1), fp) == (size_t)(n + 1);
    ok = ok && (nnz == 0 || fread(col.data(), 4, (size_t)nnz, fp) == (size_t)nnz);
    ok = ok && (nnz == 0 || fread(val.data(), 4, (size_t)nnz, fp) == (size_t)nnz);
    ok = ok && fread(z.data(), 8, (size_t)n, fp) == (size_t)n;
    ok = ok && fread(u.data(), 8, (size_t)n, fp) == (size_t)n;
    ok = ok && fread(g.data(), 8, (size_t)n, fp) == (size_t)n;
    if (!ok) return fail(nullptr, PXSNE_E_ARG, "%s: truncated", path);
    unsigned char extra;
    if (fread(&extra, 1, 1, fp) != 0) return fail(nullptr, PXSNE_E_ARG, "%s: trailing bytes", path);
    Fnv64Words f;
    f.add(rp.data(), 8 * (size_t)(n + 1));
    f.add(col.data(), 4 * (size_t)nnz);
    f.add(val.data(), 4 * (size_t)nnz);
    f.add(z.data(), 8 * (size_t)n);
    f.add(u.data(), 8 * (size_t)n);
    f.add(g.data(), 8 * (size_t)n);
    if (f.done() != h.checksum) return fail(nullptr, PXSNE_E_ARG, "%s: checksum mismatch", path);
    pxsne_ctx *c = nullptr;
    if ((rc = pxsne_create(&c, &h.params, stream))) return rc;
    rc = pxsne_set_P(c, n, rp.data(), col.data(), val.data());
    if (!rc) rc = pxsne_set_state(c, z.data(), h.s, u.data(), g.data(), h.t);
    if (rc) {
        fail(nullptr, rc, "%s: %s", path, c->err.c_str());
        pxsne_destroy(c);
        return rc;
    }
    *out = c;
    return PXSNE_OK;
}

int pxsne_get_params(const pxsne_ctx *c, pxsne_params *p) {
    if (!c || !p) return PXSNE_E_ARG;
    *p = c->p;
    return PXSNE_OK;
}

int pxsne_test_stack_limit(pxsne_ctx *c, int32_t entries) {
    if (!c) return PXSNE_E_ARG;
    if (entries != 0 && (entries < 4 || entries > kTravStack))
        return fail(c, PXSNE_E_ARG, "entries must be 0 or in [4, %d]", kTravStack);
    const int lim = entries;  // 0: the full stack
    CK(c, cudaMemcpyAsync(&c->sc->stack_limit, &lim, sizeof(int), cudaMemcpyHostToDevice,
                          c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return PXSNE_OK;
}

int pxsne_get_tree3(pxsne_ctx *c, int32_t level, uint32_t *cnt, uint64_t *sx, uint64_t *sy,
                    uint64_t *sz, uint32_t *morton) {
    int rc = need_state(c);
    if (rc) return rc;
    if (!is3(c)) return fail(c, PXSNE_E_UNSUPPORTED, "pxsne_get_tree3: 3-D embeddings only");
    if (level < 0 || level > c->L) return fail(c, PXSNE_E_ARG, "level out of range");
    cudaStream_t st = c->stream;
    const size_t cells = size_t(1) << (3 * level);
    const int64_t at = level_offset3(level);
    if (level < c->L) {
        if (cnt) CK(c, cudaMemcpyAsync(cnt, c->cnt3 + at, cells * 4, cudaMemcpyDeviceToHost, st));
    } else {
        // the leaves: rebuilt from z (the iteration clears its own once read)
        uint32_t *dc = nullptr;
        u64 *ds = nullptr;
        CK(c, cudaMallocAsync(&dc, cells * 4, st));
        CK(c, cudaMallocAsync(&ds, cells * 24, st));
        CK(c, launch_leaf_hist3(c, dc, ds));
        if (cnt) CK(c, cudaMemcpyAsync(cnt, dc, cells * 4, cudaMemcpyDeviceToHost, st));
        uint64_t *out[3] = {sx, sy, sz};
        for (int d = 0; d < 3; d++)
            if (out[d])
                CK(c, cudaMemcpyAsync(out[d], ds + d * cells, cells * 8, cudaMemcpyDeviceToHost,
                                      st));
        CK(c, cudaFreeAsync(dc, st));
        CK(c, cudaFreeAsync(ds, st));
    }
    if (morton) {
        uint32_t *d = nullptr;
        CK(c, cudaMallocAsync(&d, (size_t)c->n * 4, st));
        CK(c, launch_morton3(c, d));
        CK(c, cudaMemcpyAsync(morton, d, (size_t)c->n * 4, cudaMemcpyDeviceToHost, st));
        CK(c, cudaFreeAsync(d, st));
    }
    return check_device(c, nullptr);
}
