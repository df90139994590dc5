/*
 * pxsne.h - C ABI of the GB300 (sm_103a) PixelSNE library.
 *
 * PixelSNE (Kim et al., arXiv 1611.02568) is t-SNE whose 2-D output lives on a
 * screen of r x r pixels (Sec. 3.1, Eq. z1/z2).  Each gradient iteration
 * assigns the points to a fixed pixel-aligned quadtree (Sec. 4.1), takes the
 * Barnes-Hut repulsion against it (Sec. 3.3, Eq. bh_criteria), the attraction
 * over the sparse affinity matrix P (Sec. 3.3, Eq. grad) and a gradient step
 * followed by the screen-driven rescale (Sec. 4.2).  This library runs all of
 * it in hand-written CUDA kernels on one GPU.
 *
 * Conventions shared by every call:
 *  - Return value: PXSNE_OK (0) or a negative PXSNE_E_* code; the message of the
 *    last failure is available from pxsne_last_error().  No C++ exception
 *    crosses this boundary.
 *  - Device work is enqueued on the context's CUDA stream.  Calls that return
 *    data to the host synchronise that stream; errors raised on the device
 *    (non-finite gradient, traversal stack overflow) are reported by the next
 *    synchronising call as PXSNE_E_DEVICE.
 *  - Pointers marked "host or device" are read as device pointers when the
 *    matching *_on_device flag is non-zero (they must then be device memory of
 *    the context's device, ordered before the call on the context's stream or
 *    already complete); otherwise as host memory.
 *  - The caller owns every buffer it passes; the library copies what it needs
 *    and keeps no pointer to caller memory after a call returns.  The library
 *    owns, and frees in pxsne_destroy(), all device memory it allocates.
 *  - One context may be used by one host thread at a time.
 *
 * Positions.  The state holds each point as unsigned 32-bit fixed point per
 * axis: z_d in [0, R_d) ulps, pixel = z_d >> (32 - L) in [0, r_d) for an
 * r_1 x r_2 screen (R_d = r_d 2^(32 - L); 2^32 for a 2^L x 2^L screen).
 * t-SNE's own coordinates are y_d = s_d * z_d (+ an arbitrary offset), where the
 * per-axis scale s_d (y-units per ulp) carries the compensation of
 * Eq. beta_scaling (s_d^2 = beta_d).
 */
#ifndef PXSNE_H
#define PXSNE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PXSNE_OK 0
#define PXSNE_E_ARG (-1)         /* invalid argument */
#define PXSNE_E_OOM (-2)         /* device or host allocation failed */
#define PXSNE_E_CUDA (-3)        /* a CUDA runtime call failed */
#define PXSNE_E_STATE (-4)       /* call out of order (e.g. step before init) */
#define PXSNE_E_DEVICE (-5)      /* error flagged by a kernel */
#define PXSNE_E_UNSUPPORTED (-6) /* a valid request this library does not support */

/* Device error flags, read back by pxsne_sync (and by every synchronising
 * call, which then returns PXSNE_E_DEVICE and clears them). */
#define PXSNE_DEVERR_NONFINITE 1u   /* non-finite gradient or step */
#define PXSNE_DEVERR_STACK 2u       /* BH traversal stack overflow */
#define PXSNE_DEVERR_BISECT 4u      /* a perplexity row did not converge */
#define PXSNE_DEVERR_RANGE 8u       /* step clamped: |u / s| beyond 2^58 ulps */
#define PXSNE_DEVERR_TIMEOUT 16u    /* a bounded wait on the tensor cores gave up */

typedef struct pxsne_ctx pxsne_ctx;

/* Parameters of one embedding.  Defaults (pxsne_default_params): L = 11,
 * theta = 0.5, eta = 200, exaggeration 12 for 250 iterations, momentum 0.5
 * then 0.8 from iteration 250, min_gain 0.01, k = 90, perplexity 30,
 * init_sigma 1e-4, centre of mass, a square 2^L x 2^L screen.
 *
 * Screens of r_1 x r_2 pixels (Sec. 4.2's per-axis r_d; e.g. 1024 x 768 with
 * L = 10) keep the quadtree's root at the padded 2^L x 2^L square, so the
 * tree's depth is L on both axes; axis d then spans R_d = r_d 2^(32 - L) ulps,
 * z_d in [0, R_d) and its pixel z_d >> (32 - L) in [0, r_d).  The init map
 * and the rescale use R_d in place of 2^32 (pxsne_init, pxsne_step).
 *
 * dim = 3 embeds in 3-D (the extension of the paper's introduction): a voxel
 * grid of 2^L per axis (1 <= L <= 9, no screen_x / screen_y), each point z_d
 * in [0, 2^32) ulps on three axes, the quadtree an octree of eight children
 * per cell (Morton bits x, y, z from the least significant), the cell
 * diagonal of Eq. bh_criteria W sqrt(s_0^2 + s_1^2 + s_2^2); every other step
 * is the 2-D method with a third coordinate.  With dim = 3 the buffers of
 * pxsne_init (Y0, which must be given), pxsne_get_Y, pxsne_get_state,
 * pxsne_set_state and pxsne_get_forces hold three values per point and s
 * three; pxsne_get_tree3 reads the octree; the geometric-centre tree,
 * pxsne_step_profiled, the counters, pxsne_nbr_precision, checkpoints and
 * pxsne_kl_noalloc are 2-D only (PXSNE_E_UNSUPPORTED). */
typedef struct pxsne_params {
    int32_t log2_r;          /* L: screen is 2^L x 2^L pixels, 1 <= L <= 14 (Sec. 4.1 depth) */
    float theta;             /* Barnes-Hut threshold, >= 0 (Eq. bh_criteria) */
    float eta;               /* learning rate (y-units) */
    float exaggeration;      /* factor on P in the attraction while t < exag_iters */
    int32_t exag_iters;
    float momentum0;         /* momentum while t < momentum_switch */
    float momentum1;         /* momentum from then on */
    int32_t momentum_switch;
    float min_gain;          /* lower bound of the per-coordinate gains */
    int32_t k;               /* neighbours per row of P; >= 1 and < n */
    float perplexity;        /* target perplexity u of each row, 0 < u <= k */
    float init_sigma;        /* std-dev of the random initial embedding */
    int32_t centre_mode;     /* 0: cell centre of mass; 1: geometric cell centre (Sec. 4.1) */
    int32_t screen_x;        /* screen width r_1 in pixels, 1 <= r_1 <= 2^L; 0: 2^L */
    int32_t screen_y;        /* screen height r_2 in pixels, 1 <= r_2 <= 2^L; 0: 2^L */
    int32_t knn_probe;       /* 0: exact neighbour search; W in [ceil(k / 128) + 1,
                                1792]: approximate (see pxsne_affinities) */
    int32_t dim;             /* embedding dimension: 2 (0 means 2) or 3 (see below) */
    int32_t knn_explore;     /* rounds of neighbour exploring after an approximate
                                search, 0 .. 8 (needs knn_probe > 0; see
                                pxsne_affinities) */
} pxsne_params;

void pxsne_default_params(pxsne_params *p);

/* Create a context on the current CUDA device.  p is copied.  stream: a
 * cudaStream_t to enqueue on, or NULL to let the library create its own
 * non-blocking stream.  Fails with PXSNE_E_ARG on out-of-range parameters. */
int pxsne_create(pxsne_ctx **out, const pxsne_params *p, void *stream);

/* Free all device memory and the context.  NULL is ignored. */
void pxsne_destroy(pxsne_ctx *ctx);

/* Message of the last failure on ctx (or of the last failed pxsne_create when
 * ctx is NULL).  Valid until the next call on the same context. */
const char *pxsne_last_error(const pxsne_ctx *ctx);

/* Build the sparse affinity matrix P (Sec. 3.2-3.3; Sec. 4.3 replaces the
 * neighbour search, here done exactly by brute force):
 *   - the k nearest neighbours of each row of X by squared Euclidean
 *     distance, self excluded, ties to the lower index;
 *   - p_{j|i} proportional to exp(-beta_i d2_ij) with beta_i set by bisection
 *     so that each row's entropy is ln(perplexity);
 *   - p_ij = (p_{j|i} + p_{i|j}) / (2n) on the union pattern, stored as CSR.
 * With knn_probe = W > 0 the neighbour search is approximate (the role of
 * Sec. 4.3's random-projection trees): each pivot cell of the search's
 * locality order is split further by random-projection hyperplanes (each
 * bisecting two of the segment's rows) into tiles of 128 nearby rows, and the
 * rows of a tile are searched only against the W tiles whose centroids are
 * nearest to their tile's (their own tile first), with exact FP32 distances;
 * the neighbour lists are then the k nearest within those tiles, the same on
 * every run (tensor-core search only; the FP32 check path stays exact).  W
 * must be at least ceil(k / 128) + 1, so that W tiles hold k other rows even
 * when the own tile is the last, partial one.  knn_explore = R > 0 then
 * refines them by R rounds of Sec. 4.3's neighbour exploring (LargeVis'
 * "a neighbour of my neighbour is likely my neighbour"): in each round every
 * row tests, with the same exact FP32 distance, every entry of the lists of
 * its first min(k, 16) neighbours, and keeps the k nearest of its list and
 * those (each round reads the previous round's lists only, so a round's
 * result does not depend on the order of the rows).
 * X: host or device, row-major n x D float32, 2 <= n <= 2^24, 1 <= D <= 256
 * (the shared-memory tiles of the search bound D further for large k; an
 * unsupported size returns an error).  perplexity <= 0 uses the
 * context's parameter.  Replaces any previous P and clears the embedding
 * state.  Synchronises.  A non-finite entry of X (checked on the device)
 * returns PXSNE_E_ARG and leaves the context as it was.  Row convergence
 * failures set PXSNE_DEVERR_BISECT and return PXSNE_E_DEVICE (P is still
 * built from the last bracket). */
int pxsne_affinities(pxsne_ctx *ctx, const float *X, int64_t n, int32_t D,
                     float perplexity, int x_on_device);

/* Start an embedding (Sec. 3.1, Eq. z1/z2): Y0 (host or device, n x 2 float32,
 * y-units) is mapped per axis onto the fixed-point screen,
 *   z_d = min(R_d - 1, floor((y_d - min_d) * R_d / (max_d - min_d))),
 *   s_d = (max_d - min_d) / R_d,
 * in FP64, R_d the axis' extent in ulps (2^32 on a square 2^L screen; an axis
 * with zero extent maps to z_d = 0, s_d = 1 / R_d).  Y0 == NULL
 * draws Y0 ~ N(0, init_sigma^2 I) from `seed` with Philox4x32-10 (Salmon et al.
 * 2011) and the Box-Muller transform.  Velocities are zeroed, gains set to 1,
 * the iteration counter to 0, and the forces of the initial state computed.
 * Requires P (pxsne_affinities or pxsne_set_P). */
int pxsne_init(pxsne_ctx *ctx, const float *Y0, int y_on_device, uint64_t seed);

/* Run `iters` >= 0 gradient iterations, asynchronously on the context's
 * stream.  Iteration t: g = 4 (alpha_t Fattr - Frep / Z) (Eq. grad), the
 * gains/momentum step u = mu_t u - eta gain g, zhat = z + rint(u / s), then the
 * screen-driven rescale z_d = floor((zhat_d - min_d) R_d / (max_d - min_d + 1)),
 * s_d <- (s_d (max_d - min_d + 1)) / R_d (Sec. 4.2; R_d = 2^32 on a square
 * 2^L screen, r_d 2^(32 - L) in general), then the pixel-aligned tree
 * and forces of the new state (Sec. 4.1, Eq. bh_criteria, Eq. grad).
 * Returns enqueue errors only. */
int pxsne_step(pxsne_ctx *ctx, int32_t iters);

/* Checkpoint and resume (Sec. 5 runs the method for a fixed number of
 * iterations; a long run can be stopped and continued).  pxsne_save writes P
 * (as CSR), the state (z, s, u, gains, t) and the parameters and schedule of
 * ctx to one file at `path` (written under path + ".tmp", then renamed over
 * path); the iteration needs nothing else, so a run continued from the file
 * reproduces the one that wrote it bit for bit.  The neighbour lists of the
 * last pxsne_affinities are not kept (pxsne_nbr_precision of a loaded context
 * needs the caller's lists).  Synchronises.  Returns PXSNE_E_STATE before
 * pxsne_init, PXSNE_E_ARG if the file cannot be written.
 *
 * File layout (byte order of the writing host, little-endian on every
 * supported one): a 144-byte header {char magic[8] = "PXSNECK\0"; uint32
 * version = 1; uint32 header bytes = 144; pxsne_params (72 bytes);
 * int64 n, nnz; int32 t, 0; double s[2]; uint64 payload bytes; uint64
 * checksum}, then row_ptr[n+1] int64, col[nnz] int32, val[nnz] float32,
 * z[2n] uint32, u[2n] float32, gains[2n] float32.  The checksum is FNV-1a
 * (64-bit offset basis and prime) over the payload taken as little-endian
 * 64-bit words, the last one zero-padded. */
int pxsne_save(pxsne_ctx *ctx, const char *path);

/* Create a context from a file written by pxsne_save, on the current device
 * (stream as in pxsne_create), with the file's parameters, P and state.  The
 * header, sizes and checksum are checked before any device work: a bad or
 * truncated file returns PXSNE_E_ARG (PXSNE_E_UNSUPPORTED for another
 * version) with the reason in pxsne_last_error(NULL); *out stays NULL on
 * every failure. */
int pxsne_load(pxsne_ctx **out, const char *path, void *stream);

/* The parameters and schedule ctx runs with (after pxsne_set_schedule or
 * pxsne_load). */
int pxsne_get_params(const pxsne_ctx *ctx, pxsne_params *p);

/* Change the optimiser schedule of an existing context (learning rate,
 * exaggeration and its length, momenta and switch, minimum gain) without
 * rebuilding P; e.g. refining a warm start without exaggeration.  Takes effect
 * at the next pxsne_step.  Other fields of p are ignored. */
int pxsne_set_schedule(pxsne_ctx *ctx, const pxsne_params *p);

/* KL divergence of the current state (Eq. cost_func) in FP64, with Z the
 * Barnes-Hut normalisation of the current tree and the un-exaggerated P.
 * Synchronises. */
int pxsne_kl(pxsne_ctx *ctx, double *out);

/* Current embedding.  Y (host or device, n x 2 float32, may be NULL) gets
 * y = s * z minus the per-axis mean (t-SNE coordinates, centred); pix (host or
 * device, n x 2 int32, may be NULL) gets the pixel coordinates z >> (32 - L).
 * on_device: 0 host buffers, 1 device buffers; both synchronise.  2: device
 * buffers, enqueued on the context's stream without synchronising (the
 * buffers hold the frame once the stream reaches this point; a device error
 * flag raised meanwhile is reported by the next synchronising call), so a
 * caller can copy frame t to the host on a stream of its own while step t + 1
 * runs. */
int pxsne_get_Y(pxsne_ctx *ctx, float *Y, int32_t *pix, int on_device);

/* Neighbourhood precision of the current embedding (Eq. nei_prec):
 * (1/(k n)) sum_i |N_D^k(i) ∩ N_d^k(i)|.  N_D^k(i) = the first k entries of row
 * i of knn_hd (n x kh int32, host or device per on_device, neighbours in
 * ascending distance; NULL = the lists of the last pxsne_affinities).
 * N_d^k(i) = the exact k nearest points of i in the 2-D embedding by squared
 * y-space distance (FP64), ties to the lower index.  1 <= k <= min(32, kh)
 * and k < n.
 * hits (host, n int32, may be NULL) gets |N_D^k(i) ∩ N_d^k(i)| per point.
 * Synchronises. */
int pxsne_nbr_precision(pxsne_ctx *ctx, int32_t k, const int32_t *knn_hd, int32_t kh,
                        int on_device, double *precision, int32_t *hits);

/* Wait for the context's stream; returns PXSNE_E_DEVICE if a kernel flagged
 * an error since the last check (flags in *dev_errors when non-NULL). */
int pxsne_sync(pxsne_ctx *ctx, uint32_t *dev_errors);

/* ------------------------------------------------------------------------
 * Inspection and injection (host buffers; all synchronise).  They expose the
 * internal state at the boundary so that each step can be compared with an
 * independent implementation.
 * ------------------------------------------------------------------------ */

/* Number of points and non-zeros of P (0 before affinities). */
int pxsne_get_sizes(pxsne_ctx *ctx, int64_t *n, int64_t *nnz);

/* P as CSR: row_ptr[n+1] int64, col[nnz] int32, val[nnz] float32, with nnz
 * from pxsne_get_sizes.  Rows are as built by pxsne_affinities (columns
 * ascending) or as given to pxsne_set_P.  Any pointer may be NULL. */
int pxsne_get_P(pxsne_ctx *ctx, int64_t *row_ptr, int32_t *col, float *val);

/* Replace P by a caller CSR (2 <= n <= 2^24; row_ptr[n+1] int64 with
 * row_ptr[0] = 0 and non-decreasing, col int32 in [0, n) with no self
 * entries, val float32 finite and >= 0).  P is used as given: it is neither
 * symmetrised nor normalised.  Arguments are checked on the host
 * (PXSNE_E_ARG names the first bad row).  Clears the embedding state. */
int pxsne_set_P(pxsne_ctx *ctx, int64_t n, const int64_t *row_ptr, const int32_t *col,
                const float *val);

/* The neighbour lists of the last pxsne_affinities: idx[n*k] int32 and
 * d2[n*k] float32 (FP32 squared distances), ascending per row; beta[n]
 * float32 (the bisection result).  Any pointer may be NULL. */
int pxsne_get_knn(pxsne_ctx *ctx, int32_t *idx, float *d2, float *beta);

/* Overwrite the embedding state: z[n*2] u32 fixed point, s[2] y-units per
 * ulp, u[n*2] velocities (y-units, NULL = 0), gains[n*2] (NULL = 1), and the
 * iteration counter t; then build the tree and forces of that state. */
int pxsne_set_state(pxsne_ctx *ctx, const uint32_t *z, const double *s, const float *u,
                    const float *gains, int32_t t);

/* Read the embedding state (any pointer may be NULL). */
int pxsne_get_state(pxsne_ctx *ctx, uint32_t *z, double *s, float *u, float *gains,
                    int32_t *t);

/* The tree of the current state at one level l (0 = root .. L = pixels), in
 * Morton order (x bits at even positions): cnt[4^l] u32 cell counts N_c and,
 * for l = L only, sx/sy[4^l] u64 exact sums of the fixed-point coordinates of
 * the points in each pixel (NULL to skip).  Pixel Morton keys per point go to
 * morton[n] when non-NULL.  With centre_mode = 1 the tree keeps counts only:
 * asking for sx or sy fails with PXSNE_E_UNSUPPORTED. */
int pxsne_get_tree(pxsne_ctx *ctx, int32_t level, uint32_t *cnt, uint64_t *sx,
                   uint64_t *sy, uint32_t *morton);

/* The octree of a 3-D state (dim = 3) at one level l (0 = root .. L =
 * voxels), in Morton order: cnt[8^l] cell counts and, for l = L only,
 * sx/sy/sz[8^l] exact sums of the fixed-point coordinates (NULL to skip);
 * voxel Morton keys per point to morton[n] when non-NULL.  Synchronises. */
int pxsne_get_tree3(pxsne_ctx *ctx, int32_t level, uint32_t *cnt, uint64_t *sx, uint64_t *sy,
                    uint64_t *sz, uint32_t *morton);

/* Forces of the current state: Frep[n*2] = sum over accepted cells of
 * N w^2 (y_i - y_c) (un-normalised), Zi[n] = sum of N w, Fattr[n*2] =
 * sum_j p_ij w_ij (y_i - y_j) (un-exaggerated), Z = sum_i Zi (FP64).  Any
 * pointer may be NULL. */
int pxsne_get_forces(pxsne_ctx *ctx, float *Frep, float *Zi, float *Fattr, double *Z);

/* Tracing: run `iters` >= 1 iterations like pxsne_step, without the CUDA
 * graph, with CUDA events recorded on the context's stream around each kernel
 * group of an iteration (no synchronisation between iterations).  group_ms
 * (n_groups >= 8 slots) receives the summed milliseconds of each group over
 * all iterations and total_ms (may be NULL) the elapsed time of the whole
 * run.  Group g is named by pxsne_kernel_group_name(g).  Synchronises. */
int pxsne_step_profiled(pxsne_ctx *ctx, int32_t iters, double *group_ms, int32_t n_groups,
                        double *total_ms);

/* Name of kernel group g (0 <= g < 8), or NULL. */
const char *pxsne_kernel_group_name(int32_t g);

/* Work counters of the Barnes-Hut traversal of the state set by pxsne_init or
 * pxsne_set_state, or, after pxsne_step_profiled, their sums over the states
 * of all its iterations (each counted by one extra traversal after that
 * iteration's timed groups): n_accept =
 * accepted (point, cell) pairs (the interactions of Eq. bh_criteria), n_test =
 * tested pairs (accepted + opened + own-pixel), n_warp_steps = warp-level
 * (node, non-empty child) steps, n_nodes = stack entries popped.  Any pointer
 * may be NULL.  Synchronises. */
int pxsne_get_counters(pxsne_ctx *ctx, uint64_t *n_accept, uint64_t *n_test,
                       uint64_t *n_warp_steps, uint64_t *n_nodes);

/* The traversal's work counters by level l of the tested cell (1 = the
 * root's children .. L = pixels): counts[3 l + 0] tested and counts[3 l + 1]
 * accepted (point, cell) pairs, counts[3 l + 2] warp-level steps, over the
 * same states as pxsne_get_counters (the state of the last pxsne_init /
 * pxsne_set_state, or the sum over the iterations of the last
 * pxsne_step_profiled).  levels >= L + 1 entries of three; the rest are
 * zeroed.  Synchronises. */
int pxsne_get_level_counters(pxsne_ctx *ctx, uint64_t *counts, int32_t levels);

/* Work counters of the last neighbour search: exact FP32 distances computed
 * and list insertions over all rows (tensor-core search only; 0 otherwise),
 * and the search used (1 tensor cores, 0 FP32 CUDA cores, -1 none).
 * Synchronises. */
int pxsne_get_knn_counters(pxsne_ctx *ctx, uint64_t *exact, uint64_t *inserted, int32_t *path);

/* Tile pruning of the last tensor-core neighbour search: (query tile,
 * candidate tile) pairs of 128 x 128 rows it skipped because the triangle
 * inequality on the tiles' centroids and radii put every candidate beyond the
 * query rows' current k-th distances, and the number of pairs (T^2).  Both 0
 * after the FP32 search.  Any pointer may be NULL.  Synchronises. */
int pxsne_get_knn_pruning(pxsne_ctx *ctx, uint64_t *skipped_pairs, uint64_t *pairs);

/* Device time in milliseconds of the last neighbour-search kernel (the brute
 * force of Sec. 3.3's kNN pattern; CUDA events around its launch on the
 * context's stream).  PXSNE_E_STATE if no search has run.  Synchronises. */
int pxsne_get_knn_time(pxsne_ctx *ctx, double *search_ms);

/* Test hook of the bounded waits (no counterpart in the paper): one kernel
 * waits on an mbarrier that nothing arrives at, for at most `polls` polls of
 * at most 100 ns each (1 <= polls <= 65536), the way the tensor-core kernels
 * wait on their pipelines; it then sets PXSNE_DEVERR_TIMEOUT and returns.
 * flags (may be NULL) receives the device error flags read back.  Returns
 * PXSNE_E_DEVICE when the wait ran out (the expected outcome), PXSNE_OK if it
 * did not, PXSNE_E_ARG on a bad polls.  The context stays usable.
 * Synchronises. */
int pxsne_test_bounded_wait(pxsne_ctx *ctx, int32_t polls, uint32_t *flags);

/* Measurement (no counterpart in the paper): the peaks that the iteration's
 * rooflines are taken against, measured on the current device by plain
 * kernels timed with CUDA events on `stream` (a cudaStream_t, NULL = the
 * legacy default stream), best of five launches after one warm-up, and the
 * best over a few launch shapes:
 *   - l2_read_gbs: read bandwidth of 16-byte loads that bypass L1 from
 *     buffers (resident in L2) of 1/4, 1/2 and all of the largest power of
 *     two within a quarter of L2, 2, 4 or 8 CTAs of 512 threads per SM;
 *   - fp32_tflops / fp32_packed_tflops: 16 independent chains of FP32 FMAs
 *     per thread as scalar FMAs / as packed pairs (2 FLOP per FMA), 4, 8 or
 *     16 CTAs of 256 threads per SM;
 *   - sm_count and l2_bytes: from the device properties.
 * Any pointer may be NULL (that measurement is skipped).  Allocates and frees
 * a buffer of at most a quarter of L2.  Synchronises the stream.  Returns
 * PXSNE_E_CUDA / PXSNE_E_OOM on failure. */
int pxsne_measure_peaks(void *stream, double *l2_read_gbs, double *fp32_tflops,
                        double *fp32_packed_tflops, int32_t *sm_count, int64_t *l2_bytes);

/* Test hook of the traversal's stack guard (no counterpart in the paper):
 * the Barnes-Hut traversal keeps at most `entries` (4 <= entries <= 48) nodes
 * on a warp's stack, the room a screen of depth L needs being 3 L - 2
 * entries; 0 restores the full stack.  With too little room a warp stops
 * its walk, sets PXSNE_DEVERR_STACK and writes the forces gathered so far,
 * and the next synchronising call returns PXSNE_E_DEVICE; the context stays
 * usable.  Takes effect from the next traversal.  Synchronises. */
int pxsne_test_stack_limit(pxsne_ctx *ctx, int32_t entries);

/* Total bytes of device memory the context holds. */
int64_t pxsne_device_bytes(const pxsne_ctx *ctx);

/* ------------------------------------------------------------------------
 * Learned warm start (not in the paper): an MLP d -> 256 -> 256 -> 2 with the
 * exact GELU g(z) = z Phi(z), BF16 weights and activations as tensor-core
 * operands, FP32 accumulation, FP32 master weights and Adam (beta 0.9 / 0.999,
 * eps 1e-8).  It is trained with the mean squared error
 * L = (1/m) sum_r ||y_r - t_r||^2 on 2-D embeddings the method produced, and
 * its output initialises pxsne_init.  Parameters are one flat FP32 vector,
 * row-major: W1[256 x d], b1[256], W2[256 x 256], b2[256], W3[2 x 256], b3[2].
 * All calls synchronise the model's stream; X (n x d) and T / Y (n x 2) are
 * float32, host or device per on_device.
 * ------------------------------------------------------------------------ */
typedef struct pxsne_mlp pxsne_mlp;

/* d in [1, 1024]; He-normal weights drawn from `seed`, zero biases.  stream:
 * a cudaStream_t or NULL for a private one.  Returns PXSNE_E_ARG, _OOM or
 * _CUDA on failure (*out stays NULL). */
int pxsne_mlp_create(pxsne_mlp **out, int32_t d, uint64_t seed, void *stream);
void pxsne_mlp_destroy(pxsne_mlp *m);
const char *pxsne_mlp_last_error(const pxsne_mlp *m);
int64_t pxsne_mlp_num_params(const pxsne_mlp *m);
/* Set / read the flat FP32 parameters (host).  Setting resets Adam. */
int pxsne_mlp_set_params(pxsne_mlp *m, const float *params);
int pxsne_mlp_get_params(pxsne_mlp *m, float *params);

/* Loss and its gradient with respect to the flat parameters on one batch of
 * 1 <= n <= 8192 rows (no update).  grad (host, num_params floats) may be
 * NULL. */
int pxsne_mlp_loss_grad(pxsne_mlp *m, const float *X, const float *T, int64_t n, float *grad,
                        double *loss, int on_device);

/* `epochs` passes of Adam (learning rate lr) over the n rows in minibatches of
 * `batch` <= 8192 rows, shuffled with `shuffle_seed`; final_loss (may be NULL)
 * gets the mean batch loss of the last epoch. */
int pxsne_mlp_train(pxsne_mlp *m, const float *X, const float *T, int64_t n, int32_t epochs,
                    int32_t batch, float lr, uint64_t shuffle_seed, double *final_loss,
                    int on_device);

/* Y = MLP(X) for n rows. */
int pxsne_mlp_predict(pxsne_mlp *m, const float *X, int64_t n, float *Y, int on_device);

/* PCA pre-processing (Sec. 5.1.1 reduces every dataset to 50 dimensions
 * before P): Xout (n x dout) = (X - mean) V with V the dout leading
 * eigenvectors of the sample covariance (X - mean)^T (X - mean) / (n - 1).
 * Mean and covariance are formed on the GPU (FP32 tiles, FP64 sums); V comes
 * from block subspace iteration with a Rayleigh-Ritz step on the host in FP64
 * (start drawn from `seed`); each eigenvector's largest component is positive.
 * components (host, D x dout row-major) and eigenvalues (host, dout,
 * descending) may be NULL.  X / Xout host or device per on_device. */
int pxsne_pca(const float *X, int64_t n, int32_t D, int32_t dout, float *Xout,
              float *components, float *eigenvalues, int on_device, uint64_t seed);

/* Normalise an embedding Y (n x 2) to zero mean and unit RMS per coordinate
 * (isotropic scale) and, when Yref is non-NULL, apply the orthogonal map
 * (rotation or reflection) that best aligns it with the normalised Yref in the
 * least-squares sense (2 x 2 orthogonal Procrustes, closed form).  Row i of Y
 * and row i of Yref must be the same point (e.g. an embedding and a network's
 * prediction for the same rows).  Used to put the warm start's training
 * embeddings in one frame.  Yout may alias Y.  Host or device buffers per
 * on_device. */
int pxsne_embed_align(const float *Y, const float *Yref, int64_t n, float *Yout, int on_device);

/* ------------------------------------------------------------------------
 * Allocation-free KL.  The paper has no counterpart: this is a service for
 * callers that cannot call cudaMalloc/cudaFree, e.g. code running while a
 * framework's caching allocator owns the device memory, or a loop that must not
 * take the implicit device synchronisation those calls imply.
 *
 * Computes the same value as pxsne_kl for the embedding given by the caller:
 * C = sum_ij p_ij ln(p_ij Z / w_ij), w_ij = 1 / (1 + s0^2 dz_x^2 + s1^2 dz_y^2),
 * enqueued on `stream` (a cudaStream_t; NULL = the legacy default stream) of
 * the current device.  All pointers are device pointers owned by the caller:
 * row_ptr[n+1] int64 (non-decreasing, within col/val: not checked) and
 * col[nnz] int32 and val[nnz] float32 of P, z[n*2] u32 fixed-point positions;
 * s0, s1 are the y-units per ulp and Z the normalisation (e.g. from
 * pxsne_get_forces), each finite and > 0.  The result is written to out[0]
 * (device) when the stream reaches it.  An entry whose column lies outside
 * [0, n) is skipped without reading z, and the result is then NaN.
 *
 * No memory is allocated: the reduction's scratch is one file-scope device
 * array of 128 KiB (8192 block partials) that every GPU which loads the
 * library holds until the process exits, so n is limited to
 * pxsne_kl_noalloc_max_rows() = 16,777,216 rows (larger n returns
 * PXSNE_E_ARG).  The first call on a device looks the array's address up on
 * that device and keeps it (make that first call before any stream capture;
 * after a cudaDeviceReset of that device the kept address is stale, so do not
 * call this entry point on that device again in the process).  All calls
 * share the array: calls whose executions overlap on the GPU (other streams,
 * other threads) race and must be serialised by the caller.  Returns
 * PXSNE_E_ARG for bad arguments and PXSNE_E_CUDA if the launch fails; there is
 * no context, so no message is kept. */
int pxsne_kl_noalloc(const int64_t *row_ptr, const int32_t *col, const float *val, int64_t n,
                     const uint32_t *z, double s0, double s1, double Z, double *out,
                     void *stream);

/* Largest n that pxsne_kl_noalloc accepts. */
int64_t pxsne_kl_noalloc_max_rows(void);

#ifdef __cplusplus
}
#endif
#endif /* PXSNE_H */
