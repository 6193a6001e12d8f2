/*
 * tsne.h -- C ABI of libtsne.so: exact t-SNE on NVIDIA B300 (sm_103a).
 *
 * The CudaMon paper (Sec. 3-4; Table 1, step 7 "Umap + t-sne", run on PCA
 * scores of 1M cells) uses t-SNE without defining it.  This library computes
 * the textbook exact t-SNE (van der Maaten & Hinton 2008, with the
 * kNN-sparse input affinities of van der Maaten 2014):
 *
 *   kNN        for every point the k nearest other points of its sample by
 *              squared Euclidean distance, ordered by (distance, index);
 *   affinities p_{j|i} = exp(-beta_i d_ij^2) / sum_l exp(-beta_i d_il^2) over
 *              the k neighbours, beta_i set so exp(H(p_{.|i})) = perplexity;
 *              P = (P_cond + P_cond^T) / (2 n_s), n_s the sample's size;
 *   gradient   w_ij = 1 / (1 + |y_i - y_j|^2), Z = sum_{i != j} w_ij,
 *              dC/dy_i = 4 sum_{j != i} (alpha p_ij - w_ij / Z) w_ij (y_i - y_j)
 *                      = 4 (alpha Fa_i - Fr_i / Z),
 *              Fa_i = sum_j p_ij w_ij (y_i - y_j), Fr_i = sum_j w_ij^2 (y_i - y_j);
 *   objective  KL_alpha = sum p log p + alpha sum p log(1 + d^2) + log Z
 *              (KL(P||Q) at alpha = 1), whose gradient is the line above;
 *   optimiser  alpha = ee for iter < ee_iters else 1; mu = mom0 for
 *              iter < mom_switch else mom1; gain <- gain + 0.2 where g*u < 0,
 *              else gain * 0.8, floored at min_gain; u <- mu u - eta gain g;
 *              y <- y + u; eta = lr, or n_s / 12 when lr <= 0.
 *
 * Conventions for every entry point:
 *   - Array pointers are DEVICE pointers owned by the caller, unless a comment
 *     says HOST.  Arrays are dense row-major: X is n x d float32, Y n x 2
 *     float32 (x, y interleaved), neighbour lists n x k.
 *   - Work is enqueued asynchronously on `stream` (0 = legacy default stream);
 *     only tsne_run synchronises.  When the symmetric repulsion kernel is in
 *     use (TSNE_VARIANT_SYM / SYM4 / SYM4_FX, or AUTO when the largest sample
 *     has at least 16384 points),
 *     tsne_kl_grad and tsne_step fork their
 *     attraction kernel onto a side stream of the calling host thread (one
 *     non-blocking stream per thread and device, created on the thread's first
 *     such call and kept for its lifetime) and join it back into `stream`
 *     before they return, so every call stays ordered on `stream`; under stream
 *     capture the fork and join become edges of the graph.  No entry point allocates device memory
 *     except tsne_run; scratch comes from a caller workspace `ws` of at least
 *     tsne_workspace_size(...) bytes, 256-byte aligned.
 *   - Return value: TSNE_OK, or a negative TSNE_ERR_* code for errors detected
 *     on the host before anything is enqueued (bad arguments, small
 *     workspace) or reported by the CUDA runtime at launch.
 *   - Errors found by kernels (corrupt indices, capacity overflow, bounded
 *     waits that ran out) are OR-ed as TSNE_STATUS_* bits into the caller's
 *     device word `dev_status` (int32, may be NULL to skip reporting); the
 *     kernel skips the offending access and carries on.  Kernels never trap.
 *   - Several independent samples ("batch", S >= 1) are laid out back to back:
 *     sample s owns points [pt_off[s], pt_off[s+1]); neighbour indices and
 *     CSR column indices are global point indices inside the owner's sample.
 *     A NULL tsne_batch means one sample holding all n points.
 *   - Deterministic: no floating-point atomics; identical inputs give
 *     bitwise-identical outputs on the same device and tile configuration.
 *   - Testing hooks (environment, read at each call): TSNE_FAULT =
 *     "<entry>:<code>[,...]" makes the named entry point return <code> at
 *     once (host-side fault injection); TSNE_WAIT_LIMIT = cycles a bounded
 *     device wait may spin before it gives up with TSNE_STATUS_TIMEOUT (the
 *     persistent batched step's update slots, the tcgen05 kNN's pipeline
 *     waits; the drains of work already issued keep their own long bound).
 */
#ifndef TSNE_H_
#define TSNE_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* cudaStream_t-compatible handle (pass a cudaStream_t or torch stream pointer). */
typedef struct CUstream_st* tsne_stream_t;

enum {
  TSNE_OK = 0,
  TSNE_ERR_ARG = -1,           /* invalid argument, detected on the host             */
  TSNE_ERR_CAPACITY = -2,      /* an output buffer is smaller than required          */
  TSNE_ERR_CUDA = -3,          /* the CUDA runtime reported an error                 */
  TSNE_ERR_TIMEOUT = -4,       /* a bounded device wait ran out                      */
  TSNE_ERR_NOT_CONVERGED = -5, /* warning: some rows missed the perplexity target    */
  TSNE_ERR_WORKSPACE = -6,     /* workspace NULL, misaligned or too small            */
  TSNE_ERR_DEVICE = -7,        /* current device is not sm_103 / library not usable  */
  TSNE_ERR_DEVICE_STATUS = -8  /* tsne_run: a kernel set a bit in the status word    */
};

/* Bits OR-ed into *dev_status by kernels. */
enum {
  TSNE_STATUS_BAD_INDEX = 1,   /* a neighbour / CSR column index outside its sample  */
  TSNE_STATUS_CAPACITY = 2,    /* CSR capacity too small for the symmetrised P       */
  TSNE_STATUS_TIMEOUT = 4,     /* a bounded wait gave up                             */
  TSNE_STATUS_NONFINITE = 8    /* a non-finite value reached an output               */
};

enum { TSNE_KNN_FP32 = 0, TSNE_KNN_BF16_RERANK = 1 };

enum {
  TSNE_OP_KNN = 1,        /* tsne_knn                                      */
  TSNE_OP_AFFINITIES = 2, /* tsne_affinities                               */
  TSNE_OP_KL_GRAD = 3,    /* tsne_kl_grad and tsne_step (same workspace)   */
  TSNE_OP_PLAIN = 4,      /* tsne_kl_grad_plain and tsne_step_plain        */
  TSNE_OP_PCA = 5,        /* tsne_pca (n rows, d = g columns)              */
  TSNE_OP_PCA_TRANSFORM = 6, /* tsne_pca_transform (n rows, d = g columns) */
  TSNE_OP_KNN_GRAPH = 7,  /* tsne_knn_graph (same as TSNE_OP_AFFINITIES)   */
  TSNE_OP_UMAP_LAYOUT = 8, /* tsne_umap_layout (n points)                  */
  TSNE_OP_UMAP_INIT = 9    /* tsne_umap_init (n points)                    */
};

/* Repulsion kernel variants (tsne_params.variant).  The symmetric split keeps
   one float2 partial per point and group pair (16 B x N^2 / 1024 scratch: 7.8 GB
   at N = 1M); SYM4_FX sums the same partials into two 64-bit fixed-point
   accumulators per point (16 B x N scratch, bitwise reproducible, absolute error
   per coordinate <= (G - 1) 2^-(S+1) with S = 62 - bitlen(N), G = N / 1024
   groups).  The symmetric forms also take each diagonal group's own pairs once,
   in the same launch.  AUTO takes the symmetric split from N = 16,384: the
   fixed-point form, in tiles of 4 x 4 group pairs, once the call has at least
   eight waves of tiles (three per SM; about 400k points), else the partial
   buffers, which it also leaves for the fixed-point form past 32 GiB.  Below
   16,384 points AUTO (and TSNE_VARIANT_DIRECT) takes the direct form with its
   tile shape by problem size; under 4e8 pairs the attraction and the direct
   repulsion run in one launch. */
enum {
  TSNE_VARIANT_AUTO = -1,     /* pick by problem size                           */
  TSNE_VARIANT_DIRECT = 0,    /* direct form, tile shape picked by problem size */
  TSNE_VARIANT_DIRECT_L = 1,  /* direct form, 256 threads x 8 rows, 1024-column tiles */
  TSNE_VARIANT_DIRECT_S = 2,  /* direct form, 128 threads x 4 rows, 256-column tiles  */
  TSNE_VARIANT_SYM = 3,       /* unordered pairs once (groups of 2048)                */
  TSNE_VARIANT_DIRECT_M = 4,  /* direct form, 256 threads x 4 rows, 512-column tiles   */
  TSNE_VARIANT_SYM4 = 5,      /* unordered pairs once (groups of 1024)                */
  TSNE_VARIANT_FUSED = 6,     /* tsne_step: one persistent launch per iteration over all
                                 samples (symmetric split, groups of 1024); elsewhere
                                 like DIRECT_S                                        */
  TSNE_VARIANT_SYM4_FX = 7    /* SYM4 with fixed-point sums: O(N) scratch             */
};

#define TSNE_MAX_SAMPLES 512

/* Symmetric P in CSR form.  row_ptr int64[n+1], col int32[cap], val float32[cap];
 * columns ascending within a row, no diagonal.  row_ptr[n] is the number of
 * stored entries; `nnz` is informational (filled only by synchronous calls).  */
typedef struct tsne_csr {
  int64_t n;
  int64_t nnz;
  int64_t cap;
  int64_t* row_ptr;
  int32_t* col;
  float* val;
} tsne_csr;

/* Samples of a batch: HOST array pt_off[n_samples+1], pt_off[0] = 0,
 * non-decreasing, pt_off[n_samples] = n, 1 <= n_samples <= TSNE_MAX_SAMPLES (512). */
typedef struct tsne_batch {
  int n_samples;
  const int64_t* pt_off;
} tsne_batch;

/* Parameters of affinities and optimisation.  tsne_params_default fills the
 * values of the common exact t-SNE setting (perplexity 30, k 90, 750
 * iterations, exaggeration 12 for 250, momentum 0.5 then 0.8, lr n/12) and
 * selects the BF16 tensor-core kNN with an exact FP32 re-rank of 2k
 * candidates. */
typedef struct tsne_params {
  float perplexity;   /* target perplexity, 1 < perplexity < k                 */
  int k;              /* neighbours per point                                   */
  int knn_mode;       /* TSNE_KNN_FP32 or TSNE_KNN_BF16_RERANK                  */
  float cand_mult;    /* BF16 mode: candidates per row = cand_mult * k          */
  float calib_tol;    /* |H - log perplexity| tolerance in nats                 */
  int calib_max_iter; /* root-finding steps per row                             */
  int n_iter;         /* optimisation iterations                                */
  int ee_iters;       /* iterations with exaggeration                           */
  float ee;           /* exaggeration factor alpha                              */
  int mom_switch;     /* iteration from which mom1 is used                      */
  float mom0, mom1;   /* momentum before / after mom_switch                     */
  float lr;           /* learning rate eta; <= 0 means n_s / 12 per sample      */
  float min_gain;     /* gain floor                                             */
  int kl_every;       /* tsne_run: record KL every kl_every iterations (0: off) */
  int variant;        /* repulsion kernel variant, TSNE_VARIANT_*; AUTO picks the
                         symmetric form once the largest sample has >= 16384
                         points, else the direct form with its tile shape by
                         problem size (never the fused launch, which is taken
                         only when asked for or chosen by the autotuner)       */
  int use_graph;      /* tsne_run: capture iterations in CUDA graphs            */
} tsne_params;

void tsne_params_default(tsne_params* p);

/* Static description of an error code. */
const char* tsne_strerror(int code);

/* Library version string. */
const char* tsne_version(void);

/* Bytes of workspace needed by operation `op` (TSNE_OP_*) for n points of
 * dimension d with k neighbours, batch B (NULL = one sample) and parameters
 * `prm` (NULL = defaults).  Depends on the current device's SM count. */
size_t tsne_workspace_size(int op, int64_t n, int d, int k, const tsne_batch* B,
                           const tsne_params* prm);

/* Brute-force kNN (the t-SNE input affinities need the k nearest neighbours;
 * van der Maaten 2014 Sec. 3): for every point i the k nearest points j != i of the
 * same sample by squared Euclidean distance over the d features, ordered by
 * (d2, j).  X: n x d float32.  Out: nbr_idx int32 n x k (global indices),
 * nbr_d2 float32 n x k.  TSNE_KNN_FP32: exact FP32 brute force.
 * Requires 1 <= k < min sample size, 1 <= d <= 1024. */
int tsne_knn(const float* X, int64_t n, int d, int k, const tsne_batch* B, int knn_mode,
             float cand_mult, int32_t* nbr_idx, float* nbr_d2, void* ws, size_t ws_bytes,
             int32_t* dev_status, tsne_stream_t stream);

/* Affinities (van der Maaten & Hinton 2008 Sec. 2; sparse form, van der
 * Maaten 2014 Sec. 3): per-row beta by a bracketed Newton search (bisection
 * where a Newton step leaves the bracket) so that exp(H) = perplexity within
 * `tol` nats (at most max_iter steps), p_{j|i} over the k
 * neighbours, then P = (P_cond + P_cond^T) / (2 n_s) on the union pattern.
 * Rows whose target is unreachable (>= perplexity neighbours tied at the
 * minimum distance) get uniform weight on the tied set and beta = +inf.
 * Out: P (row_ptr, col, val written; P->cap >= 2 n k required), beta float32
 * [n] (nullable), n_bad int64 device counter (nullable; incremented by the
 * number of rows that did not converge or were unreachable). */
int tsne_affinities(const int32_t* nbr_idx, const float* nbr_d2, int64_t n, int k,
                    const tsne_batch* B, float perplexity, float tol, int max_iter,
                    tsne_csr* P, float* beta, int64_t* n_bad, void* ws, size_t ws_bytes,
                    int32_t* dev_status, tsne_stream_t stream);

/* Exact KL gradient (van der Maaten & Hinton 2008, Eq. 5 with exaggeration
 * alpha): grad n x 2 float32 (nullable) = 4 (alpha Fa - Fr / Z_s); Z_s double
 * per sample (device [S], required); kl double per sample (device [S],
 * nullable) = KL_alpha.  All O(n_s^2) pairs are evaluated. */
int tsne_kl_grad(const tsne_csr* P, const tsne_batch* B, const float* Y, float alpha,
                 float* grad, double* Z, double* kl, const tsne_params* prm, void* ws,
                 size_t ws_bytes, int32_t* dev_status, tsne_stream_t stream);

/* Same result through the plain GPU form (one thread per row, global loads,
 * separate kernels, no tiling): the comparison baseline for the tiled path. */
int tsne_kl_grad_plain(const tsne_csr* P, const tsne_batch* B, const float* Y, float alpha,
                       float* grad, double* Z, void* ws, size_t ws_bytes,
                       int32_t* dev_status, tsne_stream_t stream);

/* One optimiser iteration through the plain GPU form: the plain gradient at
 * alpha(iter), then a one-thread-per-point update with the same gains,
 * momentum and position rule as tsne_step (van der Maaten & Hinton 2008,
 * Sec. 3.4).  iter >= 0 (host numbering only); Y, uY, gains n x 2 float32 in
 * place.  Workspace: TSNE_OP_PLAIN.  The comparison baseline for whole
 * iterations of the tiled path. */
int tsne_step_plain(const tsne_csr* P, const tsne_batch* B, float* Y, float* uY, float* gains,
                    int iter, const tsne_params* prm, void* ws, size_t ws_bytes,
                    int32_t* dev_status, tsne_stream_t stream);

/* One optimiser iteration (van der Maaten & Hinton 2008 Sec. 3.4 with gains):
 * gradient at exaggeration alpha(iter), then gains, momentum and position
 * update of Y, uY (velocity) and gains, all n x 2 float32 in place.
 * iter >= 0: iteration number given by the host.  iter == -1: the iteration
 * number is read from, and advanced in, a counter kept in the workspace
 * (reset by tsne_step_reset), so a captured CUDA graph of repeated calls
 * follows the schedule.  Z (device [S], nullable) receives Z_s of the Y the
 * gradient was taken at; kl (device double [S * n_kl], nullable) receives
 * KL(P||Q) (alpha = 1) of that Y at iterations with (iter+1) % kl_every == 0,
 * at slot ((iter+1)/kl_every - 1) * S + s. */
int tsne_step(const tsne_csr* P, const tsne_batch* B, float* Y, float* uY, float* gains,
              int iter, const tsne_params* prm, double* Z, double* kl, void* ws,
              size_t ws_bytes, int32_t* dev_status, tsne_stream_t stream);

/* Allocation-free gradient.  The paper has no counterpart: this entry exists
 * for callers that cannot allocate device memory (an embedding application
 * whose own allocator owns all device memory, or a loop that cannot pay
 * cudaMalloc's implicit synchronisation) and so cannot hold the workspace
 * tsne_kl_grad needs.  Same inputs and outputs as tsne_kl_grad for one sample
 * (no batch, no params): grad n x 2 (nullable), Z double [1] (required), kl
 * double [1] (nullable, KL_alpha).  Scratch is a fixed device array of
 * TSNE_NOALLOC_SCRATCH_BYTES inside the library, present on every device that
 * loads it until the process exits; no memory is allocated.
 *   - n < 2 returns TSNE_ERR_ARG, as tsne_kl_grad does; n > TSNE_NOALLOC_MAX_N
 *     returns TSNE_ERR_CAPACITY (nothing enqueued in either case);
 *   - all calls share the array: calls that overlap on the GPU race, so order
 *     them on one stream;
 *   - the first call under each CUDA context (the primary context of a device,
 *     a caller's own driver-API context, or the new primary context after a
 *     device reset) looks up the array's device address in that context and
 *     caches it under the context's unique ID; make that first call before any
 *     stream capture begins.
 * Results equal tsne_kl_grad's up to summation order. */
#define TSNE_NOALLOC_MAX_N 65536
#define TSNE_NOALLOC_SCRATCH_BYTES (6u << 20)
int tsne_kl_grad_noalloc(const tsne_csr* P, const float* Y, float alpha, float* grad, double* Z,
                         double* kl, int32_t* dev_status, tsne_stream_t stream);

/* Fuzzy neighbour graph for UMAP / Leiden (the pipeline's step 6; UMAP's
 * fuzzy simplicial set, McInnes, Healy & Melville 2018, Sec. 3.1) from the
 * output of tsne_knn (self excluded, d2 ascending per row), k >= 2:
 *   d_j = sqrt(d2_j); rho_i = smallest positive d_j (0 if none);
 *   sigma_i solves sum_j exp(-max(0, d_j - rho_i) / sigma_i) = log2(k)
 *     (FP32 bisection to |f - log2 k| <= tol; rows whose ties at rho reach
 *     log2 k take sigma = 0, weight 1 on those ties, and count in *n_bad);
 *   w_ij = exp(-max(0, d_ij - rho_i) / sigma_i);
 *   G = fuzzy union: g_ij = w_ij + w_ji - w_ij w_ji (w = 0 off the kNN lists),
 * symmetric CSR like tsne_affinities' P (G->cap >= 2 n k).  rho, sigma
 * (FP32, n, nullable), n_bad (int64, zeroed by the caller, nullable): DEVICE.
 * Workspace: tsne_workspace_size(TSNE_OP_KNN_GRAPH, n, 0, k, B, NULL). */
int tsne_knn_graph(const int32_t* nbr_idx, const float* nbr_d2, int64_t n, int k,
                   const tsne_batch* B, float tol, int max_iter, tsne_csr* G, float* rho,
                   float* sigma, int64_t* n_bad, void* ws, size_t ws_bytes, int32_t* dev_status,
                   tsne_stream_t stream);

/* UMAP layout of a fuzzy neighbour graph (the pipeline's step 7 for UMAP;
 * McInnes, Healy & Melville 2018, Sec. 3.2 and their embedding optimisation
 * algorithm), epochs epoch0 .. epoch0 + n_run - 1 of an n_epochs schedule, on
 * Y (n x 2 float32, device, in place; any initial layout).
 *   Phi(d) = 1 / (1 + a d^(2b)) (a, b > 0: the curve fitted to min_dist and
 *   spread); alpha_e = alpha0 (1 - e / n_epochs).  Each directed entry (i, j)
 *   of G (symmetric CSR, weights in (0, 1]) is taken with probability g_ij;
 *   a taken entry adds to y_i the attraction
 *     clip(-2ab d^(2b-2) / (1 + a d^(2b)) (y_i - y_j))          (0 if d = 0)
 *   and, for n_neg vertices c drawn uniformly from i's sample (c == i skipped),
 *     clip(2b / ((1e-3 + d^2)(1 + a d^(2b))) (y_i - y_c)),
 *   every coordinate clipped to [-4, 4].  Epochs are synchronous: all terms of
 *   epoch e use the positions at its start; y_i += alpha_e (their sum) at its
 *   end.  Draws are counter-based (splitmix64 of ((e << 40) + (q << 4) + s) xor
 *   seed, q the CSR entry, s = 0 for the entry, 1..n_neg for its negatives:
 *   taken when (h >> 40) 2^-24 < g_q; negative p0 + ((h >> 32) n_s >> 32)), so
 *   a run is reproducible bit for bit and equals the same epochs run one by one.
 * Batch: negatives stay inside each sample.  Workspace: TSNE_OP_UMAP_LAYOUT
 * (n float2 of scratch positions).  Errors (host, before any launch):
 * TSNE_ERR_ARG for n_epochs < 1 or >= 2^24, epoch0 < 0, n_run < 0,
 * epoch0 + n_run > n_epochs, a or b not positive and finite, alpha0 not
 * positive and finite, n_neg outside [0, 15], G or Y missing.  Device status:
 * TSNE_STATUS_BAD_INDEX for a column outside [0, n) (entry skipped),
 * TSNE_STATUS_NONFINITE for a non-finite position written. */
int tsne_umap_layout(const tsne_csr* G, const tsne_batch* B, float* Y, int n_epochs, int epoch0,
                     int n_run, float a, float b, float alpha0, int n_neg, uint64_t seed, void* ws,
                     size_t ws_bytes, int32_t* dev_status, tsne_stream_t stream);

/* (a, b) of UMAP's low-dimensional membership Phi(d) = 1 / (1 + a d^(2b))
 * (McInnes, Healy & Melville 2018, Sec. 3.2): the least-squares fit to
 * Psi(d) = 1 for d < min_dist and exp(-(d - min_dist) / spread) beyond, on 300
 * evenly spaced d in [0, 3 spread]; Levenberg-Marquardt in FP64 from (1, 1).
 * HOST computation (no device needed); a, b: HOST doubles.  TSNE_ERR_ARG for
 * min_dist < 0, spread <= 0, a non-finite input or a NULL output;
 * TSNE_ERR_NOT_CONVERGED if the fit leaves a, b > 0. */
int tsne_umap_ab(float min_dist, float spread, double* a, double* b);

/* Initial UMAP layout from PCA scores (the pipeline's start in place of a
 * spectral one): U (n x 2 float32, device) = the first two columns of scores
 * (n rows of stride ld >= 2 floats, device), centred on their FP64 means and
 * scaled so that max |U| = 10.  Workspace: TSNE_OP_UMAP_INIT.  Fixed-order
 * reductions: the result does not depend on the device.  Device status:
 * TSNE_STATUS_NONFINITE for a non-finite score. */
int tsne_umap_init(const float* scores, int64_t n, int64_t ld, float* U, void* ws,
                   size_t ws_bytes, int32_t* dev_status, tsne_stream_t stream);

/* Set the workspace iteration counter used by tsne_step(iter = -1). */
int tsne_step_reset(void* ws, size_t ws_bytes, int iter, tsne_stream_t stream);

/* Whole embedding: kNN, affinities, then prm->n_iter iterations from the
 * initial Y (uY = 0, gains = 1).  X (n x d) and Y (n x 2, in: Y0, out: final
 * embedding) may be HOST or DEVICE pointers.  kl_trace: HOST double array of
 * (n_iter / kl_every) * S entries (nullable).  Allocates its scratch with
 * stream-ordered allocation and frees it before returning; synchronises
 * `stream`.  Returns TSNE_ERR_DEVICE_STATUS if a kernel reported a problem
 * (the bits are then in *status_out, HOST, nullable), TSNE_ERR_NOT_CONVERGED
 * if calibration missed rows (result still produced). */
int tsne_run(const float* X, int64_t n, int d, const tsne_batch* B, const tsne_params* prm,
             float* Y, double* kl_trace, int32_t* status_out, tsne_stream_t stream);

/* ---- principal component analysis (the pipeline step before the neighbour
 * graph and the embeddings; the paper's Table 1, step 5) -------------------
 * Exact definition: with the column means mu and Ac = A - 1 mu^T, the k
 * principal axes are the unit eigenvectors of Ac^T Ac for its k largest
 * eigenvalues lambda_c; scores T = Ac V^T.  Computed by randomized subspace
 * iteration with a TSNE_PCA_SKETCH-column sketch, n_power power iterations
 * and a Rayleigh-Ritz step (Halko, Martinsson & Tropp 2011, Alg. 4.4 / 5.1);
 * with a gap after lambda_k it converges to the exact axes.  The products
 * with A run on the tensor cores: each centred value of A and of the sketch
 * is split into BF16 hi + lo parts (to about 2^-17 relative) on the fly,
 * FP32 accumulation.
 *
 * tsne_pca: A n x g FP32 (row stride lda >= g floats), DEVICE, read in
 *   place by TMA: A 16-byte aligned and lda a multiple of 4 (else
 *   TSNE_ERR_ARG); n >= 65, g >= 64, 1 <= k <= 64.  omega: g x 64 FP32 Gaussian test matrix (DEVICE,
 *   row-major; the caller draws it).  Outputs (DEVICE): scores n x k FP32,
 *   components k x g FP32 (one axis per row, each flipped so that its
 *   largest-magnitude entry -- lowest index among ties -- is positive),
 *   sigma[k] = sqrt(lambda) FP64 (nullable), explained_var[k] = lambda /
 *   (n - 1) FP64 (nullable), mean[g] FP64 (nullable), total_var[1] = trace /
 *   (n - 1) FP64.  Workspace: tsne_workspace_size(TSNE_OP_PCA, n, g, ...)
 *   (about 1 KB per row of A: sketches and partial products; A is not copied).
 *   A failed Cholesky (rank-deficient sketch even after shifting) sets
 *   TSNE_STATUS_NONFINITE in dev_status.
 * tsne_pca_transform: scores = (A - mean) components^T for new rows (same
 *   layouts and alignment rule; mean FP64 g, components k x g); workspace
 *   TSNE_OP_PCA_TRANSFORM. */
#define TSNE_PCA_SKETCH 64
int tsne_pca(const float* A, int64_t n, int g, int64_t lda, int k, int n_power,
             const float* omega, float* scores, float* components, double* sigma,
             double* explained_var, double* mean, double* total_var, void* ws, size_t ws_bytes,
             int32_t* dev_status, tsne_stream_t stream);
int tsne_pca_transform(const float* A, int64_t n, int g, int64_t lda, const double* mean,
                       const float* components, int k, float* scores, void* ws, size_t ws_bytes,
                       int32_t* dev_status, tsne_stream_t stream);

/* ---- GPU telemetry sampler (the paper's CudaMon monitor, Sec. 2) --------
 * Host-only.  A background thread reads, every `period_s` seconds (>= 1 ms),
 * GPU utilisation %, memory-controller utilisation %, memory in use (MiB),
 * temperature (C), power draw (W) and SM clock (MHz) of NVML device
 * `device_index` -- read-only queries; no device setting is changed.  NVML is
 * opened at run time (libnvidia-ml.so.1, or the file named by $TSNE_NVML_LIB).
 * Times are seconds since tsne_mon_start on a monotonic clock.  A field whose
 * query failed is -1.
 *
 * tsne_mon_start  returns a handle owned by the caller (release it with
 *                 tsne_mon_free), or NULL with *err = TSNE_ERR_DEVICE (NVML
 *                 missing / init failed) or TSNE_ERR_ARG (bad index, period or
 *                 csv_path).  csv_path (nullable): the trace is also streamed
 *                 there, one "sample" or "event" line per record.
 * tsne_mon_mark   records a named timestamp (the paper's timestamp verb).
 * tsne_mon_stop   stops sampling and closes the CSV; idempotent.
 * tsne_mon_count  what = 0: samples so far, 1: events so far.
 * tsne_mon_samples copies min(count, cap_rows) samples into out (HOST,
 *                 row-major cap_rows x 7: t, gpu %, mem %, MiB, C, W, MHz).
 * tsne_mon_event  event i: its time and name (truncated to cap bytes).     */
typedef struct tsne_mon tsne_mon;
tsne_mon* tsne_mon_start(int device_index, double period_s, const char* csv_path, int* err);
int tsne_mon_mark(tsne_mon* mon, const char* name);
int tsne_mon_stop(tsne_mon* mon);
int64_t tsne_mon_count(tsne_mon* mon, int what);
int tsne_mon_samples(tsne_mon* mon, double* out, int64_t cap_rows);
int tsne_mon_event(tsne_mon* mon, int64_t i, double* t, char* name, int cap);
void tsne_mon_free(tsne_mon* mon);

#ifdef __cplusplus
}
#endif
#endif /* TSNE_H_ */
