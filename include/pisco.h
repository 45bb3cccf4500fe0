/*
 * pisco.h -- C ABI of a GB300 (sm_103a) implementation of the nullspace / ESPIRiT-equivalent
 * coil-sensitivity estimator with the PISCO accelerations (Lobos, Chan & Haldar,
 * arXiv 2302.13431).
 *
 * One call to pisco_estimate runs, on one GPU and on the plan's CUDA stream:
 *   (a) the Gram C^H C of the calibration matrix C (Eq. C) by zero-padded DFTs without
 *       forming C (Sec. V-A; the masking is neglected, so the Gram is C_full^H C_full);
 *   (b) its approximate nullspace, thresholded at sigma_n < thr * sigma_1 (footnote of
 *       Sec. III-B), with the split decided on FP64 Rayleigh quotients;
 *   (c) G(x) = H(x)^H H(x) on the reduced grid straight from the collapsed filter kernel
 *       (Sec. V-C, Eq. 24), never forming H(x);
 *   (d) simultaneous power iteration for the eigenvector of G(x) with the smallest
 *       eigenvalue, on B(x) = I - G(x)/|Lambda| (Sec. V-E, Eq. esp_null);
 *   (e) the smooth phase alpha(x) from an apodised low-resolution coil combination, periodic-
 *       sinc interpolation to the full grid (Sec. V-D) and per-pixel unit-norm output.
 *
 * Conventions shared by every entry point:
 *   - Arrays are C-ordered with x fastest.  Multichannel arrays put the coil index first:
 *     calibration data is complex64 [Q][Nc_z][Nc_y][Nc_x] with its DC sample at index
 *     floor(Nc/2) on every axis; maps are complex64 [Q][N_z][N_y][N_x].  complex64 means two
 *     consecutive IEEE floats (re, im).  In 2D N_z = Nc_z = 1.
 *   - Image-grid point j of an axis of length N sits at x_j = (j - N/2)/N (the FOV is the
 *     unit cube, Sec. III-A).  The reduced grid has N/f points per axis and its points
 *     coincide with every f-th full-grid point.
 *   - Functions never print, never abort and never throw; they return a pisco_status.
 *   - Device pointers are owned by the caller.  The plan owns its own workspace, which it
 *     allocates in pisco_plan; pisco_estimate allocates nothing.
 */
#ifndef PISCO_H_
#define PISCO_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PISCO_OK = 0,
  PISCO_ERR_ARG = 1,            /* invalid parameter or pointer; nothing was launched        */
  PISCO_ERR_CUDA = 2,           /* a CUDA runtime call failed (launch, copy, sync)            */
  PISCO_ERR_OOM = 3,            /* workspace allocation failed in pisco_plan                  */
  PISCO_ERR_RANK = 4,           /* R < Q-1: the necessary condition of Sec. III-B fails.  The
                                   outputs are still written (they are not identifiable).    */
  PISCO_ERR_TIMEOUT = 5,        /* a bounded device-side wait expired                         */
  PISCO_ERR_NOT_CONVERGED = 6,  /* block eigensolver saturated even at the largest block, or
                                   the FP64 residual bounds do not certify the threshold split
                                   (Sec. III-B footnote) after the largest automatic iteration
                                   count (or after an explicit eig_iters).  The outputs are
                                   still written with the uncertified split.                 */
  PISCO_ERR_UNSUPPORTED = 7,    /* valid request outside what this build implements          */
  PISCO_ERR_TOO_LARGE = 8       /* request needs more than the fixed scratch of
                                   pisco_gram_lags_noalloc (nothing was launched)            */
} pisco_status;

typedef enum { PISCO_KERNEL_RECT = 0, PISCO_KERNEL_ELLIPSOID = 1 } pisco_kernel_shape;

/* flags */
#define PISCO_FLAG_HOST_IO 0x1u  /* allocate pinned/device staging for pisco_estimate_host   */
#define PISCO_FLAG_TC_GFIELD 0x2u /* build G(x) (Sec. V-C, Eq. 24 in its lag form) with two
                                     tensor-core GEMMs: P = U diag(w) U^H, folded onto the lags of
                                     Lambda-Lambda, then G = |Lambda| I - E K with E the lag-to-
                                     pixel exponentials.  Products in split-precision TF32
                                     (three TF32 passes per product: head*head + head*tail +
                                     tail*head), FP32 accumulate.  Default: CUDA-core FP32.     */
#define PISCO_FLAG_TC_EIG 0x4u    /* the n x n by n x m block products of the nullspace
                                     eigensolver on the tensor cores, same split precision.
                                     The threshold split itself stays FP64 (Sec. III-B).       */
#define PISCO_FLAG_MASKED_GRAM 0x10u /* exact Gram of the masked calibration matrix (only the
                                     rows n with n - Lambda inside the calibration box: Eq. C as
                                     written, before Sec. V-A neglects the masking), from
                                     FP64 summed-area tables of the lagged products instead of
                                     the FFT route.  Needs prod(Nc) <= 14528 (one shared-memory
                                     tile of 227 KB; 24^3 fits); PISCO_ERR_UNSUPPORTED otherwise. */
#define PISCO_FLAG_BLOCK_PI 0x20u  /* power iteration on a two-vector block (Gram-Schmidt every
                                     step, 2x2 Rayleigh-Ritz at the end) for pixels whose two
                                     smallest eigenvalues of G(x) are close: convergence set by
                                     the third eigenvalue (Sec. V-E's iteration on a block);
                                     twice the work of the plain iteration                    */
#define PISCO_FLAG_GRAM_DF 0x40u  /* the FFT route of Sec. V-A and the band products of the
                                     FP64 Rayleigh quotients in double-float arithmetic (each
                                     value an unevaluated sum of two FP32 numbers, Dekker's
                                     error-free products and Knuth's two-sum; about 48
                                     significant bits) instead of FP64: GB300's FP64 rate is
                                     about 1/58 of FP32.  The lag table, the Gram and the
                                     quotients are stored and compared in FP64.               */
#define PISCO_FLAG_TC_THIN 0x80u  /* with PISCO_FLAG_TC_EIG: also the thin block products of the
                                     eigensolver (block Grams Y^H Y, Y R^-1, the Rayleigh-Ritz
                                     products) on the tensor cores, same split precision      */
#define PISCO_FLAG_TC_INTERP 0x100u /* the last periodic-sinc interpolation pass (Sec. V-D) as one
                                     batched tensor-core GEMM per estimate (maps_q = M T_q for
                                     every coil, split TF32), followed by the per-pixel
                                     normalisation of Sec. VI                                  */
#define PISCO_FLAG_G_DENSE 0x200u   /* with PISCO_FLAG_TC_GFIELD in 2D: evaluate the lag sums of
                                     G(x) (Sec. V-C) as the dense tensor-core product
                                     E(x, d) K(d, pq) instead of the default separable DFT
                                     passes over the lag rows and columns (3D always uses the
                                     dense product)                                           */
#define PISCO_FLAG_TC_1PASS 0x8u  /* with TC_GFIELD / TC_EIG: one TF32 pass per product (about
                                     11 significant bits) instead of three; for error studies */

typedef struct {
  int ndim;               /* 2 or 3                                                          */
  int grid[3];            /* full image grid N_x, N_y, N_z (N_z = 1 in 2D)                    */
  int calib[3];           /* calibration box Nc_x, Nc_y, Nc_z (Nc_z = 1 in 2D), centred       */
  int num_coils;          /* Q, 2 <= Q <= 64                                                  */
  int kernel_shape;       /* PISCO_KERNEL_RECT: ||n||_inf <= tau;  PISCO_KERNEL_ELLIPSOID:
                             sum_d (n_d/tau_d)^2 <= 1 (equal radii: ||n||_2 <= tau, Sec. V-B) */
  int kernel_radius[3];   /* tau_x, tau_y, tau_z (tau_z = 0 in 2D)                            */
  double null_threshold;  /* thr in (0,1): sigma_n < thr*sigma_1 is null (paper: 0.05)        */
  int grid_reduction;     /* f >= 1; every grid[d] must be divisible by f                     */
  int power_iters;        /* number of power iterations, >= 1 (paper: 10)                     */
  unsigned long long seed;/* start vector: v0[j][q] = u(2q) + i u(2q+1), u(t) from
                             SplitMix64(seed*2^40 + j*2^8 + t), a 24-bit uniform in [-1,1)   */
  unsigned flags;         /* PISCO_FLAG_*                                                     */
  int eig_block;          /* block size of the nullspace eigensolver (0: automatic)           */
  int eig_iters;          /* subspace iterations of the eigensolver (0: automatic: 6, doubled
                             up to 48 while the split is not certified; > 0: fixed)          */
  int tc_splits;          /* K splits of the tensor-core GEMMs (PISCO_FLAG_TC_*; 0: automatic) */
  int gemm_splits;        /* split-K cap of the CUDA-core block products (0: automatic, about
                             two CTAs per SM; small values suit batches of concurrent plans)  */
  int gemm_tile;          /* tile of the CUDA-core block products: 0 automatic, 32 or 64      */
  int batch_group;        /* batches (pisco_batch_plan): most items of identical parameters that
                             one batched pass estimates together, every stage one launch over
                             all of them (0: automatic = 64; 1: one launch chain per item).
                             Batched passes need PISCO_FLAG_TC_GFIELD and neither
                             PISCO_FLAG_MASKED_GRAM nor PISCO_FLAG_BLOCK_PI; other items run
                             one chain each.  Ignored by pisco_plan.                          */
} pisco_params;

typedef struct pisco_plan_s* pisco_plan_t;

/* Validate `p`, build the index tables, allocate the device workspace and bind the plan to
 * `cuda_stream` (a cudaStream_t; NULL = the legacy default stream).  Rejected with
 * PISCO_ERR_ARG: ndim not 2/3, Q outside [2,64], Nc <= 2*tau on some axis, Nc > N, N not
 * divisible by f, N/f < 2*tau+1, thr outside (0,1), power_iters < 1.  On success *out owns
 * the workspace until pisco_destroy. */
pisco_status pisco_plan(const pisco_params* p, void* cuda_stream, pisco_plan_t* out);

/* Run the whole path on the plan's stream.
 *   d_calib: device, complex64 [Q][Nc_z][Nc_y][Nc_x], read only.
 *   d_maps:  device, complex64 [Q][N_z][N_y][N_x], written: unit 2-norm per pixel (all zero
 *            where the interpolated vector vanishes), phase fixed by alpha(x) of Sec. V-D.
 *   d_eig:   device, float [N_z/f][N_y/f][N_x/f] or NULL: lambda_min(G(x))/|Lambda| in [0,1]
 *            on the reduced grid (Rayleigh quotient after the last power iteration).
 * Synchronises the stream once at the end to read the device status word.  Pointers must
 * be 8-byte aligned.  Not thread-safe for one plan; distinct plans may run concurrently.
 * After one call with a given (d_calib, d_maps, d_eig), the next call with the same pointers
 * captures the whole path into a CUDA graph on the plan's stream and later calls with those
 * pointers replay it (one graph launch instead of ~80 kernel launches); other pointers run
 * eagerly.  The stream must not be under capture by the caller. */
pisco_status pisco_estimate(pisco_plan_t plan, const void* d_calib, void* d_maps, float* d_eig);

/* Same as pisco_estimate with HOST buffers of the same layouts: copies the calibration block
 * to the device, runs the path, copies maps (and eig if non-NULL) back, all on the plan's
 * stream.  Needs PISCO_FLAG_HOST_IO at plan time (PISCO_ERR_ARG otherwise).  Host buffers
 * may be pageable; pinned buffers give overlap-free full-bandwidth copies. */
pisco_status pisco_estimate_host(pisco_plan_t plan, const void* h_calib, void* h_maps, float* h_eig);

/* Free the plan and its workspace.  NULL-safe. */
void pisco_destroy(pisco_plan_t plan);

/* Static English description of a status code. */
const char* pisco_status_string(pisco_status s);

/* Sizes chosen by the plan and results of the last estimate: R (nullspace dimension) and
 * k (signal dimension, R + k = Q|Lambda|) are valid after a successful estimate (-1 before),
 * workspace_bytes is the device memory the plan holds.  Any output pointer may be NULL. */
pisco_status pisco_plan_info(pisco_plan_t plan, int* R, int* k, size_t* workspace_bytes);

/* Intermediate results of the last estimate, for stage-by-stage verification.  Returns a
 * device pointer into the plan's workspace (valid until the next call on the plan) and its
 * size in bytes.  Layouts:
 *   PISCO_BUF_LAGS   complex128 [Q][Q][B_z][B_y][B_x], the correlation
 *                    R_pq[d] = sum_k conj(s_p[k]) s_q[k+d] on the box |d| <= 2 tau (Sec. V-A);
 *                    only p <= q is written.  B = 4 tau + 1.
 *   PISCO_BUF_GRAM   complex128 [Q|Lambda|][Q|Lambda|] C^H C, index q*|Lambda| + i.
 *   PISCO_BUF_SIGNAL complex64 [Q|Lambda|][m] signal-subspace basis (column j is used when
 *                    PISCO_BUF_WEIGHTS[j] = 1), Lambda in lexicographic order, x fastest.
 *   PISCO_BUF_WEIGHTS float [m] 1 for signal columns, 0 otherwise.
 *   PISCO_BUF_RITZ   double [m] Ritz values of C^H C (FP64 Rayleigh quotients where decided).
 *   PISCO_BUF_G      complex64 [Nr][Q][Q], G_pq(x) on the reduced grid (Nr pixels).
 *   PISCO_BUF_V      complex64 [Q][Nr] phase-aligned power-iteration vectors.
 *   PISCO_BUF_Y      complex64 [Q][Nr] apodised low-resolution coil images (Sec. V-D).
 *   PISCO_BUF_BLOCK  complex64 [Q|Lambda|][m] orthonormal block before the Rayleigh-Ritz step.
 *   PISCO_BUF_RITZ32 float [m] FP32 Ritz values of C^H C / scale, descending.
 *   PISCO_BUF_SCALE  double: scale = max diagonal entry of C^H C. */
enum {
  PISCO_BUF_LAGS = 0, PISCO_BUF_GRAM = 1, PISCO_BUF_SIGNAL = 2, PISCO_BUF_WEIGHTS = 3,
  PISCO_BUF_RITZ = 4, PISCO_BUF_G = 5, PISCO_BUF_V = 6, PISCO_BUF_Y = 7, PISCO_BUF_BLOCK = 8,
  PISCO_BUF_RITZ32 = 9, PISCO_BUF_SCALE = 10
};
pisco_status pisco_debug_buffer(pisco_plan_t plan, int which, void** dptr, size_t* bytes);

/* Counters of the last estimate. */
typedef struct {
  int launches;       /* CUDA kernels enqueued by the last pisco_estimate (all retries)   */
  int eig_block;      /* block size m of the nullspace eigensolver actually used          */
  int eig_iters;      /* subspace iterations per solve                                   */
  int jacobi_sweeps;  /* sweeps of the last small Rayleigh-Ritz eigensolve                */
  int nband;          /* Ritz values decided on FP64 Rayleigh quotients                   */
  double lambda_max;  /* largest eigenvalue of C^H C (sigma_1^2), FP64                     */
  int signal_dim;     /* k = Q|Lambda| - R                                                 */
  int filter_len;     /* |Lambda|                                                          */
  int warm_fallback;  /* pixels re-solved from the plain start (warm start only)            */
  double cert_margin; /* certificate of the threshold split: min over the Ritz values decided
                         in FP64 of (|mu - theta| - b) / theta, theta = thr^2 lambda_1 and b
                         the FP64 residual (Kato-Temple) bound; > 0 means certified        */
  double band_resid;  /* largest FP64 residual ||A x - mu x|| / lambda_1 of those vectors   */
} pisco_stats;
pisco_status pisco_get_stats(pisco_plan_t plan, pisco_stats* out);

/* Operation timing with CUDA events on the plan's stream.  When enabled, every operation of
 * pisco_estimate (a kernel, or a GEMM with its split-K reduction) is bracketed by two events
 * and, after the estimate's final synchronisation, its elapsed time is added to a per-name
 * total.  pisco_profile_entry enumerates the totals (idx = 0, 1, ... until PISCO_ERR_ARG);
 * `name` points to a static string.  Timing adds two event records per operation. */
pisco_status pisco_set_profiling(pisco_plan_t plan, int enable);
pisco_status pisco_profile_reset(pisco_plan_t plan);
pisco_status pisco_profile_entry(pisco_plan_t plan, int idx, const char** name, double* total_ms,
                                 int* count);

/* Batches of independent estimates (many slices or volumes, sizes and coil counts may
 * differ; the database setting of Sec. I).  pisco_batch_plan groups the items: items of identical
 * parameters (up to params.batch_group of them) share one plan whose passes run every stage as
 * ONE launch over all of them (item-strided workspace; each item's result is bitwise the one
 * pisco_estimate gives it alone), other items get a plan each.  pisco_batch_estimate captures
 * every group's pass into ONE CUDA graph whose branches (one per group) run concurrently on the
 * GPU, launches it on `cuda_stream`, synchronises once and reports each item's status in
 * item_status[i] (may be NULL).  The graph is replayed while
 * the pointer arrays stay the same.  Pointer arrays hold `count` device pointers with the
 * layouts of pisco_estimate (d_eig may be NULL, or hold NULL entries).  An item whose signal
 * dimension saturates its eigensolver block, or whose threshold split is not certified yet with
 * the automatic iteration count, is re-run alone with a larger block or more iterations (its
 * group keeps the larger setting for later calls).  Returns the
 * most severe item status.  The _host variant takes host pointers (pinned memory for full
 * copy bandwidth): the host->device copies are enqueued on the batch's stream ahead of the graph,
 * the device->host copies right after it (copy-engine copies that overlap the computation of
 * the next host-I/O batch, which is ordered after this batch's computation).  pisco_batch_item exposes item i's plan for
 * pisco_plan_info / pisco_debug_buffer / pisco_get_stats (owned by the batch; for an item of a
 * group, a one-item view into the group's workspace). */
typedef struct pisco_batch_s* pisco_batch_t;
pisco_status pisco_batch_plan(const pisco_params* params, int count, void* cuda_stream,
                              pisco_batch_t* out);
pisco_status pisco_batch_estimate(pisco_batch_t b, const void* const* d_calib, void* const* d_maps,
                                  float* const* d_eig, pisco_status* item_status);
pisco_status pisco_batch_estimate_host(pisco_batch_t b, const void* const* h_calib,
                                       void* const* h_maps, float* const* h_eig,
                                       pisco_status* item_status);
/* The host-buffer call split in two, so that a caller can keep two batch objects in flight and
 * overlap one step's host copies with the next step's computation: pisco_batch_launch_host
 * enqueues the whole batch (host->device copies, estimates, device->host copies) on the batch's
 * private stream and returns at once; pisco_batch_wait blocks until it has finished and fills
 * item_status as pisco_batch_estimate_host does.  The host buffers must stay valid and
 * untouched until the wait returns.  One launch per batch object may be in flight
 * (PISCO_ERR_ARG for a second launch, or for a wait without a launch). */
pisco_status pisco_batch_launch_host(pisco_batch_t b, const void* const* h_calib,
                                     void* const* h_maps, float* const* h_eig);
/* pisco_batch_estimate split the same way: the batch is enqueued after the work already on the
 * plan's (caller's) stream, that stream is made to wait for its completion, and the call
 * returns without synchronising; pisco_batch_wait decodes the item statuses.  A caller keeps
 * the GPU fed by launching the next batch object before waiting for this one. */
pisco_status pisco_batch_launch(pisco_batch_t b, const void* const* d_calib, void* const* d_maps,
                                float* const* d_eig);
pisco_status pisco_batch_wait(pisco_batch_t b, pisco_status* item_status);
pisco_status pisco_batch_info(pisco_batch_t b, int* count, int* launches, size_t* workspace_bytes);
pisco_status pisco_batch_item(pisco_batch_t b, int i, pisco_plan_t* plan);
/* Operation timing of a batch (as pisco_set_profiling for one plan): while enabled, batch calls
 * run eagerly (no graph) and every operation of every group's pass, each one launch over the
 * group's items, is bracketed by CUDA events on the group's stream; totals per operation name
 * are summed over the groups and enumerated by pisco_batch_profile_entry (idx = 0, 1, ... until
 * PISCO_ERR_ARG).  pisco_batch_groups reports the number of groups and the items of the
 * largest. */
pisco_status pisco_batch_set_profiling(pisco_batch_t b, int enable);
pisco_status pisco_batch_profile_reset(pisco_batch_t b);
pisco_status pisco_batch_profile_entry(pisco_batch_t b, int idx, const char** name, double* total_ms,
                                       int* count);
pisco_status pisco_batch_groups(pisco_batch_t b, int* groups, int* largest);
void pisco_batch_destroy(pisco_batch_t b);

/* Allocation-free variant of stage (a).  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory when they need the result -- code
 * under a fixed-budget or custom allocator that forbids cudaMalloc/cudaFree on its hot path,
 * pipelines that must not synchronise the device (cudaFree does), or embedded hosts that hand
 * in pre-sized buffers.  It computes the same lag table as pisco_estimate (PISCO_BUF_LAGS):
 *   d_calib: device, complex64 [Q][Nc_z][Nc_y][Nc_x] (8-byte aligned), read only;
 *   d_lags:  device, complex128 [Q][Q][B_z][B_y][B_x] with B = 4 tau + 1 (16-byte aligned),
 *            written in full: R_pq[d] for p <= q, zero for p > q.
 * Only p->ndim, calib, num_coils and kernel_radius are read.  Every intermediate lives in one
 * 32 MiB scratch array compiled into the library, which each GPU that loads the library
 * holds until the process exits; requests that need more return PISCO_ERR_TOO_LARGE (the 2D
 * 32x32 Q=32 radius-3 case needs about 20 MiB).  No cudaMalloc, cudaFree or allocating
 * library call is made.  The first call on a device resolves the scratch array's device
 * address for that device (cudaGetSymbolAddress, with that device current), so make that
 * first call before any stream capture.  All calls share the scratch and it keeps the last
 * call's contents; calls that overlap on the GPU (two streams, two threads) race.
 * Work is enqueued on `cuda_stream` (NULL: legacy default stream); returns without
 * synchronising. */
pisco_status pisco_gram_lags_noalloc(const pisco_params* p, const void* d_calib, void* d_lags,
                                     void* cuda_stream);

/* Reduced-grid support mask from an eigenvalue map (as pisco_estimate writes it):
 * d_mask[i] = 1 where d_eig[i] < threshold, else 0.  lambda_min(G)/|Lambda| is ~0 inside the
 * object, where the maps are identifiable (Sec. II), and grows outside; 0.05 mirrors the
 * nullspace threshold.  d_eig: device float[n]; d_mask: device uint8[n]; enqueued on
 * cuda_stream, no synchronisation. */
pisco_status pisco_support_mask(const float* d_eig, long long n, float threshold, unsigned char* d_mask,
                                void* cuda_stream);

/* ---- Learned warm start of the power iteration (an addition of this library; the paper
 * starts every pixel from an arbitrary vector, Sec. V-E) ------------------------------------
 * A per-pixel MLP maps the patch of normalised low-resolution coil vectors around the pixel
 * (Sec. V-D's apodised images; see pisco_warm_start_patch_features: (2r+1)^D neighbours of 2Q
 * reals, real and imaginary parts interleaved per coil) through two ReLU hidden layers to a
 * proposed start vector (2Q reals):
 *     h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), out = s(x) + W3 h2 + b3,
 * the skip term s(x) = the middle block of x (the centre pixel's own normalised vector) when
 * n_in is an odd multiple of n_out, else absent (with W3 = 0, b3 = 0 the network returns the
 * heuristic start).  Parameters travel as one FP32 blob [W1 | b1 | W2 | b2 | W3 | b3], weights
 * row-major (W1: n_hidden x n_in, W2: n_hidden x n_hidden, W3: n_out x n_hidden).  Every layer
 * product runs on the tensor cores with FP16 operands (the weights stored in FP16, the
 * activations and per-sample gradients rounded to FP16 where they enter a product) and FP32
 * accumulation; biases, activations and the Adam state (FP32 master weights) stay FP32.
 * n_in in [1, 4096], n_hidden and n_out in [1, 128].  Calls are enqueued on the stream given
 * at creation. */
typedef struct pisco_mlp_s* pisco_mlp_t;

/* Create a network with the given parameters (host blob, copied) and device workspace for
 * batches of up to max_batch samples (<= 4,000,000). */
pisco_status pisco_mlp_create(int n_in, int n_hidden, int n_out, const float* h_params,
                              long long max_batch, void* cuda_stream, pisco_mlp_t* out);
/* Replace the parameters (host blob) and reset the Adam moments and step count. */
pisco_status pisco_mlp_write(pisco_mlp_t mlp, const float* h_params);
/* d_out[b][:] = network(d_x[b][:]); device FP32 arrays [batch][n_in] and [batch][n_out]. */
pisco_status pisco_mlp_forward(pisco_mlp_t mlp, const float* d_x, long long batch, float* d_out);
/* Forward and backward pass of L = (1/batch) sum_b l(out_b, t_b) for device FP32 inputs d_x
 * [batch][n_in] and targets d_target [batch][n_out]: l = ||out - t||^2 (loss kind 0, the
 * default) or the direction loss l = 1 - |<o, t>| / (||o|| ||t||) of the complex vectors o, t
 * (kind 1; <o, t> = sum_q conj(o_q) t_q over the n_out/2 interleaved entries; l = 0 and no
 * gradient where o or t is zero).  The gradient of every parameter is kept in the network
 * (pisco_mlp_read which = 1).  h_loss (optional): L, after a synchronisation. */
pisco_status pisco_mlp_backward(pisco_mlp_t mlp, const float* d_x, const float* d_target,
                                long long batch, double* h_loss);
/* Loss of pisco_mlp_backward: 0 squared error, 1 direction loss (needs an even n_out). */
pisco_status pisco_mlp_set_loss(pisco_mlp_t mlp, int kind);
/* One Adam step (bias-corrected) with the last gradient. */
pisco_status pisco_mlp_adam(pisco_mlp_t mlp, float lr, float beta1, float beta2, float eps);
/* Copy the FP32 parameters (which = 0) or the last gradient (which = 1) into a host blob;
 * synchronises. */
pisco_status pisco_mlp_read(pisco_mlp_t mlp, int which, float* h_out);
void pisco_mlp_destroy(pisco_mlp_t mlp); /* NULL-safe */
/* The network's input features, as the estimate computes them, from low-resolution coil images
 * d_y (device complex64 [Q][npix], the layout of PISCO_BUF_Y) on the reduced grid dims
 * (ndim = 2: {N_y, N_x}; 3: {N_z, N_y, N_x}; periodic) to d_x (device FP32
 * [npix][(2r+1)^ndim][2Q]): for every neighbour o of the pixel j (z slowest, x fastest; radius
 * r in [0, 3]) the vector y(j+o) conj(y_0(j)) / (|y_0(j)| ||y(j)||), real and imaginary parts
 * interleaved (no rotation where y_0(j) = 0; zeros where y(j) = 0). */
pisco_status pisco_warm_start_patch_features(const void* d_y, int Q, const int* dims, int ndim,
                                             int radius, float* d_x, void* cuda_stream);
/* The radius-0 features of npix pixels: y_j conj(y_0j) / (|y_0j| ||y_j||), [npix][2Q]. */
pisco_status pisco_warm_start_features(const void* d_y, int Q, long long npix, float* d_x,
                                       void* cuda_stream);

/* Use `mlp` (n_out = 2Q, n_in = (2r+1)^D 2Q for a patch radius r in [0, 3]; copied into the
 * plan; one-item plans only; NULL switches the warm start off) to
 * start the power iteration of every reduced-grid pixel, run `iters` iterations, and
 * re-solve from the plain start vector with `fallback_iters` iterations every pixel whose
 * residual ||G v - lambda |Lambda| v|| / |Lambda| exceeds `gate` (gate <= 0: no fallback).
 * The number of re-solved pixels of the last estimate is in pisco_stats.warm_fallback. */
pisco_status pisco_set_warm_start(pisco_plan_t plan, pisco_mlp_t mlp, int iters, float gate,
                                  int fallback_iters);

/* The dense complex contraction behind PISCO_FLAG_TC_GFIELD / PISCO_FLAG_TC_EIG /
 * PISCO_FLAG_TC_INTERP, exposed for testing and reuse: C = alpha * A * op(B) + beta * C on the
 * tensor cores (tcgen05, TF32 operands, FP32 accumulation in tensor memory).  The operands are
 * first split into TF32 head/tail arrays in the caller's workspace (the tensor core's K-major
 * layout), then TMA loads feed a shared-memory ring consumed by tcgen05.mma.  K may be split over
 * `splits` CTAs per tile (partials summed in a fixed order, deterministic).
 *   nterms: 3 = each FP32 operand split into a TF32 head and tail, three products per entry
 *           (close to FP32 accuracy); 1 = one TF32 product (about 11 significant bits);
 *   A: device complex64 M x K, row-major, leading dimension lda >= K;
 *   opB 0: B is device complex64 K x N row-major, ldb >= N;
 *   opB 1: op(B) = conj(Bs^T) with Bs device complex64 N x K row-major, ldb >= K;
 *   C: device complex64 M x N row-major, ldc >= N, read when beta != 0, written;
 *   alpha, beta: host float[2] (real, imaginary);
 *   d_workspace: device, 16-byte aligned, at least
 *           pisco_tc_cgemm_pipelined_workspace(nterms, M, N, K, splits) bytes;
 *   d_status: optional device int; bit 16 is OR-ed in if a bounded device wait expired.
 * A, B, C 8-byte aligned (PISCO_ERR_ARG otherwise, nothing launched).  Enqueued on
 * `cuda_stream`; returns without synchronising.  The first call sets kernel attributes, so
 * make it outside stream capture. */
size_t pisco_tc_cgemm_pipelined_workspace(int nterms, int M, int N, int K, int splits);
/* Test hook of the bounded device waits (the paper has no counterpart): while enabled, the
 * tensor-core products launched by this process issue none of their shared-memory loads and
 * give up waiting after about 10 ms, so every such launch ends with its wait expired (bit 16 of
 * the status word: pisco_estimate returns PISCO_ERR_TIMEOUT) and its tensor memory freed.
 * Nothing else changes; disabling it restores normal products.  Not for production use. */
void pisco_test_stall_tensor_loads(int enable);
pisco_status pisco_tc_cgemm_pipelined(int nterms, int M, int N, int K, const float* alpha,
                                      const void* d_A, int lda, const void* d_B, int ldb, int opB,
                                      const float* beta, void* d_C, int ldc, int splits,
                                      void* d_workspace, size_t workspace_bytes, int* d_status,
                                      void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* PISCO_H_ */
