// Shared device helpers and internal launcher declarations of the PISCO GB300 path.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pisco.h"

namespace pisco {

// kernels enqueued by the calling thread (read by the host orchestration per estimate)
inline thread_local int g_launches = 0;

// ---------------------------------------------------------------------------------------
// complex arithmetic on float2 / double2
// ---------------------------------------------------------------------------------------
template <typename T> struct cplx;
template <> struct cplx<float> { using type = float2; };
template <> struct cplx<double> { using type = double2; };
template <typename T> using cpx = typename cplx<T>::type;

__host__ __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
__host__ __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) { return mk(a.x + b.x, a.y + b.y); }
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) { return mk(a.x - b.x, a.y - b.y); }
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
  return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __host__ __device__ __forceinline__ C cconj(C a) { return mk(a.x, -a.y); }
// acc += a * b
template <typename C> __device__ __forceinline__ void cfma(C& acc, C a, C b) {
  acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a) * b
template <typename C> __device__ __forceinline__ void cfmac(C& acc, C a, C b) {
  acc.x = fma(a.x, b.x, acc.x); acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y); acc.y = fma(-a.y, b.x, acc.y);
}
__device__ __forceinline__ float2 to_c(double2 a) { return make_float2((float)a.x, (float)a.y); }
__device__ __forceinline__ double2 to_z(float2 a) { return make_double2(a.x, a.y); }

// ---------------------------------------------------------------------------------------
// SplitMix64 (Steele, Lea & Flood 2014): one output for a 64-bit counter.
// ---------------------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
// 24-bit uniform in [-1, 1) for counter (seed, index, t); exact in FP32.
__host__ __device__ __forceinline__ float counter_uniform(uint64_t seed, uint64_t index, uint64_t t) {
  uint64_t r = splitmix64((seed << 40) + (index << 8) + t) >> 40;
  return (float)((int64_t)r - (1ll << 23)) * (1.0f / 8388608.0f);
}

// ---------------------------------------------------------------------------------------
// device status word (written by kernels, read once per estimate)
// ---------------------------------------------------------------------------------------
enum : int {
  ST_RANK = 1,          // R < Q-1
  ST_SATURATED = 2,     // signal dimension reached the eigensolver block
  ST_CHOL = 4,          // non-positive pivot clamped in a Cholesky factorisation
  ST_ZERO = 8,          // calibration data identically zero
  ST_TIMEOUT = 16,      // a bounded wait of a tensor-core kernel expired
  ST_UNCERTIFIED = 32,  // FP64 residual bounds do not certify the threshold split
};
struct DevStatus {
  int flags;            // ST_* bits
  int k;                // signal dimension decided by the eigensolver
  int nband;            // Ritz values refined in FP64
  int jacobi_sweeps;    // sweeps used by the last small eigensolve
  double lambda_max;    // largest eigenvalue of C^H C (FP64 Rayleigh quotient)
  int ws_fallback;      // pixels re-solved after the warm start's residual gate
  double cert_margin;   // min over the band of (|mu - theta| - bound) / theta (certificate)
  double band_resid;    // max FP64 residual of the band vectors / lambda_1
};

// ---------------------------------------------------------------------------------------
// launchers (all asynchronous on `st`; return cudaGetLastError())
// ---------------------------------------------------------------------------------------
// Generic "apply a matrix along one axis": out[b][a2][o][a0] = sum_i M[o][i] in[b][a2][i][a0]
// for a 5-level view (batch, outer, axis, inner); element types given by the template.
struct AxisView {
  long long batch;   // number of independent batches
  long long outer;   // product of the axis lengths before the transformed axis
  int n_in;          // transformed axis length on input
  int n_out;         // transformed axis length on output
  long long inner;   // product of the axis lengths after the transformed axis
  int pixel_major = 0;  // 1 (needs outer == 1): write out[(o*inner + ii)*batch + b] instead
  int mt = 0;        // 1: the matrix is stored transposed, M[i][o] ([n_in][n_out]); for
                     // inner == 1 passes this makes a warp's matrix reads contiguous
  int pm_group = 0;  // pixel_major with batch = items x pm_group: item-major blocks, each
                     // [n_out * inner][pm_group] (0: one block of the whole batch)
};
cudaError_t apply_axis_c2z(const float2* in, const double2* M, double2* out, AxisView v, cudaStream_t st);
cudaError_t apply_axis_z(const double2* in, const double2* M, double2* out, AxisView v, cudaStream_t st);
cudaError_t apply_axis_c(const float2* in, const float2* M, float2* out, AxisView v, cudaStream_t st);

// a1: pair products and Gram expansion.  `it.n` independent Grams per launch (grid z or y is
// the item); item i of each per-item buffer starts i * stride elements after item 0.
struct GramItems {
  int n = 1;
  long long calib = 0;   // calibration blocks
  long long S = 0;       // spectra [Q][nfreq]
  long long P = 0;       // pair products [npairs][nfreq]
  long long Rp = 0;      // pair lag boxes [npairs][nbox]
  long long lags = 0;    // lag tables [Q][Q][nbox] (FP64 and double-float)
  long long A = 0;       // Gram and its FP32 copy (entries)
  long long scale = 0;
};
cudaError_t gram_pair_products(const double2* S, int Q, long long nfreq, double2* P, cudaStream_t st,
                               const GramItems& it = GramItems{});
cudaError_t gram_scatter_pairs(const double2* Rpairs, int Q, int nbox, double2* lags, cudaStream_t st,
                               const GramItems& it = GramItems{});
cudaError_t gram_scale(const double2* lags, int Q, int nbox, int lag0, double* scale, cudaStream_t st,
                       const GramItems& it = GramItems{});
cudaError_t gram_expand(const double2* lags, const int* lag_of_ij, int Q, int L, int nbox,
                        const double* scale, double2* A, float2* A32, cudaStream_t st,
                        const GramItems& it = GramItems{});

// dense complex GEMM: C = alpha*op(A)*op(B) + beta*C, row-major, op in {'N','C'}
// Split-K partials go to splitk_ws (ws_elems entries); tile_count must hold 4096 zeroed ints
// (the kernel returns them to zero).  With splitk_ws == nullptr there is no split.
// max_splits caps the split-K factor (0: automatic, about two CTAs per SM): many splits cut the
// latency of one product, few splits its SM-time (what a batch of concurrent estimates needs)
template <typename T>
cudaError_t cgemm(char opA, char opB, int M, int N, int K, cpx<T> alpha, const cpx<T>* A, int lda,
                  const cpx<T>* B, int ldb, cpx<T> beta, cpx<T>* C, int ldc, cpx<T>* splitk_ws,
                  size_t ws_elems, int* tile_count, cudaStream_t st, int max_splits = 0, int tile = 0,
                  int items = 1, long long sA = 0, long long sB = 0, long long sC = 0);

// a2: block eigensolver pieces.  Every launcher runs `it.n` independent solves in one launch
// (grid dimension z, or y for the multi-CTA kernels, indexes the item); item i of a per-item
// buffer starts i * stride elements after item 0.
struct EigItems {
  int n = 1;              // items
  long long mm = 0;       // m x m blocks (Gram of the block, Rinv / L, Rayleigh-Ritz matrix)
  long long vj = 0;       // Jacobi output + scratch (2 m_max^2)
  long long vec = 0;      // m-vectors (scalings, diag(R), Ritz values, weights, FP64 Ritz values)
  long long nm = 0;       // n x m blocks
  long long nb = 0;       // band blocks (n x 8)
  long long band = 0;     // band index vectors
  long long a = 0;        // FP64 / double-float Gram (entries)
  long long scale = 0;    // Gram scale
};
cudaError_t eig_random_block(float2* X, int n, int m, unsigned long long seed, cudaStream_t st);
// thin block products for m <= 64 (FP32, CUDA cores): C = Y^H Z (m x m over n rows; ws holds
// items * eig_thin_chunks(n) * m * m partials, tickets one zeroed int per item) and X = Y W
int eig_thin_chunks(int n);
cudaError_t eig_thin_gram(const float2* Y, long long sY, const float2* Z, long long sZ, int n, int m, float2* C,
                          long long sC, float2* ws, int* tickets, int items, cudaStream_t st);
cudaError_t eig_thin_apply(const float2* Y, long long sY, const float2* W, long long sW, int n, int m, float2* X,
                           long long sX, int items, cudaStream_t st);

cudaError_t eig_chol(const float2* Gm, int m, const float* dscale, float shift_rel,
                     const float* acc_in, float2* L, float* dout, float* diagR, DevStatus* status,
                     cudaStream_t st, const EigItems& it = EigItems{});
cudaError_t eig_trsm(const float2* Y, const float2* L, const float* ds, int n, int m, float2* X,
                     cudaStream_t st, const EigItems& it = EigItems{});
cudaError_t eig_chol_inv_blocked(const float2* Gm, int m, const float* dscale, float shift_rel,
                                 const float* acc_in, float2* Rinv, float* diagR, DevStatus* status,
                                 cudaStream_t st, const EigItems& it = EigItems{});
cudaError_t eig_jacobi(const float2* B, int m, float* mu, float2* V, int max_sweeps,
                       float skip_rel, float stop_rel, DevStatus* status, cudaStream_t st,
                       const EigItems& it = EigItems{});
cudaError_t eig_band_matvec(const double2* A, const double2* Xb, int n, int nb, const int* band_idx,
                            double2* Zb, cudaStream_t st, const EigItems& it = EigItems{});
cudaError_t eig_select_band(const float* mu, int m, double thr2, int nb_max, int* band_idx,
                            cudaStream_t st, const EigItems& it = EigItems{});
cudaError_t eig_gather_band(const float2* X, int n, int m, const int* band_idx, int nb_max,
                            double2* Xb, cudaStream_t st, const EigItems& it = EigItems{});
cudaError_t eig_decide(const float* mu, int m, const int* band_idx, int nb_max, const double2* Xb,
                       const double2* Zb, int n, double thr2, int Q, const double* scale,
                       float* weights, double* ritz, DevStatus* status, cudaStream_t st,
                       const EigItems& it = EigItems{});

// a3: collapsed kernel and G field
cudaError_t gassembly_kernel(const float2* U, const float* w, int Q, int L, int m,
                             const int* lag_ptr, const int* lag_ent, int nbox, float2* K,
                             cudaStream_t st);
cudaError_t gassembly_add_identity(float2* G, int Q, long long npix, float lam_size, cudaStream_t st);
// the folded lag table KT [nlag][Q*Q] spread onto the lag box K [Q*Q][nbox] (zero where box_lag < 0)
cudaError_t gassembly_scatter_box(const float2* KT, const int* box_lag, int QQ, int nbox, float2* K, cudaStream_t st,
                                  int items = 1, long long sKT = 0, long long sK = 0);
cudaError_t gassembly_collapse(const float2* P, int n, int Q, int L, const int* lagc_ptr,
                               const int* lag_ent, int nlag, float2* KT, cudaStream_t st, int items = 1,
                               long long sP = 0, long long sKT = 0);

// the Gram's FFT route in double-float arithmetic (kernels_gram_df.cu); tables and buffers hold
// {Re hi, Re lo, Im hi, Im lo} float quadruples in the storage of the FP64 path
cudaError_t apply_axis_c2df(const float2* in, const void* M, void* out, AxisView v, cudaStream_t st);
cudaError_t apply_axis_df(const void* in, const void* M, void* out, AxisView v, cudaStream_t st);
cudaError_t gram_pair_products_df(const void* S, int Q, long long nfreq, void* P, cudaStream_t st,
                                  const GramItems& it = GramItems{});
// the lag table is written twice: FP64 (lags) and double-float (lags_df, for the expansion)
cudaError_t gram_scatter_pairs_df(const void* Rp, int Q, int nbox, double2* lags, void* lags_df, cudaStream_t st,
                                  const GramItems& it = GramItems{});
// A kept as double-float quadruples (no FP64 arithmetic per entry); A32 = A / scale
cudaError_t gram_expand_df(const void* lags_df, const int* lag_of_ij, int Q, int L, int nbox, const double* scale,
                           void* A, float2* A32, cudaStream_t st, const GramItems& it = GramItems{});
cudaError_t df_to_fp64(const void* in, long long count, double2* out, cudaStream_t st);
// a_df: A holds double-float quadruples, else FP64
cudaError_t eig_band_matvec_df(const void* A, bool a_df, const double2* Xb, int n, int nb, const int* band_idx,
                               double2* Zb, cudaStream_t st, const EigItems& it = EigItems{});

// exact Gram of the masked calibration matrix (kernels_gram.cu): A (FP64 n x n), scale, A32
// the masked Gram's summed-area table of one (pair, lag) holds every calibration sample in shared
// memory (16 bytes each): up to 227 KB, i.e. 14528 samples (24^3 = 13824 fits)
constexpr int kMaskedMaxSamples = 14528;
cudaError_t gram_masked(const float2* calib, int Q, const int* Nc, const int* lo, const int* hi, const int* lam,
                        int L, const int* lag_ids, const int* lagc_ptr, const int* lag_ent, int nlag, const int* tau,
                        const int* B, double2* A, double* scale, float2* A32, cudaStream_t st);
cudaError_t gram_masked_prepare(int nvol);
size_t gram_masked_smem(int nvol);

cudaError_t normalize_maps(float2* maps, int Q, long long npix, cudaStream_t st, int items = 1, long long sM = 0,
                           float2* const* maps_tab = nullptr);

// 2D double-float Gram pairs stage fused per pair (kernels_gram_df.cu): pair product, both
// inverse lag passes, lag table lags[(p,q)][B1*B2] for p <= q in FP64 and in double-float
constexpr int kPairsInverseDfMaxSmem = 200 * 1024;
bool gram_pairs_inverse_df_supported(int Lp1, int Lp2, int B1, int B2);
// 2D double-float forward stage fused per coil: S[q][Lp1][Lp2] from calib[q][Nc1][Nc2]
bool gram_forward_df_supported(int Nc1, int Nc2, int Lp1, int Lp2);
cudaError_t gram_forward_df(const float2* calib, int Q, int Nc1, int Nc2, const void* fwdT2, int Lp2, const void* fwd1,
                            int Lp1, void* S, cudaStream_t st, const GramItems& it = GramItems{});
cudaError_t gram_pairs_inverse_df(const void* S, int Q, int Lp1, int Lp2, const void* invT2, int B2, const void* inv1,
                                  int B1, double2* lags, void* lags_df, cudaStream_t st,
                                  const GramItems& it = GramItems{});

// 2D G(x) from the collapsed lag kernel KT[nlag][Q*Q] by two separable DFT passes
// (kernels_gassembly.cu); row_ptr[B1+1] groups the lags by row, lag_b2 their column
constexpr int kGfieldSep2MaxSmem = 200 * 1024;
bool gassembly_field_sep2_supported(int nlag, int Nr1, int B1, int Nr2, int B2);
cudaError_t gassembly_field_sep2(const float2* KT, int Q, int nlag, const int* row_ptr, const int* lag_b2,
                                 const float2* E1, int Nr1, int B1, const float2* E2, int B2, int Nr2,
                                 float lam_size, float2* G, cudaStream_t st, int items = 1, long long sKT = 0,
                                 long long sG = 0);

// warm-start MLP (kernels_mlp.cu): n_in -> H -> H -> n_out (n_in <= 4096, H and n_out <= 128);
// w32 is the FP32 parameter blob [W1 | b1 | W2 | b2 | W3 | b3] (row-major weights), w16 its
// FP16 copy (the matrices are read from w16, the biases from w32)
struct MlpView {
  int n_in, H, n_out;
  const float* w32;
  const __half* w16;
};
MlpView mlp_view(const pisco_mlp_s* m);
void mlp_dims(const pisco_mlp_s* m, int* n_in, int* H, int* n_out, size_t* nparam);
cudaError_t mlp_prepare();
size_t mlp_param_count(int n_in, int H, int n_out);
size_t mlp_part_floats(long long max_batch, int n_in, int H, int n_out);
cudaError_t mlp_forward(const MlpView& m, const float* X, long long B, float* H1, float* H2, float* out,
                        cudaStream_t st);
cudaError_t mlp_backward(const MlpView& m, const float* X, const float* T, long long B, float* H1, float* H2,
                         float* out, float* dO, float* dH2, float* dH1, float* part, float* grad,
                         float* loss_part, int loss_blocks, int loss_kind, cudaStream_t st);
cudaError_t mlp_adam(float* w32, __half* w16, const float* g, float* m1, float* m2, long long n, float lr,
                     float b1, float b2, float eps, int step, cudaStream_t st);
cudaError_t mlp_to_half(const float* w32, __half* w16, long long n, cudaStream_t st);
cudaError_t mlp_features(const float2* Y, int Q, long long npix, float* X, cudaStream_t st);
// patch features on the reduced grid dims (z, y, x) of D dimensions, radius r: [npix][(2r+1)^D 2Q]
cudaError_t mlp_patch_features(const float2* Y, int Q, const int dims[3], int r, int D, float* X, cudaStream_t st);
// column offset of the skip term in x (the middle block when n_in is an odd multiple of n_out), or -1
int mlp_skip_offset(int n_in, int n_out);

// TMA-fed tensor-core complex GEMM over operands split once in global memory (kernels_tc2.cu).
// A' head/tail: [M][tc2_k2p(K)] floats; B' head/tail: [2 tc2_np(N)][tc2_k2p(K)] floats
// (lo pointers may be null for one pass).  splits > 1 needs ws of splits*M*N complex.
int tc2_k2p(int K);
int tc2_np(int N);
cudaError_t tc2_prepare();
// test hook: while set, tensor-core GEMM launches issue no TMA loads and wait ~10 ms at most, so
// their bounded waits expire with nothing in flight (bit 16 of err, TMEM freed as always)
void tc2_set_stall(bool on);
// The split kernels take `items` independent operands (inputs item_stride elements apart, the
// split arrays one after another).
cudaError_t tc2_split_a(const float2* A, int lda, const float* kscale, int M, int K, float* hi, float* lo,
                        cudaStream_t st, int items = 1, long long a_stride = 0, long long w_stride = 0);
// cg > 0 (opB 0): column c of B is column c % cg of block c / cg, blocks cgs elements apart
cudaError_t tc2_split_b(const float2* B, int ldb, int opB, int K, int N, float* hi, float* lo, cudaStream_t st,
                        int nbatch = 1, long long b_stride = 0, int cg = 0, long long cgs = 0);
cudaError_t tc2_split_at(const float2* Y, int ldy, int M, int K, float* hi, float* lo, cudaStream_t st,
                         int items = 1, long long y_stride = 0);
// nbatch > 1: gridDim.z runs nbatch products C_b = A_b B_b (B' items of 2 Np rows one after
// another; A shared, or with a_per_item one A' of M rows per item; C_b at C + b c_stride, or at
// c_tab[b / c_div] + (b % c_div) c_stride; no split-K)
cudaError_t tc2_gemm(int nterms, int M, int N, int K, const float* Ahi, const float* Alo, const float* Bhi,
                     const float* Blo, float2 alpha, float2 beta, float2* C, int ldc, float diag_val,
                     int diag_stride, int diag_limit, int splits, float2* ws, int* err, cudaStream_t st,
                     int nbatch = 1, long long c_stride = 0, int a_per_item = 0, float2* const* c_tab = nullptr,
                     int c_div = 1, int b_per_item = 1, const float2* a_fp32 = nullptr, int lda_fp32 = 0,
                     int rg = 0, int rg_rows = 0, long long rg_plane = 0, int rg_norm = 0);
// rg > 0 (nbatch 1): the rows of C are (item, y, q) triples, rg_rows = rows per item, rg = Q;
// row (item, y, q) goes to (c_tab[item] or C + item c_stride) + q rg_plane + y ldc, and with
// rg_norm (rg dividing 128) each column of a q-group is divided by its 2-norm
// a_fp32: A given as FP32 complex rows (leading dimension lda_fp32, even; items lda_fp32 * M apart
// with a_per_item) and split into head and tail in shared memory (three passes only); Ahi/Alo unused
bool tc2_conv_ok(int K, int lda_fp32, const void* a_fp32);


// a4+a5: power iteration with the phase step
cudaError_t power_iteration_block2(const float2* G, const float2* Y, int Q, long long npix, int iters,
                                   float lam_size, unsigned long long seed, float2* V, float* eig, cudaStream_t st);
cudaError_t support_mask(const float* eig, long long n, float thr, unsigned char* mask, cudaStream_t st);
// warm-start options of the power iteration: v0 [npix][2Q] start proposals (null: counter
// start); gate > 0 flags pixels with residual above it (flags [npix], count += flagged);
// only != null re-solves only the pixels with only[x] != 0
struct PiOpts {
  const float* v0 = nullptr;
  float gate = 0.f;
  int* flags = nullptr;
  int* count = nullptr;
  const int* only = nullptr;
  // independent estimates in one launch (grid y = item): G, Y, V of item i start i * sG, sY, sV
  // elements after item 0; its eigenvalues go to eig_tab[i] (or eig + i * sE)
  int items = 1;
  long long sG = 0, sY = 0, sV = 0, sE = 0;
  float* const* eig_tab = nullptr;
};
cudaError_t power_iteration(const float2* G, const float2* Y, int Q, long long npix, int iters,
                            float lam_size, unsigned long long seed, float2* V, float* eig,
                            cudaStream_t st, const PiOpts& opt = PiOpts{});

// a6: final interpolation pass along the slowest axis fused with unit-norm normalisation
// (items independent outputs: T of item i at T + i * sT, maps at maps_tab[i] or maps + i * sM)
cudaError_t interp_final_normalize(const float2* T, const float2* M, int Q, long long outer_dummy,
                                   int n_in, int n_out, long long inner, float2* maps,
                                   cudaStream_t st, int items = 1, long long sT = 0, long long sM = 0,
                                   float2* const* maps_tab = nullptr);

}  // namespace pisco
