// C ABI and host orchestration of the PISCO GB300 path (see include/pisco.h).
//
// pisco_plan validates the request, builds the index tables (Lambda, lag indices) and the
// small DFT / interpolation matrices on the host in FP64, uploads them and allocates every
// device buffer the path needs.  pisco_estimate then only enqueues kernels on the plan's
// stream: Gram (a), nullspace (b), G(x) (c), power iteration + phase (d), interpolation and
// normalisation (e).  It reads one device status word at the end.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "common.cuh"

using namespace pisco;

namespace {

constexpr int kNbMax = 8;       // Ritz vectors refined in FP64 per decision
constexpr int kThinSplits = 8;  // K splits of the tensor-core m x m x n block Grams
constexpr int kMmax = 128;   // largest eigensolver block
constexpr int kItersMax = 48;  // largest automatic subspace iteration count

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace

struct pisco_plan_s {
  pisco_params prm;
  cudaStream_t st = nullptr;
  // batched stages: one pass estimates `items` map sets of this shape; every per-item buffer
  // holds the items one after another (item_elems: elements per item, keyed by the member's
  // offset in this struct).  A view is a one-item plan into item i of a group's buffers.
  int items = 1;
  bool view = false;
  std::unordered_map<size_t, std::pair<size_t, size_t>> item_elems;  // (elements, bytes) per item
  // per-item inputs and outputs of a group (device tables, with the host copies they hold)
  const float2** in_tab = nullptr;
  float2** maps_tab = nullptr;
  float** eig_tab = nullptr;
  std::vector<const void*> h_in;
  std::vector<void*> h_maps;
  std::vector<float*> h_eig;
  float2* X0 = nullptr;  // orthonormalised random start block (shared by the items)
  int D = 2;
  // internal axis order: [0] = z, [1] = y, [2] = x
  int N[3], Nc[3], tau[3], Nr[3], Lp[3], B[3];
  int Q = 0, L = 0, n = 0, nbox = 0, npairs = 0;
  int m = 0, m_max = 0, eig_iters = 10;
  long long npix = 0, npix_red = 0, nfreq = 0;
  std::vector<int> lam;        // L x 3 (z,y,x)
  std::vector<int> lag_of_ij;  // L x L
  std::vector<int> lag_ptr, lag_ent;  // CSR: entries (b*L + a) with m_b - m_a = lag
  // device tables
  double2* fwd[3] = {nullptr, nullptr, nullptr};
  double2* inv[3] = {nullptr, nullptr, nullptr};
  float2* gdft[3] = {nullptr, nullptr, nullptr};
  // transposed copies ([n_in][n_out]) of the tables of the contiguous axis (inner == 1 passes)
  double2 *fwdT = nullptr, *invT = nullptr;
  float2 *gdftT = nullptr, *ydftT = nullptr, *interpT = nullptr;
  float2* ydft[3] = {nullptr, nullptr, nullptr};
  float2* interp[3] = {nullptr, nullptr, nullptr};
  int* d_lag_of_ij = nullptr;
  int *d_lag_ptr = nullptr, *d_lag_ent = nullptr;
  // tensor-core routes (PISCO_FLAG_TC_*): lags of Lambda-Lambda only (compressed CSR), the
  // lag-to-pixel exponentials E [npix_red][nlag] and the folded lag table KT [nlag][Q*Q]
  bool tc_g = false, tc_eig = false;
  bool a_conv = false;  // A X on the tensor cores reads A32 and splits it into tensor memory
  bool masked = false;                 // PISCO_FLAG_MASKED_GRAM
  bool block_pi = false;               // PISCO_FLAG_BLOCK_PI
  bool gram_df = false;                // PISCO_FLAG_GRAM_DF: double-float DFT tables below
  float4 *fwdT_df = nullptr, *fwd_df[3] = {nullptr, nullptr, nullptr};
  float4 *invT_df = nullptr, *inv_df[3] = {nullptr, nullptr, nullptr};
  int lam_lo[3] = {0, 0, 0}, lam_hi[3] = {0, 0, 0};
  int *d_lam = nullptr, *d_lag_ids = nullptr;
  int tc_terms = 3;
  int nlag = 0;
  std::vector<int> lagc_ptr, lag_ids;
  int* d_lagc_ptr = nullptr;
  float2* E = nullptr;
  float2* KT = nullptr;
  // split operands of the TMA-fed tensor-core GEMMs (head/tail arrays) and split-K scratch
  int tc_splits_ax = 4, tc_splits_g = 1;
  int gemm_splits = 0;  // split-K cap of the CUDA-core block products (0: automatic)
  int gemm_tile = 0;    // CUDA-core block product tile: 0 automatic, 32 or 64
  bool tc_thin = false; // thin block products (n x m x m, m x m x n) on the tensor cores too
  bool tc_interp = false;  // last interpolation pass as a batched tensor-core GEMM
  bool a_df = false;       // A holds double-float quadruples (double-float Gram route, unmasked)
  void* lags_df = nullptr;
  double2* A64 = nullptr;  // FP64 Gram built from the double-float one on request (debug accessor)
  bool g_sep = false;      // 2D G(x) from KT by separable DFT passes instead of the dense lag GEMM
  bool g_box = false;      // 3D G(x) from KT spread onto the lag box, then separable DFT passes
  int* d_box_lag = nullptr;  // lag box entry -> compressed lag index (-1: not a lag)
  int *d_sep_rows = nullptr, *d_sep_b2 = nullptr;
  float *IAh = nullptr, *IAl = nullptr, *IBh = nullptr, *IBl = nullptr;
  float2* interpA = nullptr;  // the last axis's interpolation matrix (split into IAh/IAl)
  // first interpolation axis as one tensor-core GEMM over all rows of V (B' of interpT)
  float *IXh = nullptr, *IXl = nullptr;
  bool tc_rows2d = false;  // 2D: both interpolation axes on the tensor cores, normalisation fused
  float *TAh = nullptr, *TAl = nullptr, *TBh = nullptr, *TBl = nullptr;  // their split operands
  float *Ah = nullptr, *Al = nullptr, *Xh = nullptr, *Xl = nullptr;        // A32 and the block
  float *Eh = nullptr, *El = nullptr, *KTh = nullptr, *KTl = nullptr;      // E and the lag table
  float *UAh = nullptr, *UAl = nullptr, *UBh = nullptr, *UBl = nullptr;    // U diag(w), conj(U)^T
  float2* tc_ws = nullptr;
  float2* thin_ws = nullptr;  // partial Grams of the CUDA-core thin products (m <= 64)
  int* thin_tk = nullptr;     // their per-item ticket counters
  size_t tc_ws_elems = 0;
  // learned warm start of the power iteration (pisco_set_warm_start)
  bool ws_on = false;
  int ws_iters = 0, ws_fb_iters = 0, ws_H = 0;
  int ws_nin = 0, ws_r = 0, ws_cap = 0;  // network input width, patch radius, allocated input width
  float ws_gate = 0.f;
  float* ws_w32 = nullptr;
  __half* ws_w16 = nullptr;
  float *ws_X = nullptr, *ws_H1 = nullptr, *ws_H2 = nullptr, *ws_out = nullptr;
  int* fb_flags = nullptr;
  // device buffers
  double2 *gA = nullptr, *gB = nullptr, *S = nullptr, *P = nullptr, *Rp = nullptr, *lags = nullptr;
  double2* A = nullptr;
  float2* A32 = nullptr;
  float2 *X = nullptr, *Y = nullptr, *Z = nullptr, *U = nullptr;
  float2 *Gm = nullptr, *Rinv = nullptr, *Bm = nullptr, *Vj = nullptr;
  float* mu = nullptr;
  float *dR0 = nullptr, *dR1 = nullptr;  // diag(R) of the last orthonormalisation (ping-pong)
  float* dsc = nullptr;                    // column scaling used by the last Cholesky
  double* gscale = nullptr;                // max diag of C^H C (A32 = A / gscale)
  int* tiles = nullptr;                    // split-K tile counters
  float* w = nullptr;
  double* ritz = nullptr;
  int* band = nullptr;
  double2 *Xb = nullptr, *Zb = nullptr;
  float2* ws32 = nullptr;
  size_t ws32_elems = 0;
  double2* ws64 = nullptr;
  size_t ws64_elems = 0;
  float2 *K = nullptr, *T1 = nullptr, *T2 = nullptr, *G = nullptr;
  float2 *Ya = nullptr, *Yb = nullptr, *Yf = nullptr;
  float2* V = nullptr;
  float* eig_tmp = nullptr;
  float2 *I1 = nullptr, *I2 = nullptr;
  DevStatus* dstatus = nullptr;
  DevStatus* hstatus = nullptr;  // pinned
  float2* calib_stage = nullptr;  // every estimate reads its calibration block from here
  // host IO staging
  float2 *io_calib = nullptr, *io_maps = nullptr;
  float* io_eig = nullptr;
  std::vector<void*> allocs;
  size_t ws_bytes = 0;
  int last_R = -1, last_k = -1;
  int last_launches = 0;
  DevStatus last_status{};
  // profiling: CUDA events around every operation, accumulated per tag
  bool prof = false;
  std::vector<cudaEvent_t> ev;        // pairs (start, end)
  std::vector<const char*> ev_tag;    // tag per pair
  int ev_used = 0;
  // CUDA graph of the whole path (captured after one eager run with the same arguments) on a
  // private non-blocking stream (the caller's stream may be the uncapturable legacy stream)
  cudaStream_t cap_st = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  bool use_graph = true;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  const void* g_calib = nullptr;
  void* g_maps = nullptr;
  float* g_eig = nullptr;
  int g_m = -1;
  bool g_prof = false;
  int g_launches = 0;
  int g_events = 0;
  const void* eager_calib = nullptr;  // arguments of the last eager run
  void* eager_maps = nullptr;
  float* eager_eig = nullptr;
  int eager_m = -1;
  bool eager_prof = false;
  std::vector<const char*> prof_name;
  std::vector<double> prof_ms;
  std::vector<int> prof_cnt;
};

namespace {

// a buffer shared by all items of the plan (tables, constants, counters)
template <typename T>
bool dalloc_shared(pisco_plan_s* pl, T** p, size_t count) {
  if (count == 0) count = 1;
  void* q = nullptr;
  if (cudaMalloc(&q, count * sizeof(T)) != cudaSuccess) return false;
  pl->allocs.push_back(q);
  pl->ws_bytes += count * sizeof(T);
  *p = reinterpret_cast<T*>(q);
  return true;
}

// a per-item buffer of `count` elements per item (p is a member of *pl)
template <typename T>
bool dalloc(pisco_plan_s* pl, T** p, size_t count) {
  if (count == 0) count = 1;
  if (!dalloc_shared(pl, p, count * (size_t)pl->items)) return false;
  pl->item_elems[(size_t)(reinterpret_cast<char*>(p) - reinterpret_cast<char*>(pl))] = {count, count * sizeof(T)};
  return true;
}

// elements per item of the per-item buffer held by member `m` (0 for shared buffers)
template <typename T>
long long IS(const pisco_plan_s* pl, T* const& m) {
  const auto it = pl->item_elems.find((size_t)(reinterpret_cast<const char*>(&m) - reinterpret_cast<const char*>(pl)));
  return it == pl->item_elems.end() ? 0 : (long long)it->second.first;
}

template <typename T>
bool upload(pisco_plan_s* pl, T** p, const std::vector<T>& h) {
  if (!dalloc_shared(pl, p, h.size())) return false;
  return cudaMemcpy(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice) == cudaSuccess;
}

// FP64 table -> double-float {Re hi, Re lo, Im hi, Im lo}: hi = fl32(x), lo = fl32(x - hi)
std::vector<float4> to_df(const std::vector<double2>& M) {
  std::vector<float4> out(M.size());
  for (size_t i = 0; i < M.size(); ++i) {
    const float rh = (float)M[i].x, ih = (float)M[i].y;
    out[i] = make_float4(rh, (float)(M[i].x - (double)rh), ih, (float)(M[i].y - (double)ih));
  }
  return out;
}

template <typename T>
std::vector<T> transposed(const std::vector<T>& M, int rows, int cols) {
  std::vector<T> out((size_t)rows * cols);
  for (int r = 0; r < rows; ++r)
    for (int c = 0; c < cols; ++c) out[(size_t)c * rows + r] = M[(size_t)r * cols + c];
  return out;
}

const double kPi = 3.14159265358979323846;

// zero-padded forward DFT along one axis: F[f][n] = exp(-i 2 pi f n / Lp), n = array index
std::vector<double2> fwd_matrix(int Lp, int Nc) {
  std::vector<double2> M((size_t)Lp * Nc);
  for (int f = 0; f < Lp; ++f)
    for (int n = 0; n < Nc; ++n) {
      const double a = -2.0 * kPi * (double)((long long)f * n % Lp) / Lp;
      M[(size_t)f * Nc + n] = make_double2(cos(a), sin(a));
    }
  return M;
}
// inverse DFT at lags d = -2tau..2tau: M[d][f] = exp(+i 2 pi f d / Lp) / Lp
std::vector<double2> inv_matrix(int Lp, int tau) {
  const int Bn = 4 * tau + 1;
  std::vector<double2> M((size_t)Bn * Lp);
  for (int t = 0; t < Bn; ++t) {
    const int d = t - 2 * tau;
    for (int f = 0; f < Lp; ++f) {
      long long ph = ((long long)f * d) % Lp;
      if (ph < 0) ph += Lp;
      const double a = 2.0 * kPi * (double)ph / Lp;
      M[(size_t)t * Lp + f] = make_double2(cos(a) / Lp, sin(a) / Lp);
    }
  }
  return M;
}
// lag sum onto the reduced grid: M[j][d] = exp(+i 2 pi d x_j), x_j = (j - Nr/2)/Nr
std::vector<float2> gdft_matrix(int Nr, int tau) {
  const int Bn = 4 * tau + 1;
  std::vector<float2> M((size_t)Nr * Bn);
  for (int j = 0; j < Nr; ++j)
    for (int t = 0; t < Bn; ++t) {
      const long long d = t - 2 * tau;
      long long num = d * (long long)(j - Nr / 2);
      num %= Nr;
      if (num < 0) num += Nr;
      const double a = 2.0 * kPi * (double)num / Nr;
      M[(size_t)j * Bn + t] = make_float2((float)cos(a), (float)sin(a));
    }
  return M;
}
// apodised low-resolution image: M[j][n] = a[n] exp(+i 2 pi n x_j), n centred index,
// a[n] = exp(-(n/(Nc/4))^2 / 2)
std::vector<float2> ydft_matrix(int Nr, int Nc) {
  std::vector<float2> M((size_t)Nr * Nc);
  const double width = Nc / 4.0;
  for (int j = 0; j < Nr; ++j)
    for (int idx = 0; idx < Nc; ++idx) {
      const long long nn = idx - Nc / 2;
      const double apo = exp(-0.5 * (nn / width) * (nn / width));
      long long num = nn * (long long)(j - Nr / 2);
      num %= Nr;
      if (num < 0) num += Nr;
      const double a = 2.0 * kPi * (double)num / Nr;
      M[(size_t)j * Nc + idx] = make_float2((float)(apo * cos(a)), (float)(apo * sin(a)));
    }
  return M;
}
// periodic-sinc interpolation n_in -> n_out (Sec. V-D): DFT of the coarse samples, band
// k in [-n_in/2, n_in - n_in/2), Nyquist coefficient split between +-n_in/2 for even n_in,
// evaluated at the fine points.  Computed in FP64 as an explicit matrix.
// lag-to-pixel exponentials of the tensor-core G route: E[j][l] = exp(+i 2 pi d_l . x_j) with
// x_j = (j - Nr/2)/Nr per axis (the points of the separable lag sums), phases reduced exactly
// in integers before the FP64 sine and cosine
std::vector<float2> lag_pixel_matrix(const int* Nr, const int* B, const int* tau,
                                     const std::vector<int>& lag_ids) {
  const long long np = (long long)Nr[0] * Nr[1] * Nr[2];
  const int nl = (int)lag_ids.size();
  std::vector<float2> E((size_t)np * nl);
  for (long long x = 0; x < np; ++x) {
    const long long j[3] = {x / ((long long)Nr[1] * Nr[2]), (x / Nr[2]) % Nr[1], x % Nr[2]};
    for (int l = 0; l < nl; ++l) {
      const int t = lag_ids[l];
      const long long d[3] = {t / (B[1] * B[2]) - 2 * tau[0], (t / B[2]) % B[1] - 2 * tau[1],
                              t % B[2] - 2 * tau[2]};
      double frac = 0.0;
      for (int a = 0; a < 3; ++a) {
        long long num = (d[a] * (j[a] - Nr[a] / 2)) % Nr[a];
        if (num < 0) num += Nr[a];
        frac += (double)num / Nr[a];
      }
      const double ang = 2.0 * kPi * frac;
      E[(size_t)x * nl + l] = make_float2((float)cos(ang), (float)sin(ang));
    }
  }
  return E;
}

std::vector<float2> interp_matrix(int n_in, int n_out) {
  std::vector<float2> M((size_t)n_out * n_in);
  const int k0 = -(n_in / 2), k1 = n_in - n_in / 2;
  for (int i = 0; i < n_out; ++i) {
    const double xi = (double)(i - n_out / 2) / n_out;
    for (int j = 0; j < n_in; ++j) {
      const double xj = (double)(j - n_in / 2) / n_in;
      double re = 0.0, im = 0.0;
      for (int k = k0; k < k1; ++k) {
        const double a = -2.0 * kPi * k * xj;  // forward coefficient
        double er, ei;
        if (n_in % 2 == 0 && k == k0 && n_out != n_in) {
          // split Nyquist: (e^{-i pi n_in x} + e^{+i pi n_in x})/2 = cos(pi n_in x)
          er = cos(kPi * n_in * xi);
          ei = 0.0;
        } else {
          const double b = 2.0 * kPi * k * xi;
          er = cos(b);
          ei = sin(b);
        }
        const double fr = cos(a) / n_in, fi = sin(a) / n_in;
        re += er * fr - ei * fi;
        im += er * fi + ei * fr;
      }
      M[(size_t)i * n_in + j] = make_float2((float)re, (float)im);
    }
  }
  return M;
}

void build_support(pisco_plan_s* pl) {
  pl->lam.clear();
  const int* t = pl->tau;
  const bool ell = pl->prm.kernel_shape == PISCO_KERNEL_ELLIPSOID;
  for (int z = -t[0]; z <= t[0]; ++z)
    for (int y = -t[1]; y <= t[1]; ++y)
      for (int x = -t[2]; x <= t[2]; ++x) {
        if (ell) {
          // sum (n_d/tau_d)^2 <= 1 evaluated exactly in integers:
          // sum n_d^2 * prod_{e != d} tau_e^2 <= prod tau_e^2 over the axes with tau > 0
          long long lhs = 0, prod = 1;
          const int v[3] = {z, y, x};
          for (int d = 0; d < 3; ++d)
            if (t[d] > 0) prod *= (long long)t[d] * t[d];
          for (int d = 0; d < 3; ++d) {
            if (t[d] == 0) continue;
            lhs += (long long)v[d] * v[d] * (prod / ((long long)t[d] * t[d]));
          }
          if (lhs > prod) continue;
        }
        pl->lam.push_back(z);
        pl->lam.push_back(y);
        pl->lam.push_back(x);
      }
  pl->L = (int)pl->lam.size() / 3;
  pl->lag_of_ij.assign((size_t)pl->L * pl->L, 0);
  for (int i = 0; i < pl->L; ++i)
    for (int j = 0; j < pl->L; ++j) {
      const int dz = pl->lam[3 * i] - pl->lam[3 * j] + 2 * t[0];
      const int dy = pl->lam[3 * i + 1] - pl->lam[3 * j + 1] + 2 * t[1];
      const int dx = pl->lam[3 * i + 2] - pl->lam[3 * j + 2] + 2 * t[2];
      pl->lag_of_ij[(size_t)i * pl->L + j] = (dz * pl->B[1] + dy) * pl->B[2] + dx;
    }
  // CSR lists of the (b, a) pairs per lag box entry, in increasing b*L + a
  const int nbox = pl->B[0] * pl->B[1] * pl->B[2];
  pl->lag_ptr.assign(nbox + 1, 0);
  for (int e = 0; e < pl->L * pl->L; ++e) pl->lag_ptr[pl->lag_of_ij[e] + 1]++;
  for (int t = 0; t < nbox; ++t) pl->lag_ptr[t + 1] += pl->lag_ptr[t];
  pl->lag_ent.assign((size_t)pl->L * pl->L, 0);
  std::vector<int> fill(pl->lag_ptr.begin(), pl->lag_ptr.end() - 1);
  for (int e = 0; e < pl->L * pl->L; ++e) pl->lag_ent[fill[pl->lag_of_ij[e]]++] = e;
  // the same lists restricted to the lags that occur (Lambda - Lambda), same entry order
  pl->lagc_ptr.assign(1, 0);
  pl->lag_ids.clear();
  for (int t = 0; t < nbox; ++t)
    if (pl->lag_ptr[t + 1] > pl->lag_ptr[t]) {
      pl->lag_ids.push_back(t);
      pl->lagc_ptr.push_back(pl->lag_ptr[t + 1]);
    }
  pl->nlag = (int)pl->lag_ids.size();
}

pisco_status validate(const pisco_params* p) {
  if (!p) return PISCO_ERR_ARG;
  if (p->ndim != 2 && p->ndim != 3) return PISCO_ERR_ARG;
  if (p->num_coils < 2 || p->num_coils > 64) return PISCO_ERR_ARG;
  if (p->kernel_shape != PISCO_KERNEL_RECT && p->kernel_shape != PISCO_KERNEL_ELLIPSOID) return PISCO_ERR_ARG;
  if (!(p->null_threshold > 0.0 && p->null_threshold < 1.0)) return PISCO_ERR_ARG;
  if (p->grid_reduction < 1 || p->power_iters < 1) return PISCO_ERR_ARG;
  const int nd = p->ndim;
  for (int d = 0; d < 3; ++d) {
    const bool used = d < nd;
    if (!used) {
      if (p->grid[d] != 1 || p->calib[d] != 1 || p->kernel_radius[d] != 0) return PISCO_ERR_ARG;
      continue;
    }
    const int N = p->grid[d], Nc = p->calib[d], t = p->kernel_radius[d];
    if (N < 1 || Nc < 1 || t < 0 || t > 16) return PISCO_ERR_ARG;
    if (Nc <= 2 * t) return PISCO_ERR_ARG;
    if (Nc > N) return PISCO_ERR_ARG;
    if (N % p->grid_reduction != 0) return PISCO_ERR_ARG;
    if (N / p->grid_reduction < 2 * t + 1) return PISCO_ERR_ARG;
  }
  if (p->eig_block < 0 || p->eig_block > kMmax || (p->eig_block % 2) != 0) return PISCO_ERR_ARG;
  if (p->eig_iters < 0 || p->eig_iters > 100) return PISCO_ERR_ARG;
  if (p->batch_group < 0) return PISCO_ERR_ARG;
  return PISCO_OK;
}

#define CK(x)                                   \
  do {                                          \
    cudaError_t e__ = (x);                      \
    if (e__ != cudaSuccess) return PISCO_ERR_CUDA; \
  } while (0)

int prof_begin(pisco_plan_s* pl, const char* tag) {
  if (!pl->prof) return -1;
  if (pl->ev_used * 2 + 2 > (int)pl->ev.size()) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return -1;
    if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return -1; }
    pl->ev.push_back(a);
    pl->ev.push_back(b);
    pl->ev_tag.push_back(nullptr);
  }
  const int i = pl->ev_used++;
  pl->ev_tag[i] = tag;
  cudaEventRecord(pl->ev[2 * i], pl->st);
  return i;
}
void prof_end(pisco_plan_s* pl, int i) {
  if (i >= 0) cudaEventRecord(pl->ev[2 * i + 1], pl->st);
}
// after the stream has been synchronised: fold the recorded pairs into the per-tag totals
void prof_collect(pisco_plan_s* pl, int count) {
  for (int i = 0; i < count; ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, pl->ev[2 * i], pl->ev[2 * i + 1]) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    size_t k = 0;
    while (k < pl->prof_name.size() && strcmp(pl->prof_name[k], pl->ev_tag[i]) != 0) ++k;
    if (k == pl->prof_name.size()) {
      pl->prof_name.push_back(pl->ev_tag[i]);
      pl->prof_ms.push_back(0.0);
      pl->prof_cnt.push_back(0);
    }
    pl->prof_ms[k] += ms;
    pl->prof_cnt[k] += 1;
  }
}

void graph_reset(pisco_plan_s* pl) {
  if (pl->gexec) cudaGraphExecDestroy(pl->gexec);
  if (pl->graph) cudaGraphDestroy(pl->graph);
  pl->gexec = nullptr;
  pl->graph = nullptr;
  pl->g_m = -1;
}

// the eigensolver's block size and iteration count, which a captured graph bakes in
int solve_key(const pisco_plan_s* pl) { return pl->m * 1024 + pl->eig_iters; }

// An uncertified split with the automatic iteration count: double the subspace iterations (up
// to kItersMax) for this and later estimates.  Returns false when no retry is left.
bool retry_iters(pisco_plan_s* pl) {
  if (pl->prm.eig_iters > 0 || pl->eig_iters >= kItersMax) return false;
  pl->eig_iters = std::min(2 * pl->eig_iters, kItersMax);
  return true;
}

#define OP(tag, x)                                   \
  do {                                               \
    const int i__ = prof_begin(pl, tag);             \
    cudaError_t e__ = (x);                           \
    if (e__ != cudaSuccess) return PISCO_ERR_CUDA;   \
    prof_end(pl, i__);                               \
  } while (0)

// ---------------------------------------------------------------------------------------
// the path
// ---------------------------------------------------------------------------------------
// strides of the Gram stage's per-item buffers (the axis passes write their outputs packed)
GramItems gram_items(const pisco_plan_s* pl) {
  GramItems it;
  it.n = pl->items;
  it.calib = IS(pl, pl->calib_stage);
  it.S = (long long)pl->Q * pl->nfreq;
  it.P = (long long)pl->npairs * pl->nfreq;
  it.Rp = (long long)pl->npairs * pl->nbox;
  it.lags = IS(pl, pl->lags);
  it.A = IS(pl, pl->A);
  it.scale = 1;
  return it;
}

pisco_status run_gram(pisco_plan_s* pl, const float2* calib) {
  cudaStream_t st = pl->st;
  const int Q = pl->Q;
  const int* Nc = pl->Nc;
  const int* Lp = pl->Lp;
  const GramItems gi = gram_items(pl);
  const long long QI = (long long)Q * pl->items;            // coils of all items
  const long long NPI = (long long)pl->npairs * pl->items;  // coil pairs of all items
  if (pl->masked) {
    OP("gram_masked_fp64", gram_masked(calib, Q, Nc, pl->lam_lo, pl->lam_hi, pl->d_lam, pl->L, pl->d_lag_ids,
                                       pl->d_lagc_ptr, pl->d_lag_ent, pl->nlag, pl->tau, pl->B, pl->A, pl->gscale,
                                       pl->A32, st));
    return PISCO_OK;
  }
  const int* B = pl->B;
  if (pl->gram_df) {
    // the same passes in double-float arithmetic (FP64 storage reused; lags written in FP64)
    if (pl->D == 2 && gram_forward_df_supported(Nc[1], Nc[2], Lp[1], Lp[2])) {
      OP("gram_dft_df", gram_forward_df(calib, Q, Nc[1], Nc[2], pl->fwdT_df, Lp[2], pl->fwd_df[1], Lp[1], pl->gB, st, gi));
    } else {
      OP("gram_dft_df", apply_axis_c2df(calib, pl->fwdT_df, pl->gA, AxisView{QI, (long long)Nc[0] * Nc[1], Nc[2], Lp[2], 1, 0, 1}, st));
      OP("gram_dft_df", apply_axis_df(pl->gA, pl->fwd_df[1], pl->gB, AxisView{QI, Nc[0], Nc[1], Lp[1], Lp[2]}, st));
    }
    const void* S = pl->gB;
    if (pl->D == 3) {
      OP("gram_dft_df", apply_axis_df(pl->gB, pl->fwd_df[0], pl->S, AxisView{QI, 1, Nc[0], Lp[0], (long long)Lp[1] * Lp[2]}, st));
      S = pl->S;
    }
    if (pl->D == 2 && gram_pairs_inverse_df_supported(Lp[1], Lp[2], B[1], B[2])) {
      OP("gram_pairs_df", gram_pairs_inverse_df(S, Q, Lp[1], Lp[2], pl->invT_df, B[2], pl->inv_df[1], B[1], pl->lags,
                                                pl->lags_df, st, gi));
    } else {
    OP("gram_pair_products", gram_pair_products_df(S, Q, pl->nfreq, pl->P, st, gi));
    OP("gram_dft_df", apply_axis_df(pl->P, pl->invT_df, pl->gA, AxisView{NPI, (long long)Lp[0] * Lp[1], Lp[2], B[2], 1, 0, 1}, st));
    if (pl->D == 3) {
      OP("gram_dft_df", apply_axis_df(pl->gA, pl->inv_df[1], pl->gB, AxisView{NPI, Lp[0], Lp[1], B[1], B[2]}, st));
      OP("gram_dft_df", apply_axis_df(pl->gB, pl->inv_df[0], pl->Rp, AxisView{NPI, 1, Lp[0], B[0], (long long)B[1] * B[2]}, st));
    } else {
      OP("gram_dft_df", apply_axis_df(pl->gA, pl->inv_df[1], pl->Rp, AxisView{NPI, 1, Lp[1], B[1], B[2]}, st));
    }
    OP("gram_scatter", gram_scatter_pairs_df(pl->Rp, Q, pl->nbox, pl->lags, pl->lags_df, st, gi));
    }
    const int lag0 = (2 * pl->tau[0] * B[1] + 2 * pl->tau[1]) * B[2] + 2 * pl->tau[2];
    OP("gram_expand", gram_scale(pl->lags, Q, pl->nbox, lag0, pl->gscale, st, gi));
    OP("gram_expand", gram_expand_df(pl->lags_df, pl->d_lag_of_ij, Q, pl->L, pl->nbox, pl->gscale, pl->A, pl->A32, st, gi));
    return PISCO_OK;
  }
  // forward zero-padded DFT of every channel: x, y, z
  OP("gram_dft_fp64", apply_axis_c2z(calib, pl->fwdT, pl->gA, AxisView{QI, (long long)Nc[0] * Nc[1], Nc[2], Lp[2], 1, 0, 1}, st));
  OP("gram_dft_fp64", apply_axis_z(pl->gA, pl->fwd[1], pl->gB, AxisView{QI, Nc[0], Nc[1], Lp[1], Lp[2]}, st));
  const double2* S = pl->gB;
  if (pl->D == 3) {
    OP("gram_dft_fp64", apply_axis_z(pl->gB, pl->fwd[0], pl->S, AxisView{QI, 1, Nc[0], Lp[0], (long long)Lp[1] * Lp[2]}, st));
    S = pl->S;
  }
  OP("gram_pair_products", gram_pair_products(S, Q, pl->nfreq, pl->P, st, gi));
  OP("gram_dft_fp64", apply_axis_z(pl->P, pl->invT, pl->gA, AxisView{NPI, (long long)Lp[0] * Lp[1], Lp[2], B[2], 1, 0, 1}, st));
  if (pl->D == 3) {
    OP("gram_dft_fp64", apply_axis_z(pl->gA, pl->inv[1], pl->gB, AxisView{NPI, Lp[0], Lp[1], B[1], B[2]}, st));
    OP("gram_dft_fp64", apply_axis_z(pl->gB, pl->inv[0], pl->Rp, AxisView{NPI, 1, Lp[0], B[0], (long long)B[1] * B[2]}, st));
  } else {
    OP("gram_dft_fp64", apply_axis_z(pl->gA, pl->inv[1], pl->Rp, AxisView{NPI, 1, Lp[1], B[1], B[2]}, st));
  }
  OP("gram_scatter", gram_scatter_pairs(pl->Rp, Q, pl->nbox, pl->lags, st, gi));
  const int lag0 = (2 * pl->tau[0] * B[1] + 2 * pl->tau[1]) * B[2] + 2 * pl->tau[2];
  OP("gram_expand", gram_scale(pl->lags, Q, pl->nbox, lag0, pl->gscale, st, gi));
  OP("gram_expand", gram_expand(pl->lags, pl->d_lag_of_ij, Q, pl->L, pl->nbox, pl->gscale, pl->A, pl->A32, st, gi));
  return PISCO_OK;
}

// strides of the eigensolver's per-item buffers
EigItems eig_items(const pisco_plan_s* pl) {
  EigItems it;
  it.n = pl->items;
  it.mm = IS(pl, pl->Gm);
  it.vj = IS(pl, pl->Vj);
  it.vec = IS(pl, pl->mu);
  it.nm = IS(pl, pl->X);
  it.nb = IS(pl, pl->Xb);
  it.band = IS(pl, pl->band);
  it.a = IS(pl, pl->A);
  it.scale = IS(pl, pl->gscale);
  return it;
}

// Thin block products on the tensor cores (PISCO_FLAG_TC_THIN): C = Y^H Z (m x m over n rows,
// conj_a) or C = Y W (n x m by m x m), operands split into the plan's thin buffers; Y, Z, W, C
// of item i are sY, sZ, sC elements after item 0 (sY = 0: one Y shared by the items)
cudaError_t thin_product(pisco_plan_s* pl, bool conj_a, const float2* Y, const float2* Z, float2* C, long long sY,
                         long long sZ, long long sC, int items) {
  const int n = pl->n, m = pl->m;
  const bool tt = pl->tc_terms == 3;
  const float2 one = make_float2(1.f, 0.f), zero = make_float2(0.f, 0.f);
  const int ap = sY != 0 ? 1 : 0;
  const int ai = sY != 0 ? items : 1;
  cudaError_t e;
  if (conj_a) {
    if ((e = tc2_split_at(Y, m, m, n, pl->TAh, tt ? pl->TAl : nullptr, pl->st, ai, sY)) != cudaSuccess) return e;
    if ((e = tc2_split_b(Z, m, 0, n, m, pl->TBh, tt ? pl->TBl : nullptr, pl->st, items, sZ)) != cudaSuccess) return e;
    return tc2_gemm(pl->tc_terms, m, m, n, pl->TAh, pl->TAl, pl->TBh, pl->TBl, one, zero, C, m, 0.f, 0, 0,
                    kThinSplits, pl->tc_ws, &pl->dstatus->flags, pl->st, items, sC, ap);
  }
  if ((e = tc2_split_a(Y, m, nullptr, n, m, pl->TAh, tt ? pl->TAl : nullptr, pl->st, ai, sY)) != cudaSuccess) return e;
  if ((e = tc2_split_b(Z, m, 0, m, m, pl->TBh, tt ? pl->TBl : nullptr, pl->st, items, sZ)) != cudaSuccess) return e;
  return tc2_gemm(pl->tc_terms, n, m, m, pl->TAh, pl->TAl, pl->TBh, pl->TBl, one, zero, C, m, 0.f, 0, 0, 1, nullptr,
                  &pl->dstatus->flags, pl->st, items, sC, ap);
}

// C = Y^H Z (m x m) or C = Y W (n x m by m x m) for every item: tensor cores or CUDA cores
cudaError_t block_product(pisco_plan_s* pl, bool conj_a, const float2* Y, const float2* Z, float2* C, long long sY,
                          long long sZ, long long sC, int items) {
  if (pl->tc_thin) return thin_product(pl, conj_a, Y, Z, C, sY, sZ, sC, items);
  const int n = pl->n, m = pl->m;
  if (m <= 64) {
    if (conj_a) return eig_thin_gram(Y, sY, Z, sZ, n, m, C, sC, pl->thin_ws, pl->thin_tk, items, pl->st);
    return eig_thin_apply(Y, sY, Z, sZ, n, m, C, sC, items, pl->st);
  }
  const float2 one = make_float2(1.f, 0.f), zero = make_float2(0.f, 0.f);
  if (conj_a)
    return cgemm<float>('C', 'N', m, m, n, one, Y, m, Z, m, zero, C, m, pl->ws32, pl->ws32_elems * pl->items,
                        pl->tiles, pl->st, pl->gemm_splits, pl->gemm_tile, items, sY, sZ, sC);
  return cgemm<float>('N', 'N', n, m, m, one, Y, m, Z, m, zero, C, m, pl->ws32, pl->ws32_elems * pl->items,
                      pl->tiles, pl->st, pl->gemm_splits, pl->gemm_tile, items, sY, sZ, sC);
}

// Xout = (Yin D^-1) L^-H for the Cholesky factor L of the Hermitian matrix held in pl->Gm
// (D^-1 Gm D^-1 = L L^H).  dscale: optional column scaling D; shift_rel: optional shift;
// acc_in: diagonal of earlier factors of the same product; diag(L) D acc goes to diag_out.
pisco_status chol_apply(pisco_plan_s* pl, const float2* Yin, float2* Xout, int m, const float* dscale,
                        float shift_rel, const float* acc_in, float* diag_out, int items) {
  cudaStream_t st = pl->st;
  const int n = pl->n;
  EigItems it = eig_items(pl);
  it.n = items;
  const long long snm = IS(pl, pl->X), smm = IS(pl, pl->Gm);
  if (m <= 64) {
    OP("eig_chol", eig_chol_inv_blocked(pl->Gm, m, dscale, shift_rel, acc_in, pl->Rinv, diag_out, pl->dstatus, st, it));
    OP(pl->tc_thin ? "eig_gemm_thin_tc" : "eig_gemm_thin_fp32", block_product(pl, false, Yin, pl->Rinv, Xout, snm, smm, snm, items));
  } else {
    OP("eig_chol", eig_chol(pl->Gm, m, dscale, shift_rel, acc_in, pl->Rinv, pl->dsc, diag_out, pl->dstatus, st, it));
    OP("eig_trsm", eig_trsm(Yin, pl->Rinv, pl->dsc, n, m, Xout, st, it));
  }
  return PISCO_OK;
}

// One Cholesky-QR pass: Xout = (Yin D^-1) L^-H with orthonormal columns, L L^H the Gram matrix
// of Yin D^-1.  dscale: optional column scaling D (previous diag(R)); shift_rel: optional shift;
// acc_in: diag(R) of earlier factors of the same product; diag(R) of the whole factorisation goes
// to diag_out.  items: the plan's items (per-item Yin), or 1 for the shared start block.
pisco_status cholqr(pisco_plan_s* pl, const float2* Yin, float2* Xout, int m, const float* dscale,
                    float shift_rel, const float* acc_in, float* diag_out, int items) {
  const long long snm = IS(pl, pl->X), smm = IS(pl, pl->Gm);
  OP(pl->tc_thin ? "eig_gemm_thin_tc" : "eig_gemm_thin_fp32", block_product(pl, true, Yin, Yin, pl->Gm, snm, snm, smm, items));
  return chol_apply(pl, Yin, Xout, m, dscale, shift_rel, acc_in, diag_out, items);
}

// Y = A32 X (n x n by n x m) for every item: tensor cores (split TF32) or CUDA cores (FP32);
// sX = 0: one X shared by the items
cudaError_t ax_product(pisco_plan_s* pl, const float2* X, float2* Y, long long sX) {
  const int n = pl->n, m = pl->m, items = pl->items;
  const float2 one = make_float2(1.f, 0.f), zero = make_float2(0.f, 0.f);
  const long long snm = IS(pl, pl->X);
  if (pl->tc_eig) {
    const int xi = sX != 0 ? items : 1;
    cudaError_t e = tc2_split_b(X, m, 0, n, m, pl->Xh, pl->tc_terms == 3 ? pl->Xl : nullptr, pl->st, xi, sX);
    if (e != cudaSuccess) return e;
    // sX == 0: every item multiplies the same block (B' of item 0 for all); a_conv: A read as
    // FP32 and split into tensor memory
    return tc2_gemm(pl->tc_terms, n, m, n, pl->Ah, pl->Al, pl->Xh, pl->Xl, one, zero, Y, m, 0.f, 0, 0,
                    pl->tc_splits_ax, pl->tc_ws, &pl->dstatus->flags, pl->st, items, snm, 1, nullptr, 1,
                    sX != 0 ? 1 : 0, pl->a_conv ? pl->A32 : nullptr, n);
  }
  return cgemm<float>('N', 'N', n, m, n, one, pl->A32, n, X, m, zero, Y, m, pl->ws32, pl->ws32_elems * pl->items,
                      pl->tiles, pl->st, pl->gemm_splits, pl->gemm_tile, items, IS(pl, pl->A32), sX, snm);
}

// Nullspace of the Gram (Sec. III-A, threshold footnote of Sec. III-B): orthogonal
// iteration on an m-column block in FP32, one Gram product per orthonormalisation with the
// block rescaled by the previous Ritz values or diag(R) (keeps Cholesky-QR well conditioned),
// one Rayleigh-Ritz at the end, and the threshold split decided on FP64 Rayleigh quotients
// against the FP64 Gram, with FP64 residuals certifying the decision.
//
// The start equilibrates the first product: A X0 of an orthonormalised random block X0 spans the
// dominant directions so unevenly (condition number up to lambda_1/lambda_m, 1e4 and more on
// these spectra) that even shifted Cholesky-QR leaves a block at the FP32 limit of the next pass.
// With B = X0^H A X0 = L L^H (positive definite: A is, X0 has full rank), Z L^-H with Z = A X0 has
// about the square root of that condition number, well inside one FP32 Cholesky-QR pass, and
// diag(L) times that pass's diag(R) is the diag(R) of the whole product (the next scaling).  X0
// depends on the seed only, so the items of a batched pass share it.
pisco_status run_eig(pisco_plan_s* pl) {
  cudaStream_t st = pl->st;
  const int n = pl->n, m = pl->m, items = pl->items;
  const double thr2 = pl->prm.null_threshold * pl->prm.null_threshold;
  const EigItems it = eig_items(pl);
  const long long snm = IS(pl, pl->X), smm = IS(pl, pl->Gm), svj = IS(pl, pl->Vj);
  pisco_status s;
  OP("eig_misc", eig_random_block(pl->Y, n, m, pl->prm.seed, st));
  if (pl->tc_eig && !pl->a_conv)  // the Gram's TF32 head/tail split, shared by every product of the solve
    OP("eig_gemm_AX", tc2_split_a(pl->A32, n, nullptr, n, n, pl->Ah, pl->tc_terms == 3 ? pl->Al : nullptr, st, items,
                                  IS(pl, pl->A32)));
  // X0 = orth(random block): well conditioned (kappa ~ (1 + sqrt(m/n)) / (1 - sqrt(m/n)))
  if ((s = cholqr(pl, pl->Y, pl->X0, m, nullptr, 0.f, nullptr, pl->dR1, 1)) != PISCO_OK) return s;
  // the equilibrated first power step: Z = A X0, B = X0^H Z = L L^H, Y = Z L^-H, X1 = orth(Y)
  OP("eig_gemm_AX", ax_product(pl, pl->X0, pl->Z, 0));
  OP(pl->tc_thin ? "eig_gemm_thin_tc" : "eig_gemm_thin_fp32", block_product(pl, true, pl->X0, pl->Z, pl->Gm, 0, snm, smm, items));
  if ((s = chol_apply(pl, pl->Z, pl->Y, m, nullptr, 0.f, nullptr, pl->dR0, items)) != PISCO_OK) return s;
  if ((s = cholqr(pl, pl->Y, pl->X, m, nullptr, 0.f, pl->dR0, pl->dR1, items)) != PISCO_OK) return s;
  float* dprev = pl->dR1;
  float* dnext = pl->dR0;
  // orthogonal iteration: X <- orth(A X diag(R)^-1), diag(R) of the previous orthonormalisation
  // approximating the Ritz values of the block columns
  for (int k = 1; k < pl->eig_iters; ++k) {
    OP("eig_gemm_AX", ax_product(pl, pl->X, pl->Y, snm));
    if ((s = cholqr(pl, pl->Y, pl->X, m, dprev, 0.f, nullptr, dnext, items)) != PISCO_OK) return s;
    std::swap(dprev, dnext);
  }
  // Rayleigh-Ritz on the block
  OP("eig_gemm_AX", ax_product(pl, pl->X, pl->Z, snm));
  OP(pl->tc_thin ? "eig_gemm_thin_tc" : "eig_gemm_thin_fp32", block_product(pl, true, pl->X, pl->Z, pl->Bm, snm, snm, smm, items));
  OP("eig_jacobi", eig_jacobi(pl->Bm, m, pl->mu, pl->Vj, 30, (float)(0.05 * thr2), (float)(0.5 * thr2), pl->dstatus, st, it));
  OP(pl->tc_thin ? "eig_gemm_thin_tc" : "eig_gemm_thin_fp32", block_product(pl, false, pl->X, pl->Vj, pl->U, snm, svj, snm, items));
  // FP64 Rayleigh quotients of the Ritz vectors that decide the split
  OP("eig_misc", eig_select_band(pl->mu, m, thr2, kNbMax, pl->band, st, it));
  OP("eig_misc", eig_gather_band(pl->U, n, m, pl->band, kNbMax, pl->Xb, st, it));
  if (pl->gram_df)
    OP("eig_rayleigh_df", eig_band_matvec_df(pl->A, pl->a_df, pl->Xb, n, kNbMax, pl->band, pl->Zb, st, it));
  else
    OP("eig_rayleigh_fp64", eig_band_matvec(pl->A, pl->Xb, n, kNbMax, pl->band, pl->Zb, st, it));
  OP("eig_decide_fp64", eig_decide(pl->mu, m, pl->band, kNbMax, pl->Xb, pl->Zb, n, thr2, pl->Q, pl->gscale,
                pl->w, pl->ritz, pl->dstatus, st, it));
  return PISCO_OK;
}

pisco_status run_gfield(pisco_plan_s* pl) {
  cudaStream_t st = pl->st;
  const int Q = pl->Q, items = pl->items;
  const int* B = pl->B;
  const int* Nr = pl->Nr;
  const long long QQ = (long long)Q * Q;
  if (pl->tc_g) {
    // P = U diag(w) U^H into the (now free) FP32 Gram buffer, fold onto the lags, then
    // G = |Lambda| I - E KT, all products on the tensor cores
    const int n = pl->n;
    int* err = &pl->dstatus->flags;
    const float2 one = make_float2(1.f, 0.f), zero = make_float2(0.f, 0.f), mone = make_float2(-1.f, 0.f);
    const bool tt = pl->tc_terms == 3;
    const long long snm = IS(pl, pl->U), snn = IS(pl, pl->A32), skt = IS(pl, pl->KT), sg = IS(pl, pl->G);
    OP("g_herk_tc", tc2_split_a(pl->U, pl->m, pl->w, n, pl->m, pl->UAh, tt ? pl->UAl : nullptr, st, items, snm,
                                IS(pl, pl->w)));
    OP("g_herk_tc", tc2_split_b(pl->U, pl->m, 1, pl->m, n, pl->UBh, tt ? pl->UBl : nullptr, st, items, snm));
    OP("g_herk_tc", tc2_gemm(pl->tc_terms, n, n, pl->m, pl->UAh, pl->UAl, pl->UBh, pl->UBl, one, zero, pl->A32, n,
                             0.f, 0, 0, 1, nullptr, err, st, items, snn, 1));
    OP("g_collapse", gassembly_collapse(pl->A32, n, Q, pl->L, pl->d_lagc_ptr, pl->d_lag_ent, pl->nlag, pl->KT, st,
                                        items, snn, skt));
    if (pl->g_sep) {
      OP("g_field_sep", gassembly_field_sep2(pl->KT, Q, pl->nlag, pl->d_sep_rows, pl->d_sep_b2, pl->gdft[1], Nr[1], B[1],
                                             pl->gdft[2], B[2], Nr[2], (float)pl->L, pl->G, st, items, skt, sg));
      return PISCO_OK;
    }
    if (pl->g_box) {
      // lag box, then x, y, z passes (the last one pixel-major per item), then |Lambda| I - G
      const long long QI = QQ * items;
      OP("g_field_sep", gassembly_scatter_box(pl->KT, pl->d_box_lag, (int)QQ, pl->nbox, pl->K, st, items, skt,
                                              IS(pl, pl->K)));
      OP("g_field_sep", apply_axis_c(pl->K, pl->gdftT, pl->T1, AxisView{QI, (long long)B[0] * B[1], B[2], Nr[2], 1, 0, 1}, st));
      OP("g_field_sep", apply_axis_c(pl->T1, pl->gdft[1], pl->T2, AxisView{QI, B[0], B[1], Nr[1], Nr[2]}, st));
      AxisView vz{QI, 1, B[0], Nr[0], (long long)Nr[1] * Nr[2], 1};
      vz.pm_group = (int)QQ;
      OP("g_field_sep", apply_axis_c(pl->T2, pl->gdft[0], pl->G, vz, st));
      OP("g_field_sep", gassembly_add_identity(pl->G, Q, pl->npix_red * items, (float)pl->L, st));
      return PISCO_OK;
    }
    OP("g_field_tc", tc2_split_b(pl->KT, (int)QQ, 0, pl->nlag, (int)QQ, pl->KTh, tt ? pl->KTl : nullptr, st, items, skt));
    OP("g_field_tc", tc2_gemm(pl->tc_terms, (int)pl->npix_red, (int)QQ, pl->nlag, pl->Eh, pl->El, pl->KTh, pl->KTl,
                              mone, zero, pl->G, (int)QQ, (float)pl->L, Q + 1, (int)QQ, pl->tc_splits_g, pl->tc_ws,
                              err, st, items, sg));
    return PISCO_OK;
  }
  if (items > 1) return PISCO_ERR_UNSUPPORTED;  // batched groups take the tensor-core G route
  OP("g_kernel", gassembly_kernel(pl->U, pl->w, Q, pl->L, pl->m, pl->d_lag_ptr, pl->d_lag_ent, pl->nbox, pl->K, st));
  OP("g_dft", apply_axis_c(pl->K, pl->gdftT, pl->T1, AxisView{QQ, (long long)B[0] * B[1], B[2], Nr[2], 1, 0, 1}, st));
  if (pl->D == 3) {
    OP("g_dft", apply_axis_c(pl->T1, pl->gdft[1], pl->T2, AxisView{QQ, B[0], B[1], Nr[1], Nr[2]}, st));
    OP("g_dft", apply_axis_c(pl->T2, pl->gdft[0], pl->G, AxisView{QQ, 1, B[0], Nr[0], (long long)Nr[1] * Nr[2], 1}, st));
  } else {
    OP("g_dft", apply_axis_c(pl->T1, pl->gdft[1], pl->G, AxisView{QQ, 1, B[1], Nr[1], Nr[2], 1}, st));
  }
  OP("g_identity", gassembly_add_identity(pl->G, Q, pl->npix_red, (float)pl->L, st));
  return PISCO_OK;
}

pisco_status run_lowres(pisco_plan_s* pl, const float2* calib) {
  cudaStream_t st = pl->st;
  const long long QI = (long long)pl->Q * pl->items;  // the items' coils one after another
  const int* Nc = pl->Nc;
  const int* Nr = pl->Nr;
  OP("lowres_dft", apply_axis_c(calib, pl->ydftT, pl->Ya, AxisView{QI, (long long)Nc[0] * Nc[1], Nc[2], Nr[2], 1, 0, 1}, st));
  if (pl->D == 3) {
    OP("lowres_dft", apply_axis_c(pl->Ya, pl->ydft[1], pl->Yb, AxisView{QI, Nc[0], Nc[1], Nr[1], Nr[2]}, st));
    OP("lowres_dft", apply_axis_c(pl->Yb, pl->ydft[0], pl->Yf, AxisView{QI, 1, Nc[0], Nr[0], (long long)Nr[1] * Nr[2]}, st));
  } else {
    OP("lowres_dft", apply_axis_c(pl->Ya, pl->ydft[1], pl->Yf, AxisView{QI, 1, Nc[1], Nr[1], Nr[2]}, st));
  }
  return PISCO_OK;
}

// maps: the output of a one-item plan; a group writes item i's maps to maps_tab[i]
pisco_status run_interp(pisco_plan_s* pl, float2* maps) {
  cudaStream_t st = pl->st;
  const int Q = pl->Q, items = pl->items;
  const long long QI = (long long)Q * items;
  const int* N = pl->N;
  const int* Nr = pl->Nr;
  float2* const* tab = items > 1 ? pl->maps_tab : nullptr;
  if (pl->prm.grid_reduction == 1) {
    OP("interp_final_norm", interp_final_normalize(pl->V, nullptr, Q, 0, 1, 1, pl->npix, maps, st, items,
                                                   IS(pl, pl->V), 0, tab));
    return PISCO_OK;
  }
  if (pl->tc_rows2d) {
    // 2D on the tensor cores, axis 1 first: W[y][(q, r2)] = M1 V_q for every item (B' of V read
    // with grouped columns), then one product over the rows (item, y, q) of W: maps rows =
    // W interpT, each pixel's Q coil rows in one tile and normalised in its epilogue
    const float2 one = make_float2(1.f, 0.f), zero = make_float2(0.f, 0.f);
    const long long wrows = (long long)N[1] * Q;
    OP("interp_split", tc2_split_b(pl->V, Nr[2], 0, Nr[1], Q * Nr[2], pl->IBh, pl->IBl, st, items, IS(pl, pl->V), Nr[2],
                                   (long long)Nr[1] * Nr[2]));
    OP("interp_axis1_tc", tc2_gemm(3, N[1], Q * Nr[2], Nr[1], pl->IAh, pl->IAl, pl->IBh, pl->IBl, one, zero, pl->I1,
                             Q * Nr[2], 0.f, 0, 0, 1, nullptr, &pl->dstatus->flags, st, items, wrows * Nr[2], 0,
                             nullptr, 1, 1));
    const bool fused = 128 % Q == 0;
    OP("interp_rows_tc", tc2_gemm(3, (int)(wrows * items), N[2], Nr[2], nullptr, nullptr, pl->IXh, pl->IXl, one, zero, maps,
                             N[2], 0.f, 0, 0, 1, nullptr, &pl->dstatus->flags, st, 1, (long long)Q * pl->npix, 0, tab,
                             1, 0, pl->I1, Nr[2], Q, (int)wrows, (long long)N[1] * N[2], fused ? 1 : 0));
    if (!fused) OP("interp_final_norm", normalize_maps(maps, Q, pl->npix, st, items, 0, tab));
    return PISCO_OK;
  }
  const long long rows1 = QI * Nr[0] * Nr[1];
  if (pl->IXh && tc2_conv_ok(Nr[2], Nr[2], pl->V) && (rows1 + 127) / 128 <= 65535) {
    const float2 one = make_float2(1.f, 0.f), zero = make_float2(0.f, 0.f);
    OP("interp_axis_tc", tc2_gemm(3, (int)rows1, N[2], Nr[2], nullptr, nullptr, pl->IXh, pl->IXl, one, zero, pl->I1,
                                  N[2], 0.f, 0, 0, 1, nullptr, &pl->dstatus->flags, st, 1, 0, 0, nullptr, 1, 0, pl->V,
                                  Nr[2]));
  } else {
    OP("interp_axis", apply_axis_c(pl->V, pl->interpT, pl->I1, AxisView{QI, (long long)Nr[0] * Nr[1], Nr[2], N[2], 1, 0, 1}, st));
  }
  if (pl->tc_interp) {
    // maps_q = M T_q for every coil q (one batched tensor-core GEMM), then the per-pixel norm
    const bool tt = pl->tc_terms == 3;
    const float2 one = make_float2(1.f, 0.f), zero = make_float2(0.f, 0.f);
    const float2* T = pl->I1;
    if (pl->D == 3) {
      OP("interp_axis", apply_axis_c(pl->I1, pl->interp[1], pl->I2, AxisView{QI, Nr[0], Nr[1], N[1], N[2]}, st));
      T = pl->I2;
    }
    const int ax = pl->D == 3 ? 0 : 1;
    const long long inner = pl->D == 3 ? (long long)N[1] * N[2] : N[2];
    OP("interp_final_tc", tc2_split_b(T, (int)inner, 0, Nr[ax], (int)inner, pl->IBh, tt ? pl->IBl : nullptr, st, (int)QI,
                                      (long long)Nr[ax] * inner));
    OP("interp_final_tc", tc2_gemm(pl->tc_terms, N[ax], (int)inner, Nr[ax], pl->IAh, pl->IAl, pl->IBh, pl->IBl, one,
                                   zero, maps, (int)inner, 0.f, 0, 0, 1, nullptr, &pl->dstatus->flags, st, (int)QI,
                                   (long long)N[ax] * inner, 0, tab, Q));
    OP("interp_final_norm", normalize_maps(maps, Q, pl->npix, st, items, 0, tab));
    return PISCO_OK;
  }
  if (pl->D == 3) {
    OP("interp_axis", apply_axis_c(pl->I1, pl->interp[1], pl->I2, AxisView{QI, Nr[0], Nr[1], N[1], N[2]}, st));
    OP("interp_final_norm", interp_final_normalize(pl->I2, pl->interp[0], Q, 0, Nr[0], N[0], (long long)N[1] * N[2],
                                                   maps, st, items, (long long)Q * Nr[0] * N[1] * N[2], 0, tab));
  } else {
    OP("interp_final_norm", interp_final_normalize(pl->I1, pl->interp[1], Q, 0, Nr[1], N[1], N[2], maps, st, items,
                                                   (long long)Q * Nr[1] * N[2], 0, tab));
  }
  return PISCO_OK;
}

// The whole path.  One-item plans read `calib` and write maps / eig directly; a group reads its
// items' calibration blocks from calib_stage (staged by the batch launcher) and writes through
// maps_tab / eig_tab (maps and eig unused).
pisco_status run_all(pisco_plan_s* pl, const float2* calib, float2* maps, float* eig) {
  cudaStream_t st = pl->st;
  const int items = pl->items;
  g_launches = 0;
  CK(cudaMemsetAsync(pl->dstatus, 0, sizeof(DevStatus) * items, st));
  pisco_status s;
  if ((s = run_gram(pl, calib)) != PISCO_OK) return s;
  if ((s = run_eig(pl)) != PISCO_OK) return s;
  if ((s = run_gfield(pl)) != PISCO_OK) return s;
  if ((s = run_lowres(pl, calib)) != PISCO_OK) return s;
  if (items > 1) {
    PiOpts o;
    o.items = items;
    o.sG = IS(pl, pl->G);
    o.sY = IS(pl, pl->Yf);
    o.sV = IS(pl, pl->V);
    o.sE = IS(pl, pl->eig_tmp);
    o.eig_tab = pl->eig_tab;
    OP("power_iteration", power_iteration(pl->G, pl->Yf, pl->Q, pl->npix_red, pl->prm.power_iters, (float)pl->L,
                                          pl->prm.seed, pl->V, pl->eig_tmp, st, o));
  } else if (pl->ws_on) {
    // learned start vectors, fewer iterations, residual-gated re-solve from the plain start
    const MlpView mv{pl->ws_nin, pl->ws_H, 2 * pl->Q, pl->ws_w32, pl->ws_w16};
    const int rdims[3] = {pl->Nr[0], pl->Nr[1], pl->Nr[2]};
    OP("warm_start_mlp", mlp_patch_features(pl->Yf, pl->Q, rdims, pl->ws_r, pl->D, pl->ws_X, st));
    OP("warm_start_mlp", mlp_forward(mv, pl->ws_X, pl->npix_red, pl->ws_H1, pl->ws_H2, pl->ws_out, st));
    PiOpts o1;
    o1.v0 = pl->ws_out;
    o1.gate = pl->ws_gate;
    o1.flags = pl->fb_flags;
    o1.count = &pl->dstatus->ws_fallback;
    if (o1.gate <= 0.f) o1.flags = nullptr, o1.count = nullptr;
    OP("power_iteration", power_iteration(pl->G, pl->Yf, pl->Q, pl->npix_red, pl->ws_iters, (float)pl->L,
                                          pl->prm.seed, pl->V, eig ? eig : pl->eig_tmp, st, o1));
    if (o1.gate > 0.f) {
      PiOpts o2;
      o2.only = pl->fb_flags;
      OP("pi_fallback", power_iteration(pl->G, pl->Yf, pl->Q, pl->npix_red, pl->ws_fb_iters, (float)pl->L,
                                        pl->prm.seed, pl->V, eig ? eig : pl->eig_tmp, st, o2));
    }
  } else if (pl->block_pi) {
    OP("power_iteration", power_iteration_block2(pl->G, pl->Yf, pl->Q, pl->npix_red, pl->prm.power_iters,
                                                 (float)pl->L, pl->prm.seed, pl->V, eig ? eig : pl->eig_tmp, st));
  } else {
    OP("power_iteration", power_iteration(pl->G, pl->Yf, pl->Q, pl->npix_red, pl->prm.power_iters, (float)pl->L,
                                          pl->prm.seed, pl->V, eig ? eig : pl->eig_tmp, st));
  }
  if ((s = run_interp(pl, maps)) != PISCO_OK) return s;
  CK(cudaMemcpyAsync(pl->hstatus, pl->dstatus, sizeof(DevStatus) * items, cudaMemcpyDeviceToHost, st));
  return PISCO_OK;
}

}  // namespace

extern "C" {

const char* pisco_status_string(pisco_status s) {
  switch (s) {
    case PISCO_OK: return "ok";
    case PISCO_ERR_ARG: return "invalid argument";
    case PISCO_ERR_CUDA: return "CUDA runtime error";
    case PISCO_ERR_OOM: return "device allocation failed";
    case PISCO_ERR_RANK: return "nullspace dimension R < Q-1 (maps not identifiable)";
    case PISCO_ERR_TIMEOUT: return "bounded device wait expired";
    case PISCO_ERR_NOT_CONVERGED: return "eigensolver block saturated at its largest size";
    case PISCO_ERR_UNSUPPORTED: return "request outside this build";
    case PISCO_ERR_TOO_LARGE: return "request exceeds the fixed scratch of the no-allocation entry point";
  }
  return "unknown status";
}

void pisco_destroy(pisco_plan_t pl) {
  if (!pl) return;
  if (pl->st) cudaStreamSynchronize(pl->st);
  graph_reset(pl);
  if (pl->cap_st) { cudaStreamSynchronize(pl->cap_st); cudaStreamDestroy(pl->cap_st); }
  if (pl->ev_in) cudaEventDestroy(pl->ev_in);
  if (pl->ev_out) cudaEventDestroy(pl->ev_out);
  for (cudaEvent_t e : pl->ev) cudaEventDestroy(e);
  for (void* p : pl->allocs) cudaFree(p);  // a view owns only what was allocated for it
  if (pl->hstatus && !pl->view) cudaFreeHost(pl->hstatus);
  delete pl;
}

}  // extern "C"

// a plan whose passes estimate `items` map sets of the shape p at once (items == 1: pisco_plan)
static pisco_status plan_create(const pisco_params* p, cudaStream_t cuda_stream, int items, pisco_plan_s** out) {
  if (!out || items < 1) return PISCO_ERR_ARG;
  *out = nullptr;
  pisco_status s = validate(p);
  if (s != PISCO_OK) return s;
  pisco_plan_s* pl = new (std::nothrow) pisco_plan_s();
  if (!pl) return PISCO_ERR_OOM;
  pl->items = items;
  pl->prm = *p;
  pl->st = (cudaStream_t)cuda_stream;
  pl->D = p->ndim;
  for (int d = 0; d < 3; ++d) {  // params are x,y,z; internal z,y,x
    pl->N[2 - d] = p->grid[d];
    pl->Nc[2 - d] = p->calib[d];
    pl->tau[2 - d] = p->kernel_radius[d];
  }
  const int f = p->grid_reduction;
  pl->Q = p->num_coils;
  for (int d = 0; d < 3; ++d) {
    pl->Nr[d] = pl->N[d] / f;
    if (pl->N[d] == 1) pl->Nr[d] = 1;
    pl->Lp[d] = pl->Nc[d] + 2 * pl->tau[d];
    pl->B[d] = 4 * pl->tau[d] + 1;
  }
  build_support(pl);
  pl->n = pl->Q * pl->L;
  pl->nbox = pl->B[0] * pl->B[1] * pl->B[2];
  pl->npairs = pl->Q * (pl->Q + 1) / 2;
  pl->npix = (long long)pl->N[0] * pl->N[1] * pl->N[2];
  pl->npix_red = (long long)pl->Nr[0] * pl->Nr[1] * pl->Nr[2];
  pl->nfreq = (long long)pl->Lp[0] * pl->Lp[1] * pl->Lp[2];
  // shared-memory budget of the G-kernel build (two staged column chunks + the L x L block)
  if ((2 * (size_t)pl->L * 32 + (size_t)pl->L * pl->L) * sizeof(float2) > 220 * 1024) {
    delete pl;
    return PISCO_ERR_UNSUPPORTED;
  }
  int mmax = std::min(kMmax, pl->n - (pl->n % 2));
  pl->m_max = mmax;
  pl->m = p->eig_block > 0 ? std::min(p->eig_block, mmax) : std::min(64, mmax);
  if (pl->m < 2) { delete pl; return PISCO_ERR_ARG; }
  // 6 products keep the signal projector within 2e-6 of the FP64 oracle's on every tested
  // workload (10x inside its gate; 4 products are not enough)
  pl->eig_iters = p->eig_iters > 0 ? p->eig_iters : 6;
  pl->gemm_splits = p->gemm_splits > 0 ? std::min(p->gemm_splits, 64) : 0;
  pl->gemm_tile = (p->gemm_tile == 32 || p->gemm_tile == 64) ? p->gemm_tile : 0;
  pl->tc_thin = (p->flags & PISCO_FLAG_TC_THIN) != 0 && (p->flags & PISCO_FLAG_TC_EIG) != 0;
  pl->tc_interp = (p->flags & PISCO_FLAG_TC_INTERP) != 0 && p->grid_reduction > 1;
  if (pl->tc_interp && tc2_prepare() != cudaSuccess) {
    cudaGetLastError();
    delete pl;
    return PISCO_ERR_CUDA;
  }
  pl->masked = (p->flags & PISCO_FLAG_MASKED_GRAM) != 0;
  pl->block_pi = (p->flags & PISCO_FLAG_BLOCK_PI) != 0;
  pl->gram_df = (p->flags & PISCO_FLAG_GRAM_DF) != 0;
  if (pl->masked) {
    const int nvol = pl->Nc[0] * pl->Nc[1] * pl->Nc[2];
    if (nvol > kMaskedMaxSamples) {
      delete pl;
      return PISCO_ERR_UNSUPPORTED;
    }
    for (int d = 0; d < 3; ++d) {
      pl->lam_lo[d] = 1 << 20;
      pl->lam_hi[d] = -(1 << 20);
      for (int i = 0; i < pl->L; ++i) {
        pl->lam_lo[d] = std::min(pl->lam_lo[d], pl->lam[3 * i + d]);
        pl->lam_hi[d] = std::max(pl->lam_hi[d], pl->lam[3 * i + d]);
      }
    }
    if (gram_masked_prepare(nvol) != cudaSuccess) {
      cudaGetLastError();
      delete pl;
      return PISCO_ERR_CUDA;
    }
  }
  pl->tc_g = (p->flags & PISCO_FLAG_TC_GFIELD) != 0;
  pl->tc_eig = (p->flags & PISCO_FLAG_TC_EIG) != 0;
  pl->tc_terms = (p->flags & PISCO_FLAG_TC_1PASS) ? 1 : 3;
  pl->a_conv = pl->tc_eig && pl->tc_terms == 3 && (pl->n % 2) == 0;
  if ((pl->tc_g || pl->tc_eig) && tc2_prepare() != cudaSuccess) {
    cudaGetLastError();
    delete pl;
    return PISCO_ERR_CUDA;
  }

  const int Q = pl->Q, n = pl->n, np = pl->npairs;
  const int* Nc = pl->Nc;
  const int* Lp = pl->Lp;
  const int* B = pl->B;
  const int* Nr = pl->Nr;
  const int* N = pl->N;
  bool ok = true;
  // tables
  for (int d = 0; d < 3; ++d) {
    ok = ok && upload(pl, &pl->fwd[d], fwd_matrix(Lp[d], Nc[d]));
    ok = ok && upload(pl, &pl->inv[d], inv_matrix(Lp[d], pl->tau[d]));
    ok = ok && upload(pl, &pl->gdft[d], gdft_matrix(Nr[d], pl->tau[d]));
    ok = ok && upload(pl, &pl->ydft[d], ydft_matrix(Nr[d], Nc[d]));
    ok = ok && upload(pl, &pl->interp[d], interp_matrix(Nr[d], N[d]));
  }
  ok = ok && upload(pl, &pl->fwdT, transposed(fwd_matrix(Lp[2], Nc[2]), Lp[2], Nc[2]));
  ok = ok && upload(pl, &pl->invT, transposed(inv_matrix(Lp[2], pl->tau[2]), B[2], Lp[2]));
  ok = ok && upload(pl, &pl->gdftT, transposed(gdft_matrix(Nr[2], pl->tau[2]), Nr[2], B[2]));
  ok = ok && upload(pl, &pl->ydftT, transposed(ydft_matrix(Nr[2], Nc[2]), Nr[2], Nc[2]));
  ok = ok && upload(pl, &pl->interpT, transposed(interp_matrix(Nr[2], N[2]), N[2], Nr[2]));
  if (pl->gram_df) {
    ok = ok && upload(pl, &pl->fwdT_df, to_df(transposed(fwd_matrix(Lp[2], Nc[2]), Lp[2], Nc[2])));
    ok = ok && upload(pl, &pl->invT_df, to_df(transposed(inv_matrix(Lp[2], pl->tau[2]), B[2], Lp[2])));
    for (int d = 0; d < 2; ++d) {
      ok = ok && upload(pl, &pl->fwd_df[d], to_df(fwd_matrix(Lp[d], Nc[d])));
      ok = ok && upload(pl, &pl->inv_df[d], to_df(inv_matrix(Lp[d], pl->tau[d])));
    }
  }
  ok = ok && upload(pl, &pl->d_lag_of_ij, pl->lag_of_ij);
  ok = ok && upload(pl, &pl->d_lag_ptr, pl->lag_ptr) && upload(pl, &pl->d_lag_ent, pl->lag_ent);
  ok = ok && upload(pl, &pl->d_lagc_ptr, pl->lagc_ptr) && upload(pl, &pl->d_lag_ids, pl->lag_ids) &&
       upload(pl, &pl->d_lam, pl->lam);
  // Gram
  const long long gA = std::max((long long)Q * Nc[0] * Nc[1] * Lp[2], (long long)np * Lp[0] * Lp[1] * B[2]);
  const long long gB = std::max((long long)Q * Nc[0] * Lp[1] * Lp[2], (long long)np * Lp[0] * B[1] * B[2]);
  ok = ok && dalloc(pl, &pl->gA, gA) && dalloc(pl, &pl->gB, gB);
  ok = ok && dalloc(pl, &pl->S, (size_t)Q * pl->nfreq) && dalloc(pl, &pl->P, (size_t)np * pl->nfreq);
  ok = ok && dalloc(pl, &pl->Rp, (size_t)np * pl->nbox) && dalloc(pl, &pl->lags, (size_t)Q * Q * pl->nbox);
  pl->a_df = pl->gram_df && !pl->masked;
  if (pl->a_df) ok = ok && dalloc(pl, reinterpret_cast<double2**>(&pl->lags_df), (size_t)Q * Q * pl->nbox);
  ok = ok && dalloc(pl, &pl->A, (size_t)n * n) && dalloc(pl, &pl->A32, (size_t)n * n);
  // eigensolver (sized for the largest block)
  const int M = pl->m_max;
  ok = ok && dalloc(pl, &pl->X, (size_t)n * M) && dalloc(pl, &pl->Y, (size_t)n * M);
  ok = ok && dalloc(pl, &pl->Z, (size_t)n * M) && dalloc(pl, &pl->U, (size_t)n * M);
  ok = ok && dalloc(pl, &pl->Gm, (size_t)M * M) && dalloc(pl, &pl->Rinv, (size_t)M * M);
  {
    const size_t mt = (size_t)std::min(M, 64);
    ok = ok && dalloc(pl, &pl->thin_ws, (size_t)eig_thin_chunks(pl->n) * mt * mt) && dalloc(pl, &pl->thin_tk, 1);
    if (ok) ok = cudaMemset(pl->thin_tk, 0, sizeof(int) * (size_t)pl->items) == cudaSuccess;
  }
  ok = ok && dalloc(pl, &pl->Bm, (size_t)M * M) && dalloc(pl, &pl->Vj, (size_t)2 * M * M);
  ok = ok && dalloc(pl, &pl->mu, (size_t)M) && dalloc(pl, &pl->w, (size_t)M) && dalloc(pl, &pl->ritz, (size_t)M);
  ok = ok && dalloc(pl, &pl->band, (size_t)kNbMax);
  ok = ok && dalloc(pl, &pl->dR0, (size_t)M) && dalloc(pl, &pl->dR1, (size_t)M) && dalloc(pl, &pl->dsc, (size_t)M);
  ok = ok && dalloc(pl, &pl->tiles, (size_t)4096);  // split-K tile counters, 4096 per item
  ok = ok && dalloc_shared(pl, &pl->X0, (size_t)n * M);
  ok = ok && dalloc(pl, &pl->gscale, (size_t)1);
  ok = ok && dalloc(pl, &pl->Xb, (size_t)n * kNbMax) && dalloc(pl, &pl->Zb, (size_t)n * kNbMax);
  pl->ws32_elems = (size_t)16 * n * M;
  pl->ws64_elems = (size_t)16 * kNbMax;  // FP64 split-K scratch (the band product has its own kernel)
  ok = ok && dalloc(pl, &pl->ws32, pl->ws32_elems) && dalloc(pl, &pl->ws64, pl->ws64_elems);
  // G field
  const long long QQ = (long long)Q * Q;
  ok = ok && dalloc(pl, &pl->K, (size_t)(QQ * pl->nbox));
  ok = ok && dalloc(pl, &pl->T1, (size_t)(QQ * B[0] * B[1] * Nr[2]));
  ok = ok && dalloc(pl, &pl->T2, (size_t)(QQ * B[0] * Nr[1] * Nr[2]));
  ok = ok && dalloc(pl, &pl->G, (size_t)(QQ * pl->npix_red));
  if (ok && (pl->tc_g || pl->tc_eig)) {
    if (p->tc_splits > 0) pl->tc_splits_ax = std::min(p->tc_splits, 64);
    const size_t k2n = (size_t)tc2_k2p(n), k2m = (size_t)tc2_k2p(pl->m_max);
    const size_t lo_n = pl->tc_terms == 3 ? 1 : 0;
    pl->tc_ws_elems = std::max<size_t>((size_t)pl->tc_splits_ax * n * pl->m_max,
                                       pl->tc_splits_g > 1 ? (size_t)(pl->tc_splits_g * pl->npix_red * QQ) : 0);
    if (pl->tc_thin) pl->tc_ws_elems = std::max<size_t>(pl->tc_ws_elems, (size_t)kThinSplits * pl->m_max * pl->m_max);
    ok = dalloc(pl, &pl->tc_ws, pl->tc_ws_elems);
    if (ok && pl->tc_thin) {
      const size_t ta = std::max((size_t)n * k2m, (size_t)pl->m_max * k2n);
      const size_t tb = (size_t)2 * tc2_np(pl->m_max) * std::max(k2n, k2m);
      ok = dalloc(pl, &pl->TAh, ta) && dalloc(pl, &pl->TAl, lo_n * ta) && dalloc(pl, &pl->TBh, tb) &&
           dalloc(pl, &pl->TBl, lo_n * tb);
    }
    if (ok && pl->tc_eig)
      ok = dalloc(pl, &pl->Ah, (size_t)n * k2n) && dalloc(pl, &pl->Al, lo_n * n * k2n) &&
           dalloc(pl, &pl->Xh, (size_t)2 * tc2_np(pl->m_max) * k2n) &&
           dalloc(pl, &pl->Xl, lo_n * 2 * tc2_np(pl->m_max) * k2n);
    pl->g_sep = pl->tc_g && pl->D == 2 && (p->flags & PISCO_FLAG_G_DENSE) == 0 &&
                gassembly_field_sep2_supported(pl->nlag, Nr[1], B[1], Nr[2], B[2]);
    if (ok && pl->g_sep) {
      // lags grouped by row b1 (lag_ids ascend in b1, then b2)
      std::vector<int> rows(B[1] + 1, 0), b2(pl->nlag);
      for (int l = 0; l < pl->nlag; ++l) {
        const int t = pl->lag_ids[l];
        rows[(t / B[2]) % B[1] + 1]++;
        b2[l] = t % B[2];
      }
      for (int r = 0; r < B[1]; ++r) rows[r + 1] += rows[r];
      const size_t k2m2 = (size_t)tc2_k2p(pl->m_max);
      ok = upload(pl, &pl->d_sep_rows, rows) && upload(pl, &pl->d_sep_b2, b2) &&
           dalloc(pl, &pl->KT, (size_t)pl->nlag * QQ) && dalloc(pl, &pl->UAh, (size_t)n * k2m2) &&
           dalloc(pl, &pl->UAl, lo_n * n * k2m2) && dalloc(pl, &pl->UBh, (size_t)2 * tc2_np(n) * k2m2) &&
           dalloc(pl, &pl->UBl, lo_n * 2 * tc2_np(n) * k2m2);
    } else if (ok && pl->tc_g && pl->D == 3 && (p->flags & PISCO_FLAG_G_DENSE) == 0) {
      // 3D: the lag sums as three separable DFT passes over the 13^3 lag box (CUDA cores)
      pl->g_box = true;
      std::vector<int> box_lag(pl->nbox, -1);
      for (int l = 0; l < pl->nlag; ++l) box_lag[pl->lag_ids[l]] = l;
      ok = upload(pl, &pl->d_box_lag, box_lag) && dalloc(pl, &pl->KT, (size_t)pl->nlag * QQ) &&
           dalloc(pl, &pl->UAh, (size_t)n * k2m) && dalloc(pl, &pl->UAl, lo_n * n * k2m) &&
           dalloc(pl, &pl->UBh, (size_t)2 * tc2_np(n) * k2m) && dalloc(pl, &pl->UBl, lo_n * 2 * tc2_np(n) * k2m);
    } else if (ok && pl->tc_g) {
      const size_t k2l = (size_t)tc2_k2p(pl->nlag);
      ok = upload(pl, &pl->E, lag_pixel_matrix(Nr, B, pl->tau, pl->lag_ids)) &&
           dalloc(pl, &pl->KT, (size_t)pl->nlag * QQ) && dalloc_shared(pl, &pl->Eh, (size_t)pl->npix_red * k2l) &&
           dalloc_shared(pl, &pl->El, lo_n * pl->npix_red * k2l) && dalloc(pl, &pl->KTh, (size_t)2 * tc2_np((int)QQ) * k2l) &&
           dalloc(pl, &pl->KTl, lo_n * 2 * tc2_np((int)QQ) * k2l) && dalloc(pl, &pl->UAh, (size_t)n * k2m) &&
           dalloc(pl, &pl->UAl, lo_n * n * k2m) && dalloc(pl, &pl->UBh, (size_t)2 * tc2_np(n) * k2m) &&
           dalloc(pl, &pl->UBl, lo_n * 2 * tc2_np(n) * k2m);
      // the lag exponentials never change: split them once here
      ok = ok && tc2_split_a(pl->E, pl->nlag, nullptr, (int)pl->npix_red, pl->nlag, pl->Eh,
                             pl->tc_terms == 3 ? pl->El : nullptr, nullptr) == cudaSuccess;
    }
  }
  // low-res images, PI output, interpolation intermediates
  ok = ok && dalloc(pl, &pl->Ya, (size_t)Q * Nc[0] * Nc[1] * Nr[2]);
  ok = ok && dalloc(pl, &pl->Yb, (size_t)Q * Nc[0] * Nr[1] * Nr[2]);
  ok = ok && dalloc(pl, &pl->Yf, (size_t)(Q * pl->npix_red));
  ok = ok && dalloc(pl, &pl->V, (size_t)(Q * pl->npix_red));
  ok = ok && dalloc(pl, &pl->eig_tmp, (size_t)pl->npix_red);
  ok = ok && dalloc(pl, &pl->I1, (size_t)Q * Nr[0] * Nr[1] * N[2]);
  ok = ok && dalloc(pl, &pl->I2, (size_t)Q * Nr[0] * N[1] * N[2]);
  if (ok && pl->tc_interp) {
    // last interpolation axis: 0 in 3D, 1 in 2D (the axis kernels run the faster ones)
    const int ax = pl->D == 3 ? 0 : 1;
    const long long inner = pl->D == 3 ? (long long)N[1] * N[2] : N[2];
    const size_t k2 = (size_t)tc2_k2p(Nr[ax]);
    const size_t lo_n = pl->tc_terms == 3 ? 1 : 0;
    const size_t nb = (size_t)Q * 2 * tc2_np((int)inner) * k2;
    ok = upload(pl, &pl->interpA, interp_matrix(Nr[ax], N[ax])) && dalloc_shared(pl, &pl->IAh, (size_t)N[ax] * k2) &&
         dalloc_shared(pl, &pl->IAl, lo_n * N[ax] * k2) && dalloc(pl, &pl->IBh, nb) && dalloc(pl, &pl->IBl, lo_n * nb);
    ok = ok && tc2_split_a(pl->interpA, Nr[ax], nullptr, N[ax], Nr[ax], pl->IAh, lo_n ? pl->IAl : nullptr,
                           nullptr) == cudaSuccess;
    // the first (contiguous) axis: I1 = V interpT with V's rows read as FP32 and split in shared
    // memory (three passes only; rows of 16-byte multiples, item blocks 16-byte aligned)
    if (ok && pl->tc_terms == 3 && Nr[2] % 2 == 0 && ((long long)Q * pl->npix_red) % 2 == 0) {
      const size_t nx = (size_t)2 * tc2_np(N[2]) * tc2_k2p(Nr[2]);
      ok = dalloc_shared(pl, &pl->IXh, nx) && dalloc_shared(pl, &pl->IXl, nx) &&
           tc2_split_b(pl->interpT, N[2], 0, Nr[2], N[2], pl->IXh, pl->IXl, nullptr, 1, 0) == cudaSuccess;
      // 2D: W (N1 x Q Nr2 per item, in I1) must fit I1 and keep its item blocks 16-byte aligned;
      // the row-grouped product needs its rows (items N1 Q) within the grid's y limit
      const long long wsz = (long long)N[1] * Q * Nr[2];
      pl->tc_rows2d = ok && pl->D == 2 && wsz <= IS(pl, pl->I1) && wsz % 2 == 0 && IS(pl, pl->I1) % 2 == 0 &&
                      ((long long)N[1] * Q * items + 127) / 128 <= 65535 &&
                      (size_t)2 * tc2_np(Q * Nr[2]) * k2 <= nb;
    }
  }
  ok = ok && dalloc(pl, &pl->dstatus, 1);
  ok = ok && dalloc(pl, &pl->calib_stage, (size_t)Q * Nc[0] * Nc[1] * Nc[2]);
  if (ok && (p->flags & PISCO_FLAG_HOST_IO)) {
    ok = dalloc(pl, &pl->io_calib, (size_t)Q * Nc[0] * Nc[1] * Nc[2]) &&
         dalloc(pl, &pl->io_maps, (size_t)(Q * pl->npix)) && dalloc(pl, &pl->io_eig, (size_t)pl->npix_red);
  }
  if (ok) ok = cudaMallocHost((void**)&pl->hstatus, sizeof(DevStatus) * items) == cudaSuccess;
  if (ok && items > 1)
    ok = dalloc_shared(pl, &pl->in_tab, (size_t)items) && dalloc_shared(pl, &pl->maps_tab, (size_t)items) &&
         dalloc_shared(pl, &pl->eig_tab, (size_t)items);
  if (ok) ok = cudaStreamCreateWithFlags(&pl->cap_st, cudaStreamNonBlocking) == cudaSuccess &&
               cudaEventCreateWithFlags(&pl->ev_in, cudaEventDisableTiming) == cudaSuccess &&
               cudaEventCreateWithFlags(&pl->ev_out, cudaEventDisableTiming) == cudaSuccess;
  for (int i = 0; ok && i < 2 * 160; ++i) {  // event pool for operation timing
    cudaEvent_t e;
    ok = cudaEventCreate(&e) == cudaSuccess;
    if (ok) pl->ev.push_back(e);
    if (ok && (i & 1)) pl->ev_tag.push_back(nullptr);
  }
  if (ok) ok = cudaMemset(pl->lags, 0, sizeof(double2) * (size_t)Q * Q * pl->nbox * items) == cudaSuccess;
  if (ok) ok = cudaMemset(pl->tiles, 0, sizeof(int) * 4096 * items) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    pisco_destroy(pl);
    return PISCO_ERR_OOM;
  }
  if (cudaDeviceSynchronize() != cudaSuccess) {
    pisco_destroy(pl);
    return PISCO_ERR_CUDA;
  }
  *out = pl;
  return PISCO_OK;
}

extern "C" {

pisco_status pisco_plan(const pisco_params* p, void* cuda_stream, pisco_plan_t* out) {
  return plan_create(p, (cudaStream_t)cuda_stream, 1, out);
}

pisco_status pisco_estimate(pisco_plan_t pl, const void* d_calib, void* d_maps, float* d_eig) {
  if (!pl || !d_calib || !d_maps) return PISCO_ERR_ARG;
  if (((uintptr_t)d_calib | (uintptr_t)d_maps | (uintptr_t)d_eig) & 7) return PISCO_ERR_ARG;
  // the path (and its graph) always reads the plan's staging copy of the calibration block
  if (d_calib != pl->calib_stage &&
      cudaMemcpyAsync(pl->calib_stage, d_calib,
                      sizeof(float2) * (size_t)pl->Q * pl->Nc[0] * pl->Nc[1] * pl->Nc[2],
                      cudaMemcpyDeviceToDevice, pl->st) != cudaSuccess)
    return PISCO_ERR_CUDA;
  d_calib = pl->calib_stage;
  for (;;) {
    const bool same_as_graph = pl->gexec && pl->g_calib == d_calib && pl->g_maps == d_maps &&
                               pl->g_eig == d_eig && pl->g_m == solve_key(pl) && pl->g_prof == pl->prof;
    const bool same_as_eager = pl->eager_calib == d_calib && pl->eager_maps == d_maps &&
                               pl->eager_eig == d_eig && pl->eager_m == solve_key(pl) && pl->eager_prof == pl->prof;
    // profiled calls always run eagerly: their per-operation events time individual launches
    if (pl->use_graph && !pl->prof && !same_as_graph && same_as_eager) {
      // capture the path once the same arguments have run eagerly (attributes set, sizes settled)
      graph_reset(pl);
      pl->ev_used = 0;
      if (cudaStreamBeginCapture(pl->cap_st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        cudaStream_t user = pl->st;
        pl->st = pl->cap_st;
        pisco_status s = run_all(pl, (const float2*)d_calib, (float2*)d_maps, d_eig);
        pl->st = user;
        cudaGraph_t g = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(pl->cap_st, &g);
        if (s == PISCO_OK && ec == cudaSuccess && g &&
            cudaGraphInstantiate(&pl->gexec, g, 0) == cudaSuccess) {
          pl->graph = g;
          pl->g_calib = d_calib; pl->g_maps = d_maps; pl->g_eig = d_eig;
          pl->g_m = solve_key(pl); pl->g_prof = pl->prof;
          pl->g_launches = g_launches;
          pl->g_events = pl->ev_used;
        } else {
          if (g) cudaGraphDestroy(g);
          pl->gexec = nullptr;
          pl->use_graph = false;  // fall back to eager launches for this plan
          cudaGetLastError();
        }
      } else {
        pl->use_graph = false;
        cudaGetLastError();
      }
    }
    const bool replay = pl->use_graph && !pl->prof && pl->gexec && pl->g_calib == d_calib && pl->g_maps == d_maps &&
                        pl->g_eig == d_eig && pl->g_m == solve_key(pl) && pl->g_prof == pl->prof;
    if (replay) {
      // order the graph after earlier work on the caller's stream, and the caller after it
      if (cudaEventRecord(pl->ev_in, pl->st) != cudaSuccess ||
          cudaStreamWaitEvent(pl->cap_st, pl->ev_in, 0) != cudaSuccess ||
          cudaGraphLaunch(pl->gexec, pl->cap_st) != cudaSuccess ||
          cudaEventRecord(pl->ev_out, pl->cap_st) != cudaSuccess ||
          cudaStreamWaitEvent(pl->st, pl->ev_out, 0) != cudaSuccess)
        return PISCO_ERR_CUDA;
      if (cudaStreamSynchronize(pl->st) != cudaSuccess) return PISCO_ERR_CUDA;
      pl->last_launches = pl->g_launches;
      if (pl->prof) prof_collect(pl, pl->g_events);
    } else {
      pl->ev_used = 0;
      pisco_status s = run_all(pl, (const float2*)d_calib, (float2*)d_maps, d_eig);
      if (s != PISCO_OK) return s;
      if (cudaStreamSynchronize(pl->st) != cudaSuccess) return PISCO_ERR_CUDA;
      pl->last_launches = g_launches;
      if (pl->prof) prof_collect(pl, pl->ev_used);
      pl->eager_calib = d_calib; pl->eager_maps = d_maps; pl->eager_eig = d_eig;
      pl->eager_m = solve_key(pl); pl->eager_prof = pl->prof;
    }
    const DevStatus h = *pl->hstatus;
    pl->last_status = h;
    if (h.flags & ST_TIMEOUT) return PISCO_ERR_TIMEOUT;
    if ((h.flags & ST_SATURATED) && pl->m < pl->m_max) {
      pl->m = std::min(pl->m * 2, pl->m_max);
      continue;
    }
    if ((h.flags & ST_UNCERTIFIED) && !(h.flags & ST_SATURATED) && retry_iters(pl)) continue;
    pl->last_k = h.k;
    pl->last_R = pl->n - h.k;
    if (h.flags & (ST_SATURATED | ST_UNCERTIFIED)) return PISCO_ERR_NOT_CONVERGED;
    if (h.flags & ST_RANK) return PISCO_ERR_RANK;
    return PISCO_OK;
  }
}

pisco_status pisco_estimate_host(pisco_plan_t pl, const void* h_calib, void* h_maps, float* h_eig) {
  if (!pl || !h_calib || !h_maps) return PISCO_ERR_ARG;
  if (!pl->io_calib) return PISCO_ERR_ARG;
  const size_t cb = sizeof(float2) * (size_t)pl->Q * pl->Nc[0] * pl->Nc[1] * pl->Nc[2];
  const size_t mb = sizeof(float2) * (size_t)pl->Q * pl->npix;
  if (cudaMemcpyAsync(pl->calib_stage, h_calib, cb, cudaMemcpyHostToDevice, pl->st) != cudaSuccess)
    return PISCO_ERR_CUDA;
  pisco_status s = pisco_estimate(pl, pl->calib_stage, pl->io_maps, h_eig ? pl->io_eig : nullptr);
  if (s != PISCO_OK && s != PISCO_ERR_RANK) return s;
  if (cudaMemcpyAsync(h_maps, pl->io_maps, mb, cudaMemcpyDeviceToHost, pl->st) != cudaSuccess)
    return PISCO_ERR_CUDA;
  if (h_eig && cudaMemcpyAsync(h_eig, pl->io_eig, sizeof(float) * pl->npix_red, cudaMemcpyDeviceToHost,
                               pl->st) != cudaSuccess)
    return PISCO_ERR_CUDA;
  if (cudaStreamSynchronize(pl->st) != cudaSuccess) return PISCO_ERR_CUDA;
  return s;
}

pisco_status pisco_plan_info(pisco_plan_t pl, int* R, int* k, size_t* workspace_bytes) {
  if (!pl) return PISCO_ERR_ARG;
  if (R) *R = pl->last_R;
  if (k) *k = pl->last_k;
  if (workspace_bytes) *workspace_bytes = pl->ws_bytes;
  return PISCO_OK;
}

pisco_status pisco_debug_buffer(pisco_plan_t pl, int which, void** dptr, size_t* bytes) {
  if (!pl || !dptr || !bytes) return PISCO_ERR_ARG;
  const size_t n = pl->n;
  switch (which) {
    case PISCO_BUF_LAGS: *dptr = pl->lags; *bytes = sizeof(double2) * (size_t)pl->Q * pl->Q * pl->nbox; break;
    case PISCO_BUF_GRAM:
      if (pl->a_df) {
        // the double-float Gram as FP64 (hi + lo is exact in FP64), built on request
        if (!pl->A64 && !dalloc(pl, &pl->A64, n * n)) return PISCO_ERR_OOM;
        if (df_to_fp64(pl->A, (long long)(n * n), pl->A64, pl->st) != cudaSuccess ||
            cudaStreamSynchronize(pl->st) != cudaSuccess)
          return PISCO_ERR_CUDA;
        *dptr = pl->A64;
      } else {
        *dptr = pl->A;
      }
      *bytes = sizeof(double2) * n * n;
      break;
    case PISCO_BUF_SIGNAL: *dptr = pl->U; *bytes = sizeof(float2) * n * pl->m; break;
    case PISCO_BUF_WEIGHTS: *dptr = pl->w; *bytes = sizeof(float) * pl->m; break;
    case PISCO_BUF_RITZ: *dptr = pl->ritz; *bytes = sizeof(double) * pl->m; break;
    case PISCO_BUF_G: *dptr = pl->G; *bytes = sizeof(float2) * (size_t)pl->Q * pl->Q * pl->npix_red; break;
    case PISCO_BUF_V: *dptr = pl->V; *bytes = sizeof(float2) * (size_t)pl->Q * pl->npix_red; break;
    case PISCO_BUF_Y: *dptr = pl->Yf; *bytes = sizeof(float2) * (size_t)pl->Q * pl->npix_red; break;
    case PISCO_BUF_BLOCK: *dptr = pl->X; *bytes = sizeof(float2) * n * pl->m; break;
    case PISCO_BUF_RITZ32: *dptr = pl->mu; *bytes = sizeof(float) * pl->m; break;
    case PISCO_BUF_SCALE: *dptr = pl->gscale; *bytes = sizeof(double); break;
    default: return PISCO_ERR_ARG;
  }
  return PISCO_OK;
}

pisco_status pisco_get_stats(pisco_plan_t pl, pisco_stats* out) {
  if (!pl || !out) return PISCO_ERR_ARG;
  out->launches = pl->last_launches;
  out->eig_block = pl->m;
  out->eig_iters = pl->eig_iters;
  out->jacobi_sweeps = pl->last_status.jacobi_sweeps;
  out->nband = pl->last_status.nband;
  out->lambda_max = pl->last_status.lambda_max;
  out->signal_dim = pl->last_k;
  out->filter_len = pl->L;
  out->warm_fallback = pl->ws_on ? pl->last_status.ws_fallback : 0;
  out->cert_margin = pl->last_status.cert_margin;
  out->band_resid = pl->last_status.band_resid;
  return PISCO_OK;
}

pisco_status pisco_set_warm_start(pisco_plan_t pl, pisco_mlp_t mlp, int iters, float gate, int fallback_iters) {
  if (!pl) return PISCO_ERR_ARG;
  if (!mlp) {
    pl->ws_on = false;
    graph_reset(pl);
    pl->eager_calib = nullptr;
    return PISCO_OK;
  }
  int n_in, H, n_out;
  size_t np;
  mlp_dims(mlp, &n_in, &H, &n_out, &np);
  if (n_out != 2 * pl->Q || n_in % n_out != 0 || iters < 0 || fallback_iters < 1 || !(gate == gate)) return PISCO_ERR_ARG;
  // the input: the (2r+1)^D patch of normalised low-resolution vectors around the pixel
  int r = -1;
  for (int t = 0; t <= 3; ++t) {
    const int w = 2 * t + 1;
    if (n_in / n_out == (pl->D == 3 ? w * w * w : w * w)) r = t;
  }
  if (r < 0) return PISCO_ERR_ARG;
  if (pl->block_pi) return PISCO_ERR_UNSUPPORTED;  // the block iteration draws its own two starts
  if (pl->items > 1) return PISCO_ERR_UNSUPPORTED;
  if (cudaStreamSynchronize(pl->st) != cudaSuccess) return PISCO_ERR_CUDA;
  const size_t nr = (size_t)pl->npix_red;
  if (!pl->ws_H1) {
    const bool ok = dalloc(pl, &pl->ws_H1, nr * 128) && dalloc(pl, &pl->ws_H2, nr * 128) &&
                    dalloc(pl, &pl->ws_out, nr * 2 * pl->Q) && dalloc(pl, &pl->fb_flags, nr);
    if (!ok) {
      cudaGetLastError();
      return PISCO_ERR_OOM;
    }
  }
  if (n_in > pl->ws_cap) {  // (a narrower earlier buffer stays allocated until the plan is destroyed)
    const size_t npmax = mlp_param_count(n_in, 128, n_out);
    if (!(dalloc(pl, &pl->ws_w32, npmax) && dalloc(pl, &pl->ws_w16, npmax) && dalloc(pl, &pl->ws_X, nr * n_in))) {
      cudaGetLastError();
      return PISCO_ERR_OOM;
    }
    pl->ws_cap = n_in;
  }
  const MlpView src = mlp_view(mlp);
  if (cudaMemcpy(pl->ws_w32, src.w32, sizeof(float) * np, cudaMemcpyDeviceToDevice) != cudaSuccess ||
      cudaMemcpy(pl->ws_w16, src.w16, sizeof(__half) * np, cudaMemcpyDeviceToDevice) != cudaSuccess)
    return PISCO_ERR_CUDA;
  pl->ws_H = H;
  pl->ws_nin = n_in;
  pl->ws_r = r;
  pl->ws_iters = iters;
  pl->ws_gate = gate;
  pl->ws_fb_iters = fallback_iters;
  pl->ws_on = true;
  graph_reset(pl);
  pl->eager_calib = nullptr;  // the next call runs eagerly, the one after captures the new sequence
  return PISCO_OK;
}

pisco_status pisco_set_profiling(pisco_plan_t pl, int enable) {
  if (!pl) return PISCO_ERR_ARG;
  pl->prof = enable != 0;
  return PISCO_OK;
}

pisco_status pisco_profile_reset(pisco_plan_t pl) {
  if (!pl) return PISCO_ERR_ARG;
  pl->prof_name.clear();
  pl->prof_ms.clear();
  pl->prof_cnt.clear();
  return PISCO_OK;
}

pisco_status pisco_profile_entry(pisco_plan_t pl, int idx, const char** name, double* total_ms, int* count) {
  if (!pl || idx < 0 || idx >= (int)pl->prof_name.size()) return PISCO_ERR_ARG;
  if (name) *name = pl->prof_name[idx];
  if (total_ms) *total_ms = pl->prof_ms[idx];
  if (count) *count = pl->prof_cnt[idx];
  return PISCO_OK;
}

// ---------------------------------------------------------------------------------------
// Batches.  Items of identical parameters form groups of up to batch_group items; a group is
// one plan whose passes run every stage once over all of its items (item-strided buffers,
// per-item inputs and outputs through device pointer tables), and each of its items is
// reached through a one-item view into the group's buffers (statuses, statistics, debug
// buffers and re-runs of single items).  A group of one item is an ordinary plan.  All groups
// are captured into one CUDA graph whose branches (one per group) run concurrently; it is
// replayed while the pointer sets stay the same.
// ---------------------------------------------------------------------------------------
struct pisco_batch_s {
  std::vector<pisco_plan_s*> items;    // per item: its one-item plan (a view, or the group itself)
  std::vector<pisco_plan_s*> groups;   // owning: one plan per group
  std::vector<pisco_plan_s*> views;    // owning: views of groups with more than one item
  std::vector<int> group_of, slot_of;  // item -> group, item -> index inside its group
  std::vector<std::vector<int>> members;  // group -> its items
  std::vector<cudaStream_t> streams;   // one per group
  std::vector<cudaEvent_t> join;       // one per group
  cudaEvent_t fork = nullptr;
  cudaStream_t main = nullptr;   // private non-blocking stream: capture and graph launch
  cudaStream_t user = nullptr;   // the caller's stream
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  // host-I/O graphs: recorded after the graph (every item's compute done), before the
  // device->host copies; the next host-I/O graph of another batch waits on it (compute
  // chained, the copies of one batch overlapping the compute of the next)
  cudaEvent_t ev_compute = nullptr;
  cudaStream_t in_st = nullptr;  // host-I/O input copies (kept apart from the output copies)
  cudaEvent_t ev_staged = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  std::vector<const void*> g_in;
  std::vector<void*> g_out;
  std::vector<float*> g_eig;
  bool g_host = false;
  int launches = 0;
  bool warmed = false;  // one eager run first: kernel attributes are set outside any capture
  // the launched, not yet waited-for call (pointers kept for status decoding and re-runs)
  bool pending = false, pend_host = false;
  std::vector<const void*> pend_in;
  std::vector<void*> pend_out;
  std::vector<float*> pend_eig;
  bool prof = false;  // operation timing: eager calls, events around every operation
};

// the compute-done event of the last host-I/O graph launched by any batch
std::mutex g_chain_mu;
cudaEvent_t g_chain_ev = nullptr;
const pisco_batch_s* g_chain_owner = nullptr;

namespace {

constexpr int kAutoGroup = 64;

bool same_params(const pisco_params& a, const pisco_params& b) {
  bool s = a.ndim == b.ndim && a.num_coils == b.num_coils && a.kernel_shape == b.kernel_shape &&
           a.null_threshold == b.null_threshold && a.grid_reduction == b.grid_reduction &&
           a.power_iters == b.power_iters && a.seed == b.seed && a.flags == b.flags && a.eig_block == b.eig_block &&
           a.eig_iters == b.eig_iters && a.tc_splits == b.tc_splits && a.gemm_splits == b.gemm_splits &&
           a.gemm_tile == b.gemm_tile && a.batch_group == b.batch_group;
  for (int d = 0; d < 3; ++d)
    s = s && a.grid[d] == b.grid[d] && a.calib[d] == b.calib[d] && a.kernel_radius[d] == b.kernel_radius[d];
  return s;
}

// items of these parameters may share a batched pass
int group_cap(const pisco_params& p) {
  if (!(p.flags & PISCO_FLAG_TC_GFIELD) || (p.flags & (PISCO_FLAG_MASKED_GRAM | PISCO_FLAG_BLOCK_PI))) return 1;
  return p.batch_group > 0 ? p.batch_group : kAutoGroup;
}

// a one-item view of item i of group g: the group's plan state with every per-item buffer
// pointer moved to item i; it shares the group's tables and owns nothing at creation
pisco_plan_s* make_view(pisco_plan_s* g, int i, cudaStream_t st) {
  pisco_plan_s* v = new (std::nothrow) pisco_plan_s(*g);
  if (!v) return nullptr;
  v->items = 1;
  v->view = true;
  v->allocs.clear();
  v->ws_bytes = 0;
  v->item_elems.clear();
  v->in_tab = nullptr;
  v->maps_tab = nullptr;
  v->eig_tab = nullptr;
  v->h_in.clear();
  v->h_maps.clear();
  v->h_eig.clear();
  v->st = st;
  v->ev.clear();
  v->ev_tag.clear();
  v->ev_used = 0;
  v->prof = false;
  v->cap_st = nullptr;
  v->ev_in = v->ev_out = nullptr;
  v->use_graph = false;
  v->graph = nullptr;
  v->gexec = nullptr;
  v->g_m = -1;
  v->eager_calib = nullptr;
  v->prof_name.clear();
  v->prof_ms.clear();
  v->prof_cnt.clear();
  v->hstatus = g->hstatus + i;
  for (const auto& f : g->item_elems) {
    char** field = reinterpret_cast<char**>(reinterpret_cast<char*>(v) + f.first);
    *field += (size_t)i * f.second.second;
  }
  return v;
}

// uploads a group's pointer tables when the pointer set changed (no call of this batch is in
// flight, so the previous graph no longer reads them)
pisco_status set_tables(pisco_plan_s* g, const std::vector<const void*>& in, const std::vector<void*>& out,
                        const std::vector<float*>& eig) {
  if (g->items == 1) return PISCO_OK;
  if (g->h_in == in && g->h_maps == out && g->h_eig == eig) return PISCO_OK;
  const size_t n = (size_t)g->items;
  if (cudaMemcpy(g->in_tab, in.data(), n * sizeof(void*), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(g->maps_tab, out.data(), n * sizeof(void*), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(g->eig_tab, eig.data(), n * sizeof(void*), cudaMemcpyHostToDevice) != cudaSuccess)
    return PISCO_ERR_CUDA;
  g->h_in = in;
  g->h_maps = out;
  g->h_eig = eig;
  return PISCO_OK;
}

// calibration blocks of a group's items into its staging buffer, one launch
__global__ void gather_inputs_kernel(const float2* const* __restrict__ src, float2* __restrict__ dst,
                                     long long elems) {
  const float2* s = src[blockIdx.y];
  float2* d = dst + blockIdx.y * elems;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < elems; e += (long long)gridDim.x * blockDim.x)
    d[e] = s[e];
}

pisco_status gather_inputs(pisco_plan_s* g) {
  const long long elems = IS(g, g->calib_stage);
  long long blocks = (elems + 255) / 256;
  if (blocks > 64) blocks = 64;
  gather_inputs_kernel<<<dim3((unsigned)blocks, g->items), 256, 0, g->st>>>(g->in_tab, g->calib_stage, elems);
  ++g_launches;
  return cudaGetLastError() == cudaSuccess ? PISCO_OK : PISCO_ERR_CUDA;
}

}  // namespace

static void batch_graph_reset(pisco_batch_s* b) {
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->gexec = nullptr;
  b->graph = nullptr;
  b->g_in.clear();
  b->g_out.clear();
  b->g_eig.clear();
}

void pisco_batch_destroy(pisco_batch_t b) {
  if (!b) return;
  if (b->main) cudaStreamSynchronize(b->main);
  batch_graph_reset(b);
  {
    std::lock_guard<std::mutex> lk(g_chain_mu);
    if (g_chain_owner == b) {
      g_chain_owner = nullptr;
      g_chain_ev = nullptr;
    }
  }
  if (b->main) cudaStreamDestroy(b->main);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_compute) cudaEventDestroy(b->ev_compute);
  if (b->in_st) {
    cudaStreamSynchronize(b->in_st);
    cudaStreamDestroy(b->in_st);
  }
  if (b->ev_staged) cudaEventDestroy(b->ev_staged);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  for (auto* v : b->views) pisco_destroy(v);
  for (auto* pl : b->groups) pisco_destroy(pl);
  for (auto s : b->streams) if (s) cudaStreamDestroy(s);
  for (auto e : b->join) if (e) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  delete b;
}

pisco_status pisco_batch_plan(const pisco_params* params, int count, void* cuda_stream,
                              pisco_batch_t* out) {
  if (!out || !params || count < 1 || count > 4096) return PISCO_ERR_ARG;
  *out = nullptr;
  for (int i = 0; i < count; ++i) {
    pisco_status s = validate(&params[i]);
    if (s != PISCO_OK) return s;
  }
  pisco_batch_s* b = new (std::nothrow) pisco_batch_s();
  if (!b) return PISCO_ERR_OOM;
  b->user = (cudaStream_t)cuda_stream;
  if (cudaStreamCreateWithFlags(&b->main, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_compute, cudaEventDisableTiming) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->in_st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_staged, cudaEventDisableTiming) != cudaSuccess) {
    pisco_batch_destroy(b);
    return PISCO_ERR_CUDA;
  }
  // groups of identical parameters, in item order
  b->group_of.assign(count, -1);
  b->slot_of.assign(count, 0);
  for (int i = 0; i < count; ++i) {
    int g = -1;
    for (int j = 0; j < (int)b->members.size() && g < 0; ++j) {
      const int first = b->members[j][0];
      if (same_params(params[first], params[i]) && (int)b->members[j].size() < group_cap(params[i])) g = j;
    }
    if (g < 0) {
      g = (int)b->members.size();
      b->members.emplace_back();
    }
    b->group_of[i] = g;
    b->slot_of[i] = (int)b->members[g].size();
    b->members[g].push_back(i);
  }
  b->items.assign(count, nullptr);
  for (int g = 0; g < (int)b->members.size(); ++g) {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
      if (st) cudaStreamDestroy(st);
      pisco_batch_destroy(b);
      return PISCO_ERR_CUDA;
    }
    b->streams.push_back(st);
    b->join.push_back(ev);
    const std::vector<int>& mem = b->members[g];
    pisco_params pi = params[mem[0]];
    pi.flags |= PISCO_FLAG_HOST_IO;
    pisco_plan_s* pl = nullptr;
    pisco_status s = plan_create(&pi, st, (int)mem.size(), &pl);
    if (s != PISCO_OK) {
      pisco_batch_destroy(b);
      return s;
    }
    pl->use_graph = false;
    b->groups.push_back(pl);
    if (mem.size() == 1) {
      b->items[mem[0]] = pl;
      continue;
    }
    for (int k = 0; k < (int)mem.size(); ++k) {
      pisco_plan_s* v = make_view(pl, k, st);
      if (!v) {
        pisco_batch_destroy(b);
        return PISCO_ERR_OOM;
      }
      b->views.push_back(v);
      b->items[mem[k]] = v;
    }
  }
  *out = b;
  return PISCO_OK;
}

// the pointer tables of every group for this call (device or host I/O) and, per group, the
// work of one pass: one-item groups copy their input and run as a plan; larger groups gather
// their inputs (device I/O) and run one batched pass.  host_inline: issue the host copies of
// host-I/O calls on the group streams too (eager first call); otherwise the caller does.
static pisco_status enqueue_groups(pisco_batch_s* b, const void* const* in, void* const* outp, float* const* eig,
                                   bool host_io, bool host_inline, int* launches) {
  int total = 0;
  for (int g = 0; g < (int)b->groups.size(); ++g) {
    pisco_plan_s* gp = b->groups[g];
    cudaStream_t st = gp->st;
    if (cudaStreamWaitEvent(st, b->fork, 0) != cudaSuccess) return PISCO_ERR_CUDA;
    const std::vector<int>& mem = b->members[g];
    const size_t cb = sizeof(float2) * (size_t)gp->Q * gp->Nc[0] * gp->Nc[1] * gp->Nc[2];
    const size_t mb = sizeof(float2) * (size_t)gp->Q * gp->npix;
    // inputs
    for (int k = 0; k < (int)mem.size(); ++k) {
      const int i = mem[k];
      pisco_plan_s* it = b->items[i];
      if (host_io && host_inline &&
          cudaMemcpyAsync(it->calib_stage, in[i], cb, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return PISCO_ERR_CUDA;
      if (!host_io && mem.size() == 1 &&
          cudaMemcpyAsync(it->calib_stage, in[i], cb, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return PISCO_ERR_CUDA;
    }
    gp->ev_used = 0;
    pisco_status s;
    if (mem.size() == 1) {
      const int i = mem[0];
      float2* maps_dst = host_io ? gp->io_maps : (float2*)outp[i];
      float* eig_dst = eig && eig[i] ? (host_io ? gp->io_eig : eig[i]) : nullptr;
      s = run_all(gp, gp->calib_stage, maps_dst, eig_dst);
      if (s != PISCO_OK) return s;
      total += g_launches;
    } else {
      int extra = 0;
      if (!host_io) {
        g_launches = 0;
        if ((s = gather_inputs(gp)) != PISCO_OK) return s;
        extra = g_launches;
      }
      s = run_all(gp, gp->calib_stage, nullptr, nullptr);
      if (s != PISCO_OK) return s;
      total += g_launches + extra;
    }
    // host-I/O results of the eager call
    if (host_io && host_inline) {
      for (int k = 0; k < (int)mem.size(); ++k) {
        const int i = mem[k];
        pisco_plan_s* it = b->items[i];
        if (cudaMemcpyAsync(outp[i], it->io_maps, mb, cudaMemcpyDeviceToHost, st) != cudaSuccess) return PISCO_ERR_CUDA;
        if (eig && eig[i] &&
            cudaMemcpyAsync(eig[i], it->io_eig, sizeof(float) * it->npix_red, cudaMemcpyDeviceToHost, st) != cudaSuccess)
          return PISCO_ERR_CUDA;
      }
    }
    if (cudaEventRecord(b->join[g], st) != cudaSuccess || cudaStreamWaitEvent(b->main, b->join[g], 0) != cudaSuccess)
      return PISCO_ERR_CUDA;
  }
  if (launches) *launches = total;
  return PISCO_OK;
}

// the tables of every group with more than one item for this pointer set
static pisco_status batch_tables(pisco_batch_s* b, const void* const* in, void* const* outp, float* const* eig,
                                 bool host_io) {
  for (int g = 0; g < (int)b->groups.size(); ++g) {
    pisco_plan_s* gp = b->groups[g];
    if (gp->items == 1) continue;
    const std::vector<int>& mem = b->members[g];
    std::vector<const void*> ti(mem.size());
    std::vector<void*> tm(mem.size());
    std::vector<float*> te(mem.size());
    for (size_t k = 0; k < mem.size(); ++k) {
      const int i = mem[k];
      pisco_plan_s* it = b->items[i];
      ti[k] = host_io ? it->calib_stage : in[i];
      tm[k] = host_io ? (void*)it->io_maps : outp[i];
      te[k] = eig && eig[i] ? (host_io ? it->io_eig : eig[i]) : nullptr;
    }
    const pisco_status s = set_tables(gp, ti, tm, te);
    if (s != PISCO_OK) return s;
  }
  return PISCO_OK;
}

// Enqueue the whole batch (capture on the second call with a new pointer set, replay after);
// order_user: order the batch after the caller's stream and the caller's stream after it
// (device buffers); host-buffer launches skip that so two batches can be in flight at once.
static pisco_status batch_launch(pisco_batch_s* b, const void* const* in, void* const* outp,
                                 float* const* eig, bool host_io, bool order_user) {
  const int n = (int)b->items.size();
  for (int i = 0; i < n; ++i)
    if (!in[i] || !outp[i]) return PISCO_ERR_ARG;
  bool same = b->gexec && b->g_host == host_io && (int)b->g_in.size() == n && !b->prof;
  for (int i = 0; same && i < n; ++i)
    same = b->g_in[i] == in[i] && b->g_out[i] == outp[i] && b->g_eig[i] == (eig ? eig[i] : nullptr);
  if (!same) {
    // the tables of the new pointer set (the previous call has been waited for)
    if (cudaStreamSynchronize(b->main) != cudaSuccess) return PISCO_ERR_CUDA;
    const pisco_status s = batch_tables(b, in, outp, eig, host_io);
    if (s != PISCO_OK) return s;
  }
  if (order_user && (cudaEventRecord(b->ev_in, b->user) != cudaSuccess ||
                     cudaStreamWaitEvent(b->main, b->ev_in, 0) != cudaSuccess))
    return PISCO_ERR_CUDA;
  if (!same && (!b->warmed || b->prof)) {
    // first call (and profiled calls): every group eagerly on its own stream (same work as the graph)
    if (cudaEventRecord(b->fork, b->main) != cudaSuccess) return PISCO_ERR_CUDA;
    const pisco_status s = enqueue_groups(b, in, outp, eig, host_io, true, nullptr);
    if (s != PISCO_OK) return s;
    b->warmed = true;
  } else if (!same) {
    batch_graph_reset(b);
    if (cudaStreamBeginCapture(b->main, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return PISCO_ERR_CUDA;
    int total_launches = 0;
    pisco_status s = PISCO_OK;
    if (cudaEventRecord(b->fork, b->main) != cudaSuccess) s = PISCO_ERR_CUDA;
    // host I/O: the copies stay outside the graph (issued around each launch)
    if (s == PISCO_OK) s = enqueue_groups(b, in, outp, eig, host_io, false, &total_launches);
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(b->main, &g);
    if (s != PISCO_OK || ec != cudaSuccess || !g) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return s != PISCO_OK ? s : PISCO_ERR_CUDA;
    }
    if (cudaGraphInstantiate(&b->gexec, g, 0) != cudaSuccess) {
      cudaGraphDestroy(g);
      b->gexec = nullptr;
      return PISCO_ERR_CUDA;
    }
    b->graph = g;
    b->launches = total_launches;
    b->g_host = host_io;
    for (int i = 0; i < n; ++i) {
      b->g_in.push_back(in[i]);
      b->g_out.push_back(outp[i]);
      b->g_eig.push_back(eig ? eig[i] : nullptr);
    }
  }
  if (b->gexec && host_io) {
    // inputs staged, compute chained after the previous host-I/O batch's compute, then this
    // batch's output copies on its own stream (copy-engine copies overlap the next compute)
    // the inputs first, on their own stream (not queued behind this batch's pending output
    // copies), so that they are staged while the previous batch still computes
    if (cudaEventRecord(b->ev_staged, b->main) != cudaSuccess || cudaStreamWaitEvent(b->in_st, b->ev_staged, 0) != cudaSuccess)
      return PISCO_ERR_CUDA;
    for (int i = 0; i < n; ++i) {
      pisco_plan_s* pl = b->items[i];
      const size_t cb = sizeof(float2) * (size_t)pl->Q * pl->Nc[0] * pl->Nc[1] * pl->Nc[2];
      if (cudaMemcpyAsync(pl->calib_stage, in[i], cb, cudaMemcpyHostToDevice, b->in_st) != cudaSuccess)
        return PISCO_ERR_CUDA;
    }
    if (cudaEventRecord(b->ev_staged, b->in_st) != cudaSuccess || cudaStreamWaitEvent(b->main, b->ev_staged, 0) != cudaSuccess)
      return PISCO_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_chain_mu);
    if (g_chain_ev && g_chain_owner != b && cudaStreamWaitEvent(b->main, g_chain_ev, 0) != cudaSuccess)
      return PISCO_ERR_CUDA;
    if (cudaGraphLaunch(b->gexec, b->main) != cudaSuccess || cudaEventRecord(b->ev_compute, b->main) != cudaSuccess)
      return PISCO_ERR_CUDA;
    g_chain_ev = b->ev_compute;
    g_chain_owner = b;
    for (int i = 0; i < n; ++i) {
      pisco_plan_s* pl = b->items[i];
      const size_t mb = sizeof(float2) * (size_t)pl->Q * pl->npix;
      if (cudaMemcpyAsync(outp[i], pl->io_maps, mb, cudaMemcpyDeviceToHost, b->main) != cudaSuccess)
        return PISCO_ERR_CUDA;
      if (eig && eig[i] &&
          cudaMemcpyAsync(eig[i], pl->io_eig, sizeof(float) * pl->npix_red, cudaMemcpyDeviceToHost, b->main) != cudaSuccess)
        return PISCO_ERR_CUDA;
    }
  } else if (b->gexec && cudaGraphLaunch(b->gexec, b->main) != cudaSuccess) {
    return PISCO_ERR_CUDA;
  }
  if (order_user && (cudaEventRecord(b->ev_out, b->main) != cudaSuccess ||
                     cudaStreamWaitEvent(b->user, b->ev_out, 0) != cudaSuccess))
    return PISCO_ERR_CUDA;
  b->pend_in.assign(in, in + n);
  b->pend_out.assign(outp, outp + n);
  b->pend_eig.assign(n, nullptr);
  if (eig)
    for (int i = 0; i < n; ++i) b->pend_eig[i] = eig[i];
  b->pend_host = host_io;
  b->pending = true;
  return PISCO_OK;
}

// Wait for the launched batch, then decode every item's status.  Items whose eigensolver block
// saturated, or whose split is not certified yet with the automatic iteration count, are re-run
// alone (through their view) with a larger block or more iterations; their group adopts the
// larger setting for later calls.
static pisco_status batch_finish(pisco_batch_s* b, pisco_status* item_status) {
  if (!b->pending) return PISCO_ERR_ARG;
  b->pending = false;
  const int n = (int)b->items.size();
  const bool host_io = b->pend_host;
  const void* const* in = b->pend_in.data();
  void* const* outp = b->pend_out.data();
  float* const* eig = b->pend_eig.data();
  if (cudaStreamSynchronize(b->main) != cudaSuccess) return PISCO_ERR_CUDA;
  if (b->prof)
    for (pisco_plan_s* gp : b->groups) prof_collect(gp, gp->ev_used);
  // a bounded wait of a batched tensor-core product reports on the group's first item
  for (pisco_plan_s* gp : b->groups)
    if (gp->items > 1 && (gp->hstatus[0].flags & ST_TIMEOUT))
      for (int k = 1; k < gp->items; ++k) gp->hstatus[k].flags |= ST_TIMEOUT;
  pisco_status worst = PISCO_OK;
  bool regroup = false;
  for (int i = 0; i < n; ++i) {
    pisco_plan_s* pl = b->items[i];
    const DevStatus h = *pl->hstatus;
    pl->last_status = h;
    pl->last_launches = 0;
    pisco_status si = PISCO_OK;
    if (h.flags & ST_TIMEOUT) {
      si = PISCO_ERR_TIMEOUT;
    } else if (h.flags & ST_SATURATED) {
      // the signal dimension reached the block: redo this item alone with a larger block
      if (pl->m < pl->m_max) {
        pl->m = std::min(pl->m * 2, pl->m_max);
        batch_graph_reset(b);
        regroup = true;
        si = host_io ? pisco_estimate_host(pl, in[i], outp[i], eig[i]) : pisco_estimate(pl, in[i], outp[i], eig[i]);
      } else {
        si = PISCO_ERR_NOT_CONVERGED;
      }
    } else if ((h.flags & ST_UNCERTIFIED) && retry_iters(pl)) {
      // the split is not certified yet: redo this item alone with more subspace iterations
      batch_graph_reset(b);
      regroup = true;
      si = host_io ? pisco_estimate_host(pl, in[i], outp[i], eig[i]) : pisco_estimate(pl, in[i], outp[i], eig[i]);
    } else {
      pl->last_k = h.k;
      pl->last_R = pl->n - h.k;
      if (h.flags & ST_UNCERTIFIED) si = PISCO_ERR_NOT_CONVERGED;
      else if (h.flags & ST_RANK) si = PISCO_ERR_RANK;
    }
    if (item_status) item_status[i] = si;
    if (si != PISCO_OK && (worst == PISCO_OK || worst == PISCO_ERR_RANK)) worst = si;
  }
  if (regroup) {
    // a group runs with the largest block and iteration count any of its items needed
    for (int g = 0; g < (int)b->groups.size(); ++g) {
      pisco_plan_s* gp = b->groups[g];
      if (gp->items == 1) continue;
      for (int i : b->members[g]) {
        gp->m = std::max(gp->m, b->items[i]->m);
        gp->eig_iters = std::max(gp->eig_iters, b->items[i]->eig_iters);
      }
      for (int i : b->members[g]) {
        b->items[i]->m = gp->m;
        b->items[i]->eig_iters = gp->eig_iters;
      }
    }
  }
  return worst;
}

// workspace layout of pisco_tc_cgemm_pipelined: A' head, A' tail, B' head, B' tail, partials
static void tc2_ws_layout(int nterms, int M, int N, int K, int splits, size_t off[5], size_t* total) {
  const size_t k2 = (size_t)tc2_k2p(K), np2 = 2 * (size_t)tc2_np(N);
  const size_t a = (size_t)M * k2 * sizeof(float), b = np2 * k2 * sizeof(float);
  off[0] = 0;
  off[1] = off[0] + a;
  off[2] = off[1] + (nterms == 3 ? a : 0);
  off[3] = off[2] + b;
  off[4] = off[3] + (nterms == 3 ? b : 0);
  *total = off[4] + (splits > 1 ? (size_t)splits * M * N * sizeof(float2) : 0);
}

size_t pisco_tc_cgemm_pipelined_workspace(int nterms, int M, int N, int K, int splits) {
  if (M <= 0 || N <= 0 || K < 0) return 0;
  size_t off[5], tot;
  tc2_ws_layout(nterms, M, N, K, splits, off, &tot);
  return tot;
}

pisco_status pisco_tc_cgemm_pipelined(int nterms, int M, int N, int K, const float* alpha, const void* d_A, int lda,
                                      const void* d_B, int ldb, int opB, const float* beta, void* d_C, int ldc,
                                      int splits, void* d_workspace, size_t workspace_bytes, int* d_status,
                                      void* cuda_stream) {
  if (M < 0 || N < 0 || K < 0 || (nterms != 1 && nterms != 3) || (opB != 0 && opB != 1) || splits < 1) return PISCO_ERR_ARG;
  if (M == 0 || N == 0) return PISCO_OK;
  if (!d_C || !alpha || !beta || (K > 0 && (!d_A || !d_B)) || !d_workspace) return PISCO_ERR_ARG;
  if (lda < K || ldc < N || ldb < (opB == 0 ? N : K)) return PISCO_ERR_ARG;
  if ((((uintptr_t)d_A | (uintptr_t)d_B | (uintptr_t)d_C) & 7) || ((uintptr_t)d_workspace & 15)) return PISCO_ERR_ARG;
  size_t off[5], tot;
  tc2_ws_layout(nterms, M, N, K, splits, off, &tot);
  if (workspace_bytes < tot) return PISCO_ERR_ARG;
  if (tc2_prepare() != cudaSuccess) {
    cudaGetLastError();
    return PISCO_ERR_CUDA;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  unsigned char* w = static_cast<unsigned char*>(d_workspace);
  float* ah = reinterpret_cast<float*>(w + off[0]);
  float* al = nterms == 3 ? reinterpret_cast<float*>(w + off[1]) : nullptr;
  float* bh = reinterpret_cast<float*>(w + off[2]);
  float* bl = nterms == 3 ? reinterpret_cast<float*>(w + off[3]) : nullptr;
  float2* part = splits > 1 ? reinterpret_cast<float2*>(w + off[4]) : nullptr;
  if (K > 0 && (tc2_split_a((const float2*)d_A, lda, nullptr, M, K, ah, al, st) != cudaSuccess ||
                tc2_split_b((const float2*)d_B, ldb, opB, K, N, bh, bl, st) != cudaSuccess))
    return PISCO_ERR_CUDA;
  if (tc2_gemm(nterms, M, N, K, ah, al, bh, bl, make_float2(alpha[0], alpha[1]), make_float2(beta[0], beta[1]),
               (float2*)d_C, ldc, 0.f, 0, 0, splits, part, d_status, st) != cudaSuccess)
    return PISCO_ERR_CUDA;
  return PISCO_OK;
}

void pisco_test_stall_tensor_loads(int enable) { tc2_set_stall(enable != 0); }

pisco_status pisco_support_mask(const float* d_eig, long long n, float threshold, unsigned char* d_mask,
                                void* cuda_stream) {
  if (n < 0 || !(threshold == threshold)) return PISCO_ERR_ARG;
  if (n == 0) return PISCO_OK;
  if (!d_eig || !d_mask) return PISCO_ERR_ARG;
  return support_mask(d_eig, n, threshold, d_mask, (cudaStream_t)cuda_stream) == cudaSuccess ? PISCO_OK
                                                                                           : PISCO_ERR_CUDA;
}

pisco_status pisco_batch_estimate(pisco_batch_t b, const void* const* d_calib, void* const* d_maps,
                                  float* const* d_eig, pisco_status* item_status) {
  if (!b || !d_calib || !d_maps || b->pending) return PISCO_ERR_ARG;
  const pisco_status s = batch_launch(b, d_calib, d_maps, d_eig, false, true);
  if (s != PISCO_OK) return s;
  return batch_finish(b, item_status);
}

pisco_status pisco_batch_estimate_host(pisco_batch_t b, const void* const* h_calib, void* const* h_maps,
                                       float* const* h_eig, pisco_status* item_status) {
  if (!b || !h_calib || !h_maps || b->pending) return PISCO_ERR_ARG;
  const pisco_status s = batch_launch(b, h_calib, h_maps, h_eig, true, true);
  if (s != PISCO_OK) return s;
  return batch_finish(b, item_status);
}

pisco_status pisco_batch_launch_host(pisco_batch_t b, const void* const* h_calib, void* const* h_maps,
                                     float* const* h_eig) {
  if (!b || !h_calib || !h_maps || b->pending) return PISCO_ERR_ARG;
  return batch_launch(b, h_calib, h_maps, h_eig, true, false);
}

pisco_status pisco_batch_launch(pisco_batch_t b, const void* const* d_calib, void* const* d_maps,
                                float* const* d_eig) {
  if (!b || !d_calib || !d_maps || b->pending) return PISCO_ERR_ARG;
  return batch_launch(b, d_calib, d_maps, d_eig, false, true);
}

pisco_status pisco_batch_wait(pisco_batch_t b, pisco_status* item_status) {
  if (!b) return PISCO_ERR_ARG;
  return batch_finish(b, item_status);
}

pisco_status pisco_batch_info(pisco_batch_t b, int* count, int* launches, size_t* workspace_bytes) {
  if (!b) return PISCO_ERR_ARG;
  if (count) *count = (int)b->items.size();
  if (launches) *launches = b->launches;
  if (workspace_bytes) {
    size_t t = 0;
    for (auto* pl : b->groups) t += pl->ws_bytes;
    *workspace_bytes = t;
  }
  return PISCO_OK;
}

pisco_status pisco_batch_item(pisco_batch_t b, int i, pisco_plan_t* plan) {
  if (!b || !plan || i < 0 || i >= (int)b->items.size()) return PISCO_ERR_ARG;
  *plan = b->items[i];
  return PISCO_OK;
}

pisco_status pisco_batch_set_profiling(pisco_batch_t b, int enable) {
  if (!b || b->pending) return PISCO_ERR_ARG;
  b->prof = enable != 0;
  for (pisco_plan_s* gp : b->groups) gp->prof = b->prof;
  return PISCO_OK;
}

pisco_status pisco_batch_profile_reset(pisco_batch_t b) {
  if (!b) return PISCO_ERR_ARG;
  for (pisco_plan_s* gp : b->groups) pisco_profile_reset(gp);
  return PISCO_OK;
}

pisco_status pisco_batch_profile_entry(pisco_batch_t b, int idx, const char** name, double* total_ms, int* count) {
  if (!b || idx < 0) return PISCO_ERR_ARG;
  // the operation names of all groups in first-seen order, totals summed over the groups
  std::vector<const char*> names;
  for (pisco_plan_s* gp : b->groups)
    for (const char* nm : gp->prof_name) {
      bool seen = false;
      for (const char* x : names) seen = seen || strcmp(x, nm) == 0;
      if (!seen) names.push_back(nm);
    }
  if (idx >= (int)names.size()) return PISCO_ERR_ARG;
  double ms = 0.0;
  int cnt = 0;
  for (pisco_plan_s* gp : b->groups)
    for (size_t k = 0; k < gp->prof_name.size(); ++k)
      if (strcmp(gp->prof_name[k], names[idx]) == 0) {
        ms += gp->prof_ms[k];
        cnt += gp->prof_cnt[k];
      }
  if (name) *name = names[idx];
  if (total_ms) *total_ms = ms;
  if (count) *count = cnt;
  return PISCO_OK;
}

pisco_status pisco_batch_groups(pisco_batch_t b, int* groups, int* largest) {
  if (!b) return PISCO_ERR_ARG;
  int mx = 0;
  for (pisco_plan_s* gp : b->groups) mx = std::max(mx, gp->items);
  if (groups) *groups = (int)b->groups.size();
  if (largest) *largest = mx;
  return PISCO_OK;
}

}  // extern "C"
