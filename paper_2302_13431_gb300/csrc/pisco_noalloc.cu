// Allocation-free entry point for the Gram lag table (stage (a)).
//
// Some callers cannot allocate device memory at the point where they need this result: code
// running under a custom or fixed-budget allocator that forbids cudaMalloc/cudaFree on its hot
// path, pipelines that must not synchronise the device (cudaFree does), and embedded
// runtimes that receive pre-sized buffers from their host.  pisco_gram_lags_noalloc serves
// them: it takes the caller's input and output buffers and keeps every intermediate in one
// fixed-size scratch array that is part of this library's device image, so it calls no
// cudaMalloc, cudaFree or allocating library routine.
//
// The scratch array is shared by every call in the process on a given GPU and keeps whatever
// the last call left in it; every intermediate is fully rewritten before it is read, and the
// output's p > q half is cleared explicitly.  Two calls that overlap on the GPU (different
// streams, or different host threads) race on the scratch and give undefined results.
#include <math.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"

using namespace pisco;

namespace {

// 32 MiB of complex128 scratch; every GPU that loads this library holds it until exit.
constexpr size_t kScratchElems = (size_t)32 * 1024 * 1024 / sizeof(double2);
static __device__ __align__(256) double2 g_noalloc_scratch[kScratchElems];

// Device address of g_noalloc_scratch for each device, resolved once per device with that
// device current (host code must not hand the host-side symbol to a kernel).
constexpr int kMaxDevices = 64;
double2* g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

double2* scratch_for_current_device(pisco_status* err) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    *err = PISCO_ERR_CUDA;
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      *err = PISCO_ERR_CUDA;
      return nullptr;
    }
    g_scratch_ptr[dev] = static_cast<double2*>(p);
  }
  return g_scratch_ptr[dev];
}

// forward DFT of length Lp on the array index n: M[f][n] = exp(-i 2 pi f n / Lp)
// inverse DFT at lags d = -2tau..2tau:          M[d][f] = exp(+i 2 pi f d / Lp) / Lp
__global__ void dft_tables_kernel(double2* fwd, int Lp, int Nc, double2* inv, int tau) {
  const int Bn = 4 * tau + 1;
  const int nf = Lp * Nc, ni = Bn * Lp;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nf + ni; e += gridDim.x * blockDim.x) {
    if (e < nf) {
      const int f = e / Nc, n = e % Nc;
      const long long ph = ((long long)f * n) % Lp;
      double s, c;
      sincospi(-2.0 * (double)ph / Lp, &s, &c);
      fwd[e] = make_double2(c, s);
    } else {
      const int t = (e - nf) / Lp, f = (e - nf) % Lp;
      long long ph = ((long long)f * (t - 2 * tau)) % Lp;
      if (ph < 0) ph += Lp;
      double s, c;
      sincospi(2.0 * (double)ph / Lp, &s, &c);
      inv[e - nf] = make_double2(c / Lp, s / Lp);
    }
  }
}

__global__ void zero_lower_pairs_kernel(double2* lags, int Q, int nbox) {
  const long long total = (long long)Q * Q * nbox;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long pq = idx / nbox;
    const int p = (int)(pq / Q), q = (int)(pq % Q);
    if (p > q) lags[idx] = make_double2(0.0, 0.0);
  }
}

bool basic_params_ok(const pisco_params* p) {
  if (!p || (p->ndim != 2 && p->ndim != 3)) return false;
  if (p->num_coils < 2 || p->num_coils > 64) return false;
  for (int d = 0; d < 3; ++d) {
    const int Nc = p->calib[d], t = p->kernel_radius[d];
    if (d >= p->ndim) {
      if (Nc != 1 || t != 0) return false;
      continue;
    }
    if (Nc < 1 || t < 0 || t > 16 || Nc <= 2 * t) return false;
  }
  return true;
}

}  // namespace

extern "C" pisco_status pisco_gram_lags_noalloc(const pisco_params* p, const void* d_calib,
                                                void* d_lags, void* cuda_stream) {
  if (!basic_params_ok(p) || !d_calib || !d_lags) return PISCO_ERR_ARG;
  if (((uintptr_t)d_calib & 7) || ((uintptr_t)d_lags & 15)) return PISCO_ERR_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int Q = p->num_coils, np = Q * (Q + 1) / 2;
  int Nc[3], Lp[3], B[3], tau[3];
  for (int d = 0; d < 3; ++d) {  // params are x,y,z; internal z,y,x
    Nc[2 - d] = p->calib[d];
    tau[2 - d] = p->kernel_radius[d];
  }
  for (int d = 0; d < 3; ++d) {
    Lp[d] = Nc[d] + 2 * tau[d];
    B[d] = 4 * tau[d] + 1;
  }
  const long long nfreq = (long long)Lp[0] * Lp[1] * Lp[2];
  const int nbox = B[0] * B[1] * B[2];
  // scratch layout (complex128 elements)
  size_t off[3][2], o = 0;
  for (int d = 0; d < 3; ++d) {
    off[d][0] = o; o += (size_t)Lp[d] * Nc[d];
    off[d][1] = o; o += (size_t)B[d] * Lp[d];
  }
  const size_t gA_n = (size_t)std::max((long long)Q * Nc[0] * Nc[1] * Lp[2], (long long)np * Lp[0] * Lp[1] * B[2]);
  const size_t gB_n = (size_t)std::max((long long)Q * Nc[0] * Lp[1] * Lp[2], (long long)np * Lp[0] * B[1] * B[2]);
  const size_t gA_o = o; o += gA_n;
  const size_t gB_o = o; o += gB_n;
  const size_t S_o = o; o += (p->ndim == 3) ? (size_t)Q * nfreq : 0;
  const size_t P_o = o; o += (size_t)np * nfreq;
  const size_t Rp_o = o; o += (size_t)np * nbox;
  if (o > kScratchElems) return PISCO_ERR_TOO_LARGE;
  pisco_status err = PISCO_OK;
  double2* sc = scratch_for_current_device(&err);
  if (!sc) return err;
  for (int d = 0; d < 3; ++d) {
    const int tot = Lp[d] * Nc[d] + B[d] * Lp[d];
    dft_tables_kernel<<<(tot + 255) / 256, 256, 0, st>>>(sc + off[d][0], Lp[d], Nc[d], sc + off[d][1], tau[d]);
  }
  if (cudaGetLastError() != cudaSuccess) return PISCO_ERR_CUDA;
  const float2* calib = static_cast<const float2*>(d_calib);
  double2 *gA = sc + gA_o, *gB = sc + gB_o, *S = sc + S_o, *P = sc + P_o, *Rp = sc + Rp_o;
  const double2* fwd[3] = {sc + off[0][0], sc + off[1][0], sc + off[2][0]};
  const double2* inv[3] = {sc + off[0][1], sc + off[1][1], sc + off[2][1]};
#define NA_CK(x) do { if ((x) != cudaSuccess) return PISCO_ERR_CUDA; } while (0)
  NA_CK(apply_axis_c2z(calib, fwd[2], gA, AxisView{Q, (long long)Nc[0] * Nc[1], Nc[2], Lp[2], 1}, st));
  NA_CK(apply_axis_z(gA, fwd[1], gB, AxisView{Q, Nc[0], Nc[1], Lp[1], Lp[2]}, st));
  const double2* Sp = gB;
  if (p->ndim == 3) {
    NA_CK(apply_axis_z(gB, fwd[0], S, AxisView{Q, 1, Nc[0], Lp[0], (long long)Lp[1] * Lp[2]}, st));
    Sp = S;
  }
  NA_CK(gram_pair_products(Sp, Q, nfreq, P, st));
  NA_CK(apply_axis_z(P, inv[2], gA, AxisView{np, (long long)Lp[0] * Lp[1], Lp[2], B[2], 1}, st));
  if (p->ndim == 3) {
    NA_CK(apply_axis_z(gA, inv[1], gB, AxisView{np, Lp[0], Lp[1], B[1], B[2]}, st));
    NA_CK(apply_axis_z(gB, inv[0], Rp, AxisView{np, 1, Lp[0], B[0], (long long)B[1] * B[2]}, st));
  } else {
    NA_CK(apply_axis_z(gA, inv[1], Rp, AxisView{np, 1, Lp[1], B[1], B[2]}, st));
  }
  double2* lags = static_cast<double2*>(d_lags);
  NA_CK(gram_scatter_pairs(Rp, Q, nbox, lags, st));
  const long long tot = (long long)Q * Q * nbox;
  zero_lower_pairs_kernel<<<(unsigned)std::min<long long>((tot + 255) / 256, 1024), 256, 0, st>>>(lags, Q, nbox);
  NA_CK(cudaGetLastError());
#undef NA_CK
  return PISCO_OK;
}
