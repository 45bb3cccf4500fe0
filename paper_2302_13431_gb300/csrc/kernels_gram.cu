// Stage (a): the Gram C^H C of the calibration matrix without forming C (Sec. V-A).
//
// With the masking neglected, column i of C_p^H C_q is a shift of the single correlation
// s_q (*) s_p^*[-n]; equivalently (C^H C)[(p,i),(q,j)] = R_pq[m_i - m_j] with
// R_pq[d] = sum_k conj(s_p[k]) s_q[k+d].  The host orchestrates: zero-padded forward DFT of
// every channel (separable FP64 passes), the pair products here, inverse DFT evaluated only
// on the lag box |d| <= 2 tau (separable FP64 passes), then the expansion below.
#include "common.cuh"

namespace pisco {

__device__ __forceinline__ void pair_of(int pair, int Q, int& p, int& q) {
  // pairs enumerate (p,q) with p <= q in row-major order
  int base = 0;
  p = 0;
  while (pair >= base + (Q - p)) { base += Q - p; ++p; }
  q = p + (pair - base);
}

__global__ void pair_products_kernel(const double2* __restrict__ S, int Q, long long nfreq,
                                     double2* __restrict__ P) {
  const int pair = blockIdx.y;
  int p, q;
  pair_of(pair, Q, p, q);
  const double2* Sp = S + (long long)p * nfreq;
  const double2* Sq = S + (long long)q * nfreq;
  double2* out = P + (long long)pair * nfreq;
  for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < nfreq;
       f += (long long)gridDim.x * blockDim.x) {
    double2 acc = make_double2(0.0, 0.0);
    cfmac(acc, Sp[f], Sq[f]);
    out[f] = acc;
  }
}

cudaError_t gram_pair_products(const double2* S, int Q, long long nfreq, double2* P, cudaStream_t st) {
  const int npairs = Q * (Q + 1) / 2;
  int bx = (int)((nfreq + 255) / 256);
  if (bx > 64) bx = 64;
  pair_products_kernel<<<dim3(bx, npairs), 256, 0, st>>>(S, Q, nfreq, P);
  ++g_launches;
  return cudaGetLastError();
}

__global__ void scatter_pairs_kernel(const double2* __restrict__ Rp, int Q, int nbox,
                                     double2* __restrict__ lags) {
  const int pair = blockIdx.x;
  int p, q;
  pair_of(pair, Q, p, q);
  for (int t = threadIdx.x; t < nbox; t += blockDim.x)
    lags[((long long)p * Q + q) * nbox + t] = Rp[(long long)pair * nbox + t];
}

cudaError_t gram_scatter_pairs(const double2* Rpairs, int Q, int nbox, double2* lags, cudaStream_t st) {
  scatter_pairs_kernel<<<Q * (Q + 1) / 2, 128, 0, st>>>(Rpairs, Q, nbox, lags);
  ++g_launches;
  return cudaGetLastError();
}

// scale = max_p R_pp[0] (the largest diagonal entry of C^H C); 1 if the data are all zero.
// The FP32 copy of the Gram is divided by it so that products of the iterated block stay in
// FP32 range whatever the data scale.
__global__ void gram_scale_kernel(const double2* __restrict__ lags, int Q, int nbox, int lag0,
                                  double* __restrict__ scale) {
  double mx = 0.0;
  for (int p = threadIdx.x; p < Q; p += 32) mx = fmax(mx, lags[((long long)p * Q + p) * nbox + lag0].x);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (threadIdx.x == 0) *scale = mx > 0.0 ? mx : 1.0;
}

cudaError_t gram_scale(const double2* lags, int Q, int nbox, int lag0, double* scale, cudaStream_t st) {
  gram_scale_kernel<<<1, 32, 0, st>>>(lags, Q, nbox, lag0, scale);
  ++g_launches;
  return cudaGetLastError();
}

// A[(p,i),(q,j)] = R_pq[m_i - m_j] for p <= q, and the Hermitian mirror for p > q;
// A32 = A / scale in FP32.
__global__ void gram_expand_kernel(const double2* __restrict__ lags,
                                   const int* __restrict__ lag_of_ij, int Q, int L, int nbox,
                                   const double* __restrict__ scale,
                                   double2* __restrict__ A, float2* __restrict__ A32) {
  const long long n = (long long)Q * L;
  const double inv = 1.0 / *scale;
  const long long total = n * n;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int col = (int)(idx % n);
    const int row = (int)(idx / n);
    const int p = row / L, i = row % L;
    const int q = col / L, j = col % L;
    double2 v;
    if (p <= q) {
      v = lags[((long long)p * Q + q) * nbox + lag_of_ij[i * L + j]];
    } else {
      v = cconj(lags[((long long)q * Q + p) * nbox + lag_of_ij[j * L + i]]);
    }
    A[idx] = v;
    A32[idx] = make_float2((float)(v.x * inv), (float)(v.y * inv));
  }
}

cudaError_t gram_expand(const double2* lags, const int* lag_of_ij, int Q, int L, int nbox,
                        const double* scale, double2* A, float2* A32, cudaStream_t st) {
  const long long n = (long long)Q * L;
  long long blocks = (n * n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  gram_expand_kernel<<<(unsigned)blocks, 256, 0, st>>>(lags, lag_of_ij, Q, L, nbox, scale, A, A32);
  ++g_launches;
  return cudaGetLastError();
}

}  // namespace pisco
