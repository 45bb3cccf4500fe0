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
                                     double2* __restrict__ P, GramItems it) {
  S += blockIdx.z * it.S;
  P += blockIdx.z * it.P;
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

cudaError_t gram_pair_products(const double2* S, int Q, long long nfreq, double2* P, cudaStream_t st,
                               const GramItems& it) {
  const int npairs = Q * (Q + 1) / 2;
  int bx = (int)((nfreq + 255) / 256);
  if (bx > 64) bx = 64;
  pair_products_kernel<<<dim3(bx, npairs, it.n), 256, 0, st>>>(S, Q, nfreq, P, it);
  ++g_launches;
  return cudaGetLastError();
}

__global__ void scatter_pairs_kernel(const double2* __restrict__ Rp, int Q, int nbox,
                                     double2* __restrict__ lags, GramItems it) {
  Rp += blockIdx.y * it.Rp;
  lags += blockIdx.y * it.lags;
  const int pair = blockIdx.x;
  int p, q;
  pair_of(pair, Q, p, q);
  for (int t = threadIdx.x; t < nbox; t += blockDim.x)
    lags[((long long)p * Q + q) * nbox + t] = Rp[(long long)pair * nbox + t];
}

cudaError_t gram_scatter_pairs(const double2* Rpairs, int Q, int nbox, double2* lags, cudaStream_t st,
                               const GramItems& it) {
  scatter_pairs_kernel<<<dim3(Q * (Q + 1) / 2, it.n), 128, 0, st>>>(Rpairs, Q, nbox, lags, it);
  ++g_launches;
  return cudaGetLastError();
}

// scale = max_p R_pp[0] (the largest diagonal entry of C^H C); 1 if the data are all zero.
// The FP32 copy of the Gram is divided by it so that products of the iterated block stay in
// FP32 range whatever the data scale.
__global__ void gram_scale_kernel(const double2* __restrict__ lags, int Q, int nbox, int lag0,
                                  double* __restrict__ scale, GramItems it) {
  lags += blockIdx.x * it.lags;
  scale += blockIdx.x * it.scale;
  double mx = 0.0;
  for (int p = threadIdx.x; p < Q; p += 32) mx = fmax(mx, lags[((long long)p * Q + p) * nbox + lag0].x);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (threadIdx.x == 0) *scale = mx > 0.0 ? mx : 1.0;
}

cudaError_t gram_scale(const double2* lags, int Q, int nbox, int lag0, double* scale, cudaStream_t st,
                       const GramItems& it) {
  gram_scale_kernel<<<it.n, 32, 0, st>>>(lags, Q, nbox, lag0, scale, it);
  ++g_launches;
  return cudaGetLastError();
}

// A[(p,i),(q,j)] = R_pq[m_i - m_j] for p <= q, and the Hermitian mirror for p > q;
// A32 = A / scale in FP32.
__global__ void gram_expand_kernel(const double2* __restrict__ lags,
                                   const int* __restrict__ lag_of_ij, int Q, int L, int nbox,
                                   const double* __restrict__ scale,
                                   double2* __restrict__ A, float2* __restrict__ A32, GramItems it) {
  lags += blockIdx.y * it.lags;
  scale += blockIdx.y * it.scale;
  A += blockIdx.y * it.A;
  A32 += blockIdx.y * it.A;
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
                        const double* scale, double2* A, float2* A32, cudaStream_t st, const GramItems& it) {
  const long long n = (long long)Q * L;
  long long blocks = (n * n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  blocks = (blocks + it.n - 1) / it.n;
  gram_expand_kernel<<<dim3((unsigned)blocks, it.n), 256, 0, st>>>(lags, lag_of_ij, Q, L, nbox, scale, A, A32, it);
  ++g_launches;
  return cudaGetLastError();
}

}  // namespace pisco

namespace pisco {

// Exact Gram of the masked calibration matrix (only the rows n with n - Lambda inside the box,
// the matrix of Eq. C before Sec. V-A neglects the masking):
//   A[(p,i),(q,j)] = sum_{k in W_i} conj(s_p[k]) s_q[k + d],  d = m_i - m_j,
// where W_i (array coordinates) is the box [hi - m_i, Nc - 1 + lo - m_i] per axis, lo/hi the
// extremes of Lambda.  One CTA per (pair p <= q, lag d): the product image
// T[k] = conj(s_p[k]) s_q[k+d] (zero where k+d leaves the box) and its inclusive summed-area
// table in shared memory (FP64), then every entry of that lag is an inclusion-exclusion of 8
// table values.  For p == q only i <= j is computed and mirrored, so A is exactly Hermitian and
// every entry has one writer.
__global__ void __launch_bounds__(256) masked_gram_kernel(const float2* __restrict__ calib, int Q, int3 Nc,
                                                          int3 lo, int3 hi, const int* __restrict__ lam, int L,
                                                          const int* __restrict__ lag_ids,
                                                          const int* __restrict__ lagc_ptr,
                                                          const int* __restrict__ lag_ent, int3 tau2, int B1,
                                                          int B2, double2* __restrict__ A) {
  extern __shared__ double2 S[];
  const int l = blockIdx.x;
  int p, q;
  pair_of(blockIdx.y, Q, p, q);
  const int t = lag_ids[l];
  const int dz = t / (B1 * B2) - tau2.x, dy = (t / B2) % B1 - tau2.y, dx = t % B2 - tau2.z;
  const int nvol = Nc.x * Nc.y * Nc.z;
  const float2* sp = calib + (long long)p * nvol;
  const float2* sq = calib + (long long)q * nvol;
  for (int e = threadIdx.x; e < nvol; e += blockDim.x) {
    const int z = e / (Nc.y * Nc.z), y = (e / Nc.z) % Nc.y, x = e % Nc.z;
    const int z2 = z + dz, y2 = y + dy, x2 = x + dx;
    double2 v = make_double2(0.0, 0.0);
    if (z2 >= 0 && z2 < Nc.x && y2 >= 0 && y2 < Nc.y && x2 >= 0 && x2 < Nc.z) {
      const double2 a = to_z(sp[e]), b = to_z(sq[(z2 * Nc.y + y2) * Nc.z + x2]);
      cfmac(v, a, b);
    }
    S[e] = v;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < Nc.x * Nc.y; r += blockDim.x) {  // prefix along x
    double2* row = S + r * Nc.z;
    for (int x = 1; x < Nc.z; ++x) { row[x].x += row[x - 1].x; row[x].y += row[x - 1].y; }
  }
  __syncthreads();
  for (int r = threadIdx.x; r < Nc.x * Nc.z; r += blockDim.x) {  // along y
    const int z = r / Nc.z, x = r % Nc.z;
    double2* col = S + z * Nc.y * Nc.z + x;
    for (int y = 1; y < Nc.y; ++y) {
      col[y * Nc.z].x += col[(y - 1) * Nc.z].x;
      col[y * Nc.z].y += col[(y - 1) * Nc.z].y;
    }
  }
  __syncthreads();
  if (Nc.x > 1) {
    for (int r = threadIdx.x; r < Nc.y * Nc.z; r += blockDim.x) {  // along z
      double2* col = S + r;
      const int st = Nc.y * Nc.z;
      for (int z = 1; z < Nc.x; ++z) { col[z * st].x += col[(z - 1) * st].x; col[z * st].y += col[(z - 1) * st].y; }
    }
    __syncthreads();
  }
  const long long n = (long long)Q * L;
  auto sat = [&](int z, int y, int x) -> double2 {
    if (z < 0 || y < 0 || x < 0) return make_double2(0.0, 0.0);
    return S[(z * Nc.y + y) * Nc.z + x];
  };
  for (int e = lagc_ptr[l] + threadIdx.x; e < lagc_ptr[l + 1]; e += blockDim.x) {
    const int ent = lag_ent[e];
    const int i = ent / L, j = ent % L;
    if (p == q && i > j) continue;
    const int z0 = hi.x - lam[3 * i], y0 = hi.y - lam[3 * i + 1], x0 = hi.z - lam[3 * i + 2];
    const int z1 = Nc.x - 1 + lo.x - lam[3 * i], y1 = Nc.y - 1 + lo.y - lam[3 * i + 1], x1 = Nc.z - 1 + lo.z - lam[3 * i + 2];
    double2 s = make_double2(0.0, 0.0);
    if (z1 >= z0 && y1 >= y0 && x1 >= x0) {
      const int zz[2] = {z1, z0 - 1}, yy[2] = {y1, y0 - 1}, xx[2] = {x1, x0 - 1};
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const double2 v = sat(zz[c >> 2], yy[(c >> 1) & 1], xx[c & 1]);
        const double sg = (__popc(c) & 1) ? -1.0 : 1.0;
        s.x += sg * v.x;
        s.y += sg * v.y;
      }
    }
    A[((long long)p * L + i) * n + (long long)q * L + j] = s;
    if (!(p == q && i == j)) A[((long long)q * L + j) * n + (long long)p * L + i] = cconj(s);
  }
}

// scale = max_i Re A[i][i] (1 when not positive), A32 = A / scale
__global__ void gram_finish_scale_kernel(const double2* __restrict__ A, long long n, double* __restrict__ scale) {
  __shared__ double red[256];
  double m = 0.0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, A[i * n + i].x);
  red[threadIdx.x] = m;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *scale = red[0] > 0.0 ? red[0] : 1.0;
}

__global__ void gram_finish_a32_kernel(const double2* __restrict__ A, long long total, const double* __restrict__ scale,
                                       float2* __restrict__ A32) {
  const double inv = 1.0 / *scale;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x)
    A32[e] = make_float2((float)(A[e].x * inv), (float)(A[e].y * inv));
}

size_t gram_masked_smem(int nvol) { return sizeof(double2) * (size_t)nvol; }

cudaError_t gram_masked(const float2* calib, int Q, const int* Nc, const int* lo, const int* hi, const int* lam,
                        int L, const int* lag_ids, const int* lagc_ptr, const int* lag_ent, int nlag, const int* tau,
                        const int* B, double2* A, double* scale, float2* A32, cudaStream_t st) {
  const int nvol = Nc[0] * Nc[1] * Nc[2];
  const int npairs = Q * (Q + 1) / 2;
  masked_gram_kernel<<<dim3(nlag, npairs), 256, gram_masked_smem(nvol), st>>>(
      calib, Q, make_int3(Nc[0], Nc[1], Nc[2]), make_int3(lo[0], lo[1], lo[2]), make_int3(hi[0], hi[1], hi[2]), lam, L,
      lag_ids, lagc_ptr, lag_ent, make_int3(2 * tau[0], 2 * tau[1], 2 * tau[2]), B[1], B[2], A);
  const long long n = (long long)Q * L;
  gram_finish_scale_kernel<<<1, 256, 0, st>>>(A, n, scale);
  long long blocks = (n * n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  gram_finish_a32_kernel<<<(unsigned)blocks, 256, 0, st>>>(A, n * n, scale, A32);
  g_launches += 3;
  return cudaGetLastError();
}

cudaError_t gram_masked_prepare(int nvol) {
  // the attribute is per kernel, not per plan: always allow the largest supported tile
  (void)nvol;
  return cudaFuncSetAttribute(masked_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)gram_masked_smem(kMaskedMaxSamples));
}

}  // namespace pisco
