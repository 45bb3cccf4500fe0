// Stage (c): G(x) on the reduced grid without forming H(x) (Sec. V-C).
//
// With the nullspace projector W = sum_r h_r h_r^H = I - U U^H (U: orthonormal signal
// basis), Eq. 24 collapses to a per-pair lag kernel
//     G_pq(x) = |Lambda| delta_pq - sum_{d in Lambda-Lambda} K_pq[d] exp(+i 2 pi d^T x),
//     K_pq[d] = sum_{b - a = d} sum_j w_j U[(q,b),j] conj(U[(p,a),j]),
// i.e. the ESPIRiT form B(x) = I - G(x)/|Lambda| = H_s(x)^H H_s(x)/|Lambda| (Eq. esp_null).
// This file builds K (the dense complex contraction U_q diag(w) U_p^H folded onto lags); the
// host then evaluates the lag sums on the reduced grid with separable DFT passes.
#include "common.cuh"

namespace pisco {

namespace {
constexpr int JC = 32;  // signal columns staged per pass
}

// One CTA per (p,q).  U is [n][m] row-major (row = q*L + b).  K is [Q][Q][nbox].
// P[b][a] = sum_j w_j Uq[b][j] conj(Up[a][j]) is accumulated in shared memory over column
// chunks, then every lag sums its (b,a) entries in a fixed order (CSR lists lag_ptr/lag_ent),
// so the result is bitwise reproducible.
__global__ void __launch_bounds__(256) gkernel_kernel(const float2* __restrict__ U,
                                                      const float* __restrict__ w, int Q, int L,
                                                      int m, const int* __restrict__ lag_ptr,
                                                      const int* __restrict__ lag_ent, int nbox,
                                                      float2* __restrict__ K) {
  extern __shared__ float2 sm[];
  float2* Up = sm;              // L * JC
  float2* Uq = Up + L * JC;     // L * JC
  float2* P = Uq + L * JC;      // L * L
  const int p = blockIdx.x / Q, q = blockIdx.x % Q;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < L * L; e += nt) P[e] = make_float2(0.f, 0.f);
  for (int j0 = 0; j0 < m; j0 += JC) {
    const int jc = min(JC, m - j0);
    __syncthreads();
    for (int e = tid; e < L * JC; e += nt) {
      const int a = e / JC, j = e % JC;
      float2 up = make_float2(0.f, 0.f), uq = up;
      if (j < jc) {
        const float wj = w[j0 + j];
        up = U[(long long)(p * L + a) * m + j0 + j];
        const float2 t = U[(long long)(q * L + a) * m + j0 + j];
        uq = make_float2(t.x * wj, t.y * wj);
      }
      Up[e] = up;
      Uq[e] = uq;
    }
    __syncthreads();
    for (int e = tid; e < L * L; e += nt) {
      const int b = e / L, a = e % L;
      float2 acc = P[e];
      const float2* ub = Uq + b * JC;
      const float2* ua = Up + a * JC;
#pragma unroll 8
      for (int j = 0; j < JC; ++j) cfmac(acc, ua[j], ub[j]);
      P[e] = acc;
    }
  }
  __syncthreads();
  float2* out = K + (long long)(p * Q + q) * nbox;
  for (int t = tid; t < nbox; t += nt) {
    float2 acc = make_float2(0.f, 0.f);
    for (int e = lag_ptr[t]; e < lag_ptr[t + 1]; ++e) {
      const float2 v = P[lag_ent[e]];
      acc.x += v.x;
      acc.y += v.y;
    }
    out[t] = acc;
  }
}

cudaError_t gassembly_kernel(const float2* U, const float* w, int Q, int L, int m,
                             const int* lag_ptr, const int* lag_ent, int nbox, float2* K,
                             cudaStream_t st) {
  const size_t smem = (2 * (size_t)L * JC + (size_t)L * L) * sizeof(float2);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(gkernel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    attr_set = true;
  }
  gkernel_kernel<<<Q * Q, 256, smem, st>>>(U, w, Q, L, m, lag_ptr, lag_ent, nbox, K);
  ++g_launches;
  return cudaGetLastError();
}

// G <- |Lambda| I - G  (G holds sum_d K_pq[d] e^{i 2 pi d x} on entry), layout [npix][Q][Q].
__global__ void add_identity_kernel(float2* G, int Q, long long npix, float lam_size) {
  const long long total = (long long)Q * Q * npix;
  const int QQ = Q * Q;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int pq = (int)(idx % QQ);
    const int p = pq / Q, q = pq % Q;
    float2 v = G[idx];
    G[idx] = make_float2((p == q ? lam_size : 0.f) - v.x, -v.y);
  }
}

__global__ void scatter_box_kernel(const float2* __restrict__ KT, const int* __restrict__ box_lag, int QQ, int nbox,
                                   float2* __restrict__ K, long long sKT, long long sK) {
  KT += blockIdx.y * sKT;
  K += blockIdx.y * sK;
  const long long total = (long long)QQ * nbox;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int pq = (int)(e / nbox), t = (int)(e % nbox);
    const int l = box_lag[t];
    K[e] = l >= 0 ? KT[(long long)l * QQ + pq] : make_float2(0.f, 0.f);
  }
}

cudaError_t gassembly_scatter_box(const float2* KT, const int* box_lag, int QQ, int nbox, float2* K, cudaStream_t st,
                                  int items, long long sKT, long long sK) {
  long long blocks = ((long long)QQ * nbox + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  scatter_box_kernel<<<dim3((unsigned)blocks, items), 256, 0, st>>>(KT, box_lag, QQ, nbox, K, sKT, sK);
  ++g_launches;
  return cudaGetLastError();
}

cudaError_t gassembly_add_identity(float2* G, int Q, long long npix, float lam_size, cudaStream_t st) {
  long long blocks = ((long long)Q * Q * npix + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  add_identity_kernel<<<(unsigned)blocks, 256, 0, st>>>(G, Q, npix, lam_size);
  ++g_launches;
  return cudaGetLastError();
}

}  // namespace pisco

namespace pisco {

// Tensor-core route of stage (c): with P = U diag(w) U^H (n x n, row (q,b), column (p,a)) formed
// by a tensor-core GEMM, fold P onto the lags of Lambda - Lambda:
//     KT[l][p*Q + q] = sum_{(b,a): b - a = d_l} P[(q,b)][(p,a)],
// the entries of each lag summed in the fixed CSR order (bitwise reproducible).  KT is the
// K x N operand of the second GEMM, G[x][pq] = |Lambda| delta_pq - sum_l E[x][l] KT[l][pq].
// (3D: |Lambda| = 123, the L x L block is 121 KiB of shared memory.)
// One CTA per coil pair (p, q) (grid y: item): the L x L block P[(q, b)][(p, a)] is read with
// coalesced row loads into shared memory, then each lag's entries are summed in the CSR order.
__global__ void __launch_bounds__(128) collapse_lags_kernel(const float2* __restrict__ P, int n, int Q, int L,
                                                            const int* __restrict__ lagc_ptr,
                                                            const int* __restrict__ lag_ent, int nlag,
                                                            float2* __restrict__ KT, long long sP, long long sKT) {
  extern __shared__ float2 blk[];  // [L][L]
  P += blockIdx.y * sP;
  KT += blockIdx.y * sKT;
  const int QQ = Q * Q;
  const int pq = blockIdx.x;
  const int p = pq / Q, q = pq % Q;
  const float2* src = P + (long long)q * L * n + (long long)p * L;
  for (int e = threadIdx.x; e < L * L; e += blockDim.x) {
    const int b = e / L, a = e % L;
    blk[e] = src[(long long)b * n + a];
  }
  __syncthreads();
  for (int l = threadIdx.x; l < nlag; l += blockDim.x) {
    float2 acc = make_float2(0.f, 0.f);
    for (int e = lagc_ptr[l]; e < lagc_ptr[l + 1]; ++e) {
      const float2 v = blk[lag_ent[e]];
      acc.x += v.x;
      acc.y += v.y;
    }
    KT[(long long)l * QQ + pq] = acc;
  }
}

cudaError_t gassembly_collapse(const float2* P, int n, int Q, int L, const int* lagc_ptr,
                               const int* lag_ent, int nlag, float2* KT, cudaStream_t st, int items, long long sP,
                               long long sKT) {
  const size_t smem = (size_t)L * L * sizeof(float2);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(collapse_lags_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set = true;
  }
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  collapse_lags_kernel<<<dim3(Q * Q, items), 128, smem, st>>>(P, n, Q, L, lagc_ptr, lag_ent, nlag, KT, sP, sKT);
  ++g_launches;
  return cudaGetLastError();
}

}  // namespace pisco

namespace pisco {

// 2D G(x) from the collapsed lag kernel by two separable DFT passes (the zero-padded lag sums of
// Sec. V-C evaluated on the reduced grid).  With the lags of Lambda - Lambda sorted by their
// row b1, then column b2 (row r holds lags row_ptr[r] .. row_ptr[r+1]-1),
//     S_r(x2)       = sum_{l in row r} KT[l][pq] E2[x2][b2_l],
//     G[x1,x2][pq]  = |Lambda| delta_pq - sum_r E1[x1][r] S_r(x2),
// with E_a[j][t] = exp(+i 2 pi (t - 2 tau_a) (j - Nr_a/2)/Nr_a).  A CTA owns 32 consecutive pairs
// and 8*XPT columns x2: it stages the pairs' lag kernel, both exponential tables and the lag
// columns in shared memory with one coalesced sweep; each thread then keeps the row sums of its
// pair and XPT columns in registers, and a warp stores 32 consecutive pairs (256 B) of a pixel.
template <int NB, int XPT>
__global__ void __launch_bounds__(256) gfield_sep2_kernel(const float2* __restrict__ KT, int Q, int nlag,
                                                          const int* __restrict__ row_ptr,
                                                          const int* __restrict__ lag_b2,
                                                          const float2* __restrict__ E1, int Nr1,
                                                          const float2* __restrict__ E2, int B2, int Nr2,
                                                          float lam_size, float2* __restrict__ G, long long sKT,
                                                          long long sG) {
  extern __shared__ float2 sm[];
  KT += blockIdx.z * sKT;
  G += blockIdx.z * sG;
  float2* e1s = sm;                          // [Nr1][NB]
  float2* e2s = e1s + Nr1 * NB;              // [Nr2][B2]
  float2* ks = e2s + Nr2 * B2;               // [nlag][32]
  int* b2s = reinterpret_cast<int*>(ks + nlag * 32);  // [nlag]
  const int QQ = Q * Q;
  const int pq0 = blockIdx.x * 32;
  for (int i = threadIdx.x; i < Nr1 * NB; i += blockDim.x) e1s[i] = E1[i];
  for (int i = threadIdx.x; i < Nr2 * B2; i += blockDim.x) e2s[i] = E2[i];
  for (int i = threadIdx.x; i < nlag * 32; i += blockDim.x) {
    const int l = i >> 5, j = i & 31;
    ks[i] = pq0 + j < QQ ? KT[(long long)l * QQ + pq0 + j] : make_float2(0.f, 0.f);
  }
  for (int i = threadIdx.x; i < nlag; i += blockDim.x) b2s[i] = lag_b2[i];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int pq = pq0 + lane;
  const bool live = pq < QQ;
  const int x2b = (blockIdx.y * 8 + warp) * XPT;
  int x2c[XPT];
#pragma unroll
  for (int x = 0; x < XPT; ++x) x2c[x] = min(x2b + x, Nr2 - 1) * B2;
  float2 S[NB][XPT];
#pragma unroll
  for (int r = 0; r < NB; ++r) {
#pragma unroll
    for (int x = 0; x < XPT; ++x) S[r][x] = make_float2(0.f, 0.f);
    const int l1 = row_ptr[r + 1];
#pragma unroll 4
    for (int l = row_ptr[r]; l < l1; ++l) {
      const float2 k = ks[l * 32 + lane];
      const int b2 = b2s[l];
#pragma unroll
      for (int x = 0; x < XPT; ++x) {
        const float2 e = e2s[x2c[x] + b2];
        S[r][x].x = fmaf(k.x, e.x, fmaf(-k.y, e.y, S[r][x].x));
        S[r][x].y = fmaf(k.x, e.y, fmaf(k.y, e.x, S[r][x].y));
      }
    }
  }
  const float diag = (live && pq / Q == pq % Q) ? lam_size : 0.f;
  for (int x1 = 0; x1 < Nr1; ++x1) {
    float2 g[XPT];
#pragma unroll
    for (int x = 0; x < XPT; ++x) g[x] = make_float2(0.f, 0.f);
#pragma unroll
    for (int r = 0; r < NB; ++r) {
      const float2 e = e1s[x1 * NB + r];
#pragma unroll
      for (int x = 0; x < XPT; ++x) {
        g[x].x = fmaf(e.x, S[r][x].x, fmaf(-e.y, S[r][x].y, g[x].x));
        g[x].y = fmaf(e.x, S[r][x].y, fmaf(e.y, S[r][x].x, g[x].y));
      }
    }
#pragma unroll
    for (int x = 0; x < XPT; ++x) {
      const int x2 = x2b + x;
      if (live && x2 < Nr2) G[((long long)x1 * Nr2 + x2) * QQ + pq] = make_float2(diag - g[x].x, -g[x].y);
    }
  }
}

size_t gfield_sep2_smem(int nlag, int Nr1, int B1, int Nr2, int B2) {
  return ((size_t)Nr1 * B1 + (size_t)Nr2 * B2 + (size_t)nlag * 32) * sizeof(float2) + (size_t)nlag * sizeof(int);
}

namespace {
constexpr int kSepXPT = 2;
template <int NB>
cudaError_t launch_sep2(const float2* KT, int Q, int nlag, const int* row_ptr, const int* lag_b2, const float2* E1,
                        int Nr1, const float2* E2, int B2, int Nr2, float lam_size, float2* G, cudaStream_t st,
                        int items, long long sKT, long long sG) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(gfield_sep2_kernel<NB, kSepXPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         kGfieldSep2MaxSmem);
    attr_set = true;
  }
  const dim3 grid((unsigned)((Q * Q + 31) / 32), (unsigned)((Nr2 + 8 * kSepXPT - 1) / (8 * kSepXPT)), items);
  gfield_sep2_kernel<NB, kSepXPT><<<grid, 256, gfield_sep2_smem(nlag, Nr1, NB, Nr2, B2), st>>>(
      KT, Q, nlag, row_ptr, lag_b2, E1, Nr1, E2, B2, Nr2, lam_size, G, sKT, sG);
  ++g_launches;
  return cudaGetLastError();
}
}  // namespace

bool gassembly_field_sep2_supported(int nlag, int Nr1, int B1, int Nr2, int B2) {
  return (B1 == 5 || B1 == 9 || B1 == 13 || B1 == 17 || B1 == 21 || B1 == 25) &&
         gfield_sep2_smem(nlag, Nr1, B1, Nr2, B2) <= (size_t)kGfieldSep2MaxSmem;
}

cudaError_t gassembly_field_sep2(const float2* KT, int Q, int nlag, const int* row_ptr, const int* lag_b2,
                                 const float2* E1, int Nr1, int B1, const float2* E2, int B2, int Nr2,
                                 float lam_size, float2* G, cudaStream_t st, int items, long long sKT, long long sG) {
  switch (B1) {
    case 5: return launch_sep2<5>(KT, Q, nlag, row_ptr, lag_b2, E1, Nr1, E2, B2, Nr2, lam_size, G, st, items, sKT, sG);
    case 9: return launch_sep2<9>(KT, Q, nlag, row_ptr, lag_b2, E1, Nr1, E2, B2, Nr2, lam_size, G, st, items, sKT, sG);
    case 13: return launch_sep2<13>(KT, Q, nlag, row_ptr, lag_b2, E1, Nr1, E2, B2, Nr2, lam_size, G, st, items, sKT, sG);
    case 17: return launch_sep2<17>(KT, Q, nlag, row_ptr, lag_b2, E1, Nr1, E2, B2, Nr2, lam_size, G, st, items, sKT, sG);
    case 21: return launch_sep2<21>(KT, Q, nlag, row_ptr, lag_b2, E1, Nr1, E2, B2, Nr2, lam_size, G, st, items, sKT, sG);
    case 25: return launch_sep2<25>(KT, Q, nlag, row_ptr, lag_b2, E1, Nr1, E2, B2, Nr2, lam_size, G, st, items, sKT, sG);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pisco
