// Stage (b): the approximate nullspace of C^H C (Sec. III-A) with the threshold rule
// sigma_n < thr*sigma_1 of the Sec. III-B footnote, i.e. lambda_n < thr^2 lambda_1 on the
// Gram.  The signal dimension k = n - R is small (tens) next to n = Q|Lambda| (hundreds to
// thousands), so instead of a dense O(n^3) eigensolver this uses block subspace iteration
// with Rayleigh-Ritz on an m-column block (m >= k plus a guard band):
//   - the iteration runs in FP32 (Gram rounded to FP32), CholQR2 re-orthonormalisation of
//     the Ritz-scaled block, Rayleigh-Ritz by a one-CTA parallel cyclic Jacobi;
//   - the Ritz vectors whose FP32 Ritz values lie near the threshold, and the top one that
//     fixes lambda_1, get FP64 Rayleigh quotients against the FP64 Gram; the threshold split
//     is decided on those FP64 values.
// The small dense kernels here run in one CTA (m <= 128); the large products go through the
// split-K GEMM.
#include <math.h>

#include "common.cuh"

namespace pisco {

// ---------------------------------------------------------------------------------------
// start block: counter-based uniforms (rows = filter coefficients, columns = vectors)
// ---------------------------------------------------------------------------------------
__global__ void random_block_kernel(float2* X, int n, int m, unsigned long long seed) {
  const long long total = (long long)n * m;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(idx / m), c = (int)(idx % m);
    X[idx] = make_float2(counter_uniform(seed, (uint64_t)r, 2 * c),
                         counter_uniform(seed, (uint64_t)r, 2 * c + 1));
  }
}

cudaError_t eig_random_block(float2* X, int n, int m, unsigned long long seed, cudaStream_t st) {
  long long blocks = ((long long)n * m + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  random_block_kernel<<<(unsigned)blocks, 256, 0, st>>>(X, n, m, seed ^ 0x5EEDB10Cull);
  ++g_launches;
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Cholesky-QR pieces.
// chol_kernel (1 CTA, m <= 128): factor the Gram G = Y^H Y of an n x m block,
//   - optional column scaling D = diag(dscale) (floored at 1e-6 * max, clamped to
//     [1e-18, 1e18]): G <- D^-1 G D^-1, i.e. the block Y D^-1 is factored (the rescaling of
//     orthogonal iteration by the previous diag(R), which keeps Cholesky-QR well conditioned);
//   - optional diagonal shift s*trace(G) (shifted Cholesky-QR for an ill-conditioned block,
//     Fukaya et al. 2020);
//   - right-looking Cholesky G = L L^H in shared memory, 2D thread map, pivots below
//     1e-12 * max diag clamped (status ST_CHOL);
//   - writes Lout (lower, with the column scaling folded in: Lout = D L so that
//     Y = X (D L)^H... see trsm) and diagR[j] = L_jj * d_j * (acc ? acc[j] : 1).
// trsm_rows_kernel: X = (Y D^-1) L^-H row by row, one thread per row (x L^H = y D^-1 by
// forward substitution, the row in registers, L broadcast from shared memory).
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) chol_kernel(const float2* __restrict__ Gm, int m,
                                                   const float* __restrict__ dscale,
                                                   float shift_rel,
                                                   const float* __restrict__ acc_in,
                                                   float2* __restrict__ Lout,
                                                   float* __restrict__ dout,
                                                   float* __restrict__ diagR,
                                                   DevStatus* status, EigItems it) {
  extern __shared__ float2 sm[];
  {
    const int i = blockIdx.z;
    Gm += i * it.mm;
    if (dscale) dscale += i * it.vec;
    if (acc_in) acc_in += i * it.vec;
    Lout += i * it.mm;
    dout += i * it.vec;
    diagR += i * it.vec;
    if (status) status += i;
  }
  float2* Lm = sm;                                   // m*m
  float* ds = reinterpret_cast<float*>(Lm + m * m);  // m (scaling)
  float* dg = ds + m;                                // m (pivots)
  __shared__ float s_floor, s_shift;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int tx = tid & 15, ty = tid >> 4;            // 16 x 16 map
  if (warp == 0) {
    float mx = 0.f;
    if (dscale)
      for (int i = lane; i < m; i += 32) mx = fmaxf(mx, fabsf(dscale[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) s_floor = mx;
  }
  __syncthreads();
  for (int i = tid; i < m; i += nt) {
    float d = 1.f;
    if (dscale) d = fminf(fmaxf(fmaxf(fabsf(dscale[i]), 1e-6f * s_floor), 1e-18f), 1e18f);
    if (!(d > 0.f) || !(d < 1e30f)) d = 1.f;
    ds[i] = d;
  }
  __syncthreads();
  for (int e = tid; e < m * m; e += nt) {
    const int i = e / m, j = e % m;
    const float2 g = Gm[e];
    const float sc = 1.f / (ds[i] * ds[j]);
    Lm[e] = make_float2(g.x * sc, g.y * sc);
  }
  __syncthreads();
  if (warp == 0) {
    float md = 0.f, tr = 0.f;
    for (int i = lane; i < m; i += 32) { md = fmaxf(md, Lm[i * m + i].x); tr += Lm[i * m + i].x; }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      md = fmaxf(md, __shfl_xor_sync(0xffffffffu, md, o));
      tr += __shfl_xor_sync(0xffffffffu, tr, o);
    }
    if (lane == 0) {
      s_shift = shift_rel * tr;
      s_floor = (md + s_shift > 1e-30f) ? (md + s_shift) * 1e-12f : 1.0f;  // zero Gram: factor as I
    }
  }
  __syncthreads();
  const float floor_piv = s_floor, shift = s_shift;
  for (int j = 0; j < m; ++j) {
    const float d = Lm[j * m + j].x + shift;
    const float piv = sqrtf(d > floor_piv ? d : floor_piv);
    const float inv = 1.0f / piv;
    for (int i = j + 1 + tid; i < m; i += nt) {
      const float2 v = Lm[i * m + j];
      Lm[i * m + j] = make_float2(v.x * inv, v.y * inv);
    }
    if (tid == 0) {
      dg[j] = piv;
      if (!(d > floor_piv) && status) atomicOr(&status->flags, (int)ST_CHOL);
    }
    __syncthreads();
    for (int i = j + 1 + ty; i < m; i += 16) {
      const float2 a = Lm[i * m + j];
      for (int k = j + 1 + tx; k <= i; k += 16) {
        const float2 b = Lm[k * m + j];
        float2 g = Lm[i * m + k];
        g.x -= a.x * b.x + a.y * b.y;
        g.y -= a.y * b.x - a.x * b.y;
        Lm[i * m + k] = g;
      }
    }
    __syncthreads();
  }
  for (int i = tid; i < m; i += nt) {
    diagR[i] = dg[i] * ds[i] * (acc_in ? acc_in[i] : 1.f);
    dout[i] = ds[i];
  }
  for (int e = tid; e < m * m; e += nt) {
    const int i = e / m, k = e % m;
    Lout[e] = (k < i) ? Lm[e] : (k == i ? make_float2(dg[i], 0.f) : make_float2(0.f, 0.f));
  }
}

// Blocked Cholesky-QR factor for m <= 96 (1 CTA, 256 threads, 16 x 16 blocks): the same
// inputs and scaling/shift/floor rules as chol_kernel, but the result is the explicit
// Rinv = D^-1 L^-H (upper triangular, m x m) so that X = Y * Rinv is a plain GEMM.
//   - each diagonal block is factored and inverted by warp 0 in registers (row per lane);
//   - panels L_IJ = A_IJ Linv_JJ^H and trailing updates A_IK -= L_IJ L_KJ^H are 16x16x16
//     block products over all threads;
//   - off-diagonal blocks of L^-1 follow by block diagonals:
//     Linv_IJ = -Linv_II * sum_{K=J}^{I-1} L_IK Linv_KJ.
// About 3 barriers per block column instead of 2 per column.
constexpr int CB = 16;
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // a * conj(b)
  return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

__global__ void __launch_bounds__(256) chol_inv_blocked_kernel(const float2* __restrict__ Gm, int m,
                                                               const float* __restrict__ dscale,
                                                               float shift_rel,
                                                               const float* __restrict__ acc_in,
                                                               float2* __restrict__ Rinv,
                                                               float* __restrict__ diagR,
                                                               DevStatus* status, EigItems it) {
  extern __shared__ float2 sm[];
  {
    const int i = blockIdx.z;
    Gm += i * it.mm;
    if (dscale) dscale += i * it.vec;
    if (acc_in) acc_in += i * it.vec;
    Rinv += i * it.mm;
    diagR += i * it.vec;
    if (status) status += i;
  }
  const int NB = (m + CB - 1) / CB, M = NB * CB;
  float2* A = sm;                                    // M*M, L in the lower triangle
  float2* Li = A + M * M;                            // M*M, L^-1 (lower)
  float* ds = reinterpret_cast<float*>(Li + M * M);  // M scaling
  float* piv_s = ds + M;                             // M pivots
  __shared__ float s_mx, s_shift, s_floor;
  __shared__ int s_clamp;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ei = tid >> 4, ej = tid & 15;            // element of a 16x16 block owned by this thread
  const int pr = tid >> 2, pc = (tid & 3) * 4;       // panel: row pr (0..63), columns pc..pc+3
  if (warp == 0) {
    float mx = 0.f;
    if (dscale)
      for (int i = lane; i < m; i += 32) mx = fmaxf(mx, fabsf(dscale[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) { s_mx = mx; s_clamp = 0; }
  }
  __syncthreads();
  for (int i = tid; i < M; i += 256) {
    float d = 1.f;
    if (dscale && i < m) d = fminf(fmaxf(fmaxf(fabsf(dscale[i]), 1e-6f * s_mx), 1e-18f), 1e18f);
    if (!(d > 0.f) || !(d < 1e30f)) d = 1.f;
    ds[i] = d;
  }
  __syncthreads();
  for (int r = tid >> 4; r < M; r += 16) {
    for (int c = tid & 15; c < M; c += 16) {
      float2 v = make_float2(0.f, 0.f);
      if (r < m && c < m) {
        const float2 g = Gm[r * m + c];
        const float sc = 1.f / (ds[r] * ds[c]);
        v = make_float2(g.x * sc, g.y * sc);
      } else if (r == c) {
        v = make_float2(1.f, 0.f);
      }
      A[r * M + c] = v;
      Li[r * M + c] = make_float2(0.f, 0.f);
    }
  }
  __syncthreads();
  if (warp == 0) {
    float md = 0.f, tr = 0.f;
    for (int i = lane; i < m; i += 32) { md = fmaxf(md, A[i * M + i].x); tr += A[i * M + i].x; }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      md = fmaxf(md, __shfl_xor_sync(0xffffffffu, md, o));
      tr += __shfl_xor_sync(0xffffffffu, tr, o);
    }
    if (lane == 0) {
      s_shift = shift_rel * tr;
      s_floor = (md + s_shift > 1e-30f) ? (md + s_shift) * 1e-12f : 1.0f;  // zero Gram: factor as I
    }
  }
  __syncthreads();
  for (int i = tid; i < m; i += 256) A[i * M + i].x += s_shift;
  __syncthreads();
  const float floor_piv = s_floor;
  for (int J = 0; J < NB; ++J) {
    const int j0 = J * CB;
    // (a) panel factorisation of rows j0..M-1, columns j0..j0+15: thread (pr, pc) keeps 4
    //     entries in registers; one barrier per pivot (the pivot row publishes its column)
    const int row = j0 + pr;
    const bool own = row < M;
    float2 a[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) a[t] = own ? A[row * M + j0 + pc + t] : make_float2(0.f, 0.f);
    for (int j = 0; j < CB; ++j) {
      // publish the current column j of the panel, then every thread reads the pivot and the
      // entries of column j it needs from shared memory (one barrier per pivot)
      const bool owns_j = own && ((j >> 2) == (pc >> 2));
      if (owns_j) A[row * M + j0 + j] = a[j & 3];
      __syncthreads();
      const float dj = A[(j0 + j) * M + j0 + j].x;
      const bool clamp = !(dj > floor_piv);
      const float piv = sqrtf(clamp ? floor_piv : dj);
      const float inv = 1.f / piv;
      if (tid == 0) { piv_s[j0 + j] = piv; if (clamp) s_clamp = 1; }
      if (own && pr >= j) {
        const float2 ar = A[row * M + j0 + j];
        const float2 lrj = make_float2(ar.x * inv, ar.y * inv);  // L[row][j0+j]
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int c = pc + t;
          if (c > j && c <= pr) {
            const float2 ac = A[(j0 + c) * M + j0 + j];
            const float2 lcj = make_float2(ac.x * inv, ac.y * inv);  // L[j0+c][j0+j]
            const float2 pp = cmulc(lrj, lcj);
            a[t].x -= pp.x; a[t].y -= pp.y;
          }
        }
        if (owns_j) a[j & 3] = (pr > j) ? lrj : make_float2(piv, 0.f);
      }
    }
    __syncthreads();
    if (own) {
#pragma unroll
      for (int t = 0; t < 4; ++t)
        if (pc + t <= pr) A[row * M + j0 + pc + t] = a[t];
    }
    __syncthreads();
    // (b) trailing update A_IK -= L_IJ L_KJ^H for J < K <= I
    for (int I = J + 1; I < NB; ++I)
      for (int K = J + 1; K <= I; ++K) {
        const int i = I * CB + ei, k = K * CB + ej;
        if (K == I && ej > ei) continue;
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int t = 0; t < CB; ++t) {
          const float2 p = cmulc(A[i * M + j0 + t], A[k * M + j0 + t]);
          acc.x += p.x; acc.y += p.y;
        }
        const float2 g = A[i * M + k];
        A[i * M + k] = make_float2(g.x - acc.x, g.y - acc.y);
      }
    __syncthreads();
  }
  // (c) inverses of all diagonal blocks at once: warp J inverts block J (lane c < 16: column c)
  if (warp < NB && lane < CB) {
    const int j0 = warp * CB, c = lane;
    float2 x[CB];
#pragma unroll
    for (int r = 0; r < CB; ++r) {
      float2 acc = make_float2(r == c ? 1.f : 0.f, 0.f);
#pragma unroll
      for (int k = 0; k < r; ++k) {
        const float2 l = A[(j0 + r) * M + j0 + k];
        acc.x -= l.x * x[k].x - l.y * x[k].y;
        acc.y -= l.x * x[k].y + l.y * x[k].x;
      }
      const float di = 1.f / A[(j0 + r) * M + j0 + r].x;
      x[r] = (r >= c) ? make_float2(acc.x * di, acc.y * di) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int r = 0; r < CB; ++r) Li[(j0 + r) * M + j0 + c] = x[r];
  }
  __syncthreads();
  // (d) off-diagonal blocks of L^-1 by block diagonals:
  //   T_IJ = sum_{K=J}^{I-1} L_IK Linv_KJ (staged in Li's (I,J) block), Linv_IJ = -Linv_II T_IJ
  for (int d = 1; d < NB; ++d) {
    float2 res[6];
#pragma unroll
    for (int u = 0; u < 6; ++u) {
      const int I = d + u;
      if (I >= NB) break;
      const int J = I - d;
      const int i = I * CB + ei, j = J * CB + ej;
      float2 acc = make_float2(0.f, 0.f);
      for (int K = J; K < I; ++K) {
#pragma unroll
        for (int t = 0; t < CB; ++t) {
          const float2 l = A[i * M + K * CB + t];
          const float2 xx = Li[(K * CB + t) * M + j];
          acc.x += l.x * xx.x - l.y * xx.y;
          acc.y += l.x * xx.y + l.y * xx.x;
        }
      }
      res[u] = acc;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 6; ++u) {
      const int I = d + u;
      if (I >= NB) break;
      Li[(I * CB + ei) * M + (I - d) * CB + ej] = res[u];
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 6; ++u) {
      const int I = d + u;
      if (I >= NB) break;
      const int J = I - d;
      const int i = I * CB + ei, j = J * CB + ej;
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int t = 0; t < CB; ++t) {
        const float2 l = Li[i * M + I * CB + t];
        const float2 xx = Li[(I * CB + t) * M + j];
        acc.x -= l.x * xx.x - l.y * xx.y;
        acc.y -= l.x * xx.y + l.y * xx.x;
      }
      res[u] = acc;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 6; ++u) {
      const int I = d + u;
      if (I >= NB) break;
      Li[(I * CB + ei) * M + (I - d) * CB + ej] = res[u];
    }
    __syncthreads();
  }
  for (int i = tid; i < m; i += 256) diagR[i] = piv_s[i] * ds[i] * (acc_in ? acc_in[i] : 1.f);
  for (int r = tid >> 4; r < m; r += 16)
    for (int c = tid & 15; c < m; c += 16) {
      const float2 v = Li[c * M + r];
      const float id = 1.f / ds[r];
      Rinv[r * m + c] = make_float2(v.x * id, -v.y * id);
    }
  if (tid == 0 && s_clamp && status) atomicOr(&status->flags, (int)ST_CHOL);
}

// One thread per row r: x L^H = y with y = Y[r] D^-1, i.e. for c = 0..m-1
//   x_c = (y_c - sum_{k<c} x_k conj(L[c][k])) / L[c][c].
template <int MP>
__global__ void __launch_bounds__(128) trsm_rows_kernel(const float2* __restrict__ Y,
                                                        const float2* __restrict__ Lg,
                                                        const float* __restrict__ ds, int n, int m,
                                                        float2* __restrict__ X, EigItems it) {
  extern __shared__ float2 sm[];
  Y += blockIdx.y * it.nm;
  Lg += blockIdx.y * it.mm;
  ds += blockIdx.y * it.vec;
  X += blockIdx.y * it.nm;
  float2* Ls = sm;                                       // m*m
  float* dinv = reinterpret_cast<float*>(Ls + m * m);    // m
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) Ls[e] = Lg[e];
  for (int e = threadIdx.x; e < m; e += blockDim.x) dinv[e] = 1.0f / ds[e];
  __syncthreads();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const float2* y = Y + (long long)r * m;
  float2 x[MP];
#pragma unroll
  for (int c = 0; c < MP; ++c) {
    if (c < m) {
      const float2 yc = y[c];
      float ar = yc.x * dinv[c], ai = yc.y * dinv[c];
#pragma unroll
      for (int k = 0; k < c; ++k) {
        const float2 l = Ls[c * m + k];  // x_k conj(l)
        ar -= x[k].x * l.x + x[k].y * l.y;
        ai -= x[k].y * l.x - x[k].x * l.y;
      }
      const float di = 1.0f / Ls[c * m + c].x;
      x[c] = make_float2(ar * di, ai * di);
    } else {
      x[c] = make_float2(0.f, 0.f);
    }
  }
#pragma unroll
  for (int c = 0; c < MP; ++c)
    if (c < m) X[(long long)r * m + c] = x[c];
}

// warp-per-row fallback for m > 64: lanes split the k sum, the row lives in registers
__global__ void __launch_bounds__(256) trsm_rows_warp_kernel(const float2* __restrict__ Y,
                                                             const float2* __restrict__ Lg,
                                                             const float* __restrict__ ds, int n,
                                                             int m, float2* __restrict__ X, EigItems it) {
  extern __shared__ float2 sm[];
  Y += blockIdx.y * it.nm;
  Lg += blockIdx.y * it.mm;
  ds += blockIdx.y * it.vec;
  X += blockIdx.y * it.nm;
  float2* Ls = sm;
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) Ls[e] = Lg[e];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int warps = blockDim.x >> 5;
  for (int r = blockIdx.x * warps + (threadIdx.x >> 5); r < n; r += gridDim.x * warps) {
    const float2* y = Y + (long long)r * m;
    float2 xs[4], ys[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      xs[s] = make_float2(0.f, 0.f);
      const int k = s * 32 + lane;
      ys[s] = (k < m) ? make_float2(y[k].x / ds[k], y[k].y / ds[k]) : make_float2(0.f, 0.f);
    }
    for (int c = 0; c < m; ++c) {
      float ar = 0.f, ai = 0.f;
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int k = s * 32 + lane;
        if (k < c) {
          const float2 l = Ls[c * m + k];
          ar += xs[s].x * l.x + xs[s].y * l.y;
          ai += xs[s].y * l.x - xs[s].x * l.y;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        ar += __shfl_xor_sync(0xffffffffu, ar, o);
        ai += __shfl_xor_sync(0xffffffffu, ai, o);
      }
      float2 yc = make_float2(0.f, 0.f);
#pragma unroll
      for (int s = 0; s < 4; ++s)
        if (s == (c >> 5)) {
          yc.x = __shfl_sync(0xffffffffu, ys[s].x, c & 31);
          yc.y = __shfl_sync(0xffffffffu, ys[s].y, c & 31);
        }
      const float dinv = 1.0f / Ls[c * m + c].x;
      const float2 xc = make_float2((yc.x - ar) * dinv, (yc.y - ai) * dinv);
#pragma unroll
      for (int s = 0; s < 4; ++s)
        if (s == (c >> 5) && lane == (c & 31)) xs[s] = xc;
    }
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int k = s * 32 + lane;
      if (k < m) X[(long long)r * m + k] = xs[s];
    }
  }
}

cudaError_t eig_chol(const float2* Gm, int m, const float* dscale, float shift_rel,
                     const float* acc_in, float2* L, float* dout, float* diagR, DevStatus* status,
                     cudaStream_t st, const EigItems& it) {
  if (m > 128) return cudaErrorInvalidValue;
  const size_t smem = (size_t)m * m * sizeof(float2) + 2 * m * sizeof(float);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(chol_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set = true;
  }
  chol_kernel<<<dim3(1, 1, it.n), 256, smem, st>>>(Gm, m, dscale, shift_rel, acc_in, L, dout, diagR, status, it);
  ++g_launches;
  return cudaGetLastError();
}

cudaError_t eig_chol_inv_blocked(const float2* Gm, int m, const float* dscale, float shift_rel,
                                 const float* acc_in, float2* Rinv, float* diagR, DevStatus* status,
                                 cudaStream_t st, const EigItems& it) {
  if (m > 64) return cudaErrorInvalidValue;  // the panel step covers 64 rows
  const int M = ((m + CB - 1) / CB) * CB;
  const size_t smem = 2 * (size_t)M * M * sizeof(float2) + 2 * M * sizeof(float);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(chol_inv_blocked_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set = true;
  }
  chol_inv_blocked_kernel<<<dim3(1, 1, it.n), 256, smem, st>>>(Gm, m, dscale, shift_rel, acc_in, Rinv, diagR,
                                                              status, it);
  ++g_launches;
  return cudaGetLastError();
}

cudaError_t eig_trsm(const float2* Y, const float2* L, const float* ds, int n, int m, float2* X,
                     cudaStream_t st, const EigItems& it) {
  if (m > 128) return cudaErrorInvalidValue;
  const size_t smem = (size_t)m * m * sizeof(float2) + m * sizeof(float);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(trsm_rows_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(trsm_rows_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(trsm_rows_warp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set = true;
  }
  if (m <= 32) {
    trsm_rows_kernel<32><<<dim3((n + 127) / 128, it.n), 128, smem, st>>>(Y, L, ds, n, m, X, it);
  } else if (m <= 64) {
    trsm_rows_kernel<64><<<dim3((n + 127) / 128, it.n), 128, smem, st>>>(Y, L, ds, n, m, X, it);
  } else {
    int blocks = (n + 7) / 8;
    if (blocks > 152) blocks = 152;
    trsm_rows_warp_kernel<<<dim3(blocks, it.n), 256, smem, st>>>(Y, L, ds, n, m, X, it);
  }
  ++g_launches;
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Parallel cyclic Jacobi for a small Hermitian m x m matrix (1 CTA, FP32, m even <= 128).
// Round-robin ordering: m/2 disjoint pairs per round, m-1 rounds per sweep.  For the pair
// (p,q) with b = B[p][q] = |b| e, the rotation J = [[c, -s e],[s conj(e), c]] with
// t = tan(theta) = sign(z)/(|z| + sqrt(1+z^2)), z = (B[p][p]-B[q][q])/(2|b|), zeroes B[p][q].
// A rotation is skipped when |b| <= 3e-7 sqrt(|B_pp B_qq|) + 3e-9 max|B_ii| (relative
// accuracy for the small Ritz values); the solve stops after a sweep whose rotations all had
// |b| <= 2e-6 sqrt(|B_pp B_qq|) + 3e-9 max|B_ii| (rotations at that level only stir FP32 rounding
// noise, which otherwise keeps a converged matrix rotating until the sweep limit) or joined two
// Ritz values both below stop_rel max|B_ii| (below every value the threshold split looks at: the
// unconverged bottom of the block otherwise couples back and forth with its skipped neighbours
// and converges only linearly).
// The two-sided update of a round is applied per 2x2 block (pair i rows, pair j columns):
// B_ij <- J_i^H B_ij J_j, one shared-memory pass; V <- V J likewise.  B and, when it fits
// (m <= 96), V live in shared memory.  Output: mu (descending) and V with B V = V diag(mu).
// ---------------------------------------------------------------------------------------
template <bool VSMEM>
__global__ void __launch_bounds__(512) jacobi_kernel(const float2* __restrict__ Bin, int m,
                                                     float* __restrict__ mu,
                                                     float2* __restrict__ Vout,
                                                     float2* __restrict__ Vg, int max_sweeps,
                                                     float skip_rel, float stop_rel, DevStatus* status,
                                                     EigItems it) {
  extern __shared__ float2 sm[];
  Bin += blockIdx.z * it.mm;
  mu += blockIdx.z * it.vec;
  Vout += blockIdx.z * it.vj;
  Vg += blockIdx.z * it.vj;
  if (status) status += blockIdx.z;
  float2* Bs = sm;                                         // m*m
  float2* Vw = VSMEM ? (Bs + m * m) : Vg;                  // m*m
  float* rc = reinterpret_cast<float*>(Bs + (VSMEM ? 2 : 1) * m * m);  // c, s*er, s*ei per pair (+pad)
  int* pp = reinterpret_cast<int*>(rc + 4 * (m / 2));
  int* qq = pp + m / 2;
  int* act = qq + m / 2;                                   // rotation active flag per pair
  __shared__ int s_rot;
  __shared__ float s_bnorm;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int half = m / 2;
  for (int e = tid; e < m * m; e += nt) {
    const int i = e / m, j = e % m;
    const float2 a = Bin[i * m + j], b = Bin[j * m + i];
    Bs[e] = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y - b.y));
    Vw[e] = make_float2(i == j ? 1.f : 0.f, 0.f);
  }
  __syncthreads();
  if (tid < 32) {
    float bn = 0.f;
    for (int i = tid; i < m; i += 32) bn = fmaxf(bn, fabsf(Bs[i * m + i].x));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bn = fmaxf(bn, __shfl_xor_sync(0xffffffffu, bn, o));
    if (tid == 0) { s_bnorm = bn; s_rot = 0; }
  }
  __syncthreads();
  const float abs_tol = 3e-9f * s_bnorm;
  // Ritz values below 1e-4 * max are far below any threshold split (thr^2 >= 1e-3 for the
  // supported thresholds is not assumed; the split is re-decided in FP64): rotations among
  // such vectors only reorder noise, so their relative test uses this floor.
  const float noise = 1e-4f * s_bnorm;
  // pairs whose diagonals both lie below skip_rel * max are left alone: such Ritz vectors are
  // far below the threshold split and mixing among them cannot change the signal subspace
  const float skip_below = skip_rel * s_bnorm;
  const float stop_below = stop_rel * s_bnorm;
  const int tx = tid & 31, ty = tid >> 5, nty = nt >> 5;  // 32 x (nt/32) map
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    for (int r = 0; r < m - 1; ++r) {
      for (int i = tid; i < half; i += nt) {
        const int a = (i == 0) ? 0 : 1 + (i - 1 + r) % (m - 1);
        const int b = 1 + (m - 2 - i + r) % (m - 1);
        const int p = min(a, b), q = max(a, b);
        pp[i] = p; qq[i] = q;
        const float2 bpq = Bs[p * m + q];
        const float mag = sqrtf(bpq.x * bpq.x + bpq.y * bpq.y);
        const float app = Bs[p * m + p].x, aqq = Bs[q * m + q].x;
        float c = 1.f, ser = 0.f, sei = 0.f;
        int on = 0;
        const bool both_low = fabsf(app) < skip_below && fabsf(aqq) < skip_below;
        const float rel = sqrtf(fmaxf(fabsf(app), noise) * fmaxf(fabsf(aqq), noise));
        if (!both_low && mag > 3e-7f * rel + abs_tol) {
          const float z = (app - aqq) / (2.f * mag);
          const float t = (z >= 0.f ? 1.f : -1.f) / (fabsf(z) + sqrtf(1.f + z * z));
          c = rsqrtf(1.f + t * t);
          const float sn = t * c;
          ser = sn * bpq.x / mag; sei = sn * bpq.y / mag;
          on = 1;
          if (mag > 2e-6f * rel + abs_tol && fmaxf(app, aqq) >= stop_below) s_rot = 1;
        }
        rc[4 * i] = c; rc[4 * i + 1] = ser; rc[4 * i + 2] = sei;
        act[i] = on;
      }
      __syncthreads();
      // 2x2 blocks: rows of pair i, columns of pair j
      for (int i = ty; i < half; i += nty)
      for (int j = tx; j < half; j += 32) {
        const int ai = act[i], aj = act[j];
        if (!ai && !aj) continue;
        const int pi = pp[i], qi = qq[i], pj = pp[j], qj = qq[j];
        float2 x00 = Bs[pi * m + pj], x01 = Bs[pi * m + qj], x10 = Bs[qi * m + pj], x11 = Bs[qi * m + qj];
        if (ai) {  // rows: J_i^H [x0.; x1.]: r0 = c x0 + se x1, r1 = -conj(se) x0 + c x1
          const float c = rc[4 * i];
          const float2 se = make_float2(rc[4 * i + 1], rc[4 * i + 2]);
          const float2 y00 = make_float2(c * x00.x + se.x * x10.x - se.y * x10.y, c * x00.y + se.x * x10.y + se.y * x10.x);
          const float2 y01 = make_float2(c * x01.x + se.x * x11.x - se.y * x11.y, c * x01.y + se.x * x11.y + se.y * x11.x);
          const float2 y10 = make_float2(-(se.x * x00.x + se.y * x00.y) + c * x10.x, -(se.x * x00.y - se.y * x00.x) + c * x10.y);
          const float2 y11 = make_float2(-(se.x * x01.x + se.y * x01.y) + c * x11.x, -(se.x * x01.y - se.y * x01.x) + c * x11.y);
          x00 = y00; x01 = y01; x10 = y10; x11 = y11;
        }
        if (aj) {  // columns: [x.0 x.1] J_j: k0 = c x0 + conj(se) x1, k1 = -se x0 + c x1
          const float c = rc[4 * j];
          const float2 se = make_float2(rc[4 * j + 1], rc[4 * j + 2]);
          const float2 y00 = make_float2(c * x00.x + se.x * x01.x + se.y * x01.y, c * x00.y + se.x * x01.y - se.y * x01.x);
          const float2 y01 = make_float2(-(se.x * x00.x - se.y * x00.y) + c * x01.x, -(se.x * x00.y + se.y * x00.x) + c * x01.y);
          const float2 y10 = make_float2(c * x10.x + se.x * x11.x + se.y * x11.y, c * x10.y + se.x * x11.y - se.y * x11.x);
          const float2 y11 = make_float2(-(se.x * x10.x - se.y * x10.y) + c * x11.x, -(se.x * x10.y + se.y * x10.x) + c * x11.y);
          x00 = y00; x01 = y01; x10 = y10; x11 = y11;
        }
        Bs[pi * m + pj] = x00; Bs[pi * m + qj] = x01; Bs[qi * m + pj] = x10; Bs[qi * m + qj] = x11;
      }
      // V <- V J: row k, pair j
      for (int k = ty; k < m; k += nty)
      for (int j = tx; j < half; j += 32) {
        if (!act[j]) continue;
        const int pj = pp[j], qj = qq[j];
        const float c = rc[4 * j];
        const float2 se = make_float2(rc[4 * j + 1], rc[4 * j + 2]);
        const float2 xp = Vw[k * m + pj], xq = Vw[k * m + qj];
        Vw[k * m + pj] = make_float2(c * xp.x + se.x * xq.x + se.y * xq.y, c * xp.y + se.x * xq.y - se.y * xq.x);
        Vw[k * m + qj] = make_float2(-(se.x * xp.x - se.y * xp.y) + c * xq.x, -(se.x * xp.y + se.y * xp.x) + c * xq.y);
      }
      __syncthreads();
    }
    const int any = s_rot;
    __syncthreads();
    if (tid == 0) s_rot = 0;
    __syncthreads();
    if (!any) break;
  }
  if (tid == 0 && status) status->jacobi_sweeps = sweep;
  // sort eigenvalues descending (rank by count, ties broken by index) and permute V
  int* rk = pp;  // pp, qq are contiguous: m ints
  __syncthreads();
  for (int i = tid; i < m; i += nt) {
    const float v = Bs[i * m + i].x;
    int rank = 0;
    for (int j = 0; j < m; ++j) {
      const float w = Bs[j * m + j].x;
      rank += (w > v) || (w == v && j < i);
    }
    rk[i] = rank;
    mu[rank] = v;
  }
  __syncthreads();
  for (int e = tid; e < m * m; e += nt) {
    const int k = e / m, i = e % m;
    Vout[k * m + rk[i]] = Vw[k * m + i];
  }
}

// The same cyclic Jacobi (ordering, rotation, skip and stop rules) for m <= 64, arranged for
// latency: the round schedule and the upper-triangle block list are tabulated once; each round
// updates only the 2x2 blocks (i <= j) and mirrors them (B stays exactly Hermitian); and the
// rotations of round r+1 are computed by warp 0 while the other warps apply round r to V
// (rotation parameters double-buffered), so a round costs two barriers and no serial phase.
constexpr int kJs = 65;  // padded row stride of B in shared memory
__global__ void __launch_bounds__(544) jacobi_small_kernel(const float2* __restrict__ Bin, int m,
                                                           float* __restrict__ mu, float2* __restrict__ Vout,
                                                           int max_sweeps, float skip_rel, float stop_rel,
                                                           DevStatus* status, EigItems it) {
  extern __shared__ float2 jsm[];
  float2* Bs = jsm;               // [64][kJs]
  float2* Vw = jsm + 64 * kJs;    // [64][64]
  __shared__ unsigned char sched[63 * 32 * 2];  // (p, q) of every pair of every round
  __shared__ unsigned char blk[528 * 2];        // (i, j), i <= j, of every block
  __shared__ float rc[2][32][3];                // c, Re(s e), Im(s e) per pair, two rounds
  __shared__ int act[2][32];
  __shared__ int s_rot, s_stop, s_sweeps;
  __shared__ float s_bnorm;
  Bin += blockIdx.z * it.mm;
  mu += blockIdx.z * it.vec;
  Vout += blockIdx.z * it.vj;
  if (status) status += blockIdx.z;
  const int tid = threadIdx.x, nt = blockDim.x, warp = tid >> 5, lane = tid & 31;
  const int half = m / 2, rounds = m - 1;
  const int nblk = half * (half + 1) / 2;
  for (int e = tid; e < m * m; e += nt) {
    const int i = e / m, j = e % m;
    const float2 a = Bin[i * m + j], b = Bin[j * m + i];
    Bs[i * kJs + j] = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y - b.y));
    Vw[e] = make_float2(i == j ? 1.f : 0.f, 0.f);
  }
  for (int e = tid; e < rounds * half; e += nt) {
    const int r = e / half, i = e % half;
    const int a = (i == 0) ? 0 : 1 + (i - 1 + r) % (m - 1);
    const int b = 1 + (m - 2 - i + r) % (m - 1);
    sched[2 * e] = (unsigned char)min(a, b);
    sched[2 * e + 1] = (unsigned char)max(a, b);
  }
  for (int e = tid; e < nblk; e += nt) {
    int i = 0, base = 0;
    while (e >= base + (half - i)) { base += half - i; ++i; }
    blk[2 * e] = (unsigned char)i;
    blk[2 * e + 1] = (unsigned char)(i + (e - base));
  }
  __syncthreads();
  if (warp == 0) {
    float bn = 0.f;
    for (int i = lane; i < m; i += 32) bn = fmaxf(bn, fabsf(Bs[i * kJs + i].x));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bn = fmaxf(bn, __shfl_xor_sync(0xffffffffu, bn, o));
    if (lane == 0) { s_bnorm = bn; s_rot = 0; s_stop = 0; s_sweeps = 0; }
  }
  __syncthreads();
  const float abs_tol = 3e-9f * s_bnorm;
  const float noise = 1e-4f * s_bnorm;
  const float skip_below = skip_rel * s_bnorm;
  const float stop_below = stop_rel * s_bnorm;
  // warp 0: rotations of global round g (round g % rounds of sweep g / rounds) into buffer g & 1
  auto rotations = [&](int g) {
    const int r = g % rounds, buf = g & 1;
    if (lane < half) {
      const int p = sched[2 * (r * half + lane)], q = sched[2 * (r * half + lane) + 1];
      const float2 bpq = Bs[p * kJs + q];
      // (approximate reciprocals and square roots: the rotation stays orthogonal to rounding,
      // c = 1/sqrt(1+t^2) and |e| = 1, whatever the accuracy of t; the annihilated entry is
      // set to zero below, as in the classical method)
      const float m2 = bpq.x * bpq.x + bpq.y * bpq.y;
      const float inv = rsqrtf(m2);
      const float mag = m2 > 0.f ? m2 * inv : 0.f;
      const float app = Bs[p * kJs + p].x, aqq = Bs[q * kJs + q].x;
      float c = 1.f, ser = 0.f, sei = 0.f;
      int on = 0, big = 0;
      const bool both_low = fabsf(app) < skip_below && fabsf(aqq) < skip_below;
      const float pr = fmaxf(fabsf(app), noise) * fmaxf(fabsf(aqq), noise);
      const float rel = pr * rsqrtf(pr);
      if (!both_low && mag > 3e-7f * rel + abs_tol) {
        const float z = (app - aqq) * (0.5f * inv);
        const float h = fmaf(z, z, 1.f);
        const float t = copysignf(__fdividef(1.f, fabsf(z) + h * rsqrtf(h)), z);
        c = rsqrtf(fmaf(t, t, 1.f));
        const float sn = t * c;
        ser = sn * bpq.x * inv;
        sei = sn * bpq.y * inv;
        on = 1;
        big = mag > 2e-6f * rel + abs_tol && fmaxf(app, aqq) >= stop_below;
      }
      rc[buf][lane][0] = c;
      rc[buf][lane][1] = ser;
      rc[buf][lane][2] = sei;
      act[buf][lane] = on;
      if (__any_sync(__activemask(), big) && lane == 0) s_rot = 1;
    }
  };
  const int gmax = max_sweeps * rounds;
  const int nwv = nt / 32 - 1;  // warps updating V
  if (warp == 0 && gmax > 0) rotations(0);
  // this thread's block (i <= j) of the two-sided update, fixed for the whole solve
  const bool has_blk = tid < nblk;
  const int bi = has_blk ? blk[2 * tid] : 0, bj = has_blk ? blk[2 * tid + 1] : 0;
  __syncthreads();
  int g = 0;
  for (; g < gmax; ++g) {
    const int buf = g & 1, r = g % rounds;
    const unsigned char* sp = sched + 2 * r * half;
    // (1) B <- J^H B J on the blocks i <= j, mirrored
    if (has_blk) {
      const int i = bi, j = bj;
      const int ai = act[buf][i], aj = act[buf][j];
      if (ai || aj) {
      const int pi = sp[2 * i], qi = sp[2 * i + 1], pj = sp[2 * j], qj = sp[2 * j + 1];
      float2 x00 = Bs[pi * kJs + pj], x01 = Bs[pi * kJs + qj], x10 = Bs[qi * kJs + pj], x11 = Bs[qi * kJs + qj];
      if (ai) {  // rows: r0 = c x0 + se x1, r1 = -conj(se) x0 + c x1
        const float c = rc[buf][i][0];
        const float2 se = make_float2(rc[buf][i][1], rc[buf][i][2]);
        const float2 y00 = make_float2(c * x00.x + se.x * x10.x - se.y * x10.y, c * x00.y + se.x * x10.y + se.y * x10.x);
        const float2 y01 = make_float2(c * x01.x + se.x * x11.x - se.y * x11.y, c * x01.y + se.x * x11.y + se.y * x11.x);
        const float2 y10 = make_float2(-(se.x * x00.x + se.y * x00.y) + c * x10.x, -(se.x * x00.y - se.y * x00.x) + c * x10.y);
        const float2 y11 = make_float2(-(se.x * x01.x + se.y * x01.y) + c * x11.x, -(se.x * x01.y - se.y * x01.x) + c * x11.y);
        x00 = y00; x01 = y01; x10 = y10; x11 = y11;
      }
      if (aj) {  // columns: k0 = c x0 + conj(se) x1, k1 = -se x0 + c x1
        const float c = rc[buf][j][0];
        const float2 se = make_float2(rc[buf][j][1], rc[buf][j][2]);
        const float2 y00 = make_float2(c * x00.x + se.x * x01.x + se.y * x01.y, c * x00.y + se.x * x01.y - se.y * x01.x);
        const float2 y01 = make_float2(-(se.x * x00.x - se.y * x00.y) + c * x01.x, -(se.x * x00.y + se.y * x00.x) + c * x01.y);
        const float2 y10 = make_float2(c * x10.x + se.x * x11.x + se.y * x11.y, c * x10.y + se.x * x11.y - se.y * x11.x);
        const float2 y11 = make_float2(-(se.x * x10.x - se.y * x10.y) + c * x11.x, -(se.x * x10.y + se.y * x10.x) + c * x11.y);
        x00 = y00; x01 = y01; x10 = y10; x11 = y11;
      }
      if (i == j) {  // the pair's own block: real diagonal, the rotated entry annihilated
        x00.y = 0.f;
        x11.y = 0.f;
        if (ai) x01 = make_float2(0.f, 0.f);
        x10 = make_float2(x01.x, -x01.y);
      }
      Bs[pi * kJs + pj] = x00; Bs[pi * kJs + qj] = x01; Bs[qi * kJs + pj] = x10; Bs[qi * kJs + qj] = x11;
      if (i != j) {
        Bs[pj * kJs + pi] = make_float2(x00.x, -x00.y);
        Bs[qj * kJs + pi] = make_float2(x01.x, -x01.y);
        Bs[pj * kJs + qi] = make_float2(x10.x, -x10.y);
        Bs[qj * kJs + qi] = make_float2(x11.x, -x11.y);
      }
      }
    }
    __syncthreads();
    // (2) warp 0: the next round's rotations (after a sweep, the stop test); warps 1..: V <- V J
    if (warp == 0) {
      const int gn = g + 1;
      bool stop = gn >= gmax;
      if (stop && lane == 0) s_sweeps = max_sweeps;
      if (!stop && gn % rounds == 0) {  // a sweep ended: stop if none of its rotations was large
        __syncwarp();
        const int any = s_rot;
        __syncwarp();
        if (lane == 0) { s_rot = 0; s_sweeps = gn / rounds; }
        __syncwarp();
        stop = !any;
      }
      if (stop) {
        if (lane == 0) s_stop = 1;
      } else {
        rotations(gn);
      }
    } else {
      // lane = pair (its rotation read once per round), warps 1.. step through the rows
      const int j = lane;
      if (j < half && act[buf][j]) {
        const int pj = sp[2 * j], qj = sp[2 * j + 1];
        const float c = rc[buf][j][0];
        const float2 se = make_float2(rc[buf][j][1], rc[buf][j][2]);
        for (int k = warp - 1; k < m; k += nwv) {
          const float2 xp = Vw[k * m + pj], xq = Vw[k * m + qj];
          Vw[k * m + pj] = make_float2(c * xp.x + se.x * xq.x + se.y * xq.y, c * xp.y + se.x * xq.y - se.y * xq.x);
          Vw[k * m + qj] = make_float2(-(se.x * xp.x - se.y * xp.y) + c * xq.x, -(se.x * xp.y + se.y * xp.x) + c * xq.y);
        }
      }
    }
    __syncthreads();
    if (s_stop) break;
  }
  if (tid == 0 && status) status->jacobi_sweeps = (g >= gmax) ? max_sweeps : s_sweeps;
  __syncthreads();
  // sort eigenvalues descending (rank by count, ties broken by index) and permute V
  __shared__ int rk[64];
  for (int i = tid; i < m; i += nt) {
    const float v = Bs[i * kJs + i].x;
    int rank = 0;
    for (int j = 0; j < m; ++j) {
      const float w = Bs[j * kJs + j].x;
      rank += (w > v) || (w == v && j < i);
    }
    rk[i] = rank;
    mu[rank] = v;
  }
  __syncthreads();
  for (int e = tid; e < m * m; e += nt) {
    const int k = e / m, i = e % m;
    Vout[k * m + rk[i]] = Vw[k * m + i];
  }
}

// ---------------------------------------------------------------------------------------
// Thin block products of the orthogonal iteration for m <= 64 columns, FP32 on the CUDA cores.
// 128 threads; thread (ti, tj) of a 16 x 8 grid owns a 4 x 8 block of the 64 x 64 (or 64-row x
// 64-column) output: rows 4 ti .. 4 ti + 3 and columns 2 tj + 16 u + e (u < 4, e < 2), so that the
// eight threads of a quarter-warp read 128 consecutive bytes with 16-byte shared loads.
// thin_gram: C = Y^H Z (m x m) over n rows.  CTA (split, item) runs over its share of the rows in
// chunks of kThinRows staged in shared memory; the split's partial goes to ws[item][split], and
// the last CTA of the item to finish (ticket counter, reset by that CTA) sums the partials in
// split order into C.
// thin_apply: X = Y W (n x m by m x m), CTA (chunk of rows, item).
// ---------------------------------------------------------------------------------------
constexpr int kThinRows = 64;
constexpr int kThinLd = 64 + 2;    // padded row (float2): rows stay 16-byte aligned
constexpr int kThinMaxSplits = 16;  // row splits of a thin Gram (CTAs per item)

__device__ __forceinline__ void thin_load(float2 (&v)[8], const float2* row, int tj) {
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const float4 t = *reinterpret_cast<const float4*>(row + 2 * tj + 16 * u);
    v[2 * u] = make_float2(t.x, t.y);
    v[2 * u + 1] = make_float2(t.z, t.w);
  }
}

__global__ void __launch_bounds__(128) thin_gram_kernel(const float2* __restrict__ Y, long long sY,
                                                        const float2* __restrict__ Z, long long sZ, int n, int m,
                                                        float2* __restrict__ C, long long sC,
                                                        float2* __restrict__ ws, int* __restrict__ tickets) {
  extern __shared__ __align__(16) float2 tsm[];
  float2* Ys = tsm;                       // [kThinRows][kThinLd]
  float2* Zs = tsm + kThinRows * kThinLd;
  __shared__ int s_last;
  const int item = blockIdx.y, split = blockIdx.x, nsp = gridDim.x;
  Y += item * sY;
  Z += item * sZ;
  C += item * sC;
  const int nch = (n + kThinRows - 1) / kThinRows;
  const int c0 = (int)((long long)nch * split / nsp), c1 = (int)((long long)nch * (split + 1) / nsp);
  const int tid = threadIdx.x, ti = tid >> 3, tj = tid & 7;
  float2 acc[4][8];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = make_float2(0.f, 0.f);
  for (int ch = c0; ch < c1; ++ch) {
    const int r0 = ch * kThinRows;
    const int rows = min(kThinRows, n - r0);
    __syncthreads();
    for (int e = tid; e < kThinRows * 64; e += 128) {  // zero-padded to 64 rows x 64 columns
      const int r = e >> 6, c = e & 63;
      const bool in = r < rows && c < m;
      Ys[r * kThinLd + c] = in ? Y[(long long)(r0 + r) * m + c] : make_float2(0.f, 0.f);
      Zs[r * kThinLd + c] = in ? Z[(long long)(r0 + r) * m + c] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int r = 0; r < rows; ++r) {
      const float4 y01 = *reinterpret_cast<const float4*>(Ys + r * kThinLd + 4 * ti);
      const float4 y23 = *reinterpret_cast<const float4*>(Ys + r * kThinLd + 4 * ti + 2);
      const float2 y[4] = {make_float2(y01.x, y01.y), make_float2(y01.z, y01.w), make_float2(y23.x, y23.y),
                           make_float2(y23.z, y23.w)};
      float2 z[8];
      thin_load(z, Zs + r * kThinLd, tj);
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) {  // conj(y) z
          acc[a][b].x = fmaf(y[a].x, z[b].x, fmaf(y[a].y, z[b].y, acc[a][b].x));
          acc[a][b].y = fmaf(y[a].x, z[b].y, fmaf(-y[a].y, z[b].x, acc[a][b].y));
        }
    }
  }
  const long long mm = (long long)m * m;
  float2* part = ws + ((long long)item * nsp + split) * mm;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int i = 4 * ti + a, j = 2 * tj + 16 * (b >> 1) + (b & 1);
      if (i < m && j < m) part[i * m + j] = acc[a][b];
    }
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    const int t = atomicAdd(&tickets[item], 1);
    s_last = (t == nsp - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // the last split of the item: partials summed in split order (all loads of an entry issued
  // together, up to kThinMaxSplits of them)
  const float2* base = ws + (long long)item * nsp * mm;
  for (long long e = tid; e < mm; e += 128) {
    float2 w[kThinMaxSplits];
#pragma unroll
    for (int k = 0; k < kThinMaxSplits; ++k) w[k] = k < nsp ? __ldcg(base + k * mm + e) : make_float2(0.f, 0.f);
    float2 v = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < kThinMaxSplits; ++k) {
      v.x += w[k].x;
      v.y += w[k].y;
    }
    C[e] = v;
  }
  if (tid == 0) tickets[item] = 0;
}

__global__ void __launch_bounds__(128) thin_apply_kernel(const float2* __restrict__ Y, long long sY,
                                                         const float2* __restrict__ W, long long sW, int n, int m,
                                                         float2* __restrict__ X, long long sX) {
  extern __shared__ __align__(16) float2 tsm[];
  float2* Ys = tsm;                       // [kThinRows][kThinLd]
  float2* Ws = tsm + kThinRows * kThinLd; // [64][kThinLd]
  const int item = blockIdx.y;
  Y += item * sY;
  W += item * sW;
  X += item * sX;
  const int r0 = blockIdx.x * kThinRows;
  const int rows = min(kThinRows, n - r0);
  const int tid = threadIdx.x, ti = tid >> 3, tj = tid & 7;
  for (int e = tid; e < kThinRows * 64; e += 128) {  // zero-padded
    const int r = e >> 6, c = e & 63;
    Ys[r * kThinLd + c] = (r < rows && c < m) ? Y[(long long)(r0 + r) * m + c] : make_float2(0.f, 0.f);
    Ws[r * kThinLd + c] = (r < m && c < m) ? W[r * m + c] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  float2 acc[4][8];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = make_float2(0.f, 0.f);
  for (int k = 0; k < m; ++k) {
    float2 y[4], w[8];
#pragma unroll
    for (int a = 0; a < 4; ++a) y[a] = Ys[(4 * ti + a) * kThinLd + k];
    thin_load(w, Ws + k * kThinLd, tj);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) {  // y w
        acc[a][b].x = fmaf(y[a].x, w[b].x, fmaf(-y[a].y, w[b].y, acc[a][b].x));
        acc[a][b].y = fmaf(y[a].x, w[b].y, fmaf(y[a].y, w[b].x, acc[a][b].y));
      }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int i = 4 * ti + a, j = 2 * tj + 16 * (b >> 1) + (b & 1);
      if (i < rows && j < m) X[(long long)(r0 + i) * m + j] = acc[a][b];
    }
}

int eig_thin_chunks(int n) { return (n + kThinRows - 1) / kThinRows; }
// row splits of a thin Gram: one chunk of rows each, at most kThinMaxSplits (more CTAs per item:
// each CTA is latency-bound on its own)
static int thin_splits(int n) { return std::max(1, std::min(kThinMaxSplits, eig_thin_chunks(n))); }

constexpr size_t kThinSmem = (size_t)2 * kThinRows * kThinLd * sizeof(float2);
static bool thin_attrs() {
  static const bool ok =
      cudaFuncSetAttribute(thin_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kThinSmem) ==
          cudaSuccess &&
      cudaFuncSetAttribute(thin_apply_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kThinSmem) ==
          cudaSuccess;
  return ok;
}

cudaError_t eig_thin_gram(const float2* Y, long long sY, const float2* Z, long long sZ, int n, int m, float2* C,
                          long long sC, float2* ws, int* tickets, int items, cudaStream_t st) {
  if (m > 64 || m < 1 || n < 1) return cudaErrorInvalidValue;
  if (!thin_attrs()) return cudaErrorInvalidValue;
  thin_gram_kernel<<<dim3(thin_splits(n), items), 128, kThinSmem, st>>>(Y, sY, Z, sZ, n, m, C, sC, ws, tickets);
  ++g_launches;
  return cudaGetLastError();
}

cudaError_t eig_thin_apply(const float2* Y, long long sY, const float2* W, long long sW, int n, int m, float2* X,
                           long long sX, int items, cudaStream_t st) {
  if (m > 64 || m < 1 || n < 1) return cudaErrorInvalidValue;
  if (!thin_attrs()) return cudaErrorInvalidValue;
  thin_apply_kernel<<<dim3(eig_thin_chunks(n), items), 128, kThinSmem, st>>>(Y, sY, W, sW, n, m, X, sX);
  ++g_launches;
  return cudaGetLastError();
}

cudaError_t eig_jacobi(const float2* B, int m, float* mu, float2* V, int max_sweeps,
                       float skip_rel, float stop_rel, DevStatus* status, cudaStream_t st, const EigItems& it) {
  // V must have room for 2*m*m entries: [0, m*m) output, [m*m, 2*m*m) scratch
  const bool vsmem = m <= 96;
  const size_t smem = (size_t)(vsmem ? 2 : 1) * m * m * sizeof(float2) + 4 * (m / 2) * sizeof(float) +
                      3 * (m / 2) * sizeof(int);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(jacobi_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(jacobi_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set = true;
  }
  if (m <= 64 && m % 2 == 0) {
    constexpr size_t kSmallSmem = (size_t)(64 * kJs + 64 * 64) * sizeof(float2);
    static bool small_attr = false;
    if (!small_attr) {
      cudaFuncSetAttribute(jacobi_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmallSmem);
      small_attr = true;
    }
    jacobi_small_kernel<<<dim3(1, 1, it.n), 544, kSmallSmem, st>>>(B, m, mu, V, max_sweeps, skip_rel, stop_rel, status, it);
    ++g_launches;
    return cudaGetLastError();
  }
  const int threads = 512;
  if (vsmem)
    jacobi_kernel<true><<<dim3(1, 1, it.n), threads, smem, st>>>(B, m, mu, V, V + (size_t)m * m, max_sweeps,
                                                                 skip_rel, stop_rel, status, it);
  else
    jacobi_kernel<false><<<dim3(1, 1, it.n), threads, smem, st>>>(B, m, mu, V, V + (size_t)m * m, max_sweeps,
                                                                  skip_rel, stop_rel, status, it);
  ++g_launches;
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// FP64 decision.  band_idx[0] = 0 (the top Ritz vector fixes lambda_1); the others are the
// Ritz vectors whose FP32 Ritz value lies within a factor 2 of the FP32 threshold, closest
// (in log distance) first, -1 padded.
// ---------------------------------------------------------------------------------------
__global__ void select_band_kernel(const float* __restrict__ mu, int m, double thr2, int nb_max,
                                   int* __restrict__ band_idx, EigItems it) {
  mu += blockIdx.z * it.vec;
  band_idx += blockIdx.z * it.band;
  // candidate j >= 1 with |log2(mu_j/theta)| <= 1; rank by (distance, index); the nb_max-1
  // nearest fill band_idx[1..]
  const int j = threadIdx.x;
  const float theta = (float)(thr2 * (double)mu[0]);
  for (int i = j; i < nb_max; i += blockDim.x) band_idx[i] = (i == 0) ? 0 : -1;
  __syncthreads();
  if (j >= m || j == 0) return;
  auto dist = [&](int t) -> float {
    const float v = mu[t];
    if (!(v > 0.f) || !(theta > 0.f)) return 1e30f;
    return fabsf(log2f(v / theta));
  };
  const float dj = dist(j);
  if (!(dj <= 1.0f)) return;
  int rank = 0;
  for (int t = 1; t < m; ++t) {
    const float dt = dist(t);
    rank += (dt < dj) || (dt == dj && t < j);
  }
  if (rank < nb_max - 1) band_idx[1 + rank] = j;
}

cudaError_t eig_select_band(const float* mu, int m, double thr2, int nb_max, int* band_idx,
                            cudaStream_t st, const EigItems& it) {
  select_band_kernel<<<dim3(1, 1, it.n), 128, 0, st>>>(mu, m, thr2, nb_max, band_idx, it);
  ++g_launches;
  return cudaGetLastError();
}

__global__ void gather_band_kernel(const float2* __restrict__ X, int n, int m,
                                   const int* __restrict__ band_idx, int nb_max, double2* __restrict__ Xb,
                                   EigItems it) {
  X += blockIdx.y * it.nm;
  band_idx += blockIdx.y * it.band;
  Xb += blockIdx.y * it.nb;
  const long long total = (long long)n * nb_max;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(idx / nb_max), c = (int)(idx % nb_max);
    const int j = band_idx[c];
    Xb[idx] = (j >= 0) ? to_z(X[(long long)r * m + j]) : make_double2(0.0, 0.0);
  }
}

cudaError_t eig_gather_band(const float2* X, int n, int m, const int* band_idx, int nb_max,
                            double2* Xb, cudaStream_t st, const EigItems& it) {
  long long blocks = ((long long)n * nb_max + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  gather_band_kernel<<<dim3((unsigned)blocks, it.n), 256, 0, st>>>(X, n, m, band_idx, nb_max, Xb, it);
  ++g_launches;
  return cudaGetLastError();
}

// Zb = A * Xb for the FP64 Gram A (n x n) and the nb <= 16 band columns: one warp per row of
// A (lanes stride the row, so loads are coalesced), Xb staged in shared memory in chunks,
// FP64 accumulation, warp reduction.  FP64-FMA bound: n^2 * nb complex MACs.
// Only the band columns in use (band_idx >= 0; they come first) are multiplied: the unused
// ones are zero and cost no FP64 work.
template <int NBV>
__global__ void __launch_bounds__(256) band_matvec_kernel(const double2* __restrict__ A,
                                                          const double2* __restrict__ Xb, int n,
                                                          const int* __restrict__ band_idx,
                                                          double2* __restrict__ Zb, EigItems it) {
  constexpr int KC = 256;  // rows of Xb per chunk (32 KiB of shared memory for 8 columns)
  A += blockIdx.y * it.a;
  Xb += blockIdx.y * it.nb;
  band_idx += blockIdx.y * it.band;
  Zb += blockIdx.y * it.nb;
  __shared__ double2 xs[KC * NBV];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r = blockIdx.x * 8 + warp;
  int nbu = 0;
#pragma unroll
  for (int c = 0; c < NBV; ++c)
    if (band_idx[c] >= 0) nbu = c + 1;
  double2 acc[NBV];
#pragma unroll
  for (int c = 0; c < NBV; ++c) acc[c] = make_double2(0.0, 0.0);
  for (int k0 = 0; k0 < n; k0 += KC) {
    const int kc = min(KC, n - k0);
    __syncthreads();
    for (int e = threadIdx.x; e < kc * NBV; e += blockDim.x) xs[e] = Xb[(long long)k0 * NBV + e];
    __syncthreads();
    if (r < n) {
      const double2* arow = A + (long long)r * n + k0;
      for (int k = lane; k < kc; k += 32) {
        const double2 a = arow[k];
#pragma unroll
        for (int c = 0; c < NBV; ++c)
          if (c < nbu) cfma(acc[c], a, xs[k * NBV + c]);
      }
    }
  }
#pragma unroll
  for (int c = 0; c < NBV; ++c) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      acc[c].x += __shfl_xor_sync(0xffffffffu, acc[c].x, o);
      acc[c].y += __shfl_xor_sync(0xffffffffu, acc[c].y, o);
    }
  }
  if (r < n && lane == 0) {
#pragma unroll
    for (int c = 0; c < NBV; ++c) Zb[(long long)r * NBV + c] = acc[c];
  }
}

cudaError_t eig_band_matvec(const double2* A, const double2* Xb, int n, int nb, const int* band_idx,
                            double2* Zb, cudaStream_t st, const EigItems& it) {
  if (nb != 8) return cudaErrorInvalidValue;
  band_matvec_kernel<8><<<dim3((n + 7) / 8, it.n), 256, 0, st>>>(A, Xb, n, band_idx, Zb, it);
  ++g_launches;
  return cudaGetLastError();
}

// FP64 Rayleigh quotients mu~_c = Re(x_c^H A x_c) / (x_c^H x_c) of the band vectors, then the
// threshold split on the FP64 values (band) and the FP32 values (far from the threshold).
//
// Certificate of the split.  For a Hermitian A and a unit vector x with Rayleigh quotient mu
// and residual r = ||A x - mu x||, some eigenvalue lies in [mu - r, mu + r]; when every other
// eigenvalue is at least g away from mu (g > r), that eigenvalue lies within r^2 / (g - r) of mu
// (Kato-Temple).  Each band vector's FP64 residual gives the bound b_c = min(r_c, r_c^2/(g_c - r_c))
// with g_c the distance to the nearest other Ritz value (less that value's own bound when it is
// a band value); theta = thr^2 lambda_1 inherits thr^2 b_0 from lambda_1.  The split is certified
// when every band value satisfies |mu_c - theta| > b_c + thr^2 b_0 and every Ritz value decided
// in FP32 lies outside [theta / 1.001, 1.001 theta] (FP32 Ritz values of the scaled Gram carry
// errors of order 1e-7 lambda_1, i.e. 4e-5 theta at thr = 0.05).  Otherwise ST_UNCERTIFIED.
__global__ void __launch_bounds__(256) decide_kernel(const float* __restrict__ mu, int m,
                                                     const int* __restrict__ band_idx, int nb_max,
                                                     const double2* __restrict__ Xb,
                                                     const double2* __restrict__ Zb, int n,
                                                     double thr2, int Q,
                                                     const double* __restrict__ scale,
                                                     float* __restrict__ w,
                                                     double* __restrict__ ritz, DevStatus* status,
                                                     EigItems it) {
  __shared__ double num[32], den[32], res[32], bnd[32];
  {
    const int i = blockIdx.z;
    mu += i * it.vec;
    band_idx += i * it.band;
    Xb += i * it.nb;
    Zb += i * it.nb;
    scale += i * it.scale;
    w += i * it.vec;
    ritz += i * it.vec;
    status += i;
  }
  __shared__ double s_lmax;
  __shared__ int s_uncert;
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  if (tid == 0) s_uncert = 0;
  // one warp per band column (8 warps, loop over columns)
  for (int c = warp; c < nb_max; c += blockDim.x / 32) {
    double a = 0.0, b = 0.0;
    for (int r = lane; r < n; r += 32) {
      const double2 x = Xb[(long long)r * nb_max + c], z = Zb[(long long)r * nb_max + c];
      a += x.x * z.x + x.y * z.y;
      b += x.x * x.x + x.y * x.y;
    }
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    // FP64 residual of the normalised vector: ||z - mu x||^2 / ||x||^2, summed directly
    const double muc = b > 0.0 ? a / b : 0.0;
    double e = 0.0;
    for (int r = lane; r < n; r += 32) {
      const double2 x = Xb[(long long)r * nb_max + c], z = Zb[(long long)r * nb_max + c];
      const double dx = z.x - muc * x.x, dy = z.y - muc * x.y;
      e += dx * dx + dy * dy;
    }
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if (lane == 0) {
      num[c] = a;
      den[c] = b;
      res[c] = b > 0.0 ? sqrt(e / b) : 0.0;
    }
  }
  __syncthreads();
  if (tid == 0) s_lmax = den[0] > 0.0 ? num[0] / den[0] : 0.0;
  __syncthreads();
  const double lmax = s_lmax;
  const double theta = thr2 * lmax;
  const double sc = *scale;  // FP32 Ritz values are of the Gram divided by `scale`
  for (int j = tid; j < m; j += blockDim.x) {
    double v = (double)mu[j] * sc;
    for (int c = 0; c < nb_max; ++c)
      if (band_idx[c] == j && den[c] > 0.0) v = num[c] / den[c];
    ritz[j] = v;
    bool sig;
    if (lmax > 0.0) sig = (v >= theta);
    else sig = true;  // all-zero data: nothing is strictly below 0, so nothing is null
    w[j] = sig ? 1.f : 0.f;
  }
  __syncthreads();
  // first bounds: the plain residual bound of every band value (neighbours' bounds below)
  if (tid < nb_max) bnd[tid] = res[tid];
  __syncthreads();
  if (tid < nb_max && band_idx[tid] >= 0 && den[tid] > 0.0) {
    const int c = tid, jc = band_idx[c];
    const double mc = ritz[jc], rc = res[c];
    double g = 1e300;
    for (int j = 0; j < m; ++j) {
      if (j == jc) continue;
      double d = fabs(mc - ritz[j]);
      for (int c2 = 0; c2 < nb_max; ++c2)
        if (band_idx[c2] == j && den[c2] > 0.0) d -= res[c2];
      g = fmin(g, d);
    }
    double bc = rc;
    if (g > rc) bc = fmin(rc, rc * rc / (g - rc));
    bnd[c] = bc;
  }
  __syncthreads();
  if (tid < m && lmax > 0.0) {
    const int j = tid;
    int c = -1;
    for (int c2 = 0; c2 < nb_max; ++c2)
      if (band_idx[c2] == j && den[c2] > 0.0) c = c2;
    const double v = ritz[j];
    bool ok;
    if (c == 0) ok = true;  // lambda_1 itself: its bound enters through theta
    else if (c > 0) ok = fabs(v - theta) > bnd[c] + thr2 * bnd[0];
    else ok = (v > 1.001 * theta) || (v < theta / 1.001);
    if (!ok) atomicOr(&s_uncert, 1);
  }
  __syncthreads();
  if (tid == 0) {
    int k = 0;
    for (int j = 0; j < m; ++j) k += (w[j] > 0.f);
    int flags = 0;
    if (!(lmax > 0.0)) { flags |= ST_ZERO; k = n; }
    const int guard = max(4, m / 8);
    if (k > m - guard && !(flags & ST_ZERO)) flags |= ST_SATURATED;
    const int R = n - k;
    if (R < Q - 1) flags |= ST_RANK;
    if (s_uncert && !(flags & ST_ZERO)) flags |= ST_UNCERTIFIED;
    // smallest relative certificate margin over the band (for reporting)
    double margin = 1e300, rmax = 0.0;
    for (int c = 1; c < nb_max; ++c) {
      if (band_idx[c] < 0 || !(den[c] > 0.0)) continue;
      margin = fmin(margin, (fabs(ritz[band_idx[c]] - theta) - bnd[c] - thr2 * bnd[0]) / theta);
      rmax = fmax(rmax, res[c]);
    }
    atomicOr(&status->flags, flags);
    status->k = k;
    int nb = 0;
    for (int c = 0; c < nb_max; ++c) nb += (band_idx[c] >= 0);
    status->nband = nb;
    status->lambda_max = lmax;
    status->cert_margin = lmax > 0.0 ? margin : 0.0;
    status->band_resid = lmax > 0.0 ? rmax / lmax : 0.0;
  }
}

cudaError_t eig_decide(const float* mu, int m, const int* band_idx, int nb_max, const double2* Xb,
                       const double2* Zb, int n, double thr2, int Q, const double* scale,
                       float* weights, double* ritz, DevStatus* status, cudaStream_t st, const EigItems& it) {
  decide_kernel<<<dim3(1, 1, it.n), 256, 0, st>>>(mu, m, band_idx, nb_max, Xb, Zb, n, thr2, Q, scale, weights,
                                                 ritz, status, it);
  ++g_launches;
  return cudaGetLastError();
}

}  // namespace pisco
