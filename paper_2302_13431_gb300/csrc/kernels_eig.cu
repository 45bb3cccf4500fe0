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
// Cholesky-QR pieces.  chol_kernel (1 CTA): Gm = L L^H for a small Hermitian positive
// definite m x m matrix, right-looking in shared memory, two barriers per column; pivots
// below 1e-12 * max diag are clamped (status ST_CHOL).  trsm_rows_kernel (many CTAs):
// X = Y L^{-H} row by row (x L^H = y, forward substitution), one warp per row with L staged
// in shared memory, so no explicit inverse is formed.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) chol_kernel(const float2* __restrict__ Gm, int m,
                                                    float2* __restrict__ Lout, DevStatus* status) {
  // left-looking: column j needs the finished columns k < j only.  Every warp recomputes the
  // pivot of column j itself (no extra barrier), then fills its rows of column j.
  extern __shared__ float2 sm[];
  float2* Lm = sm;  // m*m, row-major, lower triangle
  __shared__ float s_floor;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int i = tid; i < m * m; i += blockDim.x) Lm[i] = Gm[i];
  __syncthreads();
  if (tid == 0) {
    float md = 0.f;
    for (int i = 0; i < m; ++i) md = fmaxf(md, Lm[i * m + i].x);
    s_floor = fmaxf(md, 1e-30f) * 1e-12f;
  }
  __syncthreads();
  const float floor_piv = s_floor;
  for (int j = 0; j < m; ++j) {
    // pivot: G_jj - sum_{k<j} |L_jk|^2
    float sq = 0.f;
    for (int k = lane; k < j; k += 32) {
      const float2 l = Lm[j * m + k];
      sq += l.x * l.x + l.y * l.y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    const float d = Lm[j * m + j].x - sq;
    const float piv = sqrtf(d > floor_piv ? d : floor_piv);
    const float inv = 1.0f / piv;
    for (int i = j + 1 + warp; i < m; i += nw) {
      float ar = 0.f, ai = 0.f;
      for (int k = lane; k < j; k += 32) {
        const float2 a = Lm[i * m + k], b = Lm[j * m + k];  // a * conj(b)
        ar += a.x * b.x + a.y * b.y;
        ai += a.y * b.x - a.x * b.y;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        ar += __shfl_xor_sync(0xffffffffu, ar, o);
        ai += __shfl_xor_sync(0xffffffffu, ai, o);
      }
      if (lane == 0) {
        const float2 g = Lm[i * m + j];
        Lm[i * m + j] = make_float2((g.x - ar) * inv, (g.y - ai) * inv);
      }
    }
    __syncthreads();
    if (tid == 0) {
      Lm[j * m + j] = make_float2(piv, 0.f);
      if (!(d > floor_piv) && status) atomicOr(&status->flags, (int)ST_CHOL);
    }
    // the diagonal entry is not read again by later columns' off-diagonal sums (k < j' only
    // touches columns < j'), and the next pivot reads row j' only, so no barrier is needed here
  }
  __syncthreads();
  for (int e = tid; e < m * m; e += blockDim.x) {
    const int i = e / m, k = e % m;
    Lout[e] = (k <= i) ? Lm[e] : make_float2(0.f, 0.f);
  }
}

__global__ void __launch_bounds__(256) trsm_rows_kernel(const float2* __restrict__ Y,
                                                        const float2* __restrict__ Lg, int n, int m,
                                                        float2* __restrict__ X) {
  extern __shared__ float2 sm[];
  float2* Ls = sm;  // m*m
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
      ys[s] = (k < m) ? y[k] : make_float2(0.f, 0.f);
    }
    for (int c = 0; c < m; ++c) {
      // sum_{k<c} x_k conj(L[c][k]), lanes split k
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

cudaError_t eig_chol(const float2* Gm, int m, float2* L, DevStatus* status, cudaStream_t st) {
  const size_t smem = (size_t)m * m * sizeof(float2);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(chol_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set = true;
  }
  chol_kernel<<<1, 1024, smem, st>>>(Gm, m, L, status);
  ++g_launches;
  return cudaGetLastError();
}

cudaError_t eig_trsm_rows(const float2* Y, const float2* L, int n, int m, float2* X, cudaStream_t st) {
  if (m > 128) return cudaErrorInvalidValue;
  const size_t smem = (size_t)m * m * sizeof(float2);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(trsm_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set = true;
  }
  int blocks = (n + 7) / 8;
  if (blocks > 152) blocks = 152;
  trsm_rows_kernel<<<blocks, 256, smem, st>>>(Y, L, n, m, X);
  ++g_launches;
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Parallel cyclic Jacobi for a small Hermitian m x m matrix (1 CTA, FP32, m even <= 128).
// Round-robin ordering: m/2 disjoint pairs per round, m-1 rounds per sweep.  For the pair
// (p,q) with b = B[p][q] = |b| e, the rotation J = [[c, -s e],[s conj(e), c]] with
// t = tan(theta) = sign(z)/(|z| + sqrt(1+z^2)), z = (B[p][p]-B[q][q])/(2|b|), zeroes B[p][q].
// A rotation is skipped when |b| <= 3e-7 sqrt(|B_pp B_qq|) + 3e-9 max|B_ii| (relative
// accuracy for the small Ritz values); the solve stops after a sweep without rotations.
// The two-sided update of a round is applied per 2x2 block (pair i rows, pair j columns):
// B_ij <- J_i^H B_ij J_j, one shared-memory pass; V <- V J likewise.  B and, when it fits
// (m <= 96), V live in shared memory.  Output: mu (descending) and V with B V = V diag(mu).
// ---------------------------------------------------------------------------------------
template <bool VSMEM>
__global__ void __launch_bounds__(512) jacobi_kernel(const float2* __restrict__ Bin, int m,
                                                     float* __restrict__ mu,
                                                     float2* __restrict__ Vout,
                                                     float2* __restrict__ Vg, int max_sweeps,
                                                     DevStatus* status) {
  extern __shared__ float2 sm[];
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
  if (tid == 0) {
    float bn = 0.f;
    for (int i = 0; i < m; ++i) bn = fmaxf(bn, fabsf(Bs[i * m + i].x));
    s_bnorm = bn;
    s_rot = 0;
  }
  __syncthreads();
  const float abs_tol = 3e-9f * s_bnorm;
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
        if (mag > 3e-7f * sqrtf(fabsf(app * aqq)) + abs_tol) {
          const float z = (app - aqq) / (2.f * mag);
          const float t = (z >= 0.f ? 1.f : -1.f) / (fabsf(z) + sqrtf(1.f + z * z));
          c = rsqrtf(1.f + t * t);
          const float sn = t * c;
          ser = sn * bpq.x / mag; sei = sn * bpq.y / mag;
          on = 1;
          s_rot = 1;
        }
        rc[4 * i] = c; rc[4 * i + 1] = ser; rc[4 * i + 2] = sei;
        act[i] = on;
      }
      __syncthreads();
      // 2x2 blocks: rows of pair i, columns of pair j
      for (int e = tid; e < half * half; e += nt) {
        const int i = e / half, j = e % half;
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
      for (int e = tid; e < m * half; e += nt) {
        const int k = e / half, j = e % half;
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

cudaError_t eig_jacobi(const float2* B, int m, float* mu, float2* V, int max_sweeps,
                       DevStatus* status, cudaStream_t st) {
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
  const int threads = 512;
  if (vsmem)
    jacobi_kernel<true><<<1, threads, smem, st>>>(B, m, mu, V, V + (size_t)m * m, max_sweeps, status);
  else
    jacobi_kernel<false><<<1, threads, smem, st>>>(B, m, mu, V, V + (size_t)m * m, max_sweeps, status);
  ++g_launches;
  return cudaGetLastError();
}

// Y[:, j] /= max(mu_j, floor_rel*mu_0): keeps the block well conditioned for Cholesky-QR.
__global__ void scale_cols_kernel(float2* Y, int n, int m, const float* __restrict__ mu, float floor_rel) {
  const long long total = (long long)n * m;
  const float top = fmaxf(mu[0], 1e-30f);
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(idx % m);
    const float d = fmaxf(mu[c], floor_rel * top);
    float2 v = Y[idx];
    Y[idx] = make_float2(v.x / d, v.y / d);
  }
}

cudaError_t eig_scale_cols(float2* Y, int n, int m, const float* mu, float floor_rel, cudaStream_t st) {
  long long blocks = ((long long)n * m + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  scale_cols_kernel<<<(unsigned)blocks, 256, 0, st>>>(Y, n, m, mu, floor_rel);
  ++g_launches;
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// FP64 decision.  band_idx[0] = 0 (the top Ritz vector fixes lambda_1); the others are the
// Ritz vectors whose FP32 Ritz value lies within a factor 4 of the FP32 threshold, closest
// (in log distance) first, -1 padded.
// ---------------------------------------------------------------------------------------
__global__ void select_band_kernel(const float* __restrict__ mu, int m, double thr2, int nb_max,
                                   int* __restrict__ band_idx) {
  // candidate j >= 1 with |log2(mu_j/theta)| <= 2; rank by (distance, index); the nb_max-1
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
  if (!(dj <= 2.0f)) return;
  int rank = 0;
  for (int t = 1; t < m; ++t) {
    const float dt = dist(t);
    rank += (dt < dj) || (dt == dj && t < j);
  }
  if (rank < nb_max - 1) band_idx[1 + rank] = j;
}

cudaError_t eig_select_band(const float* mu, int m, double thr2, int nb_max, int* band_idx,
                            cudaStream_t st) {
  select_band_kernel<<<1, 128, 0, st>>>(mu, m, thr2, nb_max, band_idx);
  ++g_launches;
  return cudaGetLastError();
}

__global__ void gather_band_kernel(const float2* __restrict__ X, int n, int m,
                                   const int* __restrict__ band_idx, int nb_max, double2* __restrict__ Xb) {
  const long long total = (long long)n * nb_max;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(idx / nb_max), c = (int)(idx % nb_max);
    const int j = band_idx[c];
    Xb[idx] = (j >= 0) ? to_z(X[(long long)r * m + j]) : make_double2(0.0, 0.0);
  }
}

cudaError_t eig_gather_band(const float2* X, int n, int m, const int* band_idx, int nb_max,
                            double2* Xb, cudaStream_t st) {
  long long blocks = ((long long)n * nb_max + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  gather_band_kernel<<<(unsigned)blocks, 256, 0, st>>>(X, n, m, band_idx, nb_max, Xb);
  ++g_launches;
  return cudaGetLastError();
}

// FP64 Rayleigh quotients mu~_c = Re(x_c^H A x_c) / (x_c^H x_c) of the band vectors, then the
// threshold split on the FP64 values (band) and the FP32 values (far from the threshold).
__global__ void __launch_bounds__(256) decide_kernel(const float* __restrict__ mu, int m,
                                                     const int* __restrict__ band_idx, int nb_max,
                                                     const double2* __restrict__ Xb,
                                                     const double2* __restrict__ Zb, int n,
                                                     double thr2, int Q, float* __restrict__ w,
                                                     double* __restrict__ ritz, DevStatus* status) {
  __shared__ double num[32], den[32];
  __shared__ double s_lmax;
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
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
    if (lane == 0) { num[c] = a; den[c] = b; }
  }
  __syncthreads();
  if (tid == 0) s_lmax = den[0] > 0.0 ? num[0] / den[0] : 0.0;
  __syncthreads();
  const double lmax = s_lmax;
  const double theta = thr2 * lmax;
  for (int j = tid; j < m; j += blockDim.x) {
    double v = (double)mu[j];
    for (int c = 0; c < nb_max; ++c)
      if (band_idx[c] == j && den[c] > 0.0) v = num[c] / den[c];
    ritz[j] = v;
    bool sig;
    if (lmax > 0.0) sig = (v >= theta);
    else sig = true;  // all-zero data: nothing is strictly below 0, so nothing is null
    w[j] = sig ? 1.f : 0.f;
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
    atomicOr(&status->flags, flags);
    status->k = k;
    int nb = 0;
    for (int c = 0; c < nb_max; ++c) nb += (band_idx[c] >= 0);
    status->nband = nb;
    status->lambda_max = lmax;
  }
}

cudaError_t eig_decide(const float* mu, int m, const int* band_idx, int nb_max, const double2* Xb,
                       const double2* Zb, int n, double thr2, int Q, float* weights, double* ritz,
                       DevStatus* status, cudaStream_t st) {
  decide_kernel<<<1, 256, 0, st>>>(mu, m, band_idx, nb_max, Xb, Zb, n, thr2, Q, weights, ritz, status);
  ++g_launches;
  return cudaGetLastError();
}

}  // namespace pisco
