// Dense complex GEMM on the CUDA cores, FP32 or FP64:  C = alpha*op(A)*op(B) + beta*C with
// row-major operands and op in {'N' (as stored), 'C' (conjugate transpose)}.
//
// Used by the block eigensolver of stage (b): the n x n by n x m products with the Gram
// (FP32 subspace iteration, FP64 Rayleigh quotients) and the thin n x m / m x m products of
// the Rayleigh-Ritz and Cholesky-QR steps.  The shapes are skinny (m = 32..128), so a CTA
// owns a 32 x 32 (or 64 x 64) output tile and K is split across CTAs until the grid covers the
// 152 SMs; the last CTA of a tile sums the split partials in a fixed order.  `items`
// independent products (operands sA, sB, sC elements apart) run in the same launch: grid.z is
// item * splits + split.
#include <algorithm>

#include "common.cuh"

namespace pisco {

namespace {
constexpr int BM = 32, BN = 32, BK = 16;
}  // namespace
constexpr int kMaxTiles = 4096;  // tile counters the caller provides per item
namespace {

template <typename T>
__global__ void __launch_bounds__(256) cgemm_kernel(char opA, char opB, int M, int N, int K,
                                                    cpx<T> alpha, const cpx<T>* __restrict__ A,
                                                    int lda, const cpx<T>* __restrict__ B, int ldb,
                                                    cpx<T> beta, cpx<T>* __restrict__ C, int ldc,
                                                    cpx<T>* __restrict__ ws, int kchunk,
                                                    int* __restrict__ tile_count, int splits,
                                                    long long sA, long long sB, long long sC) {
  using Cx = cpx<T>;
  __shared__ Cx As[BK][BM + 1];
  __shared__ Cx Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int r0 = blockIdx.y * BM, c0 = blockIdx.x * BN;
  const int item = blockIdx.z / splits, split = blockIdx.z % splits;
  A += item * sA;
  B += item * sB;
  C += item * sC;
  const int kbeg = split * kchunk;
  const int kend = min(K, kbeg + kchunk);
  Cx acc[2][2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) acc[i][j] = mk(T(0), T(0));
  const Cx zero = mk(T(0), T(0));

  for (int k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int e = tid + 256 * s;
      int r, k;
      if (opA == 'N') { r = e / BK; k = e % BK; } else { k = e / BM; r = e % BM; }
      const int gr = r0 + r, gk = k0 + k;
      Cx v = zero;
      if (gr < M && gk < kend) {
        if (opA == 'N') v = A[(long long)gr * lda + gk];
        else v = cconj(A[(long long)gk * lda + gr]);
      }
      As[k][r] = v;
      int c;
      if (opB == 'N') { k = e / BN; c = e % BN; } else { c = e / BK; k = e % BK; }
      const int gc = c0 + c;
      const int gk2 = k0 + k;
      Cx w = zero;
      if (gc < N && gk2 < kend) {
        if (opB == 'N') w = B[(long long)gk2 * ldb + gc];
        else w = cconj(B[(long long)gc * ldb + gk2]);
      }
      Bs[k][c] = w;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      const Cx a0 = As[kk][ty * 2], a1 = As[kk][ty * 2 + 1];
      const Cx b0 = Bs[kk][tx * 2], b1 = Bs[kk][tx * 2 + 1];
      cfma(acc[0][0], a0, b0);
      cfma(acc[0][1], a0, b1);
      cfma(acc[1][0], a1, b0);
      cfma(acc[1][1], a1, b1);
    }
    __syncthreads();
  }
  if (splits == 1) {
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int gr = r0 + ty * 2 + i, gc = c0 + tx * 2 + j;
        if (gr >= M || gc >= N) continue;
        Cx out = cmul(alpha, acc[i][j]);
        if (beta.x != T(0) || beta.y != T(0)) out = cadd(out, cmul(beta, C[(long long)gr * ldc + gc]));
        C[(long long)gr * ldc + gc] = out;
      }
    return;
  }
  // split-K: publish this slice's partial tile; the last CTA of the tile sums all slices in
  // slice order (deterministic) and writes C.  No CTA waits on another.
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int gr = r0 + ty * 2 + i, gc = c0 + tx * 2 + j;
      if (gr < M && gc < N) ws[((long long)blockIdx.z * M + gr) * N + gc] = acc[i][j];
    }
  __threadfence();
  __syncthreads();
  __shared__ int s_last;
  const int tile = item * kMaxTiles + blockIdx.y * gridDim.x + blockIdx.x;
  if (tid == 0) s_last = (atomicAdd(&tile_count[tile], 1) == splits - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int gr = r0 + ty * 2 + i, gc = c0 + tx * 2 + j;
      if (gr >= M || gc >= N) continue;
      Cx sum = mk(T(0), T(0));
      for (int z = 0; z < splits; ++z) sum = cadd(sum, __ldcg(&ws[((long long)(item * splits + z) * M + gr) * N + gc]));
      Cx out = cmul(alpha, sum);
      if (beta.x != T(0) || beta.y != T(0)) out = cadd(out, cmul(beta, C[(long long)gr * ldc + gc]));
      C[(long long)gr * ldc + gc] = out;
    }
  if (tid == 0) tile_count[tile] = 0;  // ready for the next launch on the stream
}

}  // namespace

// 64 x 64 CTA tile, 4 x 4 complex outputs per thread (16 accumulators: 8 shared loads feed
// 64 FMAs per k), BK = 16.  Split-K partials go to `ws`; the last CTA of a tile reduces them
// with all its threads (independent loads, fixed slice order -> deterministic).
namespace {
constexpr int BM2 = 64, BN2 = 64, BK2 = 16;
template <typename T>
__global__ void __launch_bounds__(256) cgemm64_kernel(char opA, char opB, int M, int N, int K,
                                                      cpx<T> alpha, const cpx<T>* __restrict__ A,
                                                      int lda, const cpx<T>* __restrict__ B, int ldb,
                                                      cpx<T> beta, cpx<T>* __restrict__ C, int ldc,
                                                      cpx<T>* __restrict__ ws, int kchunk,
                                                      int* __restrict__ tile_count, int splits,
                                                      long long sA, long long sB, long long sC) {
  using Cx = cpx<T>;
  __shared__ Cx As[BK2][BM2 + 1];
  __shared__ Cx Bs[BK2][BN2 + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int r0 = blockIdx.y * BM2, c0 = blockIdx.x * BN2;
  const int item = blockIdx.z / splits, split = blockIdx.z % splits;
  A += item * sA;
  B += item * sB;
  C += item * sC;
  const int kbeg = split * kchunk;
  const int kend = min(K, kbeg + kchunk);
  Cx acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = mk(T(0), T(0));
  const Cx zero = mk(T(0), T(0));
  for (int k0 = kbeg; k0 < kend; k0 += BK2) {
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int e = tid + 256 * s;  // 1024 = 64 x 16 entries of each tile
      int r, k;
      if (opA == 'N') { r = e >> 4; k = e & 15; } else { k = e >> 6; r = e & 63; }
      Cx v = zero;
      const int gr = r0 + r, gk = k0 + k;
      if (gr < M && gk < kend) v = (opA == 'N') ? A[(long long)gr * lda + gk] : cconj(A[(long long)gk * lda + gr]);
      As[k][r] = v;
      int c;
      if (opB == 'N') { k = e >> 6; c = e & 63; } else { c = e >> 4; k = e & 15; }
      Cx w = zero;
      const int gc = c0 + c, gk2 = k0 + k;
      if (gc < N && gk2 < kend) w = (opB == 'N') ? B[(long long)gk2 * ldb + gc] : cconj(B[(long long)gc * ldb + gk2]);
      Bs[k][c] = w;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK2; ++kk) {
      Cx a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) cfma(acc[i][j], a[i], b[j]);
    }
    __syncthreads();
  }
  if (splits == 1) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int gr = r0 + ty + 16 * i, gc = c0 + tx + 16 * j;
        if (gr >= M || gc >= N) continue;
        Cx out = cmul(alpha, acc[i][j]);
        if (beta.x != T(0) || beta.y != T(0)) out = cadd(out, cmul(beta, C[(long long)gr * ldc + gc]));
        C[(long long)gr * ldc + gc] = out;
      }
    return;
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gr = r0 + ty + 16 * i, gc = c0 + tx + 16 * j;
      if (gr < M && gc < N) ws[((long long)blockIdx.z * M + gr) * N + gc] = acc[i][j];
    }
  __threadfence();
  __syncthreads();
  __shared__ int s_last;
  const int tile = item * kMaxTiles + blockIdx.y * gridDim.x + blockIdx.x;
  if (tid == 0) s_last = (atomicAdd(&tile_count[tile], 1) == splits - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const int nz = splits;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gr = r0 + ty + 16 * i, gc = c0 + tx + 16 * j;
      if (gr >= M || gc >= N) continue;
      const cpx<T>* src = ws + (long long)item * splits * M * N + (long long)gr * N + gc;
      const long long stride = (long long)M * N;
      Cx s0 = mk(T(0), T(0)), s1 = s0, s2 = s0, s3 = s0;
      int z = 0;
      for (; z + 4 <= nz; z += 4) {
        s0 = cadd(s0, __ldcg(src + (z + 0) * stride));
        s1 = cadd(s1, __ldcg(src + (z + 1) * stride));
        s2 = cadd(s2, __ldcg(src + (z + 2) * stride));
        s3 = cadd(s3, __ldcg(src + (z + 3) * stride));
      }
      for (; z < nz; ++z) s0 = cadd(s0, __ldcg(src + z * stride));
      const Cx sum = cadd(cadd(s0, s1), cadd(s2, s3));
      Cx out = cmul(alpha, sum);
      if (beta.x != T(0) || beta.y != T(0)) out = cadd(out, cmul(beta, C[(long long)gr * ldc + gc]));
      C[(long long)gr * ldc + gc] = out;
    }
  if (tid == 0) tile_count[tile] = 0;
}
}  // namespace

template <typename T>
cudaError_t cgemm(char opA, char opB, int M, int N, int K, cpx<T> alpha, const cpx<T>* A, int lda,
                  const cpx<T>* B, int ldb, cpx<T> beta, cpx<T>* C, int ldc, cpx<T>* ws,
                  size_t ws_elems, int* tile_count, cudaStream_t st, int max_splits, int tile, int items,
                  long long sA, long long sB, long long sC) {
  if (M <= 0 || N <= 0 || items < 1) return cudaSuccess;
  // automatic: 64x64 tiles only for large K (the 32x32 kernel has the lower latency for the
  // skinny shapes of one solve); tile = 64 / 32 forces one (64x64 costs less SM time per flop)
  const bool big = tile == 64 || (tile != 32 && M >= 48 && N >= 48 && K >= 4096);
  if (big) {
    // 64 x 64 tiles; split K until ~1 CTA per SM, at most 16 slices of >= 2 k-steps each
    const int tiles2 = ((M + BM2 - 1) / BM2) * ((N + BN2 - 1) / BN2);
    const int kb = K > 0 ? (K + BK2 - 1) / BK2 : 1;
    int sp = 1;
    // the split of one product does not depend on the batch (an item's result is the same
    // whether it runs alone or in a batch)
    if (ws != nullptr && tile_count != nullptr && tiles2 <= kMaxTiles) {
      sp = (152 + tiles2 - 1) / tiles2;
      sp = std::min(sp, std::max(1, kb / 2));
      sp = std::min(sp, 16);
      if (max_splits > 0) sp = std::min(sp, max_splits);
      while (sp > 1 && (size_t)sp * M * N * items > ws_elems) --sp;
    }
    const int kc = ((kb + sp - 1) / sp) * BK2;
    sp = K > 0 ? (K + kc - 1) / kc : 1;
    dim3 grid2((N + BN2 - 1) / BN2, (M + BM2 - 1) / BM2, sp * items);
    cgemm64_kernel<T><<<grid2, 256, 0, st>>>(opA, opB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, ws,
                                             kc, tile_count, sp, sA, sB, sC);
    ++g_launches;
    return cudaGetLastError();
  }
  const int tiles = ((M + BM - 1) / BM) * ((N + BN - 1) / BN);
  int splits = 1;
  const int kblocks = K > 0 ? (K + BK - 1) / BK : 1;
  if (ws != nullptr && tile_count != nullptr && tiles <= kMaxTiles) {
    splits = (2 * 152 + tiles - 1) / tiles;
    if (splits > kblocks) splits = kblocks;
    if (splits > 64) splits = 64;
    if (max_splits > 0 && splits > max_splits) splits = max_splits;
    while (splits > 1 && (size_t)splits * M * N * items > ws_elems) --splits;
    if (splits < 1) splits = 1;
  }
  const int kchunk = ((kblocks + splits - 1) / splits) * BK;
  splits = K > 0 ? (K + kchunk - 1) / kchunk : 1;
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, splits * items);
  cgemm_kernel<T><<<grid, 256, 0, st>>>(opA, opB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, ws,
                                        kchunk, tile_count, splits, sA, sB, sC);
  ++g_launches;
  return cudaGetLastError();
}

template cudaError_t cgemm<float>(char, char, int, int, int, float2, const float2*, int, const float2*,
                                  int, float2, float2*, int, float2*, size_t, int*, cudaStream_t, int, int, int,
                                  long long, long long, long long);
template cudaError_t cgemm<double>(char, char, int, int, int, double2, const double2*, int,
                                   const double2*, int, double2, double2*, int, double2*, size_t, int*,
                                   cudaStream_t, int, int, int, long long, long long, long long);

}  // namespace pisco
