// Dense complex GEMM on the CUDA cores, FP32 or FP64:  C = alpha*op(A)*op(B) + beta*C with
// row-major operands and op in {'N' (as stored), 'C' (conjugate transpose)}.
//
// Used by the block eigensolver of stage (b): the n x n by n x m products with the Gram
// (FP32 subspace iteration, FP64 Rayleigh quotients) and the thin n x m / m x m products of
// the Rayleigh-Ritz and Cholesky-QR steps.  The shapes are skinny (m = 32..128), so a CTA
// owns a 32 x 32 output tile and K is split across grid.z until the grid covers the 152 SMs;
// split partials are reduced in a second deterministic pass.
#include "common.cuh"

namespace pisco {

namespace {
constexpr int BM = 32, BN = 32, BK = 16;

template <typename T>
__global__ void __launch_bounds__(256) cgemm_kernel(char opA, char opB, int M, int N, int K,
                                                    cpx<T> alpha, const cpx<T>* __restrict__ A,
                                                    int lda, const cpx<T>* __restrict__ B, int ldb,
                                                    cpx<T> beta, cpx<T>* __restrict__ C, int ldc,
                                                    cpx<T>* __restrict__ ws, int kchunk) {
  using Cx = cpx<T>;
  __shared__ Cx As[BK][BM + 1];
  __shared__ Cx Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int r0 = blockIdx.y * BM, c0 = blockIdx.x * BN;
  const int kbeg = blockIdx.z * kchunk;
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
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int gr = r0 + ty * 2 + i, gc = c0 + tx * 2 + j;
      if (gr >= M || gc >= N) continue;
      if (gridDim.z == 1) {
        Cx out = cmul(alpha, acc[i][j]);
        if (beta.x != T(0) || beta.y != T(0)) out = cadd(out, cmul(beta, C[(long long)gr * ldc + gc]));
        C[(long long)gr * ldc + gc] = out;
      } else {
        ws[((long long)blockIdx.z * M + gr) * N + gc] = acc[i][j];
      }
    }
}

template <typename T>
__global__ void splitk_reduce_kernel(int M, int N, int splits, cpx<T> alpha,
                                     const cpx<T>* __restrict__ ws, cpx<T> beta,
                                     cpx<T>* __restrict__ C, int ldc) {
  using Cx = cpx<T>;
  const long long total = (long long)M * N;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    Cx s = mk(T(0), T(0));
    for (int z = 0; z < splits; ++z) s = cadd(s, ws[(long long)z * total + idx]);
    const int gr = (int)(idx / N), gc = (int)(idx % N);
    Cx out = cmul(alpha, s);
    if (beta.x != T(0) || beta.y != T(0)) out = cadd(out, cmul(beta, C[(long long)gr * ldc + gc]));
    C[(long long)gr * ldc + gc] = out;
  }
}
}  // namespace

template <typename T>
cudaError_t cgemm(char opA, char opB, int M, int N, int K, cpx<T> alpha, const cpx<T>* A, int lda,
                  const cpx<T>* B, int ldb, cpx<T> beta, cpx<T>* C, int ldc, cpx<T>* ws,
                  size_t ws_elems, cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  const int tiles = ((M + BM - 1) / BM) * ((N + BN - 1) / BN);
  int splits = 1;
  const int kblocks = K > 0 ? (K + BK - 1) / BK : 1;
  if (ws != nullptr) {
    splits = (2 * 152 + tiles - 1) / tiles;
    if (splits > kblocks) splits = kblocks;
    if (splits > 64) splits = 64;
    while (splits > 1 && (size_t)splits * M * N > ws_elems) --splits;
    if (splits < 1) splits = 1;
  }
  const int kchunk = ((kblocks + splits - 1) / splits) * BK;
  splits = K > 0 ? (K + kchunk - 1) / kchunk : 1;
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, splits);
  cgemm_kernel<T><<<grid, 256, 0, st>>>(opA, opB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, ws,
                                        kchunk);
  ++g_launches;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || splits == 1) return e;
  long long total = (long long)M * N;
  long long blocks = (total + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  splitk_reduce_kernel<T><<<(unsigned)blocks, 256, 0, st>>>(M, N, splits, alpha, ws, beta, C, ldc);
  ++g_launches;
  return cudaGetLastError();
}

template cudaError_t cgemm<float>(char, char, int, int, int, float2, const float2*, int, const float2*,
                                  int, float2, float2*, int, float2*, size_t, cudaStream_t);
template cudaError_t cgemm<double>(char, char, int, int, int, double2, const double2*, int,
                                   const double2*, int, double2, double2*, int, double2*, size_t,
                                   cudaStream_t);

}  // namespace pisco
