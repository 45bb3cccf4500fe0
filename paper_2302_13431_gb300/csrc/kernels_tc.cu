// Dense complex GEMM on the 5th-generation tensor cores: tcgen05.mma with TF32 operands from
// shared memory and the FP32 accumulator in tensor memory (TMEM).
//
//   C = alpha * A * op(B) + beta * C   (+ diag_val on columns c with c % diag_stride == 0,
//                                          c < diag_limit)
//   A: M x K complex64, row-major (lda), optionally with every column k scaled by kscale[k];
//   op(B) = B (K x N row-major, ldb) or conj(Bs^T) with Bs N x K row-major (ldb).
//
// Complex products as one real GEMM.  Along K, a complex64 row of A is already the interleaved
// real row A' = [Re a_0, Im a_0, Re a_1, Im a_1, ...].  For each output column c the B operand
// holds two real rows, [Re b_0, -Im b_0, ...] (accumulator column c: Re C) and
// [Im b_0, Re b_0, ...] (accumulator column 32 + c: Im C).  A CTA owns a 128 x 32 complex tile
// of C: one M = 128, N = 64 accumulator of 64 TMEM columns.
//
// Precision (the split-precision products of the G(x) assembly and the eigensolver block
// products): every FP32 operand x is split into a TF32 head h = rna(x) and a TF32 tail
// t = rna(x - h); NT = 3 issues h*h + h*t + t*h (relative error ~2^-21, close to FP32), NT = 1
// issues h*h only (~2^-11).  Accumulation is FP32 in TMEM.
//
// Data movement: each K step stages 16 complex columns (32 real) of A and B.  128 threads load
// them from global memory (L2-resident operands; 32-byte sectors fully used), split them and
// store them in the canonical no-swizzle K-major layout: 8-row x 16-byte core matrices,
// 128 contiguous bytes each, adjacent in K at 128 B (LBO) and in M/N at 1024 B (SBO).  Each
// group of 8 threads writes one whole core matrix, so the 16-byte stores are bank-conflict
// free.  Two stage buffers: the loads of step s+1 overlap the MMAs of step s; a stage buffer is
// rewritten only after the tcgen05.commit of the MMAs that read it has arrived on its mbarrier.
// Every wait is bounded; on expiry the kernel flags `err` and still frees its TMEM.
#include <stdint.h>

#include "common.cuh"

namespace pisco {

namespace {

constexpr int TC_BM = 128;       // rows of C per CTA = TMEM lanes
constexpr int TC_BN = 32;        // complex columns of C per CTA (64 accumulator columns)
constexpr int TC_BKC = 16;       // complex K per stage (32 real, 8 core matrices of 4 TF32)
constexpr int TC_THREADS = 128;  // 4 warps: warp w reads TMEM lanes 32w..32w+31
constexpr uint32_t A_BYTES = TC_BM * 2 * TC_BKC * 4;      // 16384
constexpr uint32_t B_BYTES = 2 * TC_BN * 2 * TC_BKC * 4;  // 8192
constexpr uint32_t CORE_LBO = 128;                        // next core matrix along K
constexpr uint32_t CORE_SBO = 8 * 128;                    // next 8-row group along M / N
constexpr uint32_t TMEM_COLS = 64;
constexpr long long kWaitCycles = 4000000000ll;           // ~2 s at 2 GHz

// instruction descriptor, kind::tf32: D FP32 (bits 4-5 = 1), A and B TF32 (bits 7-9, 10-12 = 2),
// both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28
constexpr uint32_t IDESC_TF32_M128_N64 =
    (1u << 4) | (2u << 7) | (2u << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor: start >> 4 (bits 0-13), LBO >> 4 (16-29), SBO >> 4 (32-45),
// descriptor version 1 (bits 46-47), base offset 0, no swizzle (bits 61-63 = 0)
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait for the completion of the phase with the given parity
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > kWaitCycles) return false;
  }
  return true;
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

// 32 lanes x 32 consecutive 32-bit TMEM columns -> 32 registers per thread
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
        "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
        "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// TF32 head of x, rounded to nearest (ties away from zero) on the 13 dropped mantissa bits
__device__ __forceinline__ float tf32_head(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

struct TcArgs {
  int M, N, K;
  const float2* A;
  int lda;
  const float* kscale;
  const float2* B;
  int ldb;
  int opB;  // 0: B[k * ldb + n]; 1: conj(B[n * ldb + k])
  float2* C;
  int ldc;
  float2 alpha, beta;
  float diag_val;
  int diag_stride, diag_limit;
  int* err;
};

// two consecutive complex values (k, k + 1) of row `row` of a row-major complex array, zero
// outside rows < nrows and columns < ncols
__device__ __forceinline__ float4 load_pair(const float2* __restrict__ p, int ld, int row, int k,
                                            int nrows, int ncols, bool vec) {
  if (row >= nrows || k >= ncols) return make_float4(0.f, 0.f, 0.f, 0.f);
  const float2* q = p + (long long)row * ld + k;
  if (vec && k + 1 < ncols) return __ldg(reinterpret_cast<const float4*>(q));
  const float2 a = __ldg(q);
  const float2 b = (k + 1 < ncols) ? __ldg(q + 1) : make_float2(0.f, 0.f);
  return make_float4(a.x, a.y, b.x, b.y);
}

__device__ __forceinline__ float2 load_one(const float2* __restrict__ p, int ld, int row, int col,
                                           int nrows, int ncols) {
  if (row >= nrows || col >= ncols) return make_float2(0.f, 0.f);
  return __ldg(p + (long long)row * ld + col);
}

// one 16-byte core-matrix row: head to `hi`, tail to `lo` (NT == 3)
template <int NT>
__device__ __forceinline__ void put_row(unsigned char* hi, unsigned char* lo, uint32_t off, float4 v) {
  float4 h = make_float4(tf32_head(v.x), tf32_head(v.y), tf32_head(v.z), tf32_head(v.w));
  *reinterpret_cast<float4*>(hi + off) = h;
  if (NT == 3) {
    float4 t = make_float4(tf32_head(v.x - h.x), tf32_head(v.y - h.y), tf32_head(v.z - h.z),
                           tf32_head(v.w - h.w));
    *reinterpret_cast<float4*>(lo + off) = t;
  }
}

// byte offset of the core-matrix row holding (row, 16-byte column j) of a 32-real-wide tile
__device__ __forceinline__ uint32_t core_off(int row, int j) {
  return (uint32_t)(((row >> 3) * 8 + j) * 128 + (row & 7) * 16);
}

template <int NT>
__global__ void __launch_bounds__(TC_THREADS, 1) tc_cgemm_kernel(TcArgs g) {
  constexpr uint32_t STAGE = (NT == 3 ? 2u : 1u) * (A_BYTES + B_BYTES);
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw_s = smem_u32(smem_raw);
  const uint32_t base_s = (raw_s + 1023u) & ~1023u;
  unsigned char* base = smem_raw + (base_s - raw_s);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(base + 2 * STAGE);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(base + 2 * STAGE + 16);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * TC_BM, n0 = blockIdx.x * TC_BN;
  const int M = g.M, N = g.N, K = g.K;
  const int nkb = (K + TC_BKC - 1) / TC_BKC;
  const bool a_vec = ((reinterpret_cast<uintptr_t>(g.A) & 15) == 0) && ((g.lda & 1) == 0);
  const bool b_vec = ((reinterpret_cast<uintptr_t>(g.B) & 15) == 0) && ((g.ldb & 1) == 0);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(smem_u32(&mbar[0]), 1);
    mbar_init(smem_u32(&mbar[1]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  bool ok = true;

  for (int kb = 0; kb < nkb; ++kb) {
    const int s = kb & 1;
    const int k0 = kb * TC_BKC;
    unsigned char* aH = base + s * STAGE;
    unsigned char* aL = aH + A_BYTES;
    unsigned char* bH = aH + (NT == 3 ? 2 * A_BYTES : A_BYTES);
    unsigned char* bL = bH + B_BYTES;
    // global -> registers (overlaps the MMAs still reading the other stage)
    float4 av[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int id = tid + TC_THREADS * i;  // rowlo = id & 7, j = (id >> 3) & 7, rowhi = id >> 6
      const int row = (id >> 6) * 8 + (id & 7), j = (id >> 3) & 7;
      const int k = k0 + 2 * j;
      float4 v = load_pair(g.A, g.lda, m0 + row, k, M, K, a_vec);
      if (g.kscale) {
        const float w0 = (k < K) ? __ldg(g.kscale + k) : 0.f;
        const float w1 = (k + 1 < K) ? __ldg(g.kscale + k + 1) : 0.f;
        v.x *= w0; v.y *= w0; v.z *= w1; v.w *= w1;
      }
      av[i] = v;
    }
    float4 bre[2], bim[2];
    int brow[2], bj[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int id = tid + TC_THREADS * i;
      if (g.opB == 0) {
        const int c = id & 31, j = id >> 5;
        const int k = k0 + 2 * j;
        const float2 b0 = load_one(g.B, g.ldb, k, n0 + c, K, N);
        const float2 b1 = load_one(g.B, g.ldb, k + 1, n0 + c, K, N);
        bre[i] = make_float4(b0.x, -b0.y, b1.x, -b1.y);
        bim[i] = make_float4(b0.y, b0.x, b1.y, b1.x);
        brow[i] = c;
        bj[i] = j;
      } else {
        const int c = (id >> 6) * 8 + (id & 7), j = (id >> 3) & 7;
        const float4 sv = load_pair(g.B, g.ldb, n0 + c, k0 + 2 * j, N, K, b_vec);
        bre[i] = sv;  // (Re b, -Im b) with b = conj(s)
        bim[i] = make_float4(-sv.y, sv.x, -sv.w, sv.z);
        brow[i] = c;
        bj[i] = j;
      }
    }
    // the MMAs issued two steps ago read this stage buffer: wait for their commit
    if (kb >= 2 && ok) ok = mbar_wait(smem_u32(&mbar[s]), (uint32_t)(((kb - 2) >> 1) & 1));
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int id = tid + TC_THREADS * i;
      const int row = (id >> 6) * 8 + (id & 7), j = (id >> 3) & 7;
      put_row<NT>(aH, aL, core_off(row, j), av[i]);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      put_row<NT>(bH, bL, core_off(brow[i], bj[i]), bre[i]);
      put_row<NT>(bH, bL, core_off(brow[i] + TC_BN, bj[i]), bim[i]);
    }
    // generic-proxy shared stores -> visible to the tensor core (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t aHs = smem_u32(aH), aLs = smem_u32(aL), bHs = smem_u32(bH), bLs = smem_u32(bL);
#pragma unroll
      for (int j = 0; j < 4; ++j) {  // one MMA covers K = 8 TF32 = 2 core matrices
        const uint64_t ah = smem_desc(aHs + 256 * j, CORE_LBO, CORE_SBO);
        const uint64_t bh = smem_desc(bHs + 256 * j, CORE_LBO, CORE_SBO);
        mma_tf32(tmem, ah, bh, IDESC_TF32_M128_N64, (kb > 0 || j > 0) ? 1u : 0u);
        if (NT == 3) {
          const uint64_t al = smem_desc(aLs + 256 * j, CORE_LBO, CORE_SBO);
          const uint64_t bl = smem_desc(bLs + 256 * j, CORE_LBO, CORE_SBO);
          mma_tf32(tmem, ah, bl, IDESC_TF32_M128_N64, 1u);
          mma_tf32(tmem, al, bh, IDESC_TF32_M128_N64, 1u);
        }
      }
      mma_commit(smem_u32(&mbar[s]));
    }
  }
  // the last commit covers every MMA issued before it
  if (nkb > 0) {
    const int last = nkb - 1;
    if (ok) ok = mbar_wait(smem_u32(&mbar[last & 1]), (uint32_t)((last >> 1) & 1));
    if (!ok) {
      if (g.err) atomicOr(g.err, 16);
      mbar_wait(smem_u32(&mbar[last & 1]), (uint32_t)((last >> 1) & 1));  // once more, bounded
    }
  }
  tc_fence_after();
  // TMEM -> registers -> shared tile [128][33] (stage buffers are free now)
  float2* tile = reinterpret_cast<float2*>(base);
  {
    const int row = warp * 32 + lane;
    uint32_t r[32];
    const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
    if (nkb > 0) {
      tmem_ld32(tl, r);
    } else {
#pragma unroll
      for (int c = 0; c < 32; ++c) r[c] = 0u;
    }
#pragma unroll
    for (int c = 0; c < 32; ++c) tile[row * 33 + c].x = __uint_as_float(r[c]);
    if (nkb > 0) {
      tmem_ld32(tl + 32, r);
    }
#pragma unroll
    for (int c = 0; c < 32; ++c) tile[row * 33 + c].y = __uint_as_float(r[c]);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
  // coalesced epilogue: warp w writes rows w, w + 4, ...; lane = column
  const bool has_beta = (g.beta.x != 0.f || g.beta.y != 0.f);
  for (int rr = warp; rr < TC_BM; rr += 4) {
    const int gm = m0 + rr, gn = n0 + lane;
    if (gm >= M || gn >= N) continue;
    const float2 acc = tile[rr * 33 + lane];
    float2 out = make_float2(g.alpha.x * acc.x - g.alpha.y * acc.y, g.alpha.x * acc.y + g.alpha.y * acc.x);
    float2* cp = g.C + (long long)gm * g.ldc + gn;
    if (has_beta) {
      const float2 c = *cp;
      out.x += g.beta.x * c.x - g.beta.y * c.y;
      out.y += g.beta.x * c.y + g.beta.y * c.x;
    }
    if (g.diag_stride > 0 && gn < g.diag_limit && gn % g.diag_stride == 0) out.x += g.diag_val;
    *cp = out;
  }
}

template <int NT>
size_t tc_smem_bytes() {
  const size_t stage = (NT == 3 ? 2u : 1u) * (A_BYTES + B_BYTES);
  return 2 * stage + 1024 + 64;
}

}  // namespace

cudaError_t tc_gemm_prepare() {
  cudaError_t e = cudaFuncSetAttribute(tc_cgemm_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)tc_smem_bytes<3>());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(tc_cgemm_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)tc_smem_bytes<1>());
}

cudaError_t tc_cgemm(int nterms, int M, int N, int K, float2 alpha, const float2* A, int lda,
                     const float* kscale, const float2* B, int ldb, int opB, float2 beta, float2* C,
                     int ldc, float diag_val, int diag_stride, int diag_limit, int* err, cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  TcArgs g{M, N, K < 0 ? 0 : K, A, lda, kscale, B, ldb, opB, C, ldc, alpha, beta,
           diag_val, diag_stride, diag_limit, err};
  dim3 grid((N + TC_BN - 1) / TC_BN, (M + TC_BM - 1) / TC_BM);
  if (nterms == 1) {
    tc_cgemm_kernel<1><<<grid, TC_THREADS, tc_smem_bytes<1>(), st>>>(g);
  } else {
    tc_cgemm_kernel<3><<<grid, TC_THREADS, tc_smem_bytes<3>(), st>>>(g);
  }
  ++g_launches;
  return cudaGetLastError();
}

}  // namespace pisco
