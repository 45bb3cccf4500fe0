// Dense complex GEMM on the tensor cores (tcgen05, TF32 with an FP32 accumulator in TMEM), fed by
// TMA, in split precision.
//
//   C = alpha * A * op(B) + beta * C  (+ diag_val on columns c % diag_stride == 0, c < diag_limit)
//
// The operands are split once, in global memory, into the real K-major layout the tensor core
// reads (tc2_split_a / tc2_split_b): A' [M][K2p] with the complex row interleaved (Re, Im),
// B' [2 Np][K2p] with, per 32-column tile t, rows 64t..64t+31 = [Re b, -Im b] (real part of
// C) and rows 64t+32..64t+63 = [Im b, Re b] (imaginary part); each as a TF32 head array and a
// TF32 tail array.  A GEMM then moves no data through registers: per K step of 32 real columns
// one thread issues the TMA loads of the step's four tiles (head/tail of A and B, 128-byte
// swizzled) into a 2- or 4-stage ring, another thread issues the tcgen05.mma instructions (TF32,
// FP32 accumulator 128 x 64 in TMEM) and releases each stage through tcgen05.commit, and the
// 4 warps read the accumulator back for the epilogue.  K may be split across gridDim.z; the
// partial tiles are then summed in a fixed order by a second kernel (deterministic).
//
// Every mbarrier wait is bounded; on expiry the kernel sets bit 16 of *err, stops issuing and
// still frees its TMEM.
//
// A variant (CONV) reads A as plain FP32 complex rows instead of split arrays: TMA brings the
// FP32 tile into the stage, four converter warps (one per TMEM lane quarter) read one row each,
// split it into TF32 head and tail (the arithmetic of the split kernels) and store both into
// tensor memory, from where the MMAs read A (lane = row, K along the columns).  A then crosses HBM
// at 8 instead of 16 bytes per complex entry and needs no separate split pass, and the split A
// takes no shared memory: the tensor core reads only B from shared memory, the converters read
// the FP32 tile once and write nothing there (the stage ring is bound by shared-memory bandwidth
// otherwise).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <atomic>
#include <mutex>

#include "common.cuh"

namespace pisco {

namespace {

constexpr int BM = 128;           // rows of C per CTA (TMEM lanes)
constexpr int BNC = 32;           // complex columns of one B' tile (64 real rows)
constexpr int BK = 32;            // real K per stage (128 bytes of FP32: one swizzle row)
constexpr uint32_t A_TILE = BM * BK * 4;        // 16384
constexpr uint32_t B_TILE = 2 * BNC * BK * 4;   // 8192 per B' tile; a CTA covers WT tiles
constexpr long long kWait = 4000000000ll;       // ~2 s at 2 GHz
constexpr long long kWaitStalled = 20000000ll;  // ~10 ms: the wait limit while loads are withheld
// instruction descriptor: FP32 accumulator, TF32 A and B, both K-major, N = 64 * WT, M = 128
template <int WT>
__device__ __forceinline__ constexpr uint32_t idesc() {
  return (1u << 4) | (2u << 7) | (2u << 10) | (((64u * WT) >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// K-major, 128-byte swizzle: start >> 4, LBO field 1 (unused for this layout), SBO 1024 B
// (next 8-row group), descriptor version 1, layout type 2 (SWIZZLE_128B)
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | (1ull << 16) | ((uint64_t)(1024u >> 4) << 32) | (1ull << 46) |
         (2ull << 61);
}

__device__ __forceinline__ void bar_init(uint32_t b, uint32_t n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(b), "r"(n) : "memory");
}
__device__ __forceinline__ bool bar_try(uint32_t b, uint32_t par) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(b), "r"(par)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool bar_wait(uint32_t b, uint32_t par, long long limit) {
  const long long t0 = clock64();
  while (!bar_try(b, par))
    if (clock64() - t0 > limit) return false;
  return true;
}
__device__ __forceinline__ void bar_expect_tx(uint32_t b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tma_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y)
      : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
template <int WT>
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc<WT>()), "r"(acc)
      : "memory");
}
// A from tensor memory (lane = row of A, K in consecutive 32-bit columns), B from shared memory
template <int WT>
__device__ __forceinline__ void mma_ts(uint32_t d, uint32_t a_tmem, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d),
      "r"(a_tmem), "l"(b), "r"(idesc<WT>()), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void commit(uint32_t b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(b) : "memory");
}
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

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
      "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, "
      "%17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
      "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]),
      "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]),
      "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
}
__device__ __forceinline__ float4 ld_shared_f4(uint32_t a) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
  return v;
}

__device__ __forceinline__ float head(float x) { return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u); }

struct Args {
  int M, N, K2;   // K2 = 2K (real columns of A' and B')
  int kpb;        // K steps per split (gridDim.z splits)
  float2* C;
  int ldc;
  float2 alpha, beta;
  float diag_val;
  int diag_stride, diag_limit;
  float2* ws;     // [splits][M][N] partial products when gridDim.z > 1 (split-K)
  int* err;
  int batched;    // 1: gridDim.z indexes independent products (no split-K)
  int b_rows;     // B' rows per batch item (2 Np)
  long long c_stride;  // C elements per batch item
  int a_rows;     // 0: every batch item shares A'; else A' rows per batch item (A' per item)
  float2* const* c_tab;  // non-null: C of batch item z is c_tab[z / c_div] + (z % c_div) * c_stride
  int c_div;
  int splits;     // K splits (gridDim.z = items * splits); partials of item b, split z at
                  // ws + (b * splits + z) * M * N
  // row groups (rg > 0, one product over all items' rows): row r is (item, y, q) with
  // item = r / rg_rows, y = (r % rg_rows) / rg, q = r % rg, written to
  // (c_tab[item] or C + item * c_stride) + q * rg_plane + y * ldc; rg_norm: every column of a
  // group of rg rows (one pixel's coils) divided by its 2-norm
  int rg, rg_rows, rg_norm;
  long long rg_plane;
  long long wait_limit;  // clock cycles a bounded mbarrier wait may take
  int no_loads;   // test hook: the producer issues no loads, so the waits on them expire
};

template <int NT, bool CONV, int WT>
__host__ __device__ constexpr uint32_t stage_bytes() {
  // split operands: [A head][A tail][B head][B tail]; CONV: [A fp32][B head][B tail] (the split A
  // goes to tensor memory)
  return CONV ? A_TILE + 2u * WT * B_TILE : (NT == 3 ? 2u : 1u) * (A_TILE + WT * B_TILE);
}

__host__ __device__ constexpr uint32_t pow2_cols(uint32_t n) { return n <= 32 ? 32 : 2 * pow2_cols((n + 1) / 2); }

// One CTA: a 128 x (32 WT) complex tile of C, accumulated in 64 WT TMEM columns (columns
// 64h .. 64h+31 hold Re, 64h+32 .. 64h+63 Im of the complex columns 32h .. 32h+31).
template <int NT, int STAGES, bool CONV, int WT>
__global__ void __launch_bounds__(CONV ? 256 : 128, 1) tc2_kernel(const __grid_constant__ CUtensorMap tAh,
                                                     const __grid_constant__ CUtensorMap tAl,
                                                     const __grid_constant__ CUtensorMap tBh,
                                                     const __grid_constant__ CUtensorMap tBl, Args g) {
  static_assert(!CONV || NT == 3, "the converting variant splits A into head and tail");
  static_assert(STAGES * stage_bytes<NT, CONV, WT>() >= 128u * (BNC * WT + 1) * 8u, "epilogue tile exceeds the ring");
  constexpr uint32_t STAGE = stage_bytes<NT, CONV, WT>();
  // the row-group epilogue keeps scales and row offsets beside the tile: converting variants whose
  // ring holds all three (the host launches row-grouped products on those only)
  constexpr bool RG_OK = CONV && STAGES * STAGE >= 128u * (BNC * WT + 1) * 8u + 128u * BNC * WT * 4u + 128u * 8u;
  constexpr uint32_t A_TAIL = A_TILE;                        // split A: head at 0, tail here
  constexpr uint32_t B_OFF = CONV ? A_TILE : (NT == 3 ? 2u : 1u) * A_TILE;
  constexpr uint32_t BT = WT * B_TILE;                      // B head (tail) bytes per stage
  constexpr uint32_t ACC_COLS = 64 * WT;
  // CONV: the split A of stage s in TMEM columns ACC_COLS + 64 s (head) and + 32 (tail)
  constexpr uint32_t TMEM_COLS = CONV ? pow2_cols(ACC_COLS + 64 * STAGES) : ACC_COLS;
  static_assert(TMEM_COLS <= 512, "tensor memory holds 512 columns");
  // warps: 0 producer, 1 MMA issuer, (CONV) 4-7 converters (TMEM lane quarter = warp - 4);
  // warps 0-3 read the accumulator (TMEM lane quarter = warp), all of them share the epilogue
  constexpr int NTHR = CONV ? 256 : 128, NWARP = NTHR / 32;
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = su32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* gbase = smem_raw + (base - raw);
  // full[S], empty[S], accum, (CONV) conv[S]
  uint64_t* bars = reinterpret_cast<uint64_t*>(gbase + STAGES * STAGE);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gbase + STAGES * STAGE + (3 * STAGES + 1) * 8);
  const uint32_t full0 = su32(&bars[0]), empty0 = su32(&bars[STAGES]), accum = su32(&bars[2 * STAGES]);
  const uint32_t conv0 = su32(&bars[2 * STAGES + 1]);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BNC * WT;
  const int total = (g.K2 + BK - 1) / BK;
  const int zb = (int)blockIdx.z / g.splits;                // batch item
  const int kb0 = ((int)blockIdx.z % g.splits) * g.kpb;    // first K step of this split
  const int nk = min(g.kpb, total - kb0);
  const int brow0 = zb * g.b_rows;                          // this item's rows of B'
  const int arow0 = zb * g.a_rows + m0;                     // this tile's first row of A'
  float2* Cb = g.c_tab ? g.c_tab[zb / g.c_div] + (long long)(zb % g.c_div) * g.c_stride
                       : g.C + (long long)zb * g.c_stride;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) {
      bar_init(full0 + 8 * s, 1);
      bar_init(empty0 + 8 * s, 1);
      if (CONV) bar_init(conv0 + 8 * s, 128);  // the converter warps
    }
    bar_init(accum, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  bool ok = true;

  if (warp == 0 && lane == 0 && nk > 0 && !g.no_loads) {
    // producer: TMA loads of the four tiles of every K step into the stage ring
    for (int i = 0; i < nk && ok; ++i) {
      const int s = i % STAGES, c = i / STAGES;
      if (i >= STAGES) ok = bar_wait(empty0 + 8 * s, (uint32_t)((c - 1) & 1), g.wait_limit);
      if (!ok) break;
      const uint32_t st = base + s * STAGE;
      const uint32_t fb = full0 + 8 * s;
      const int kx = (kb0 + i) * BK;
      if (CONV) {
        bar_expect_tx(fb, A_TILE + 2 * BT);
        tma_2d(st, &tAh, kx, arow0, fb);  // the FP32 tile
      } else {
        bar_expect_tx(fb, STAGE);
        tma_2d(st, &tAh, kx, arow0, fb);
        if (NT == 3) tma_2d(st + A_TILE, &tAl, kx, arow0, fb);
      }
      const uint32_t sb = st + B_OFF;
      tma_2d(sb, &tBh, kx, brow0 + 2 * n0, fb);
      if (NT == 3) tma_2d(sb + BT, &tBl, kx, brow0 + 2 * n0, fb);
    }
  } else if (CONV && warp >= 4 && nk > 0) {
    // converters: row r of the FP32 tile (128-byte swizzled: 16-byte chunk ch of row r at chunk
    // ch ^ (r & 7)) -> TF32 head and tail in TMEM lane r, K in consecutive columns; the waits are
    // warp-uniform, so the warp-collective TMEM stores run in every lane or in none
    const int q = warp - 4, r = 32 * q + lane;
    const uint32_t tq = tmem + ((uint32_t)(32 * q) << 16) + ACC_COLS;
    for (int i = 0; i < nk && ok; ++i) {
      const int s = i % STAGES, c = i / STAGES;
      ok = __all_sync(0xffffffffu, bar_wait(full0 + 8 * s, (uint32_t)(c & 1), g.wait_limit));
      if (!ok) break;
      const uint32_t row = base + s * STAGE + r * 128;
      uint32_t hd[32], tl[32];
#pragma unroll
      for (int ch = 0; ch < 8; ++ch) {
        const float4 v = ld_shared_f4(row + ((uint32_t)(ch ^ (r & 7)) << 4));
        const float e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float h = head(e[u]);
          hd[4 * ch + u] = __float_as_uint(h);
          tl[4 * ch + u] = __float_as_uint(head(e[u] - h));
        }
      }
      tmem_st32(tq + 64 * s, hd);
      tmem_st32(tq + 64 * s + 32, tl);
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      fence_before();
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(conv0 + 8 * s) : "memory");
    }
  } else if (warp == 1 && lane == 0 && nk > 0) {
    // MMA issuer: 4 MMAs of K = 8 per stage (x3 for the head/tail split)
    for (int i = 0; i < nk && ok; ++i) {
      const int s = i % STAGES, c = i / STAGES;
      ok = bar_wait((CONV ? conv0 : full0) + 8 * s, (uint32_t)(c & 1), g.wait_limit);
      if (!ok) break;
      fence_after();
      const uint32_t st = base + s * STAGE;
      const uint32_t sb = st + B_OFF;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint64_t bh = desc_sw128(sb + 32 * j);
        if (CONV) {
          const uint32_t ah = tmem + ACC_COLS + 64 * s + 8 * j;
          mma_ts<WT>(tmem, ah, bh, (i > 0 || j > 0) ? 1u : 0u);
          mma_ts<WT>(tmem, ah, desc_sw128(sb + BT + 32 * j), 1u);
          mma_ts<WT>(tmem, ah + 32, bh, 1u);
        } else {
          const uint64_t ah = desc_sw128(st + 32 * j);
          mma<WT>(tmem, ah, bh, (i > 0 || j > 0) ? 1u : 0u);
          if (NT == 3) {
            mma<WT>(tmem, ah, desc_sw128(sb + BT + 32 * j), 1u);
            mma<WT>(tmem, desc_sw128(st + A_TAIL + 32 * j), bh, 1u);
          }
        }
      }
      commit(empty0 + 8 * s);
    }
    commit(accum);
  }
  __syncwarp();
  if (nk > 0) {
    if (!bar_wait(accum, 0, g.wait_limit)) ok = false;
  }
  if (!ok && g.err) atomicOr(g.err, 16);
  fence_after();
  // accumulator -> registers -> shared tile [128][TS] (the stage ring is free: all MMAs done)
  constexpr int TS = BNC * WT + 1;
  float2* tile = reinterpret_cast<float2*>(gbase);
  if (warp < 4) {
    const int row = warp * 32 + lane;
    uint32_t r[32];
    const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
    for (int h = 0; h < WT; ++h) {
      if (nk > 0) tmem_ld32(tl + 64 * h, r);
      else
#pragma unroll
        for (int c = 0; c < 32; ++c) r[c] = 0u;
#pragma unroll
      for (int c = 0; c < 32; ++c) tile[row * TS + 32 * h + c].x = __uint_as_float(r[c]);
      if (nk > 0) tmem_ld32(tl + 64 * h + 32, r);
#pragma unroll
      for (int c = 0; c < 32; ++c) tile[row * TS + 32 * h + c].y = __uint_as_float(r[c]);
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
  if (g.rg > 0 && !RG_OK) {
    if (tid == 0 && g.err) atomicOr(g.err, 16);
    return;
  }
  if (RG_OK && g.rg > 0) {
    float* scl = reinterpret_cast<float*>(gbase + (size_t)BM * TS * sizeof(float2));  // [BM / rg][32 WT]
    long long* rowoff = reinterpret_cast<long long*>(scl + BM * BNC * WT);                // [BM]
    if (tid < BM) {  // each thread places one row: (item, y, q) -> offset from the item's output
      const int gm = m0 + tid;
      long long off = -1;
      if (gm < g.M) {
        const int item = gm / g.rg_rows, rem = gm % g.rg_rows;
        off = (long long)item * (1ll << 40) + (long long)(rem % g.rg) * g.rg_plane + (long long)(rem / g.rg) * g.ldc;
      }
      rowoff[tid] = off;
    }
    if (g.rg_norm) {
      const int ng = BM / g.rg;
      for (int e = tid; e < ng * BNC * WT; e += NTHR) {
        const int gi = e / (BNC * WT), c = e % (BNC * WT);
        float n2 = 0.f;
        for (int r = 0; r < g.rg; ++r) {
          const float2 v = tile[(gi * g.rg + r) * TS + c];
          n2 = fmaf(v.x, v.x, fmaf(v.y, v.y, n2));
        }
        scl[e] = n2 > 0.f ? rsqrtf(n2) : 0.f;
      }
      __syncthreads();
    }
    __syncthreads();
    for (int e = warp; e < BM * WT; e += NWARP) {
      const int rr = e / WT, gn = n0 + 32 * (e % WT) + lane;
      const long long ro = rowoff[rr];
      if (ro < 0 || gn >= g.N) continue;
      const int item = (int)(ro >> 40);
      float2* base = (g.c_tab ? g.c_tab[item] : g.C + (long long)item * g.c_stride) + (ro & ((1ll << 40) - 1));
      float2 v = tile[rr * TS + (gn - n0)];
      if (g.rg_norm) {
        const float sc = scl[(rr / g.rg) * (BNC * WT) + (gn - n0)];
        v.x *= sc;
        v.y *= sc;
      }
      __stcs(base + gn, v);
    }
    return;
  }
  if (g.splits > 1) {  // raw partial tile
    float2* out = g.ws + (long long)blockIdx.z * g.M * g.N;
    for (int e = warp; e < BM * WT; e += NWARP) {
      const int rr = e / WT, gm = m0 + rr, gn = n0 + 32 * (e % WT) + lane;
      if (gm < g.M && gn < g.N) out[(long long)gm * g.N + gn] = tile[rr * TS + (gn - n0)];
    }
    return;
  }
  const bool has_beta = (g.beta.x != 0.f || g.beta.y != 0.f);
  for (int e = warp; e < BM * WT; e += NWARP) {
    const int rr = e / WT, gm = m0 + rr, gn = n0 + 32 * (e % WT) + lane;
    if (gm >= g.M || gn >= g.N) continue;
    const float2 a = tile[rr * TS + (gn - n0)];
    float2 o = make_float2(g.alpha.x * a.x - g.alpha.y * a.y, g.alpha.x * a.y + g.alpha.y * a.x);
    float2* cp = Cb + (long long)gm * g.ldc + gn;
    if (has_beta) {
      const float2 c = *cp;
      o.x += g.beta.x * c.x - g.beta.y * c.y;
      o.y += g.beta.x * c.y + g.beta.y * c.x;
    }
    if (g.diag_stride > 0 && gn < g.diag_limit && gn % g.diag_stride == 0) o.x += g.diag_val;
    *cp = o;
  }
}

// Row-tile persistent form of the converting, row-grouped product, for K2 <= 128 (one 128-row
// tile of A covers the whole K): a CTA loads its A tile by TMA, four converter warps split it into
// TF32 head and tail in tensor memory (lane = row, K along the columns, one barrier per K step so
// the MMAs start on the first), and the CTA runs over every 64-column tile of C with B' streamed
// through a four-stage ring and the accumulator double-buffered in TMEM (2 x 128 columns), so the
// epilogue of one column tile overlaps the MMAs of the next.  The FP32 A buffer is refilled with
// the next row tile as soon as it is converted; CTAs loop over row tiles (grid <= SM count).
// Warps: 0 producer, 1 MMA issuer, 4-7 epilogue (TMEM lane quarter = warp - 4), 8-11 converters
// (lane quarter = warp - 8).  Epilogue: each warp's 32 rows; the per-pixel norm over groups of rg
// rows (8 <= rg <= 32, so a group never leaves its warp) through a per-warp shared tile; the
// stores go through the same tile transposed, so a store instruction writes two 128-byte runs of
// one output row each.
namespace rows {
constexpr int KSMAX = 4;                               // K steps of 32 real columns: K2 <= 128
constexpr int S = 4;                                   // B' ring stages
constexpr int NTHR = 384;
constexpr uint32_t BT = 2 * B_TILE;                    // one 64-column B' tile (head or tail)
constexpr uint32_t RSTAGE = 2 * BT;                    // head + tail
constexpr uint32_t R_OFF = KSMAX * A_TILE;             // after the FP32 A tile
constexpr uint32_t STG_OFF = R_OFF + S * RSTAGE;       // per warp: [32][17] float2, or [32][33] float
constexpr uint32_t STG_WARP = 32 * 17 * 8;
constexpr uint32_t SCL_OFF = STG_OFF + 4 * STG_WARP;   // per warp: [32 / rg][32] scales
constexpr uint32_t BAR_OFF = SCL_OFF + 4 * 128 * 4;
// afull, araw, aempty, done, aconv[KSMAX], bfull[S], bempty[S], accf[2], acce[2]
constexpr int NBAR = 4 + KSMAX + 2 * S + 4;
constexpr uint32_t TOTAL = BAR_OFF + NBAR * 8 + 16;
constexpr uint32_t TMEM_COLS = 512;                    // accumulators 0 / 128, split A from 256
constexpr uint32_t A_COL = 256;
static_assert(4 * STG_WARP >= 4 * 32 * 33 * 4, "norm tile exceeds the staging tile");
static_assert(A_COL + 64 * KSMAX <= TMEM_COLS, "split A exceeds tensor memory");
}  // namespace rows

__global__ void __launch_bounds__(rows::NTHR, 1) tc2_rows_kernel(const __grid_constant__ CUtensorMap tA,
                                                                 const __grid_constant__ CUtensorMap tBh,
                                                                 const __grid_constant__ CUtensorMap tBl, Args g) {
  using namespace rows;
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = su32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* gb = smem_raw + (base - raw);
  uint64_t* bars = reinterpret_cast<uint64_t*>(gb + BAR_OFF);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gb + BAR_OFF + NBAR * 8);
  const uint32_t afull = su32(&bars[0]), araw = su32(&bars[1]), aempty = su32(&bars[2]), done = su32(&bars[3]);
  const uint32_t aconv0 = su32(&bars[4]), bfull0 = su32(&bars[4 + KSMAX]), bempty0 = su32(&bars[4 + KSMAX + S]);
  const uint32_t accf0 = su32(&bars[4 + KSMAX + 2 * S]), acce0 = su32(&bars[6 + KSMAX + 2 * S]);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ks = (g.K2 + BK - 1) / BK;
  const int nct = (g.N + 63) / 64;
  const int ntiles = (g.M + BM - 1) / BM;
  const long long lim = g.wait_limit;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    bar_init(afull, 1);
    bar_init(araw, 128);
    bar_init(aempty, 1);
    bar_init(done, 1);
    for (int k = 0; k < KSMAX; ++k) bar_init(aconv0 + 8 * k, 128);
    for (int s = 0; s < S; ++s) {
      bar_init(bfull0 + 8 * s, 1);
      bar_init(bempty0 + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      bar_init(accf0 + 8 * b, 1);
      bar_init(acce0 + 8 * b, 4);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  bool ok = true;

  if (warp == 0) {
    if (lane == 0 && !g.no_loads) {
      // producer: per row tile, the FP32 A tile (once the previous one is converted), then B'
      // head and tail of every (column tile, K step) into the ring
      int it = 0, na = 0;
      for (int rt = blockIdx.x; rt < ntiles && ok; rt += gridDim.x) {
        if (na > 0 && !(ok = bar_wait(araw, (uint32_t)((na - 1) & 1), lim))) break;
        bar_expect_tx(afull, (uint32_t)ks * A_TILE);
        for (int kk = 0; kk < ks; ++kk) tma_2d(base + kk * A_TILE, &tA, kk * BK, rt * BM, afull);
        ++na;
        for (int ct = 0; ct < nct && ok; ++ct) {
          for (int kk = 0; kk < ks; ++kk) {
            const int s = it % S, c = it / S;
            if (it >= S && !(ok = bar_wait(bempty0 + 8 * s, (uint32_t)((c - 1) & 1), lim))) break;
            const uint32_t fb = bfull0 + 8 * s, sb = base + R_OFF + s * RSTAGE;
            bar_expect_tx(fb, RSTAGE);
            tma_2d(sb, &tBh, kk * BK, 128 * ct, fb);
            tma_2d(sb + BT, &tBl, kk * BK, 128 * ct, fb);
            ++it;
          }
        }
      }
      // every load this thread issued has landed before the CTA may exit (bounded)
      for (int j = it - S > 0 ? it - S : 0; j < it; ++j) bar_wait(bfull0 + 8 * (j % S), (uint32_t)((j / S) & 1), lim);
      if (na > 0) bar_wait(afull, (uint32_t)((na - 1) & 1), lim);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer: 4 x 3 MMAs (N = 128, K = 8, A from TMEM) per (column tile, K step) into
      // accumulator buffer tc & 1
      int it = 0, tc = 0, na = 0;
      bool issued = false;
      for (int rt = blockIdx.x; rt < ntiles && ok; rt += gridDim.x, ++na) {
        for (int ct = 0; ct < nct && ok; ++ct) {
          const int b = tc & 1, u = tc >> 1;
          if (tc >= 2 && !(ok = bar_wait(acce0 + 8 * b, (uint32_t)((u - 1) & 1), lim))) break;
          fence_after();
          const uint32_t d = tmem + 128u * b;
          for (int kk = 0; kk < ks; ++kk) {
            const int s = it % S, c = it / S;
            if (ct == 0 && !(ok = bar_wait(aconv0 + 8 * kk, (uint32_t)(na & 1), lim))) break;
            if (!(ok = bar_wait(bfull0 + 8 * s, (uint32_t)(c & 1), lim))) break;
            fence_after();
            const uint32_t sb = base + R_OFF + s * RSTAGE, ta = tmem + A_COL + 64 * kk;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const uint64_t bh = desc_sw128(sb + 32 * j);
              mma_ts<2>(d, ta + 8 * j, bh, (kk > 0 || j > 0) ? 1u : 0u);
              mma_ts<2>(d, ta + 8 * j, desc_sw128(sb + BT + 32 * j), 1u);
              mma_ts<2>(d, ta + 32 + 8 * j, bh, 1u);
            }
            issued = true;
            commit(bempty0 + 8 * s);
            ++it;
          }
          if (!ok) break;
          commit(accf0 + 8 * b);
          ++tc;
        }
        if (!ok) break;
        commit(aempty);  // the split A of this row tile may be overwritten once these retire
      }
      if (issued) {  // every MMA retired before TMEM is freed (bounded)
        commit(done);
        bar_wait(done, 0, lim);
      }
    }
  } else if (warp >= 8) {
    // converters: row r of the FP32 tile (128-byte swizzled: 16-byte chunk ch of row r at chunk
    // ch ^ (r & 7)) -> TF32 head and tail in TMEM lane r; waits warp-uniform, so the
    // warp-collective TMEM stores run in every lane or in none
    const int q = warp - 8, r = 32 * q + lane;
    const uint32_t tq = tmem + ((uint32_t)(32 * q) << 16) + A_COL;
    int na = 0;
    for (int rt = blockIdx.x; rt < ntiles && ok; rt += gridDim.x, ++na) {
      ok = __all_sync(0xffffffffu, bar_wait(afull, (uint32_t)(na & 1), lim));
      if (ok && na > 0) ok = __all_sync(0xffffffffu, bar_wait(aempty, (uint32_t)((na - 1) & 1), lim));
      if (!ok) break;
      fence_after();
      for (int kk = 0; kk < ks; ++kk) {
        const uint32_t row = base + kk * A_TILE + r * 128;
        uint32_t hd[32], tl[32];
#pragma unroll
        for (int ch = 0; ch < 8; ++ch) {
          const float4 v = ld_shared_f4(row + ((uint32_t)(ch ^ (r & 7)) << 4));
          const float e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float h = head(e[u]);
            hd[4 * ch + u] = __float_as_uint(h);
            tl[4 * ch + u] = __float_as_uint(head(e[u] - h));
          }
        }
        tmem_st32(tq + 64 * kk, hd);
        tmem_st32(tq + 64 * kk + 32, tl);
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        fence_before();
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(aconv0 + 8 * kk) : "memory");
      }
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(araw) : "memory");  // FP32 tile read
    }
  } else if (warp >= 4) {
    // epilogue: rows 32 (warp - 4) + lane of the tile; waits are made warp-uniform, so the
    // warp-collective TMEM loads run in every lane or in none
    const int qw = warp - 4;
    float* sq = reinterpret_cast<float*>(gb + STG_OFF + qw * STG_WARP);     // [32][33] |v|^2
    float2* stg = reinterpret_cast<float2*>(gb + STG_OFF + qw * STG_WARP);  // [32][17] values
    float* scl = reinterpret_cast<float*>(gb + SCL_OFF) + qw * 128;         // [32 / rg][32]
    const int rg = g.rg;
    const bool norm = g.rg_norm != 0;
    int tc = 0;
    for (int rt = blockIdx.x; rt < ntiles && ok; rt += gridDim.x) {
      const int gm = rt * BM + 32 * qw + lane;
      float2* rowp = nullptr;
      if (gm < g.M) {
        const int item = gm / g.rg_rows, rem = gm % g.rg_rows;
        rowp = (g.c_tab ? g.c_tab[item] : g.C + (long long)item * g.c_stride) + (long long)(rem % rg) * g.rg_plane +
               (long long)(rem / rg) * g.ldc;
      }
      for (int ct = 0; ct < nct && ok; ++ct) {
        const int b = tc & 1, u = tc >> 1;
        ok = __all_sync(0xffffffffu, bar_wait(accf0 + 8 * b, (uint32_t)(u & 1), lim));
        if (!ok) break;
        fence_after();
        const uint32_t ta = tmem + ((uint32_t)(32 * qw) << 16) + 128u * b;
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
          uint32_t re[32], im[32];
          tmem_ld32(ta + 64 * h, re);
          tmem_ld32(ta + 64 * h + 32, im);
          if (h == 1) {  // both halves read: the buffer is free for the column tile after next
            fence_before();
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(acce0 + 8 * b) : "memory");
          }
          const int x0 = 64 * ct + 32 * h;
          if (x0 >= g.N) continue;
          if (norm) {
#pragma unroll
            for (int c = 0; c < 32; ++c) {
              const float x = __uint_as_float(re[c]), y = __uint_as_float(im[c]);
              sq[lane * 33 + c] = fmaf(x, x, y * y);
            }
            __syncwarp();
            for (int gi = 0; gi < 32 / rg; ++gi) {
              float n2 = 0.f;
              for (int r = 0; r < rg; ++r) n2 += sq[(gi * rg + r) * 33 + lane];
              scl[gi * 32 + lane] = n2 > 0.f ? rsqrtf(n2) : 0.f;
            }
            __syncwarp();
            const float* sc = scl + (lane / rg) * 32;
#pragma unroll
            for (int c = 0; c < 32; ++c) {
              const float f = sc[c];
              re[c] = __float_as_uint(__uint_as_float(re[c]) * f);
              im[c] = __float_as_uint(__uint_as_float(im[c]) * f);
            }
          }
#pragma unroll
          for (int hh = 0; hh < 2; ++hh) {
#pragma unroll
            for (int j = 0; j < 16; ++j)
              stg[lane * 17 + j] = make_float2(__uint_as_float(re[16 * hh + j]), __uint_as_float(im[16 * hh + j]));
            __syncwarp();
#pragma unroll 4
            for (int i = 0; i < 16; ++i) {
              const int rr = 2 * i + (lane >> 4), col = lane & 15;
              float2* p = reinterpret_cast<float2*>(
                  __shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(rowp), rr));
              const int x = x0 + 16 * hh + col;
              if (p != nullptr && x < g.N) __stcs(p + x, stg[rr * 17 + col]);
            }
            __syncwarp();
          }
        }
        ++tc;
      }
    }
  }
  __syncwarp();
  if (!ok && g.err) atomicOr(g.err, 16);
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

// C = alpha * sum_z ws[z] + beta * C (+ diag), partials summed in z order; grid y = batch item
// (its partials at ws + item * splits * M * N, its C at C + item * c_stride)
__global__ void splitk_reduce_kernel(const float2* __restrict__ ws, int splits, int M, int N, float2 alpha,
                                     float2 beta, float2* __restrict__ C, int ldc, float diag_val, int diag_stride,
                                     int diag_limit, long long c_stride) {
  const long long total = (long long)M * N;
  ws += (long long)blockIdx.y * splits * total;
  C += blockIdx.y * c_stride;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    float2 a = make_float2(0.f, 0.f);
    for (int z = 0; z < splits; ++z) {
      const float2 v = ws[(long long)z * total + e];
      a.x += v.x;
      a.y += v.y;
    }
    const int m = (int)(e / N), n = (int)(e % N);
    float2 o = make_float2(alpha.x * a.x - alpha.y * a.y, alpha.x * a.y + alpha.y * a.x);
    float2* cp = C + (long long)m * ldc + n;
    if (beta.x != 0.f || beta.y != 0.f) {
      const float2 c = *cp;
      o.x += beta.x * c.x - beta.y * c.y;
      o.y += beta.x * c.y + beta.y * c.x;
    }
    if (diag_stride > 0 && n < diag_limit && n % diag_stride == 0) o.x += diag_val;
    *cp = o;
  }
}

// A' head/tail: A'[m][2k] = Re(A[m][k] w_k), A'[m][2k+1] = Im(...), w_k = kscale[k] (or 1);
// `items` independent operands: A, kscale and A' advance by a_stride, w_stride and M * K2p
__global__ void split_a_kernel(const float2* __restrict__ A, int lda, const float* __restrict__ kscale, int M, int K,
                               float* __restrict__ hi, float* __restrict__ lo, int K2p, int items,
                               long long a_stride, long long w_stride) {
  const long long per = (long long)M * K;
  const long long total = per * items;
  for (long long e0 = blockIdx.x * (long long)blockDim.x + threadIdx.x; e0 < total; e0 += (long long)gridDim.x * blockDim.x) {
    const long long it = e0 / per, e = e0 % per;
    const int m = (int)(e / K), k = (int)(e % K);
    float2 v = A[it * a_stride + (long long)m * lda + k];
    if (kscale) {
      const float w = kscale[it * w_stride + k];
      v.x *= w;
      v.y *= w;
    }
    const float hx = head(v.x), hy = head(v.y);
    const long long o = it * ((long long)M * K2p) + (long long)m * K2p + 2 * k;
    *reinterpret_cast<float2*>(hi + o) = make_float2(hx, hy);
    if (lo) *reinterpret_cast<float2*>(lo + o) = make_float2(head(v.x - hx), head(v.y - hy));
  }
}

// A' head/tail for A = conj(Y^T), Y K x M row-major (ldy): A'[i][2k] = Re Y[k][i],
// A'[i][2k+1] = -Im Y[k][i]
__global__ void split_at_kernel(const float2* __restrict__ Y, int ldy, int M, int K, float* __restrict__ hi,
                                float* __restrict__ lo, int K2p, int items, long long y_stride) {
  const long long per = (long long)M * K;
  const long long total = per * items;
  for (long long e0 = blockIdx.x * (long long)blockDim.x + threadIdx.x; e0 < total; e0 += (long long)gridDim.x * blockDim.x) {
    const long long it = e0 / per, e = e0 % per;
    const int k = (int)(e / M), i = (int)(e % M);
    const float2 y = Y[it * y_stride + (long long)k * ldy + i];
    const float vx = y.x, vy = -y.y;
    const float hx = head(vx), hy = head(vy);
    const long long o = it * ((long long)M * K2p) + (long long)i * K2p + 2 * k;
    *reinterpret_cast<float2*>(hi + o) = make_float2(hx, hy);
    if (lo) *reinterpret_cast<float2*>(lo + o) = make_float2(head(vx - hx), head(vy - hy));
  }
}

// B' head/tail rows (see the file comment); columns c >= N of the last tile are zero
// cg > 0 (opB 0): column c of B is column c % cg of block c / cg, the blocks cgs elements apart
__global__ void split_b_kernel(const float2* __restrict__ B, int ldb, int opB, int K, int N, int Np,
                               float* __restrict__ hi, float* __restrict__ lo, int K2p, int nbatch,
                               long long b_stride, int cg, long long cgs) {
  const long long per = (long long)Np * K;
  const long long total = per * nbatch;
  for (long long e0 = blockIdx.x * (long long)blockDim.x + threadIdx.x; e0 < total; e0 += (long long)gridDim.x * blockDim.x) {
    const long long bi = e0 / per, e = e0 % per;
    const float2* Bb = B + bi * b_stride;
    float* hb = hi + bi * (2LL * Np * K2p);
    float* lb = lo ? lo + bi * (2LL * Np * K2p) : nullptr;
    const int c = (int)(e / K), k = (int)(e % K);
    float2 b = make_float2(0.f, 0.f);
    if (c < N) {
      if (opB == 0) b = cg > 0 ? Bb[(long long)(c / cg) * cgs + (long long)k * ldb + c % cg] : Bb[(long long)k * ldb + c];
      else {
        const float2 s = Bb[(long long)c * ldb + k];
        b = make_float2(s.x, -s.y);
      }
    }
    const int t = c / BNC, cl = c % BNC;
    const long long rre = (long long)(64 * t + cl) * K2p + 2 * k;
    const long long rim = (long long)(64 * t + 32 + cl) * K2p + 2 * k;
    const float2 vre = make_float2(b.x, -b.y), vim = make_float2(b.y, b.x);
    const float2 hre = make_float2(head(vre.x), head(vre.y)), him = make_float2(head(vim.x), head(vim.y));
    *reinterpret_cast<float2*>(hb + rre) = hre;
    *reinterpret_cast<float2*>(hb + rim) = him;
    if (lb) {
      *reinterpret_cast<float2*>(lb + rre) = make_float2(head(vre.x - hre.x), head(vre.y - hre.y));
      *reinterpret_cast<float2*>(lb + rim) = make_float2(head(vim.x - him.x), head(vim.y - him.y));
    }
  }
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
// test hook (pisco_test_stall_tensor_loads): launches made while it is set withhold their loads
std::atomic<int> g_tc2_stall{0};
std::mutex g_encode_mu;

bool encode_2d(CUtensorMap* map, const float* base, int cols, int rows, int ld_floats, int box_rows) {
  if (!g_encode) {
    std::lock_guard<std::mutex> lk(g_encode_mu);
    if (!g_encode) {
      void* fn = nullptr;
      cudaDriverEntryPointQueryResult q;
      if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
          q != cudaDriverEntryPointSuccess || !fn)
        return false;
      g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
  }
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld_floats * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return g_encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int NT, int STAGES, bool CONV, int WT>
size_t smem_bytes() {
  return (size_t)STAGES * stage_bytes<NT, CONV, WT>() + 1024 + 128;
}

unsigned grid_for(long long n) {
  long long b = (n + 255) / 256;
  return (unsigned)(b > 152 * 8 ? 152 * 8 : (b < 1 ? 1 : b));
}

}  // namespace

void tc2_set_stall(bool on) { g_tc2_stall.store(on ? 1 : 0); }

bool tc2_conv_ok(int K, int lda_fp32, const void* a_fp32) {
  return a_fp32 != nullptr && (lda_fp32 % 2) == 0 && lda_fp32 >= K && ((uintptr_t)a_fp32 % 16) == 0;
}

int tc2_k2p(int K) { return ((2 * K + 3) / 4) * 4; }
int tc2_np(int N) { return ((N + BNC - 1) / BNC) * BNC; }

template <int NT, int S, bool CONV, int WT>
static cudaError_t set_smem() {
  return cudaFuncSetAttribute(tc2_kernel<NT, S, CONV, WT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem_bytes<NT, S, CONV, WT>());
}

template <int NT, int S, bool CONV, int WT>
static void launch(dim3 grid, cudaStream_t st, const CUtensorMap& a, const CUtensorMap& al, const CUtensorMap& b,
                   const CUtensorMap& bl, const Args& g) {
  tc2_kernel<NT, S, CONV, WT><<<grid, CONV ? 256 : 128, smem_bytes<NT, S, CONV, WT>(), st>>>(a, al, b, bl, g);
}

int sm_count() {
  static std::atomic<int> n{0};
  int v = n.load();
  if (v <= 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        v <= 0)
      v = 1;
    n.store(v);
  }
  return v;
}

cudaError_t tc2_prepare() {
  cudaError_t e = cudaFuncSetAttribute(tc2_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(rows::TOTAL + 1024));
  if (e == cudaSuccess) e = set_smem<3, 3, false, 2>();
  if (e == cudaSuccess) e = set_smem<3, 2, false, 1>();
  if (e == cudaSuccess) e = set_smem<1, 4, false, 2>();
  if (e == cudaSuccess) e = set_smem<1, 2, false, 1>();
  if (e == cudaSuccess) e = set_smem<3, 2, true, 2>();
  if (e == cudaSuccess) e = set_smem<3, 3, true, 1>();
  return e;
}

cudaError_t tc2_split_a(const float2* A, int lda, const float* kscale, int M, int K, float* hi, float* lo,
                        cudaStream_t st, int items, long long a_stride, long long w_stride) {
  split_a_kernel<<<grid_for((long long)M * K * items), 256, 0, st>>>(A, lda, kscale, M, K, hi, lo, tc2_k2p(K), items,
                                                                     a_stride, w_stride);
  ++g_launches;
  return cudaGetLastError();
}

cudaError_t tc2_split_at(const float2* Y, int ldy, int M, int K, float* hi, float* lo, cudaStream_t st, int items,
                         long long y_stride) {
  split_at_kernel<<<grid_for((long long)M * K * items), 256, 0, st>>>(Y, ldy, M, K, hi, lo, tc2_k2p(K), items,
                                                                      y_stride);
  ++g_launches;
  return cudaGetLastError();
}

cudaError_t tc2_split_b(const float2* B, int ldb, int opB, int K, int N, float* hi, float* lo, cudaStream_t st,
                        int nbatch, long long b_stride, int cg, long long cgs) {
  const int Np = tc2_np(N);
  split_b_kernel<<<grid_for((long long)Np * K * nbatch), 256, 0, st>>>(B, ldb, opB, K, N, Np, hi, lo, tc2_k2p(K),
                                                                      nbatch, b_stride, opB == 0 ? cg : 0, cgs);
  ++g_launches;
  return cudaGetLastError();
}

cudaError_t tc2_gemm(int nterms, int M, int N, int K, const float* Ahi, const float* Alo, const float* Bhi,
                     const float* Blo, float2 alpha, float2 beta, float2* C, int ldc, float diag_val,
                     int diag_stride, int diag_limit, int splits, float2* ws, int* err, cudaStream_t st,
                     int nbatch, long long c_stride, int a_per_item, float2* const* c_tab, int c_div,
                     int b_per_item, const float2* a_fp32, int lda_fp32, int rg, int rg_rows,
                     long long rg_plane, int rg_norm) {
  if (M <= 0 || N <= 0 || nbatch < 1) return cudaSuccess;
  if (rg > 0 && (nbatch != 1 || rg_rows <= 0 || rg_rows % rg != 0 || (rg_norm && BM % rg != 0)))
    return cudaErrorInvalidValue;
  const int K2 = 2 * K, K2p = tc2_k2p(K), Np = tc2_np(N);
  const int total = (K2 + BK - 1) / BK;
  // split-K: also in batched mode (per item), never with a C table
  if (splits < 1 || ws == nullptr || c_tab != nullptr || rg > 0) splits = 1;
  if (splits > total) splits = total > 0 ? total : 1;
  const int kpb = total > 0 ? (total + splits - 1) / splits : 0;
  if (kpb > 0) splits = (total + kpb - 1) / kpb;
  CUtensorMap mAh, mAl, mBh, mBl;
  const float* al = nterms == 3 ? Alo : Ahi;
  const float* bl = nterms == 3 ? Blo : Bhi;
  const int kcols = K2 > 0 ? K2 : 1;
  const int arows = a_per_item && nbatch > 1 ? M * nbatch : M;
  // A from FP32 complex rows, split on the way into tensor memory: three passes, rows 16-byte aligned
  const bool conv = a_fp32 != nullptr && nterms == 3 && (lda_fp32 % 2) == 0 && lda_fp32 >= K &&
                    ((uintptr_t)a_fp32 % 16) == 0;
  // the row-group epilogue keeps its scales and row offsets beside the tile: converting variants
  if (rg > 0 && !conv) return cudaErrorInvalidValue;
  if (conv) {
    if (!encode_2d(&mAh, reinterpret_cast<const float*>(a_fp32), kcols, arows, 2 * lda_fp32, BM)) return cudaErrorInvalidValue;
    mAl = mAh;
  } else if (!encode_2d(&mAh, Ahi, kcols, arows, K2p, BM) || !encode_2d(&mAl, al, kcols, arows, K2p, BM)) {
    return cudaErrorInvalidValue;
  }
  // long K loops (> 8 steps per CTA) take 64 complex columns per CTA (one N = 128 MMA: half the
  // A loads per output): split operands 3-4 stages, converting 2 stages at 2 CTAs per SM (one
  // CTA's conversions and loads fill the other's gaps on the tensor pipe); short ones 32 columns
  // and 2-3 stages, 2 CTAs per SM, so one CTA's epilogue overlaps another's loads.  Row-grouped
  // products take the 32-column form.
  const bool wide = kpb > 8 && rg == 0;
  // row-grouped products whose A tile fits shared memory whole (K2 <= 128) and whose pixel groups
  // stay within a warp (8 <= rg <= 32 when normalised): the row-tile persistent kernel
  const bool rows_res = conv && rg > 0 && K2 > 0 && K2 <= rows::KSMAX * BK && (!rg_norm || (rg >= 8 && rg <= 32));
  const int wt = (wide || rows_res) ? 2 : 1;
  if (!encode_2d(&mBh, Bhi, kcols, 2 * Np * (b_per_item ? nbatch : 1), K2p, 2 * BNC * wt) ||
      !encode_2d(&mBl, bl, kcols, 2 * Np * (b_per_item ? nbatch : 1), K2p, 2 * BNC * wt))
    return cudaErrorInvalidValue;
  Args g{M, N, K2, kpb, C, ldc, alpha, beta, diag_val, diag_stride, diag_limit, ws, err,
         nbatch > 1 ? 1 : 0, b_per_item ? 2 * Np : 0, c_stride, a_per_item && nbatch > 1 ? M : 0,
         (nbatch > 1 || rg > 0) ? c_tab : nullptr,
         c_div > 0 ? c_div : 1};
  g.rg = rg > 0 ? rg : 0;
  g.rg_rows = rg_rows;
  g.rg_norm = rg > 0 && rg_norm ? 1 : 0;
  g.rg_plane = rg_plane;
  g.splits = splits;
  g.no_loads = g_tc2_stall.load() ? 1 : 0;
  g.wait_limit = g.no_loads ? kWaitStalled : kWait;
  if (rows_res) {
    const int ntiles = (M + BM - 1) / BM, nsm = sm_count();
    tc2_rows_kernel<<<ntiles < nsm ? ntiles : nsm, rows::NTHR, rows::TOTAL + 1024, st>>>(mAh, mBh, mBl, g);
    ++g_launches;
    return cudaGetLastError();
  }
  dim3 grid((Np + BNC * wt - 1) / (BNC * wt), (M + BM - 1) / BM, nbatch * splits);
  if (conv) {
    if (wide) launch<3, 2, true, 2>(grid, st, mAh, mAl, mBh, mBl, g);
    else launch<3, 3, true, 1>(grid, st, mAh, mAl, mBh, mBl, g);
  }
  else if (nterms == 1) {
    if (wide) launch<1, 4, false, 2>(grid, st, mAh, mAl, mBh, mBl, g);
    else launch<1, 2, false, 1>(grid, st, mAh, mAl, mBh, mBl, g);
  } else {
    if (wide) launch<3, 3, false, 2>(grid, st, mAh, mAl, mBh, mBl, g);
    else launch<3, 2, false, 1>(grid, st, mAh, mAl, mBh, mBl, g);
  }
  ++g_launches;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || splits == 1) return e;
  splitk_reduce_kernel<<<dim3(grid_for((long long)M * N), nbatch), 256, 0, st>>>(
      ws, splits, M, N, alpha, beta, C, ldc, diag_val, diag_stride, diag_limit, c_stride);
  ++g_launches;
  return cudaGetLastError();
}

}  // namespace pisco
