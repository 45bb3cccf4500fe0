// Stage (e): periodic-sinc interpolation of the reduced-grid maps to the full grid
// (Sec. V-D) and the per-pixel sum-of-squares normalisation of the output (Sec. VI).
// The interpolation is separable; the host runs the passes along the faster axes with the
// generic axis kernel, and this kernel performs the pass along the slowest axis for all Q
// coils of one output pixel in one thread, so the unit-norm scaling happens in registers
// before the single write of the maps (the HBM-bound part of the stage).
#include "common.cuh"

namespace pisco {

namespace {
constexpr int QB = 32;  // coils held in registers per chunk
}

// T: [Q][n_in][inner], M: [n_out][n_in] (nullptr: identity, n_in == n_out), maps: [Q][n_out][inner]
__global__ void __launch_bounds__(128) interp_final_kernel(const float2* __restrict__ T,
                                                           const float2* __restrict__ M, int Q,
                                                           int n_in, int n_out, long long inner,
                                                           float2* __restrict__ maps, long long sT, long long sM,
                                                           float2* const* __restrict__ maps_tab) {
  T += blockIdx.y * sT;
  maps = maps_tab ? maps_tab[blockIdx.y] : maps + blockIdx.y * sM;
  const long long total = (long long)n_out * inner;
  const long long plane_in = (long long)n_in * inner, plane_out = total;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long ii = idx % inner;
    const int o = (int)(idx / inner);
    float norm2 = 0.f;
    float2 acc[QB];
    for (int q0 = 0; q0 < Q; q0 += QB) {
#pragma unroll
      for (int c = 0; c < QB; ++c) acc[c] = make_float2(0.f, 0.f);
      if (M != nullptr) {
        for (int i = 0; i < n_in; ++i) {
          const float2 mo = M[(long long)o * n_in + i];
          const float2* src = T + (long long)i * inner + ii;
#pragma unroll
          for (int c = 0; c < QB; ++c)
            if (q0 + c < Q) cfma(acc[c], mo, src[(long long)(q0 + c) * plane_in]);
        }
      } else {
#pragma unroll
        for (int c = 0; c < QB; ++c)
          if (q0 + c < Q) acc[c] = T[(long long)(q0 + c) * plane_in + (long long)o * inner + ii];
      }
#pragma unroll
      for (int c = 0; c < QB; ++c) norm2 += acc[c].x * acc[c].x + acc[c].y * acc[c].y;
      if (Q > QB) {
#pragma unroll
        for (int c = 0; c < QB; ++c)
          if (q0 + c < Q) maps[(long long)(q0 + c) * plane_out + idx] = acc[c];
      }
    }
    const float s = norm2 > 0.f ? rsqrtf(norm2) : 0.f;
    if (Q <= QB) {
#pragma unroll
      for (int c = 0; c < QB; ++c)
        if (c < Q) maps[(long long)c * plane_out + idx] = make_float2(acc[c].x * s, acc[c].y * s);
    } else {
      for (int c = 0; c < Q; ++c) {
        float2 v = maps[(long long)c * plane_out + idx];
        maps[(long long)c * plane_out + idx] = make_float2(v.x * s, v.y * s);
      }
    }
  }
}

// Tiled form for M != nullptr: a CTA computes a TO x TI tile of (output index along the axis,
// inner index) for every coil.  The TO rows of M are staged once; the coils are processed in
// chunks of QC whose T rows [n_in][TI] are staged in shared memory, so T is read from L2 once
// per tile column instead of once per output pixel.  Each thread keeps all its coils in
// registers (QB <= 64), normalises and writes the maps once.
template <int QB>
__global__ void __launch_bounds__(256) interp_tiled_kernel(const float2* __restrict__ T,
                                                           const float2* __restrict__ M, int Q,
                                                           int n_in, int n_out, long long inner,
                                                           float2* __restrict__ maps, long long sT, long long sM,
                                                           float2* const* __restrict__ maps_tab) {
  constexpr int TO = 16, TI = 16, QC = 4;
  T += blockIdx.z * sT;
  maps = maps_tab ? maps_tab[blockIdx.z] : maps + blockIdx.z * sM;
  extern __shared__ float2 sm[];
  float2* Ms = sm;                      // TO * n_in
  float2* Ts = Ms + TO * n_in;          // QC * n_in * TI
  const int tid = threadIdx.x;
  const int to = tid / TI, ti = tid % TI;
  const int o0 = blockIdx.y * TO;
  const long long i0 = (long long)blockIdx.x * TI;
  const int o = o0 + to;
  const long long ii = i0 + ti;
  const long long plane_in = (long long)n_in * inner, plane_out = (long long)n_out * inner;
  for (int e = tid; e < TO * n_in; e += 256) {
    const int r = e / n_in, c = e % n_in;
    Ms[e] = (o0 + r < n_out) ? M[(long long)(o0 + r) * n_in + c] : make_float2(0.f, 0.f);
  }
  float2 acc[QB];
#pragma unroll
  for (int c = 0; c < QB; ++c) acc[c] = make_float2(0.f, 0.f);
#pragma unroll
  for (int q0 = 0; q0 < QB; q0 += QC) {
    if (q0 >= Q) break;
    __syncthreads();
    for (int e = tid; e < QC * n_in * TI; e += 256) {
      const int c = e / (n_in * TI);
      const int rem = e % (n_in * TI);
      const int i = rem / TI, t = rem % TI;
      float2 v = make_float2(0.f, 0.f);
      if (q0 + c < Q && i0 + t < inner) v = T[(long long)(q0 + c) * plane_in + (long long)i * inner + i0 + t];
      Ts[e] = v;
    }
    __syncthreads();
    const float2* mrow = Ms + to * n_in;
    for (int i = 0; i < n_in; ++i) {
      const float2 mo = mrow[i];
#pragma unroll
      for (int c = 0; c < QC; ++c) cfma(acc[q0 + c], mo, Ts[(c * n_in + i) * TI + ti]);
    }
  }
  if (o >= n_out || ii >= inner) return;
  float n2 = 0.f;
#pragma unroll
  for (int c = 0; c < QB; ++c)
    if (c < Q) n2 += acc[c].x * acc[c].x + acc[c].y * acc[c].y;
  const float s = n2 > 0.f ? rsqrtf(n2) : 0.f;
  const long long out0 = (long long)o * inner + ii;
#pragma unroll
  for (int c = 0; c < QB; ++c)
    if (c < Q) maps[(long long)c * plane_out + out0] = make_float2(acc[c].x * s, acc[c].y * s);
}

cudaError_t interp_final_normalize(const float2* T, const float2* M, int Q, long long /*unused*/,
                                   int n_in, int n_out, long long inner, float2* maps,
                                   cudaStream_t st, int items, long long sT, long long sM, float2* const* maps_tab) {
  if (M != nullptr && n_in <= 128 && Q <= 64) {
    const size_t smem = (size_t)(16 * n_in + 4 * n_in * 16) * sizeof(float2);
    static bool attr_set = false;
    if (!attr_set) {
      cudaFuncSetAttribute(interp_tiled_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      cudaFuncSetAttribute(interp_tiled_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      attr_set = true;
    }
    dim3 grid((unsigned)((inner + 15) / 16), (unsigned)((n_out + 15) / 16), items);
    if (Q <= 32)
      interp_tiled_kernel<32><<<grid, 256, smem, st>>>(T, M, Q, n_in, n_out, inner, maps, sT, sM, maps_tab);
    else
      interp_tiled_kernel<64><<<grid, 256, smem, st>>>(T, M, Q, n_in, n_out, inner, maps, sT, sM, maps_tab);
    ++g_launches;
    return cudaGetLastError();
  }
  const long long total = (long long)n_out * inner;
  long long blocks = (total + 127) / 128;
  if (blocks > 152 * 32) blocks = 152 * 32;
  blocks = (blocks + items - 1) / items;
  interp_final_kernel<<<dim3((unsigned)blocks, items), 128, 0, st>>>(T, M, Q, n_in, n_out, inner, maps, sT, sM,
                                                                      maps_tab);
  ++g_launches;
  return cudaGetLastError();
}

}  // namespace pisco

namespace pisco {

// maps[q][x] /= ||maps[.][x]|| (sum of squares over the coils; zero pixels stay zero): the
// normalisation of Sec. VI after a final interpolation pass that wrote unnormalised maps.  One
// thread per pixel keeps its coils in registers (QB per chunk; Q <= QB reads the maps once), so the
// maps cross HBM once in each direction; grid y is the item (maps_tab[item], or maps + item * sM).
template <int QB>
__global__ void __launch_bounds__(256) normalize_maps_kernel(float2* __restrict__ maps, int Q, long long npix,
                                                             long long sM, float2* const* __restrict__ maps_tab) {
  maps = maps_tab ? maps_tab[blockIdx.y] : maps + blockIdx.y * sM;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < npix; x += (long long)gridDim.x * blockDim.x) {
    float2 v[QB];
    float n2 = 0.f;
#pragma unroll
    for (int q = 0; q < QB; ++q) {
      v[q] = q < Q ? __ldcs(maps + (long long)q * npix + x) : make_float2(0.f, 0.f);
      n2 = fmaf(v[q].x, v[q].x, fmaf(v[q].y, v[q].y, n2));
    }
    for (int q = QB; q < Q; ++q) {  // coils beyond the register chunk (read twice)
      const float2 w = maps[(long long)q * npix + x];
      n2 = fmaf(w.x, w.x, fmaf(w.y, w.y, n2));
    }
    const float s = n2 > 0.f ? rsqrtf(n2) : 0.f;
#pragma unroll
    for (int q = 0; q < QB; ++q)
      if (q < Q) __stcs(maps + (long long)q * npix + x, make_float2(v[q].x * s, v[q].y * s));
    for (int q = QB; q < Q; ++q) {
      const float2 w = maps[(long long)q * npix + x];
      maps[(long long)q * npix + x] = make_float2(w.x * s, w.y * s);
    }
  }
}

cudaError_t normalize_maps(float2* maps, int Q, long long npix, cudaStream_t st, int items, long long sM,
                           float2* const* maps_tab) {
  long long b = (npix + 255) / 256;
  if (b > 152 * 8) b = 152 * 8;
  b = (b + items - 1) / items;
  if (Q <= 16)
    normalize_maps_kernel<16><<<dim3((unsigned)b, items), 256, 0, st>>>(maps, Q, npix, sM, maps_tab);
  else
    normalize_maps_kernel<32><<<dim3((unsigned)b, items), 256, 0, st>>>(maps, Q, npix, sM, maps_tab);
  ++g_launches;
  return cudaGetLastError();
}

}  // namespace pisco
