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
                                                           float2* __restrict__ maps) {
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

cudaError_t interp_final_normalize(const float2* T, const float2* M, int Q, long long /*unused*/,
                                   int n_in, int n_out, long long inner, float2* maps,
                                   cudaStream_t st) {
  const long long total = (long long)n_out * inner;
  long long blocks = (total + 127) / 128;
  if (blocks > 152 * 32) blocks = 152 * 32;
  interp_final_kernel<<<(unsigned)blocks, 128, 0, st>>>(T, M, Q, n_in, n_out, inner, maps);
  ++g_launches;
  return cudaGetLastError();
}

}  // namespace pisco
