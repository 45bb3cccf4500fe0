// Separable small DFTs as "apply a dense matrix along one axis", in FP64 (Gram, Sec. V-A)
// and FP32 (G(x) on the reduced grid, Sec. V-C; apodised low-res images and periodic-sinc
// interpolation, Sec. V-D).  The transforms here are short (tens of points) and not powers
// of two, so each axis is a small dense matrix product; every output element is one thread,
// with the inner (fastest) index mapped to consecutive threads so loads are coalesced and
// the matrix row is a warp-wide broadcast.  Along the contiguous axis (inner == 1) consecutive
// threads are consecutive outputs instead; those passes read a transposed matrix (AxisView::mt)
// so that a warp's matrix loads stay contiguous while the input element is the broadcast.
#include <type_traits>

#include "common.cuh"

namespace pisco {

template <typename Tin, typename C>
__global__ void __launch_bounds__(256) apply_axis_kernel(const Tin* __restrict__ in,
                                                         const C* __restrict__ M,
                                                         C* __restrict__ out, AxisView v) {
  const long long total = v.batch * v.outer * (long long)v.n_out * v.inner;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    long long t = idx;
    const long long ii = t % v.inner; t /= v.inner;
    const int o = (int)(t % v.n_out); t /= v.n_out;
    const long long bo = t;  // batch*outer flattened
    const Tin* src = in + (bo * v.n_in) * v.inner + ii;
    const C* row = v.mt ? M + o : M + (long long)o * v.n_in;
    const long long mstep = v.mt ? v.n_out : 1;
    C acc = mk(decltype(acc.x)(0), decltype(acc.x)(0));
    for (int i = 0; i < v.n_in; ++i) {
      const Tin s = src[(long long)i * v.inner];
      C sv = mk(decltype(acc.x)(s.x), decltype(acc.x)(s.y));
      cfma(acc, row[(long long)i * mstep], sv);
    }
    if (v.pixel_major && v.pm_group > 0)
      out[((bo / v.pm_group) * ((long long)v.n_out * v.inner) + (long long)o * v.inner + ii) * v.pm_group +
          bo % v.pm_group] = acc;
    else if (v.pixel_major)
      out[((long long)o * v.inner + ii) * v.batch + bo] = acc;
    else
      out[(bo * v.n_out + o) * v.inner + ii] = acc;
  }
}

// FP32 contiguous-axis pass (inner == 1, transposed matrix) with a register tile of R rows:
// each matrix element, loaded once (coalesced across the warp's outputs), serves R rows whose
// input elements are warp-wide broadcasts.
template <int R>
__global__ void __launch_bounds__(256) apply_axis_rows_kernel(const float2* __restrict__ in,
                                                              const float2* __restrict__ MT,
                                                              float2* __restrict__ out, long long rows,
                                                              int n_in, int n_out) {
  const long long groups = (rows + R - 1) / R;
  const long long total = groups * n_out;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int o = (int)(idx % n_out);
    const long long r0 = (idx / n_out) * R;
    float2 acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = make_float2(0.f, 0.f);
    for (int i = 0; i < n_in; ++i) {
      const float2 m = MT[(long long)i * n_out + o];
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (r0 + r < rows) cfma(acc[r], m, in[(r0 + r) * n_in + i]);
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (r0 + r < rows) out[(r0 + r) * n_out + o] = acc[r];
  }
}

template <typename Tin, typename C>
static cudaError_t launch_apply(const Tin* in, const C* M, C* out, AxisView v, cudaStream_t st) {
  const long long total = v.batch * v.outer * (long long)v.n_out * v.inner;
  if (total <= 0) return cudaSuccess;
  if constexpr (std::is_same<Tin, float2>::value && std::is_same<C, float2>::value) {
    if (v.inner == 1 && v.mt && !v.pixel_major) {
      constexpr int R = 4;
      const long long rows = v.batch * v.outer;
      long long blocks = (((rows + R - 1) / R) * v.n_out + 255) / 256;
      if (blocks > 152 * 16) blocks = 152 * 16;
      apply_axis_rows_kernel<R><<<(unsigned)blocks, 256, 0, st>>>(in, M, out, rows, v.n_in, v.n_out);
      ++g_launches;
      return cudaGetLastError();
    }
  }
  long long blocks = (total + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  apply_axis_kernel<Tin, C><<<(unsigned)blocks, 256, 0, st>>>(in, M, out, v);
  ++g_launches;
  return cudaGetLastError();
}

cudaError_t apply_axis_c2z(const float2* in, const double2* M, double2* out, AxisView v, cudaStream_t st) {
  return launch_apply<float2, double2>(in, M, out, v, st);
}
cudaError_t apply_axis_z(const double2* in, const double2* M, double2* out, AxisView v, cudaStream_t st) {
  return launch_apply<double2, double2>(in, M, out, v, st);
}
cudaError_t apply_axis_c(const float2* in, const float2* M, float2* out, AxisView v, cudaStream_t st) {
  return launch_apply<float2, float2>(in, M, out, v, st);
}

}  // namespace pisco
