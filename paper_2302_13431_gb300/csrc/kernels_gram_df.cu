// Stage (a) in double-float arithmetic: the FFT route of Sec. V-A with every FP64 operation
// replaced by an unevaluated sum of two FP32 numbers (hi + lo, |lo| <= ulp(hi)/2) computed with
// the error-free transformations of Dekker (1971) and Knuth (TAOCP vol. 2): the product of two
// FP32 numbers is exact as (fl(a*b), fma(a, b, -fl(a*b))), the sum as Knuth's TwoSum.  About 48
// significant bits; on GB300, whose FP64 rate is about 1/58 of its FP32 rate, a complex
// double-float multiply-add (~60 FP32 operations) costs a quarter of a complex FP64 one.
// Storage is 16 bytes per complex value, the layout of the FP64 path ({Re hi, Re lo, Im hi,
// Im lo} in place of {Re, Im} doubles), and the lag table is written back in FP64.
#include "common.cuh"

namespace pisco {

namespace {

struct dfc {
  float rh, rl, ih, il;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void quick_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  e = b - (s - a);
}
// (ah, al) += (xh, xl) * (yh, yl)
__device__ __forceinline__ void df_fma(float& ah, float& al, float xh, float xl, float yh, float yl) {
  const float p = xh * yh;
  float pe = fmaf(xh, yh, -p);
  pe = fmaf(xh, yl, pe);
  pe = fmaf(xl, yh, pe);
  float s, e;
  two_sum(ah, p, s, e);
  e += al + pe;
  quick_two_sum(s, e, ah, al);
}
// acc += m * x (complex)
__device__ __forceinline__ void df_cfma(dfc& acc, const dfc& m, const dfc& x) {
  df_fma(acc.rh, acc.rl, m.rh, m.rl, x.rh, x.rl);
  df_fma(acc.rh, acc.rl, -m.ih, -m.il, x.ih, x.il);
  df_fma(acc.ih, acc.il, m.rh, m.rl, x.ih, x.il);
  df_fma(acc.ih, acc.il, m.ih, m.il, x.rh, x.rl);
}
// acc += conj(a) * b
__device__ __forceinline__ void df_cfmac(dfc& acc, const dfc& a, const dfc& b) {
  df_fma(acc.rh, acc.rl, a.rh, a.rl, b.rh, b.rl);
  df_fma(acc.rh, acc.rl, a.ih, a.il, b.ih, b.il);
  df_fma(acc.ih, acc.il, a.rh, a.rl, b.ih, b.il);
  df_fma(acc.ih, acc.il, -a.ih, -a.il, b.rh, b.rl);
}

__device__ __forceinline__ dfc load_in(const float2* p) {
  const float2 v = *p;
  return dfc{v.x, 0.f, v.y, 0.f};
}
__device__ __forceinline__ dfc load_in(const dfc* p) { return *p; }

// the axis transform of kernels_dft.cu (same index map and transposed-table option)
template <typename Tin>
__global__ void __launch_bounds__(256) apply_axis_df_kernel(const Tin* __restrict__ in, const dfc* __restrict__ M,
                                                            dfc* __restrict__ out, AxisView v) {
  const long long total = v.batch * v.outer * (long long)v.n_out * v.inner;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    long long t = idx;
    const long long ii = t % v.inner;
    t /= v.inner;
    const int o = (int)(t % v.n_out);
    t /= v.n_out;
    const long long bo = t;
    const Tin* src = in + (bo * v.n_in) * v.inner + ii;
    const dfc* row = v.mt ? M + o : M + (long long)o * v.n_in;
    const long long mstep = v.mt ? v.n_out : 1;
    dfc acc{0.f, 0.f, 0.f, 0.f};
    for (int i = 0; i < v.n_in; ++i) df_cfma(acc, row[(long long)i * mstep], load_in(src + (long long)i * v.inner));
    out[(bo * v.n_out + o) * v.inner + ii] = acc;
  }
}

__global__ void pair_products_df_kernel(const dfc* __restrict__ S, int Q, long long nfreq, dfc* __restrict__ P) {
  const int pair = blockIdx.y;
  int p = 0, base = 0;
  while (pair >= base + (Q - p)) { base += Q - p; ++p; }
  const int q = p + (pair - base);
  const dfc* Sp = S + (long long)p * nfreq;
  const dfc* Sq = S + (long long)q * nfreq;
  dfc* out = P + (long long)pair * nfreq;
  for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < nfreq; f += (long long)gridDim.x * blockDim.x) {
    dfc acc{0.f, 0.f, 0.f, 0.f};
    df_cfmac(acc, Sp[f], Sq[f]);
    out[f] = acc;
  }
}

// lags[(p,q)][t] = Rp[pair][t] as FP64 (hi + lo is exact in FP64)
__global__ void scatter_pairs_df_kernel(const dfc* __restrict__ Rp, int Q, int nbox, double2* __restrict__ lags) {
  const int pair = blockIdx.x;
  int p = 0, base = 0;
  while (pair >= base + (Q - p)) { base += Q - p; ++p; }
  const int q = p + (pair - base);
  for (int t = threadIdx.x; t < nbox; t += blockDim.x) {
    const dfc v = Rp[(long long)pair * nbox + t];
    lags[((long long)p * Q + q) * nbox + t] = make_double2((double)v.rh + (double)v.rl, (double)v.ih + (double)v.il);
  }
}

template <typename Tin>
cudaError_t launch_df(const Tin* in, const void* M, void* out, AxisView v, cudaStream_t st) {
  const long long total = v.batch * v.outer * (long long)v.n_out * v.inner;
  if (total <= 0) return cudaSuccess;
  long long blocks = (total + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  apply_axis_df_kernel<Tin><<<(unsigned)blocks, 256, 0, st>>>(in, static_cast<const dfc*>(M), static_cast<dfc*>(out), v);
  ++g_launches;
  return cudaGetLastError();
}

}  // namespace

// M tables in double-float ({Re hi, Re lo, Im hi, Im lo} per entry, 16 bytes)
cudaError_t apply_axis_c2df(const float2* in, const void* M, void* out, AxisView v, cudaStream_t st) {
  return launch_df<float2>(in, M, out, v, st);
}
cudaError_t apply_axis_df(const void* in, const void* M, void* out, AxisView v, cudaStream_t st) {
  return launch_df<dfc>(static_cast<const dfc*>(in), M, out, v, st);
}
cudaError_t gram_pair_products_df(const void* S, int Q, long long nfreq, void* P, cudaStream_t st) {
  const int npairs = Q * (Q + 1) / 2;
  int bx = (int)((nfreq + 255) / 256);
  if (bx > 64) bx = 64;
  pair_products_df_kernel<<<dim3(bx, npairs), 256, 0, st>>>(static_cast<const dfc*>(S), Q, nfreq, static_cast<dfc*>(P));
  ++g_launches;
  return cudaGetLastError();
}
cudaError_t gram_scatter_pairs_df(const void* Rp, int Q, int nbox, double2* lags, cudaStream_t st) {
  scatter_pairs_df_kernel<<<Q * (Q + 1) / 2, 128, 0, st>>>(static_cast<const dfc*>(Rp), Q, nbox, lags);
  ++g_launches;
  return cudaGetLastError();
}

}  // namespace pisco

namespace pisco {
namespace {

// (ah, al) += a * x with a = (a_hi + a_lo) double-float and x exact in FP32
__device__ __forceinline__ void df_fma1(float& ah, float& al, float a_hi, float a_lo, float x) {
  const float p = a_hi * x;
  float pe = fmaf(a_hi, x, -p);
  pe = fmaf(a_lo, x, pe);
  float s, e;
  two_sum(ah, p, s, e);
  e += al + pe;
  quick_two_sum(s, e, ah, al);
}
__device__ __forceinline__ void df_add(float& ah, float& al, float bh, float bl) {
  float s, e;
  two_sum(ah, bh, s, e);
  e += al + bl;
  quick_two_sum(s, e, ah, al);
}

// Zb = A * Xb (the band products of the FP64 Rayleigh quotients) in double-float: A's FP64
// entries split into two floats, the band vectors exact in FP32 (they come from the FP32 Ritz
// block); one warp per row of A, only the band columns in use.  Zb written in FP64.
template <int NBV>
__global__ void __launch_bounds__(256) band_matvec_df_kernel(const double2* __restrict__ A,
                                                             const double2* __restrict__ Xb, int n,
                                                             const int* __restrict__ band_idx,
                                                             double2* __restrict__ Zb) {
  constexpr int KC = 512;
  __shared__ float2 xs[KC * NBV];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r = blockIdx.x * 8 + warp;
  int nbu = 0;
#pragma unroll
  for (int c = 0; c < NBV; ++c)
    if (band_idx[c] >= 0) nbu = c + 1;
  float arh[NBV], arl[NBV], aih[NBV], ail[NBV];
#pragma unroll
  for (int c = 0; c < NBV; ++c) arh[c] = arl[c] = aih[c] = ail[c] = 0.f;
  for (int k0 = 0; k0 < n; k0 += KC) {
    const int kc = min(KC, n - k0);
    __syncthreads();
    for (int e = threadIdx.x; e < kc * NBV; e += blockDim.x) {
      const double2 v = Xb[(long long)k0 * NBV + e];
      xs[e] = make_float2((float)v.x, (float)v.y);  // exact: the band vectors are FP32 values
    }
    __syncthreads();
    if (r < n) {
      const double2* arow = A + (long long)r * n + k0;
      for (int k = lane; k < kc; k += 32) {
        const double2 a = arow[k];
        const float ahx = (float)a.x, ahy = (float)a.y;
        const float alx = (float)(a.x - (double)ahx), aly = (float)(a.y - (double)ahy);
#pragma unroll
        for (int c = 0; c < NBV; ++c) {
          if (c < nbu) {
            const float2 x = xs[k * NBV + c];
            df_fma1(arh[c], arl[c], ahx, alx, x.x);     // Re += Re a Re x
            df_fma1(arh[c], arl[c], -ahy, -aly, x.y);   //      - Im a Im x
            df_fma1(aih[c], ail[c], ahx, alx, x.y);     // Im += Re a Im x
            df_fma1(aih[c], ail[c], ahy, aly, x.x);     //      + Im a Re x
          }
        }
      }
    }
  }
#pragma unroll
  for (int c = 0; c < NBV; ++c) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float bh = __shfl_xor_sync(0xffffffffu, arh[c], o), bl = __shfl_xor_sync(0xffffffffu, arl[c], o);
      const float ch = __shfl_xor_sync(0xffffffffu, aih[c], o), cl = __shfl_xor_sync(0xffffffffu, ail[c], o);
      df_add(arh[c], arl[c], bh, bl);
      df_add(aih[c], ail[c], ch, cl);
    }
  }
  if (r < n && lane == 0) {
#pragma unroll
    for (int c = 0; c < NBV; ++c)
      Zb[(long long)r * NBV + c] = make_double2((double)arh[c] + (double)arl[c], (double)aih[c] + (double)ail[c]);
  }
}

}  // namespace

cudaError_t eig_band_matvec_df(const double2* A, const double2* Xb, int n, int nb, const int* band_idx, double2* Zb,
                               cudaStream_t st) {
  if (nb != 8) return cudaErrorInvalidValue;
  band_matvec_df_kernel<8><<<(n + 7) / 8, 256, 0, st>>>(A, Xb, n, band_idx, Zb);
  ++g_launches;
  return cudaGetLastError();
}

}  // namespace pisco
