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
// (ah, al) += (bh, bl)
__device__ __forceinline__ void df_add(float& ah, float& al, float bh, float bl) {
  float s, e;
  two_sum(ah, bh, s, e);
  e += al + bl;
  quick_two_sum(s, e, ah, al);
}
__device__ __forceinline__ dfc df_cadd(dfc a, const dfc& b) {
  df_add(a.rh, a.rl, b.rh, b.rl);
  df_add(a.ih, a.il, b.ih, b.il);
  return a;
}
// Dot2-style accumulation (Ogita, Rump & Oishi 2005) of double-float products: the running
// sum s takes the head product by TwoSum, its rounding error and the product's low-order terms
// go to a second FP32 accumulator c without renormalising every step (12 instructions per real
// term against 15 for a renormalised double-float multiply-add); s + c is normalised once.
__device__ __forceinline__ void dot2_term(float& s, float& c, float xh, float xl, float yh, float yl) {
  const float p = xh * yh;
  float q = fmaf(xh, yh, -p);
  q = fmaf(xh, yl, q);
  q = fmaf(xl, yh, q);
  float t, r;
  two_sum(s, p, t, r);
  s = t;
  c += q + r;
}
// acc (unnormalised: {s_re, c_re, s_im, c_im}) += m * x (complex)
__device__ __forceinline__ void dot2_cfma(dfc& acc, const dfc& m, const dfc& x) {
  dot2_term(acc.rh, acc.rl, m.rh, m.rl, x.rh, x.rl);
  dot2_term(acc.rh, acc.rl, -m.ih, -m.il, x.ih, x.il);
  dot2_term(acc.ih, acc.il, m.rh, m.rl, x.ih, x.il);
  dot2_term(acc.ih, acc.il, m.ih, m.il, x.rh, x.rl);
}
__device__ __forceinline__ dfc dot2_finish(const dfc& a) {
  dfc o;
  two_sum(a.rh, a.rl, o.rh, o.rl);
  two_sum(a.ih, a.il, o.ih, o.il);
  return o;
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

__global__ void pair_products_df_kernel(const dfc* __restrict__ S, int Q, long long nfreq, dfc* __restrict__ P,
                                        GramItems it) {
  S += blockIdx.z * it.S;
  P += blockIdx.z * it.P;
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
__global__ void scatter_pairs_df_kernel(const dfc* __restrict__ Rp, int Q, int nbox, double2* __restrict__ lags,
                                        dfc* __restrict__ lags_df, GramItems it) {
  Rp += blockIdx.y * it.Rp;
  lags += blockIdx.y * it.lags;
  lags_df += blockIdx.y * it.lags;
  const int pair = blockIdx.x;
  int p = 0, base = 0;
  while (pair >= base + (Q - p)) { base += Q - p; ++p; }
  const int q = p + (pair - base);
  for (int t = threadIdx.x; t < nbox; t += blockDim.x) {
    const dfc v = Rp[(long long)pair * nbox + t];
    lags[((long long)p * Q + q) * nbox + t] = make_double2((double)v.rh + (double)v.rl, (double)v.ih + (double)v.il);
    lags_df[((long long)p * Q + q) * nbox + t] = v;
  }
}

// 2D pairs stage of the double-float Gram, fused per pair (p <= q): the frequency-domain product
// conj(S_p) S_q, the inverse lag transform along the contiguous axis (Lp2 -> B2) and then along
// axis 1 (Lp1 -> B1), all in shared memory, and the FP64 lag table of the pair.
// Both inverse passes pair the lags +d and -d: with the table entry of lag d >= 0 at frequency f
// equal to (c + i s) / Lp, c = cos(2 pi f d / Lp), s = sin(2 pi f d / Lp), and that of lag -d
// equal to (c - i s) / Lp, the two outputs are C + i S and C - i S for C = sum_f c x_f and
// S = sum_f s x_f (x_f complex).  A thread computes the four real Dot2 sums (Re and Im of C and
// of S: four independent dependency chains) of one (row, d >= 0) and writes both lags: half the
// products of evaluating every lag on its own.  (For d = 0 the sine column is exactly zero.)
// invT2: [Lp2][B2] (transposed), inv1: [B1][Lp1]; B1, B2 odd (lags -2 tau .. 2 tau).
__device__ __forceinline__ void dot2_lag_pair(dfc& cs, dfc& sn, const dfc& w, const dfc& x) {
  dot2_term(cs.rh, cs.rl, w.rh, w.rl, x.rh, x.rl);
  dot2_term(cs.ih, cs.il, w.rh, w.rl, x.ih, x.il);
  dot2_term(sn.rh, sn.rl, w.ih, w.il, x.rh, x.rl);
  dot2_term(sn.ih, sn.il, w.ih, w.il, x.ih, x.il);
}
// (C + i S, C - i S) from the finished sums
__device__ __forceinline__ void lag_pair_outputs(const dfc& C, const dfc& Sx, dfc& plus, dfc& minus) {
  plus = C;
  minus = C;
  df_add(plus.rh, plus.rl, -Sx.ih, -Sx.il);
  df_add(plus.ih, plus.il, Sx.rh, Sx.rl);
  df_add(minus.rh, minus.rl, Sx.ih, Sx.il);
  df_add(minus.ih, minus.il, -Sx.rh, -Sx.rl);
}
__global__ void __launch_bounds__(256) pairs_inverse_df_kernel(const dfc* __restrict__ S, int Q, int Lp1, int Lp2,
                                                               const dfc* __restrict__ invT2, int B2,
                                                               const dfc* __restrict__ inv1, int B1,
                                                               double2* __restrict__ lags, dfc* __restrict__ lags_df,
                                                               GramItems it) {
  extern __shared__ dfc dsm[];
  S += blockIdx.y * it.S;
  lags += blockIdx.y * it.lags;
  lags_df += blockIdx.y * it.lags;
  const int ldp = Lp2 | 1;  // odd row stride (in 16-byte words): conflict-free column reads
  dfc* P = dsm;                       // [Lp1][ldp]
  dfc* T = P + Lp1 * ldp;             // [Lp1][B2]
  dfc* m2 = T + Lp1 * B2;             // [Lp2][B2]
  dfc* m1 = m2 + Lp2 * B2;            // [B1][Lp1]
  const int pair = blockIdx.x;
  int p = 0, base = 0;
  while (pair >= base + (Q - p)) { base += Q - p; ++p; }
  const int q = p + (pair - base);
  const long long nfreq = (long long)Lp1 * Lp2;
  const dfc* Sp = S + p * nfreq;
  const dfc* Sq = S + q * nfreq;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int c2 = B2 / 2, c1 = B1 / 2;  // table columns / rows of lag 0
  for (int i = tid; i < Lp2 * B2; i += nt) m2[i] = invT2[i];
  for (int i = tid; i < B1 * Lp1; i += nt) m1[i] = inv1[i];
  for (int f = tid; f < Lp1 * Lp2; f += nt) {
    dfc acc{0.f, 0.f, 0.f, 0.f};
    df_cfmac(acc, Sp[f], Sq[f]);
    P[(f / Lp2) * ldp + f % Lp2] = acc;
  }
  __syncthreads();
  for (int o = tid; o < Lp1 * (c2 + 1); o += nt) {
    const int f1 = o / (c2 + 1), d = o % (c2 + 1);
    const dfc* prow = P + f1 * ldp;
    const dfc* wcol = m2 + c2 + d;
    dfc cs{0.f, 0.f, 0.f, 0.f}, sn{0.f, 0.f, 0.f, 0.f};
    for (int f2 = 0; f2 < Lp2; ++f2) dot2_lag_pair(cs, sn, wcol[f2 * B2], prow[f2]);
    dfc plus, minus;
    lag_pair_outputs(dot2_finish(cs), dot2_finish(sn), plus, minus);
    T[f1 * B2 + c2 + d] = plus;
    if (d > 0) T[f1 * B2 + c2 - d] = minus;
  }
  __syncthreads();
  const long long ob = ((long long)p * Q + q) * B1 * B2;
  for (int o = tid; o < (c1 + 1) * B2; o += nt) {
    const int d = o / B2, b2 = o % B2;
    const dfc* mrow = m1 + (c1 + d) * Lp1;
    dfc cs{0.f, 0.f, 0.f, 0.f}, sn{0.f, 0.f, 0.f, 0.f};
    for (int f1 = 0; f1 < Lp1; ++f1) dot2_lag_pair(cs, sn, mrow[f1], T[f1 * B2 + b2]);
    dfc plus, minus;
    lag_pair_outputs(dot2_finish(cs), dot2_finish(sn), plus, minus);
    const long long op = ob + (long long)(c1 + d) * B2 + b2, om = ob + (long long)(c1 - d) * B2 + b2;
    lags[op] = make_double2((double)plus.rh + (double)plus.rl, (double)plus.ih + (double)plus.il);
    lags_df[op] = plus;
    if (d > 0) {
      lags[om] = make_double2((double)minus.rh + (double)minus.rl, (double)minus.ih + (double)minus.il);
      lags_df[om] = minus;
    }
  }
}

// 2D forward stage of the double-float Gram, fused per coil: the zero-padded DFT of one coil's
// calibration along the contiguous axis (Nc2 -> Lp2), then along axis 1 (Nc1 -> Lp1), with the
// calibration, the intermediate and both tables in shared memory.  Each output accumulates its
// terms in the order of the unfused axis passes (bitwise the same spectrum).
// fwdT2: [Nc2][Lp2] (transposed), fwd1: [Lp1][Nc1]; S: [Q][Lp1][Lp2].
__global__ void __launch_bounds__(256) forward_df_kernel(const float2* __restrict__ calib, int Nc1, int Nc2,
                                                         const dfc* __restrict__ fwdT2, int Lp2,
                                                         const dfc* __restrict__ fwd1, int Lp1, dfc* __restrict__ S,
                                                         GramItems it) {
  extern __shared__ dfc fsm[];
  calib += blockIdx.y * it.calib;
  S += blockIdx.y * it.S;
  dfc* T = fsm;                                  // [Nc1][Lp2]
  dfc* m2 = T + Nc1 * Lp2;                       // [Nc2][Lp2]
  dfc* m1 = m2 + Nc2 * Lp2;                      // [Lp1][Nc1]
  float2* cs = reinterpret_cast<float2*>(m1 + Lp1 * Nc1);  // [Nc1][Nc2]
  const int q = blockIdx.x;
  const int tid = threadIdx.x, nt = blockDim.x;
  const float2* cq = calib + (long long)q * Nc1 * Nc2;
  for (int i = tid; i < Nc1 * Nc2; i += nt) cs[i] = cq[i];
  for (int i = tid; i < Nc2 * Lp2; i += nt) m2[i] = fwdT2[i];
  for (int i = tid; i < Lp1 * Nc1; i += nt) m1[i] = fwd1[i];
  __syncthreads();
  for (int o = tid; o < Nc1 * Lp2; o += nt) {
    const int x1 = o / Lp2, f2 = o % Lp2;
    const float2* crow = cs + x1 * Nc2;
    dfc acc{0.f, 0.f, 0.f, 0.f};
    for (int x2 = 0; x2 < Nc2; ++x2) {
      const float2 v = crow[x2];
      df_cfma(acc, m2[x2 * Lp2 + f2], dfc{v.x, 0.f, v.y, 0.f});
    }
    T[o] = acc;
  }
  __syncthreads();
  dfc* out = S + (long long)q * Lp1 * Lp2;
  for (int o = tid; o < Lp1 * Lp2; o += nt) {
    const int f1 = o / Lp2, f2 = o % Lp2;
    const dfc* mrow = m1 + f1 * Nc1;
    dfc acc{0.f, 0.f, 0.f, 0.f};
    for (int x1 = 0; x1 < Nc1; ++x1) df_cfma(acc, mrow[x1], T[x1 * Lp2 + f2]);
    out[o] = acc;
  }
}

size_t forward_df_smem(int Nc1, int Nc2, int Lp1, int Lp2) {
  return ((size_t)Nc1 * Lp2 + (size_t)Nc2 * Lp2 + (size_t)Lp1 * Nc1) * sizeof(dfc) +
         (size_t)Nc1 * Nc2 * sizeof(float2);
}

size_t pairs_inverse_df_smem(int Lp1, int Lp2, int B1, int B2) {
  return ((size_t)Lp1 * (Lp2 | 1) + (size_t)Lp1 * B2 + (size_t)Lp2 * B2 + (size_t)B1 * Lp1) * sizeof(dfc);
}

// A[(p,i),(q,j)] = R_pq[m_i - m_j] (Hermitian mirror for p > q) kept in double-float, and
// A32 = A / scale in FP32, from the double-float lag table: no FP64 arithmetic per entry
__global__ void gram_expand_df_kernel(const dfc* __restrict__ lags_df, const int* __restrict__ lag_of_ij, int Q,
                                      int L, int nbox, const double* __restrict__ scale, dfc* __restrict__ A,
                                      float2* __restrict__ A32, GramItems it) {
  lags_df += blockIdx.y * it.lags;
  scale += blockIdx.y * it.scale;
  A += blockIdx.y * it.A;
  A32 += blockIdx.y * it.A;
  const long long n = (long long)Q * L;
  const float inv = (float)(1.0 / *scale);
  const long long total = n * n;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int col = (int)(idx % n);
    const int row = (int)(idx / n);
    const int p = row / L, i = row % L;
    const int q = col / L, j = col % L;
    dfc v;
    if (p <= q) {
      v = lags_df[((long long)p * Q + q) * nbox + lag_of_ij[i * L + j]];
    } else {
      v = lags_df[((long long)q * Q + p) * nbox + lag_of_ij[j * L + i]];
      v.ih = -v.ih;
      v.il = -v.il;
    }
    A[idx] = v;
    A32[idx] = make_float2(fmaf(v.rh, inv, v.rl * inv), fmaf(v.ih, inv, v.il * inv));
  }
}

__global__ void df_to_fp64_kernel(const dfc* __restrict__ in, long long count, double2* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x) {
    const dfc v = in[i];
    out[i] = make_double2((double)v.rh + (double)v.rl, (double)v.ih + (double)v.il);
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
cudaError_t gram_pair_products_df(const void* S, int Q, long long nfreq, void* P, cudaStream_t st,
                                  const GramItems& it) {
  const int npairs = Q * (Q + 1) / 2;
  int bx = (int)((nfreq + 255) / 256);
  if (bx > 64) bx = 64;
  pair_products_df_kernel<<<dim3(bx, npairs, it.n), 256, 0, st>>>(static_cast<const dfc*>(S), Q, nfreq,
                                                                  static_cast<dfc*>(P), it);
  ++g_launches;
  return cudaGetLastError();
}
cudaError_t gram_expand_df(const void* lags_df, const int* lag_of_ij, int Q, int L, int nbox, const double* scale,
                           void* A, float2* A32, cudaStream_t st, const GramItems& it) {
  const long long n = (long long)Q * L;
  long long blocks = (n * n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  blocks = (blocks + it.n - 1) / it.n;
  gram_expand_df_kernel<<<dim3((unsigned)blocks, it.n), 256, 0, st>>>(static_cast<const dfc*>(lags_df), lag_of_ij, Q,
                                                                      L, nbox, scale, static_cast<dfc*>(A), A32, it);
  ++g_launches;
  return cudaGetLastError();
}
cudaError_t df_to_fp64(const void* in, long long count, double2* out, cudaStream_t st) {
  long long blocks = (count + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  df_to_fp64_kernel<<<(unsigned)blocks, 256, 0, st>>>(static_cast<const dfc*>(in), count, out);
  ++g_launches;
  return cudaGetLastError();
}
bool gram_forward_df_supported(int Nc1, int Nc2, int Lp1, int Lp2) {
  return forward_df_smem(Nc1, Nc2, Lp1, Lp2) <= (size_t)kPairsInverseDfMaxSmem;
}
cudaError_t gram_forward_df(const float2* calib, int Q, int Nc1, int Nc2, const void* fwdT2, int Lp2, const void* fwd1,
                            int Lp1, void* S, cudaStream_t st, const GramItems& it) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(forward_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kPairsInverseDfMaxSmem);
    attr_set = true;
  }
  forward_df_kernel<<<dim3(Q, it.n), 256, forward_df_smem(Nc1, Nc2, Lp1, Lp2), st>>>(
      calib, Nc1, Nc2, static_cast<const dfc*>(fwdT2), Lp2, static_cast<const dfc*>(fwd1), Lp1, static_cast<dfc*>(S),
      it);
  ++g_launches;
  return cudaGetLastError();
}
bool gram_pairs_inverse_df_supported(int Lp1, int Lp2, int B1, int B2) {
  return pairs_inverse_df_smem(Lp1, Lp2, B1, B2) <= (size_t)kPairsInverseDfMaxSmem;
}
cudaError_t gram_pairs_inverse_df(const void* S, int Q, int Lp1, int Lp2, const void* invT2, int B2, const void* inv1,
                                  int B1, double2* lags, void* lags_df, cudaStream_t st, const GramItems& it) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(pairs_inverse_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kPairsInverseDfMaxSmem);
    attr_set = true;
  }
  pairs_inverse_df_kernel<<<dim3(Q * (Q + 1) / 2, it.n), 256, pairs_inverse_df_smem(Lp1, Lp2, B1, B2), st>>>(
      static_cast<const dfc*>(S), Q, Lp1, Lp2, static_cast<const dfc*>(invT2), B2, static_cast<const dfc*>(inv1), B1,
      lags, static_cast<dfc*>(lags_df), it);
  ++g_launches;
  return cudaGetLastError();
}
cudaError_t gram_scatter_pairs_df(const void* Rp, int Q, int nbox, double2* lags, void* lags_df, cudaStream_t st,
                                  const GramItems& it) {
  scatter_pairs_df_kernel<<<dim3(Q * (Q + 1) / 2, it.n), 128, 0, st>>>(static_cast<const dfc*>(Rp), Q, nbox, lags,
                                                                       static_cast<dfc*>(lags_df), it);
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

// an entry of A as double-float parts: FP64 storage is split here, double-float storage read as is
__device__ __forceinline__ void split_entry(const double2& a, float& rh, float& rl, float& ih, float& il) {
  rh = (float)a.x;
  ih = (float)a.y;
  rl = (float)(a.x - (double)rh);
  il = (float)(a.y - (double)ih);
}
__device__ __forceinline__ void split_entry(const float4& a, float& rh, float& rl, float& ih, float& il) {
  rh = a.x;
  rl = a.y;
  ih = a.z;
  il = a.w;
}

// Zb = A * Xb (the band products of the FP64 Rayleigh quotients) in double-float: A's entries as
// hi + lo float pairs, the band vectors exact in FP32 (they come from the FP32 Ritz block).  Each
// product term is accumulated error-free in the manner of Ogita, Rump & Oishi's Dot2 (2005): the
// exact product hi*x as (p, q) by FMA, the running sum s updated by TwoSum (s, r), and the error
// terms q + r + lo*x gathered in a second FP32 accumulator c; s + c carries about 48 bits.  One
// warp per row of A (lanes stride the row: coalesced 16-byte loads), eight rows per CTA sharing the
// band vectors staged column-major in shared memory (consecutive lanes read consecutive words),
// only the used band columns (NBU) multiplied, partial sums combined by warp shuffles.
constexpr int kBandKC = 512;      // k values of Xb staged per pass
constexpr int kBandRows = 8;      // rows per CTA (one warp each)

__device__ __forceinline__ void dot2_term(float& s, float& c, float a_hi, float a_lo, float x) {
  const float p = a_hi * x;
  const float q = fmaf(a_hi, x, -p);
  float t, r;
  two_sum(s, p, t, r);
  s = t;
  c = fmaf(a_lo, x, c + (q + r));
}
__device__ __forceinline__ void dot2_merge(float& s, float& c, float s2, float c2) {
  float t, r;
  two_sum(s, s2, t, r);
  s = t;
  c += c2 + r;
}

template <int NBV, int NBU, typename TA>
__device__ __forceinline__ void band_row_accumulate(const TA* __restrict__ arow, const float2* xs, int kc, int lane,
                                                    float (&sr)[NBV], float (&cr)[NBV], float (&si)[NBV],
                                                    float (&ci)[NBV]) {
  for (int k = lane; k < kc; k += 32) {
    float ahx, alx, ahy, aly;
    split_entry(arow[k], ahx, alx, ahy, aly);
#pragma unroll
    for (int c = 0; c < NBU; ++c) {
      const float2 x = xs[c * kBandKC + k];
      dot2_term(sr[c], cr[c], ahx, alx, x.x);     // Re += Re a Re x
      dot2_term(sr[c], cr[c], -ahy, -aly, x.y);   //      - Im a Im x
      dot2_term(si[c], ci[c], ahx, alx, x.y);     // Im += Re a Im x
      dot2_term(si[c], ci[c], ahy, aly, x.x);     //      + Im a Re x
    }
  }
}

template <int NBV, typename TA>
__global__ void __launch_bounds__(256) band_matvec_df_kernel(const TA* __restrict__ A,
                                                             const double2* __restrict__ Xb, int n,
                                                             const int* __restrict__ band_idx,
                                                             double2* __restrict__ Zb, EigItems it) {
  __shared__ float2 xs[NBV * kBandKC];  // [column][k]
  A += blockIdx.y * it.a;
  Xb += blockIdx.y * it.nb;
  band_idx += blockIdx.y * it.band;
  Zb += blockIdx.y * it.nb;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r = blockIdx.x * kBandRows + warp;
  int nbu = 0;
#pragma unroll
  for (int c = 0; c < NBV; ++c)
    if (band_idx[c] >= 0) nbu = c + 1;
  float sr[NBV], cr[NBV], si[NBV], ci[NBV];
#pragma unroll
  for (int c = 0; c < NBV; ++c) sr[c] = cr[c] = si[c] = ci[c] = 0.f;
  for (int k0 = 0; k0 < n; k0 += kBandKC) {
    const int kc = min(kBandKC, n - k0);
    __syncthreads();
    for (int e = threadIdx.x; e < kc * nbu; e += blockDim.x) {
      const int c = e / kc, k = e % kc;
      const double2 v = Xb[(long long)(k0 + k) * NBV + c];
      xs[c * kBandKC + k] = make_float2((float)v.x, (float)v.y);  // exact: the band vectors are FP32 values
    }
    __syncthreads();
    if (r < n) {
      const TA* arow = A + (long long)r * n + k0;
      switch (nbu) {
        case 1: band_row_accumulate<NBV, 1>(arow, xs, kc, lane, sr, cr, si, ci); break;
        case 2: band_row_accumulate<NBV, 2>(arow, xs, kc, lane, sr, cr, si, ci); break;
        case 3: band_row_accumulate<NBV, 3>(arow, xs, kc, lane, sr, cr, si, ci); break;
        case 4: band_row_accumulate<NBV, 4>(arow, xs, kc, lane, sr, cr, si, ci); break;
        case 5: band_row_accumulate<NBV, 5>(arow, xs, kc, lane, sr, cr, si, ci); break;
        case 6: band_row_accumulate<NBV, 6>(arow, xs, kc, lane, sr, cr, si, ci); break;
        case 7: band_row_accumulate<NBV, 7>(arow, xs, kc, lane, sr, cr, si, ci); break;
        case 8: band_row_accumulate<NBV, 8>(arow, xs, kc, lane, sr, cr, si, ci); break;
        default: break;
      }
    }
  }
  if (r >= n) return;
#pragma unroll
  for (int c = 0; c < NBV; ++c) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float a1 = __shfl_xor_sync(0xffffffffu, sr[c], o), a2 = __shfl_xor_sync(0xffffffffu, cr[c], o);
      const float b1 = __shfl_xor_sync(0xffffffffu, si[c], o), b2 = __shfl_xor_sync(0xffffffffu, ci[c], o);
      dot2_merge(sr[c], cr[c], a1, a2);
      dot2_merge(si[c], ci[c], b1, b2);
    }
  }
  if (lane == 0) {
#pragma unroll
    for (int c = 0; c < NBV; ++c)
      Zb[(long long)r * NBV + c] = make_double2((double)sr[c] + (double)cr[c], (double)si[c] + (double)ci[c]);
  }
}

}  // namespace

cudaError_t eig_band_matvec_df(const void* A, bool a_df, const double2* Xb, int n, int nb, const int* band_idx,
                               double2* Zb, cudaStream_t st, const EigItems& it) {
  if (nb != 8) return cudaErrorInvalidValue;
  const dim3 grid((unsigned)((n + kBandRows - 1) / kBandRows), it.n);
  if (a_df)
    band_matvec_df_kernel<8, float4><<<grid, 256, 0, st>>>(static_cast<const float4*>(A), Xb, n, band_idx, Zb, it);
  else
    band_matvec_df_kernel<8, double2><<<grid, 256, 0, st>>>(static_cast<const double2*>(A), Xb, n, band_idx, Zb, it);
  ++g_launches;
  return cudaGetLastError();
}

}  // namespace pisco
