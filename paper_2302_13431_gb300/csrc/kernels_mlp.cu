// The warm start's per-pixel MLP: inference inside the estimate and training kernels.
//
//   h1 = relu(W1 x + b1),  h2 = relu(W2 h1 + b2),  out = s(x) + W3 h2 + b3
//
// x: the patch of normalised low-resolution coil vectors around the pixel (K = (2r+1)^D
// neighbours of Sec. V-D's apodised images, each divided by the centre's norm and rotated by
// the centre's coil-0 phase, the neighbours as differences from the centre; real and imaginary
// parts interleaved, 2Q reals per neighbour); out:
// the proposed power-iteration start vector (Sec. V-E), 2Q reals.  s(x): the skip term, the
// middle block of x when n_in is an odd multiple of n_out (the centre pixel's own normalised
// vector, the heuristic start), else none; with a zero last layer the network returns it.
//
// Every layer product runs on the tensor cores: warp-level mma.sync m16n8k16 with FP16 operands
// (weights stored in FP16, activations and gradients rounded to FP16 where they enter a
// product) and FP32 accumulation.  Biases, activations, losses and the Adam state stay FP32.
// Weight gradients are summed over the batch in a fixed order (per-chunk partials, then an
// ordered sum scaled by 1/B), so training is bitwise reproducible.  Losses: the mean squared
// error to the target, or the phase-free direction loss 1 - |<o, t>| / (||o|| ||t||) of the
// complex vectors (the distance the power iteration cares about).
#include <cuda_fp16.h>

#include <algorithm>

#include "common.cuh"

namespace pisco {

namespace {
constexpr int TM = 64, TN = 64, TK = 32;  // CTA tile of a product; K step
constexpr int SLD = TK + 8;               // padded smem row (halves): conflict-free fragment loads
constexpr int WCH = 2048;                 // samples per weight-gradient chunk

// C[m][n] = sum_k A[m][k] B[k][n]
//   A: FP32, row-major [M][lda] (AT false) or stored transposed, A[m][k] = Ag[k * lda + m] (AT true)
//   B: FP16 weights W [N][ldb] with B[k][n] = W[n][k] (BT false), or stored [K][ldb] (BT true),
//      FP16 or FP32; bias_col >= 0: column n == bias_col of B is 1 (the bias gradient)
// Epilogues: EPI_STORE (plain, split-K partial at z), EPI_BIAS_RELU / EPI_BIAS (+ bias, ReLU,
// optional skip R[m][skip_off + n]), EPI_MASK (multiplied by Hact[m][n] > 0).
enum { EPI_STORE = 0, EPI_BIAS_RELU = 1, EPI_BIAS = 2, EPI_MASK = 3 };

struct GemmArgs {
  int M, N, K;
  const float* A;
  long long lda;
  const void* B;
  long long ldb;
  int bias_col;
  float* C;
  long long ldc;
  long long c_split;  // EPI_STORE: elements between split-K partials (blockIdx.z)
  int kchunk;         // K per blockIdx.z (split-K), else K
  const float* bias;
  const float* R;     // skip source (EPI_BIAS), row stride r_ld, column offset skip_off
  long long r_ld;
  int skip_off;
  const float* Hact;  // EPI_MASK
};

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <typename TB>
__device__ __forceinline__ float load_b(const TB* p) { return (float)p[0]; }
template <>
__device__ __forceinline__ float load_b<__half>(const __half* p) { return __half2float(p[0]); }

// 128 threads = 4 warps in 2 x 2, each warp a 32 x 32 block of the 64 x 64 tile (2 x 4 mma tiles)
template <bool AT, bool BT, typename TB, int EPI>
__global__ void __launch_bounds__(128) mlp_gemm_kernel(GemmArgs g) {
  __shared__ __align__(16) __half As[TM * SLD];  // [m][k]
  __shared__ __align__(16) __half Bs[TN * SLD];  // [n][k]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int gq = lane >> 2, tq = lane & 3;  // mma fragment row group, thread in group
  const long long m0 = (long long)blockIdx.y * TM;
  const int n0 = blockIdx.x * TN;
  const int kb = blockIdx.z * g.kchunk, ke = min(g.K, kb + g.kchunk);
  const TB* Bg = static_cast<const TB*>(g.B);
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[i][j][c] = 0.f;
  for (int k0 = kb; k0 < ke; k0 += TK) {
    __syncthreads();
    // stage A (64 x 32) and B (64 x 32) as FP16, zero outside the matrices
    for (int e = tid; e < TM * TK; e += 128) {
      int mm, kk;
      if (AT) { mm = e % TM; kk = e / TM; }   // consecutive threads along m (contiguous)
      else { kk = e % TK; mm = e / TK; }      // consecutive threads along k (contiguous)
      const long long gm = m0 + mm;
      const int gk = k0 + kk;
      float v = 0.f;
      if (gm < g.M && gk < ke) v = AT ? g.A[(long long)gk * g.lda + gm] : g.A[gm * g.lda + gk];
      As[mm * SLD + kk] = __float2half_rn(v);
    }
    for (int e = tid; e < TN * TK; e += 128) {
      int nn, kk;
      if (BT) { nn = e % TN; kk = e / TN; }
      else { kk = e % TK; nn = e / TK; }
      const int gn = n0 + nn, gk = k0 + kk;
      float v = 0.f;
      if (gk < ke) {
        if (gn == g.bias_col) v = 1.f;
        else if (gn < g.N) v = BT ? load_b<TB>(Bg + (long long)gk * g.ldb + gn) : load_b<TB>(Bg + (long long)gn * g.ldb + gk);
      }
      Bs[nn * SLD + kk] = __float2half_rn(v);
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < TK; ks += 16) {
      uint32_t af[2][4], bf[4][2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const __half* ap = As + (wm + 16 * i + gq) * SLD + ks + 2 * tq;
        af[i][0] = *reinterpret_cast<const uint32_t*>(ap);
        af[i][1] = *reinterpret_cast<const uint32_t*>(ap + 8 * SLD);
        af[i][2] = *reinterpret_cast<const uint32_t*>(ap + 8);
        af[i][3] = *reinterpret_cast<const uint32_t*>(ap + 8 * SLD + 8);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const __half* bp = Bs + (wn + 8 * j + gq) * SLD + ks + 2 * tq;
        bf[j][0] = *reinterpret_cast<const uint32_t*>(bp);
        bf[j][1] = *reinterpret_cast<const uint32_t*>(bp + 8);
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) mma16816(acc[i][j], af[i], bf[j]);
    }
  }
  // epilogue: accumulator (i, j, c) holds C[wm + 16 i + gq + 8 (c >= 2)][wn + 8 j + 2 tq + (c & 1)]
  float* C = g.C + (EPI == EPI_STORE ? (long long)blockIdx.z * g.c_split : 0);
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const long long gm = m0 + wm + 16 * i + gq + ((c >> 1) << 3);
        const int gn = n0 + wn + 8 * j + 2 * tq + (c & 1);
        const int ncols = (EPI == EPI_STORE && g.bias_col >= 0) ? g.bias_col + 1 : g.N;
        if (gm >= g.M || gn >= ncols) continue;
        float v = acc[i][j][c];
        if (EPI == EPI_BIAS_RELU) v = fmaxf(v + g.bias[gn], 0.f);
        if (EPI == EPI_BIAS) {
          v += g.bias[gn];
          if (g.R) v += g.R[gm * g.r_ld + g.skip_off + gn];
        }
        if (EPI == EPI_MASK && !(g.Hact[gm * g.ldc + gn] > 0.f)) v = 0.f;
        C[gm * g.ldc + gn] = v;
      }
}

template <bool AT, bool BT, typename TB, int EPI>
cudaError_t gemm(const GemmArgs& g, int splits, cudaStream_t st) {
  dim3 grid((unsigned)((std::max(g.N, g.bias_col + 1) + TN - 1) / TN), (unsigned)((g.M + TM - 1) / TM),
            (unsigned)splits);
  mlp_gemm_kernel<AT, BT, TB, EPI><<<grid, 128, 0, st>>>(g);
  ++g_launches;
  return cudaGetLastError();
}

// g[o][i] (i < I) and gb[o]: ordered sum of the chunk partials, scaled by inv_b (1/B: the
// per-sample gradients enter the products unscaled, so that their FP16 rounding keeps its range)
__global__ void reduce_weight_parts_kernel(const float* __restrict__ part, int nchunk, int O, int I, float inv_b,
                                           float* __restrict__ gW, float* __restrict__ gb) {
  const int W1 = I + 1;
  const int nout = O * W1;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nout; e += gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int c = 0; c < nchunk; ++c) s += part[(long long)c * nout + e];
    s *= inv_b;
    const int o = e / W1, i = e % W1;
    if (i < I) gW[o * I + i] = s;
    else gb[o] = s;
  }
}

// per-sample loss gradients (unscaled) and per-CTA partial sums of the per-sample losses
//   kind 0 (squared error): l = ||o - t||^2, dl/do = 2 (o - t)
//   kind 1 (direction): with s = <o, t> = sum_q conj(o_q) t_q over the Q complex entries,
//     l = 1 - |s| / (||o|| ||t||), dl/do = -(t e^{-i arg s} / ||o|| - |s| o / ||o||^3) / ||t||
__global__ void __launch_bounds__(256) loss_kernel(const float* __restrict__ out, const float* __restrict__ t,
                                                   long long B, int n, int kind, float* __restrict__ dout,
                                                   float* __restrict__ loss_part) {
  __shared__ float red[256];
  float acc = 0.f;
  for (long long b = blockIdx.x * 256ll + threadIdx.x; b < B; b += (long long)gridDim.x * 256) {
    const float* o = out + b * n;
    const float* tt = t + b * n;
    float* d = dout + b * n;
    if (kind == 0) {
      for (int e = 0; e < n; ++e) {
        const float df = o[e] - tt[e];
        d[e] = 2.f * df;
        acc = fmaf(df, df, acc);
      }
    } else {
      float sr = 0.f, si = 0.f, oo = 0.f, ttn = 0.f;
      for (int e = 0; e + 1 < n; e += 2) {
        const float orr = o[e], oi = o[e + 1], tr = tt[e], ti = tt[e + 1];
        sr = fmaf(orr, tr, fmaf(oi, ti, sr));   // Re conj(o) t
        si = fmaf(orr, ti, fmaf(-oi, tr, si));  // Im conj(o) t
        oo = fmaf(orr, orr, fmaf(oi, oi, oo));
        ttn = fmaf(tr, tr, fmaf(ti, ti, ttn));
      }
      const float as = sqrtf(sr * sr + si * si);
      const float no = sqrtf(oo), nt = sqrtf(ttn);
      if (no > 0.f && nt > 0.f) {
        const float er = as > 0.f ? sr / as : 1.f, ei = as > 0.f ? -si / as : 0.f;  // e^{-i arg s}
        const float c1 = 1.f / (no * nt), c2 = as / (no * no * no * nt);
        for (int e = 0; e + 1 < n; e += 2) {
          const float tr = tt[e], ti = tt[e + 1];
          d[e] = -((tr * er - ti * ei) * c1 - o[e] * c2);
          d[e + 1] = -((tr * ei + ti * er) * c1 - o[e + 1] * c2);
        }
        acc += 1.f - as / (no * nt);
      } else {
        for (int e = 0; e < n; ++e) d[e] = 0.f;
      }
    }
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) loss_part[blockIdx.x] = red[0];
}

__global__ void adam_kernel(float* __restrict__ w, __half* __restrict__ w16, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, long long n, float lr, float b1,
                            float b2, float eps, float c1, float c2) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const float ge = g[e];
    const float me = b1 * m[e] + (1.f - b1) * ge;
    const float ve = b2 * v[e] + (1.f - b2) * ge * ge;
    m[e] = me;
    v[e] = ve;
    const float mh = me / c1, vh = ve / c2;
    const float we = w[e] - lr * mh / (sqrtf(vh) + eps);
    w[e] = we;
    w16[e] = __float2half_rn(we);
  }
}

__global__ void to_half_kernel(const float* __restrict__ w, __half* __restrict__ w16, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    w16[e] = __float2half_rn(w[e]);
}

// network input from the low-resolution images Y [Q][npix] on the reduced grid dims (z, y, x;
// periodic): with u(k) = y(k) conj(y_0(j)) / (|y_0(j)| ||y(j)||), the centre block u(j) and, for
// every other neighbour o of the (2r+1)^D patch (z slowest, x fastest), u(j + o) - u(j) (small
// numbers that keep their precision when rounded to FP16 for the first product); real and
// imaginary parts interleaved; a pixel with y(j) = 0 gets zeros, a zero y_0(j) no rotation.
__global__ void patch_features_kernel(const float2* __restrict__ Y, int Q, int nz, int ny, int nx, int r, int D,
                                      float* __restrict__ X) {
  const long long npix = (long long)nz * ny * nx;
  const int w = 2 * r + 1;
  const int K = D == 3 ? w * w * w : w * w;
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < npix; j += (long long)gridDim.x * blockDim.x) {
    float n2 = 0.f;
    for (int q = 0; q < Q; ++q) {
      const float2 y = Y[(long long)q * npix + j];
      n2 = fmaf(y.x, y.x, fmaf(y.y, y.y, n2));
    }
    const float2 y0 = Y[j];
    const float a0 = sqrtf(y0.x * y0.x + y0.y * y0.y);
    const float s = n2 > 0.f ? rsqrtf(n2) : 0.f;
    // multiply by conj(y0 / |y0|) * s
    const float cr = a0 > 0.f ? y0.x / a0 * s : s, ci = a0 > 0.f ? -y0.y / a0 * s : 0.f;
    const int x = (int)(j % nx), yy = (int)((j / nx) % ny), z = (int)(j / ((long long)nx * ny));
    float* out = X + j * (long long)K * 2 * Q;
    const int kc = K / 2;  // the centre
    int k = 0;
    for (int dz = (D == 3 ? -r : 0); dz <= (D == 3 ? r : 0); ++dz)
      for (int dy = -r; dy <= r; ++dy)
        for (int dx = -r; dx <= r; ++dx, ++k) {
          const int zz = (z + dz + nz) % nz, y2 = (yy + dy + ny) % ny, x2 = (x + dx + nx) % nx;
          const long long jn = ((long long)zz * ny + y2) * nx + x2;
          for (int q = 0; q < Q; ++q) {
            const float2 v = Y[(long long)q * npix + jn];
            float ur = v.x * cr - v.y * ci, ui = v.x * ci + v.y * cr;
            if (k != kc) {
              const float2 c = Y[(long long)q * npix + j];
              ur -= c.x * cr - c.y * ci;
              ui -= c.x * ci + c.y * cr;
            }
            out[(k * Q + q) * 2] = ur;
            out[(k * Q + q) * 2 + 1] = ui;
          }
        }
  }
}

unsigned grid_for(long long n, int per) { long long b = (n + per - 1) / per; return (unsigned)(b > 152 * 16 ? 152 * 16 : (b < 1 ? 1 : b)); }

}  // namespace

cudaError_t mlp_prepare() { return cudaSuccess; }

size_t mlp_param_count(int n_in, int H, int n_out) {
  return (size_t)H * n_in + H + (size_t)H * H + H + (size_t)n_out * H + n_out;
}

// offsets of W1, b1, W2, b2, W3, b3 in the parameter blob
static void offsets(int n_in, int H, int n_out, size_t o[6]) {
  o[0] = 0;
  o[1] = o[0] + (size_t)H * n_in;
  o[2] = o[1] + H;
  o[3] = o[2] + (size_t)H * H;
  o[4] = o[3] + H;
  o[5] = o[4] + (size_t)n_out * H;
}

// the skip term's column offset in x: the middle block when n_in is an odd multiple of n_out
int mlp_skip_offset(int n_in, int n_out) {
  if (n_in % n_out != 0 || ((n_in / n_out) & 1) == 0) return -1;
  return (n_in / n_out / 2) * n_out;
}

static GemmArgs fwd_args(const float* A, long long B, int I, const __half* W, const float* bias, int O, float* Y) {
  GemmArgs g{};
  g.M = (int)B;
  g.N = O;
  g.K = I;
  g.A = A;
  g.lda = I;
  g.B = W;
  g.ldb = I;
  g.bias_col = -1;
  g.C = Y;
  g.ldc = O;
  g.kchunk = I;
  g.bias = bias;
  return g;
}

cudaError_t mlp_forward(const MlpView& m, const float* X, long long B, float* H1, float* H2, float* out,
                        cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
  size_t o[6];
  offsets(m.n_in, m.H, m.n_out, o);
  cudaError_t e = gemm<false, false, __half, EPI_BIAS_RELU>(fwd_args(X, B, m.n_in, m.w16 + o[0], m.w32 + o[1], m.H, H1), 1, st);
  if (e == cudaSuccess)
    e = gemm<false, false, __half, EPI_BIAS_RELU>(fwd_args(H1, B, m.H, m.w16 + o[2], m.w32 + o[3], m.H, H2), 1, st);
  if (e != cudaSuccess) return e;
  GemmArgs g3 = fwd_args(H2, B, m.H, m.w16 + o[4], m.w32 + o[5], m.n_out, out);
  const int so = mlp_skip_offset(m.n_in, m.n_out);
  if (so >= 0) {
    g3.R = X;
    g3.r_ld = m.n_in;
    g3.skip_off = so;
  }
  return gemm<false, false, __half, EPI_BIAS>(g3, 1, st);
}

// weight gradient of one layer: part[c][o][i] = sum over chunk c of dY[b][o] Xin[b][i], bias
// column i = I; then the ordered chunk sum / B into gW, gb
static cudaError_t weight_grad(const float* dY, long long B, int O, const float* Xin, int I, float* part,
                               float* gW, float* gb, cudaStream_t st) {
  GemmArgs g{};
  g.M = O;
  g.N = I;
  g.K = (int)B;
  g.A = dY;
  g.lda = O;
  g.B = Xin;
  g.ldb = I;
  g.bias_col = I;
  g.C = part;
  g.ldc = I + 1;
  g.c_split = (long long)O * (I + 1);
  g.kchunk = WCH;
  const int nch = (int)((B + WCH - 1) / WCH);
  cudaError_t e = gemm<true, true, float, EPI_STORE>(g, nch, st);
  if (e != cudaSuccess) return e;
  reduce_weight_parts_kernel<<<grid_for((long long)O * (I + 1), 256), 256, 0, st>>>(part, nch, O, I, 1.f / (float)B,
                                                                                  gW, gb);
  ++g_launches;
  return cudaGetLastError();
}

// dX[b][i] = (sum_o dY[b][o] W[o][i]) * (Hact[b][i] > 0)
static cudaError_t data_grad(const float* dY, long long B, int O, const __half* W, int I, const float* Hact,
                             float* dX, cudaStream_t st) {
  GemmArgs g{};
  g.M = (int)B;
  g.N = I;
  g.K = O;
  g.A = dY;
  g.lda = O;
  g.B = W;
  g.ldb = I;
  g.bias_col = -1;
  g.C = dX;
  g.ldc = I;
  g.kchunk = O;
  g.Hact = Hact;
  return gemm<false, true, __half, EPI_MASK>(g, 1, st);
}

cudaError_t mlp_backward(const MlpView& m, const float* X, const float* T, long long B, float* H1, float* H2,
                         float* out, float* dO, float* dH2, float* dH1, float* part, float* grad,
                         float* loss_part, int loss_blocks, int loss_kind, cudaStream_t st) {
  size_t o[6];
  offsets(m.n_in, m.H, m.n_out, o);
  cudaError_t e = mlp_forward(m, X, B, H1, H2, out, st);
  if (e != cudaSuccess || B <= 0) return e;
  loss_kernel<<<loss_blocks, 256, 0, st>>>(out, T, B, m.n_out, loss_kind, dO, loss_part);
  ++g_launches;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // layer 3: gW3, gb3 from dO and H2; dH2 = (dO W3) * (H2 > 0)
  if ((e = weight_grad(dO, B, m.n_out, H2, m.H, part, grad + o[4], grad + o[5], st)) != cudaSuccess) return e;
  if ((e = data_grad(dO, B, m.n_out, m.w16 + o[4], m.H, H2, dH2, st)) != cudaSuccess) return e;
  // layer 2
  if ((e = weight_grad(dH2, B, m.H, H1, m.H, part, grad + o[2], grad + o[3], st)) != cudaSuccess) return e;
  if ((e = data_grad(dH2, B, m.H, m.w16 + o[2], m.H, H1, dH1, st)) != cudaSuccess) return e;
  // layer 1
  return weight_grad(dH1, B, m.H, X, m.n_in, part, grad + o[0], grad + o[1], st);
}

cudaError_t mlp_adam(float* w32, __half* w16, const float* g, float* m1, float* m2, long long n, float lr,
                     float b1, float b2, float eps, int step, cudaStream_t st) {
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  adam_kernel<<<grid_for(n, 256), 256, 0, st>>>(w32, w16, g, m1, m2, n, lr, b1, b2, eps, c1, c2);
  ++g_launches;
  return cudaGetLastError();
}

cudaError_t mlp_to_half(const float* w32, __half* w16, long long n, cudaStream_t st) {
  to_half_kernel<<<grid_for(n, 256), 256, 0, st>>>(w32, w16, n);
  ++g_launches;
  return cudaGetLastError();
}

cudaError_t mlp_patch_features(const float2* Y, int Q, const int dims[3], int r, int D, float* X, cudaStream_t st) {
  const long long npix = (long long)dims[0] * dims[1] * dims[2];
  patch_features_kernel<<<grid_for(npix, 128), 128, 0, st>>>(Y, Q, dims[0], dims[1], dims[2], r, D, X);
  ++g_launches;
  return cudaGetLastError();
}

cudaError_t mlp_features(const float2* Y, int Q, long long npix, float* X, cudaStream_t st) {
  const int dims[3] = {1, 1, (int)npix};
  return mlp_patch_features(Y, Q, dims, 0, 2, X, st);
}

size_t mlp_part_floats(long long max_batch, int n_in, int H, int n_out) {
  const long long nch = (max_batch + WCH - 1) / WCH;
  const int w = std::max(n_in, H) + 1;
  return (size_t)nch * (size_t)std::max(H, n_out) * w;
}

}  // namespace pisco
