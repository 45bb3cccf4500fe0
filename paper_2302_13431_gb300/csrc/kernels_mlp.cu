// The warm start's per-pixel MLP: inference inside the estimate and training kernels.
//
//   h1 = relu(W1 x + b1),  h2 = relu(W2 h1 + b2),  out = x + W3 h2 + b3
//
// (the skip term x whenever the input and output widths agree: the network corrects the
// heuristic start y(x)/||y(x)||; with a zero last layer it returns it unchanged).
//
// x: the pixel's low-resolution coil vector y(x)/||y(x)|| (Sec. V-D), real and imaginary parts
// interleaved (2Q reals); out: the proposed power-iteration start vector (Sec. V-E), same
// layout.  Weight matrices are FP16 (converted to FP32 in shared memory), biases FP32, all
// accumulation FP32.  Training minimises the mean squared error to a target vector with Adam
// on FP32 master weights; the weight gradients are reduced over the batch in a fixed order
// (per-chunk partials, then an ordered sum), so training is bitwise reproducible.
//
// Layers are at most 128 wide.  A CTA owns 64 samples (rows); its 256 threads each own one
// row and every 4th output column, the layer's weights and the row tile sit in shared memory
// with odd row strides (bank-conflict-free reads).
#include <cuda_fp16.h>

#include <algorithm>

#include "common.cuh"

namespace pisco {

namespace {
constexpr int ROWS = 64;
constexpr int MAXW = 128;
constexpr int WCH = 256;  // samples per weight-gradient chunk
constexpr int WROWS = 32; // samples per shared-memory sub-chunk of the weight gradient

// Y[r][o] = act(sum_i X[r][i] W[o][i] + b[o]) (+ R[r][o] when R is given: the skip term)
template <bool RELU>
__global__ void __launch_bounds__(256) linear_fwd_kernel(const float* __restrict__ X, int B, int I,
                                                         const __half* __restrict__ W,
                                                         const float* __restrict__ bias, int O,
                                                         const float* __restrict__ R,
                                                         float* __restrict__ Y) {
  extern __shared__ float sm[];
  float* Ws = sm;                  // O x (I + 1)
  float* Xs = Ws + O * (I + 1);    // ROWS x (I + 1)
  const int tid = threadIdx.x;
  const long long r0 = (long long)blockIdx.x * ROWS;
  for (int e = tid; e < O * I; e += 256) Ws[(e / I) * (I + 1) + e % I] = __half2float(W[e]);
  for (int e = tid; e < ROWS * I; e += 256) {
    const long long r = r0 + e / I;
    Xs[(e / I) * (I + 1) + e % I] = (r < B) ? X[r * I + e % I] : 0.f;
  }
  __syncthreads();
  const int r = tid >> 2, oc = tid & 3;
  float acc[MAXW / 4];
#pragma unroll
  for (int j = 0; j < MAXW / 4; ++j) acc[j] = 0.f;
  const float* xr = Xs + r * (I + 1);
  for (int i = 0; i < I; ++i) {
    const float xv = xr[i];
#pragma unroll
    for (int j = 0; j < MAXW / 4; ++j) {
      const int o = oc + 4 * j;
      if (o < O) acc[j] = fmaf(xv, Ws[o * (I + 1) + i], acc[j]);
    }
  }
  const long long gr = r0 + r;
  if (gr < B) {
#pragma unroll
    for (int j = 0; j < MAXW / 4; ++j) {
      const int o = oc + 4 * j;
      if (o < O) {
        float v = acc[j] + bias[o];
        if (RELU) v = fmaxf(v, 0.f);
        if (R != nullptr) v += R[gr * O + o];
        Y[gr * O + o] = v;
      }
    }
  }
}

// dX[r][i] = (sum_o dY[r][o] W[o][i]) * (Xact[r][i] > 0 if Xact)
__global__ void __launch_bounds__(256) linear_bwd_data_kernel(const float* __restrict__ dY, int B, int O,
                                                              const __half* __restrict__ W, int I,
                                                              const float* __restrict__ Xact,
                                                              float* __restrict__ dX) {
  extern __shared__ float sm[];
  float* Ws = sm;                  // O x (I + 1)
  float* Ds = Ws + O * (I + 1);    // ROWS x (O + 1)
  const int tid = threadIdx.x;
  const long long r0 = (long long)blockIdx.x * ROWS;
  for (int e = tid; e < O * I; e += 256) Ws[(e / I) * (I + 1) + e % I] = __half2float(W[e]);
  for (int e = tid; e < ROWS * O; e += 256) {
    const long long r = r0 + e / O;
    Ds[(e / O) * (O + 1) + e % O] = (r < B) ? dY[r * O + e % O] : 0.f;
  }
  __syncthreads();
  const int r = tid >> 2, ic = tid & 3;
  float acc[MAXW / 4];
#pragma unroll
  for (int j = 0; j < MAXW / 4; ++j) acc[j] = 0.f;
  const float* dr = Ds + r * (O + 1);
  for (int o = 0; o < O; ++o) {
    const float dv = dr[o];
    const float* wr = Ws + o * (I + 1);
#pragma unroll
    for (int j = 0; j < MAXW / 4; ++j) {
      const int i = ic + 4 * j;
      if (i < I) acc[j] = fmaf(dv, wr[i], acc[j]);
    }
  }
  const long long gr = r0 + r;
  if (gr < B) {
#pragma unroll
    for (int j = 0; j < MAXW / 4; ++j) {
      const int i = ic + 4 * j;
      if (i < I) {
        float v = acc[j];
        if (Xact != nullptr && !(Xact[gr * I + i] > 0.f)) v = 0.f;
        dX[gr * I + i] = v;
      }
    }
  }
}

// per chunk c of WCH samples: part[c][o][i] = sum_b dY[b][o] X[b][i] (i < I), part[c][o][I] =
// sum_b dY[b][o]  (the bias gradient)
__global__ void __launch_bounds__(256) linear_bwd_weight_kernel(const float* __restrict__ dY, int B, int O,
                                                                const float* __restrict__ X, int I,
                                                                float* __restrict__ part) {
  __shared__ float Ds[WROWS][MAXW + 1];
  __shared__ float Xs[WROWS][MAXW + 1];
  const int tid = threadIdx.x;
  const int W1 = I + 1;  // I weight columns + the bias column
  const int nout = O * W1;
  float acc[(MAXW * (MAXW + 1) + 255) / 256];
  constexpr int NA = (MAXW * (MAXW + 1) + 255) / 256;
#pragma unroll
  for (int j = 0; j < NA; ++j) acc[j] = 0.f;
  const long long c0 = (long long)blockIdx.x * WCH;
  for (int s = 0; s < WCH; s += WROWS) {
    __syncthreads();
    for (int e = tid; e < WROWS * O; e += 256) {
      const long long b = c0 + s + e / O;
      Ds[e / O][e % O] = (b < B) ? dY[b * O + e % O] : 0.f;
    }
    for (int e = tid; e < WROWS * I; e += 256) {
      const long long b = c0 + s + e / I;
      Xs[e / I][e % I] = (b < B) ? X[b * I + e % I] : 0.f;
    }
    for (int e = tid; e < WROWS; e += 256) Xs[e][I] = 1.f;  // bias column
    __syncthreads();
#pragma unroll
    for (int j = 0; j < NA; ++j) {
      const int e = tid + 256 * j;
      if (e < nout) {
        const int o = e / W1, i = e % W1;
        float a = acc[j];
        for (int b = 0; b < WROWS; ++b) a = fmaf(Ds[b][o], Xs[b][i], a);
        acc[j] = a;
      }
    }
  }
  float* out = part + (long long)blockIdx.x * nout;
#pragma unroll
  for (int j = 0; j < NA; ++j) {
    const int e = tid + 256 * j;
    if (e < nout) out[e] = acc[j];
  }
}

// g[o][i] (i < I) and gb[o]: ordered sum of the chunk partials
__global__ void reduce_weight_parts_kernel(const float* __restrict__ part, int nchunk, int O, int I,
                                           float* __restrict__ gW, float* __restrict__ gb) {
  const int W1 = I + 1;
  const int nout = O * W1;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nout; e += gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int c = 0; c < nchunk; ++c) s += part[(long long)c * nout + e];
    const int o = e / W1, i = e % W1;
    if (i < I) gW[o * I + i] = s;
    else gb[o] = s;
  }
}

// dOut = 2 (out - t) / B; per-CTA partial sums of ||out - t||^2 (fixed-order tree)
__global__ void __launch_bounds__(256) mse_kernel(const float* __restrict__ out, const float* __restrict__ t,
                                                  long long n, float scale, float* __restrict__ dout,
                                                  float* __restrict__ loss_part) {
  __shared__ float red[256];
  float s = 0.f;
  for (long long e = blockIdx.x * 256ll + threadIdx.x; e < n; e += (long long)gridDim.x * 256) {
    const float d = out[e] - t[e];
    dout[e] = 2.f * d * scale;
    s = fmaf(d, d, s);
  }
  red[threadIdx.x] = s;
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

// network input from the low-resolution images Y [Q][npix]: x[j] = y_j / ||y_j||, interleaved
__global__ void mlp_features_kernel(const float2* __restrict__ Y, int Q, long long npix, float* __restrict__ X) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < npix; j += (long long)gridDim.x * blockDim.x) {
    float n2 = 0.f;
    for (int q = 0; q < Q; ++q) {
      const float2 y = Y[(long long)q * npix + j];
      n2 = fmaf(y.x, y.x, fmaf(y.y, y.y, n2));
    }
    const float s = n2 > 0.f ? rsqrtf(n2) : 0.f;
    for (int q = 0; q < Q; ++q) {
      const float2 y = Y[(long long)q * npix + j];
      X[j * 2 * Q + 2 * q] = y.x * s;
      X[j * 2 * Q + 2 * q + 1] = y.y * s;
    }
  }
}

size_t fwd_smem(int I, int O) { return sizeof(float) * ((size_t)O * (I + 1) + (size_t)ROWS * (I + 1)); }
size_t bwd_smem(int I, int O) { return sizeof(float) * ((size_t)O * (I + 1) + (size_t)ROWS * (O + 1)); }
unsigned grid_for(long long n, int per) { long long b = (n + per - 1) / per; return (unsigned)(b > 152 * 16 ? 152 * 16 : (b < 1 ? 1 : b)); }

}  // namespace

cudaError_t mlp_prepare() {
  const int big = (int)std::max(fwd_smem(MAXW, MAXW), bwd_smem(MAXW, MAXW));
  cudaError_t e = cudaFuncSetAttribute(linear_fwd_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(linear_fwd_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(linear_bwd_data_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  return e;
}

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

cudaError_t mlp_forward(const MlpView& m, const float* X, long long B, float* H1, float* H2, float* out,
                        cudaStream_t st) {
  size_t o[6];
  offsets(m.n_in, m.H, m.n_out, o);
  const unsigned blocks = (unsigned)((B + ROWS - 1) / ROWS);
  if (B <= 0) return cudaSuccess;
  const float* skip = (m.n_in == m.n_out) ? X : nullptr;  // out = x + W3 h2 + b3
  linear_fwd_kernel<true><<<blocks, 256, fwd_smem(m.n_in, m.H), st>>>(X, (int)B, m.n_in, m.w16 + o[0], m.w32 + o[1], m.H, nullptr, H1);
  linear_fwd_kernel<true><<<blocks, 256, fwd_smem(m.H, m.H), st>>>(H1, (int)B, m.H, m.w16 + o[2], m.w32 + o[3], m.H, nullptr, H2);
  linear_fwd_kernel<false><<<blocks, 256, fwd_smem(m.H, m.n_out), st>>>(H2, (int)B, m.H, m.w16 + o[4], m.w32 + o[5], m.n_out, skip, out);
  g_launches += 3;
  return cudaGetLastError();
}

cudaError_t mlp_backward(const MlpView& m, const float* X, const float* T, long long B, float* H1, float* H2,
                         float* out, float* dO, float* dH2, float* dH1, float* part, float* grad,
                         float* loss_part, int loss_blocks, cudaStream_t st) {
  size_t o[6];
  offsets(m.n_in, m.H, m.n_out, o);
  cudaError_t e = mlp_forward(m, X, B, H1, H2, out, st);
  if (e != cudaSuccess || B <= 0) return e;
  const unsigned blocks = (unsigned)((B + ROWS - 1) / ROWS);
  const unsigned nch = (unsigned)((B + WCH - 1) / WCH);
  mse_kernel<<<loss_blocks, 256, 0, st>>>(out, T, B * m.n_out, 1.0f / (float)B, dO, loss_part);
  // layer 3: gW3, gb3 from dO and H2; dH2 = (dO W3) * (H2 > 0)
  linear_bwd_weight_kernel<<<nch, 256, 0, st>>>(dO, (int)B, m.n_out, H2, m.H, part);
  reduce_weight_parts_kernel<<<grid_for((long long)m.n_out * (m.H + 1), 256), 256, 0, st>>>(part, nch, m.n_out, m.H, grad + o[4], grad + o[5]);
  linear_bwd_data_kernel<<<blocks, 256, bwd_smem(m.H, m.n_out), st>>>(dO, (int)B, m.n_out, m.w16 + o[4], m.H, H2, dH2);
  // layer 2
  linear_bwd_weight_kernel<<<nch, 256, 0, st>>>(dH2, (int)B, m.H, H1, m.H, part);
  reduce_weight_parts_kernel<<<grid_for((long long)m.H * (m.H + 1), 256), 256, 0, st>>>(part, nch, m.H, m.H, grad + o[2], grad + o[3]);
  linear_bwd_data_kernel<<<blocks, 256, bwd_smem(m.H, m.H), st>>>(dH2, (int)B, m.H, m.w16 + o[2], m.H, H1, dH1);
  // layer 1
  linear_bwd_weight_kernel<<<nch, 256, 0, st>>>(dH1, (int)B, m.H, X, m.n_in, part);
  reduce_weight_parts_kernel<<<grid_for((long long)m.H * (m.n_in + 1), 256), 256, 0, st>>>(part, nch, m.H, m.n_in, grad + o[0], grad + o[1]);
  g_launches += 8;
  return cudaGetLastError();
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

cudaError_t mlp_features(const float2* Y, int Q, long long npix, float* X, cudaStream_t st) {
  mlp_features_kernel<<<grid_for(npix, 256), 256, 0, st>>>(Y, Q, npix, X);
  ++g_launches;
  return cudaGetLastError();
}

size_t mlp_part_floats(long long max_batch, int n_in, int H, int n_out) {
  const long long nch = (max_batch + WCH - 1) / WCH;
  const int w = std::max(n_in, H) + 1;
  return (size_t)nch * (size_t)std::max(H, n_out) * w;
}

}  // namespace pisco
