// Stages (d)+(e, phase): simultaneous power iteration over all reduced-grid pixels
// (Sec. V-E) on B(x) = I - G(x)/|Lambda| (Eq. esp_null), followed by the smooth phase step
// of Sec. V-D: v <- v * rho/|rho| with rho = v^H y(x), y the apodised low-resolution coil
// images, so that the coil-combined reconstruction becomes real and non-negative.
//
// A CTA holds PIX pixels; the Q x Q matrix of every pixel is staged once in shared memory
// (pixel-major, row p contiguous) and the Q threads of a pixel each own one coil.  Thread q
// forms (G v)_q = sum_p conj(G_pq) v_p from row p (Hermitian), which makes the Q lanes read
// consecutive shared-memory words; v is broadcast from shared memory.  All iterations run
// out of shared memory, so G is read from HBM once.
#include "common.cuh"

namespace pisco {

template <int QP>
__device__ __forceinline__ float pixel_sum(float v, float* red, int xi, int q) {
  if constexpr (QP <= 32) {
#pragma unroll
    for (int o = QP / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
  } else {
    // QP == 64: two warps per pixel
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((q & 31) == 0) red[xi * 2 + (q >> 5)] = v;
    __syncthreads();
    const float s = red[xi * 2] + red[xi * 2 + 1];
    __syncthreads();
    return s;
  }
}

template <int QP>
__global__ void __launch_bounds__(256) pi_kernel(const float2* __restrict__ G,
                                                 const float2* __restrict__ Y, int Q,
                                                 long long npix, int iters, float lam_size,
                                                 unsigned long long seed, float2* __restrict__ V,
                                                 float* __restrict__ eig) {
  constexpr int PIX = 256 / QP;
  extern __shared__ float2 sm[];
  const long long QQ = (long long)Q * Q;
  const long long GST = QQ + 1;             // padded per-pixel stride (bank spread)
  float2* Gs = sm;                          // PIX * GST
  float2* vs = Gs + (size_t)PIX * GST;      // PIX * QP
  float* red = reinterpret_cast<float*>(vs + PIX * QP);  // PIX * 2
  const int tid = threadIdx.x;
  const int xi = tid / QP, q = tid % QP;
  const long long x0 = (long long)blockIdx.x * PIX;
  const long long x = x0 + xi;
  const bool live = (x < npix) && (q < Q);
  // stage G tile: global [p][q][x] -> shared [xi][p][q]
  for (long long e = tid; e < QQ * PIX; e += blockDim.x) {
    const int xx = (int)(e % PIX);
    const long long pq = e / PIX;
    float2 g = make_float2(0.f, 0.f);
    if (x0 + xx < npix) g = G[pq * npix + x0 + xx];
    Gs[(long long)xx * GST + pq] = g;
  }
  const float inv_lam = 1.0f / lam_size;
  // start vector (normalised)
  float2 v = make_float2(0.f, 0.f);
  if (live) v = make_float2(counter_uniform(seed, (uint64_t)x, 2 * q), counter_uniform(seed, (uint64_t)x, 2 * q + 1));
  {
    float n2 = pixel_sum<QP>(v.x * v.x + v.y * v.y, red, xi, q);
    const float s = n2 > 0.f ? rsqrtf(n2) : 0.f;
    v.x *= s; v.y *= s;
  }
  vs[xi * QP + q] = v;
  __syncthreads();
  const float2* Gx = Gs + (long long)xi * GST;
  float2 gv = make_float2(0.f, 0.f);
  for (int it = 0; it <= iters; ++it) {
    gv = make_float2(0.f, 0.f);
    if (q < Q) {
      for (int p = 0; p < Q; ++p) cfmac(gv, Gx[p * Q + q], vs[xi * QP + p]);
    }
    if (it == iters) break;
    float2 nv = make_float2(v.x - gv.x * inv_lam, v.y - gv.y * inv_lam);
    const float n2 = pixel_sum<QP>(nv.x * nv.x + nv.y * nv.y, red, xi, q);
    const float s = n2 > 0.f ? rsqrtf(n2) : 0.f;
    v = make_float2(nv.x * s, nv.y * s);
    __syncthreads();
    vs[xi * QP + q] = v;
    __syncthreads();
  }
  // Rayleigh quotient and phase of the coil-combined low-resolution image
  const float lam = pixel_sum<QP>(v.x * gv.x + v.y * gv.y, red, xi, q) * inv_lam;
  float2 y = make_float2(0.f, 0.f);
  if (live) y = Y[(long long)q * npix + x];
  const float rr = pixel_sum<QP>(v.x * y.x + v.y * y.y, red, xi, q);
  const float ri = pixel_sum<QP>(v.x * y.y - v.y * y.x, red, xi, q);
  const float mag = sqrtf(rr * rr + ri * ri);
  if (mag > 0.f) {
    const float cr = rr / mag, ci = ri / mag;
    v = make_float2(v.x * cr - v.y * ci, v.x * ci + v.y * cr);
  }
  if (live) {
    V[(long long)q * npix + x] = v;
    if (q == 0 && eig != nullptr) eig[x] = lam;
  }
}

template <int QP>
static cudaError_t launch_pi(const float2* G, const float2* Y, int Q, long long npix, int iters,
                             float lam_size, unsigned long long seed, float2* V, float* eig,
                             cudaStream_t st) {
  constexpr int PIX = 256 / QP;
  const size_t smem = (size_t)PIX * ((size_t)Q * Q + 1) * sizeof(float2) + PIX * QP * sizeof(float2) + PIX * 2 * sizeof(float);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(pi_kernel<QP>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set = true;
  }
  const long long blocks = (npix + PIX - 1) / PIX;
  pi_kernel<QP><<<(unsigned)blocks, 256, smem, st>>>(G, Y, Q, npix, iters, lam_size, seed, V, eig);
  ++g_launches;
  return cudaGetLastError();
}

cudaError_t power_iteration(const float2* G, const float2* Y, int Q, long long npix, int iters,
                            float lam_size, unsigned long long seed, float2* V, float* eig,
                            cudaStream_t st) {
  if (Q <= 2) return launch_pi<2>(G, Y, Q, npix, iters, lam_size, seed, V, eig, st);
  if (Q <= 4) return launch_pi<4>(G, Y, Q, npix, iters, lam_size, seed, V, eig, st);
  if (Q <= 8) return launch_pi<8>(G, Y, Q, npix, iters, lam_size, seed, V, eig, st);
  if (Q <= 16) return launch_pi<16>(G, Y, Q, npix, iters, lam_size, seed, V, eig, st);
  if (Q <= 32) return launch_pi<32>(G, Y, Q, npix, iters, lam_size, seed, V, eig, st);
  if (Q <= 64) return launch_pi<64>(G, Y, Q, npix, iters, lam_size, seed, V, eig, st);
  return cudaErrorInvalidValue;
}

}  // namespace pisco
