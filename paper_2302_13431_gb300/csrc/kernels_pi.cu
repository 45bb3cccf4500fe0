// Stages (d)+(e, phase): simultaneous power iteration over all reduced-grid pixels
// (Sec. V-E) on B(x) = I - G(x)/|Lambda| (Eq. esp_null), followed by the smooth phase step
// of Sec. V-D: v <- v * rho/|rho| with rho = v^H y(x), y the apodised low-resolution coil
// images, so that the coil-combined reconstruction becomes real and non-negative.
//
// A CTA holds PIX pixels and the Q threads of a pixel each own one coil.  G is stored
// pixel-major ([pixel][p][q]); thread q keeps column q of its pixel's G in registers, so every
// iteration (G v)_q = sum_p conj(G_pq) v_p (G Hermitian) reads only v from shared memory
// (a broadcast).  G is read from HBM once, coalesced across the Q threads.
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

// Optional warm start (PiOpts): v0 from a proposal [npix][2Q] (interleaved re/im) instead of
// the counter-based start; a residual gate that flags pixels whose final residual
// ||G v - lambda |Lambda| v|| / |Lambda| exceeds `gate`; and a fallback pass that re-solves
// only the flagged pixels (CTAs without one exit at once; the others write flagged pixels only).
// (up to 32 coils: at most 85 registers a thread, so that three CTAs share an SM; the G column
// takes 64 of them)
template <int QP>
__global__ void __launch_bounds__(256, QP <= 32 ? 3 : 1) pi_kernel(const float2* __restrict__ G,
                                                 const float2* __restrict__ Y, int Q,
                                                 long long npix, int iters, float lam_size,
                                                 unsigned long long seed, float2* __restrict__ V,
                                                 float* __restrict__ eig, PiOpts opt) {
  constexpr int PIX = 256 / QP;
  __shared__ __align__(16) float2 vs[2][PIX * QP];  // double-buffered iterate: one barrier per step
  __shared__ float red[PIX * 2];
  __shared__ int any_flag;
  {
    const int i = blockIdx.y;
    G += i * opt.sG;
    Y += i * opt.sY;
    V += i * opt.sV;
    if (opt.eig_tab) eig = opt.eig_tab[i];
    else if (eig) eig += i * opt.sE;
  }
  const int tid = threadIdx.x;
  const int xi = tid / QP, q = tid % QP;
  const long long x = (long long)blockIdx.x * PIX + xi;
  const bool live = (x < npix) && (q < Q);
  bool write = true;
  if (opt.only != nullptr) {  // fallback pass: uniform early exit for CTAs without a flagged pixel
    if (tid == 0) any_flag = 0;
    __syncthreads();
    const bool mine = (x < npix) && opt.only[x] != 0;
    if (mine && q == 0) any_flag = 1;
    __syncthreads();
    if (any_flag == 0) return;
    write = mine;
  }
  const long long QQ = (long long)Q * Q;
  float2 gcol[QP];
#pragma unroll
  for (int p = 0; p < QP; ++p) {
    gcol[p] = make_float2(0.f, 0.f);
    if (live && p < Q) gcol[p] = G[x * QQ + (long long)p * Q + q];
  }
  const float inv_lam = 1.0f / lam_size;
  float2 v = make_float2(0.f, 0.f);
  if (live) {
    if (opt.v0 != nullptr)
      v = make_float2(opt.v0[x * 2 * Q + 2 * q], opt.v0[x * 2 * Q + 2 * q + 1]);
    else
      v = make_float2(counter_uniform(seed, (uint64_t)x, 2 * q), counter_uniform(seed, (uint64_t)x, 2 * q + 1));
  }
  {
    const float n2 = pixel_sum<QP>(v.x * v.x + v.y * v.y, red, xi, q);
    const float s = n2 > 0.f ? rsqrtf(n2) : 0.f;
    v.x *= s; v.y *= s;
  }
  // a pixel's QP threads lie in one warp for QP <= 32: warp barriers suffice
  int cur = 0;
  vs[cur][xi * QP + q] = v;
  if (QP <= 32) __syncwarp(); else __syncthreads();
  float2 gv = make_float2(0.f, 0.f);
  for (int it = 0; it <= iters; ++it) {
    gv = make_float2(0.f, 0.f);
    const float4* vp = reinterpret_cast<const float4*>(&vs[cur][xi * QP]);
#pragma unroll
    for (int p = 0; p < QP / 2; ++p) {
      const float4 t = vp[p];
      cfmac(gv, gcol[2 * p], make_float2(t.x, t.y));
      cfmac(gv, gcol[2 * p + 1], make_float2(t.z, t.w));
    }
    if (it == iters) break;
    const float2 nv = make_float2(v.x - gv.x * inv_lam, v.y - gv.y * inv_lam);
    const float n2 = pixel_sum<QP>(nv.x * nv.x + nv.y * nv.y, red, xi, q);
    const float s = n2 > 0.f ? rsqrtf(n2) : 0.f;
    v = make_float2(nv.x * s, nv.y * s);
    cur ^= 1;
    vs[cur][xi * QP + q] = v;
    if (QP <= 32) __syncwarp(); else __syncthreads();
  }
  // Rayleigh quotient and phase of the coil-combined low-resolution image
  const float lraw = pixel_sum<QP>(v.x * gv.x + v.y * gv.y, red, xi, q);
  const float lam = lraw * inv_lam;
  if (opt.gate > 0.f) {
    const float rx = gv.x - lraw * v.x, ry = gv.y - lraw * v.y;
    const float r2 = pixel_sum<QP>(live ? rx * rx + ry * ry : 0.f, red, xi, q);
    const bool bad = sqrtf(r2) * inv_lam > opt.gate;
    if (x < npix && q == 0) {
      opt.flags[x] = bad ? 1 : 0;
      if (bad) atomicAdd(opt.count, 1);
    }
  }
  float2 y = make_float2(0.f, 0.f);
  if (live) y = Y[(long long)q * npix + x];
  const float rr = pixel_sum<QP>(v.x * y.x + v.y * y.y, red, xi, q);
  const float ri = pixel_sum<QP>(v.x * y.y - v.y * y.x, red, xi, q);
  const float mag = sqrtf(rr * rr + ri * ri);
  if (mag > 0.f) {
    const float cr = rr / mag, ci = ri / mag;
    v = make_float2(v.x * cr - v.y * ci, v.x * ci + v.y * cr);
  }
  if (live && write) {
    V[(long long)q * npix + x] = v;
    if (q == 0 && eig != nullptr) eig[x] = lam;
  }
}

// Block variant for pixels whose two smallest eigenvalues are close: power iteration on two
// vectors (Gram-Schmidt after every step), then Rayleigh-Ritz on the 2x2 matrix V^H G V; its
// convergence is set by lambda_3 instead of lambda_2.  The second start vector draws the
// counters 2Q..4Q-1 of the same generator.  Output as pi_kernel (phase step included).
template <int QP>
__global__ void __launch_bounds__(256) pi_block2_kernel(const float2* __restrict__ G,
                                                        const float2* __restrict__ Y, int Q,
                                                        long long npix, int iters, float lam_size,
                                                        unsigned long long seed, float2* __restrict__ V,
                                                        float* __restrict__ eig) {
  constexpr int PIX = 256 / QP;
  __shared__ float2 vs1[PIX * QP];
  __shared__ float2 vs2[PIX * QP];
  __shared__ float red[PIX * 2];
  const int tid = threadIdx.x;
  const int xi = tid / QP, q = tid % QP;
  const long long x = (long long)blockIdx.x * PIX + xi;
  const bool live = (x < npix) && (q < Q);
  const long long QQ = (long long)Q * Q;
  float2 gcol[QP];
#pragma unroll
  for (int p = 0; p < QP; ++p) {
    gcol[p] = make_float2(0.f, 0.f);
    if (live && p < Q) gcol[p] = G[x * QQ + (long long)p * Q + q];
  }
  const float inv_lam = 1.0f / lam_size;
  float2 v1 = make_float2(0.f, 0.f), v2 = v1;
  if (live) {
    v1 = make_float2(counter_uniform(seed, (uint64_t)x, 2 * q), counter_uniform(seed, (uint64_t)x, 2 * q + 1));
    v2 = make_float2(counter_uniform(seed, (uint64_t)x, 2 * Q + 2 * q),
                     counter_uniform(seed, (uint64_t)x, 2 * Q + 2 * q + 1));
  }
  auto orth = [&](float2& a, float2& b) {
    const float n1 = pixel_sum<QP>(a.x * a.x + a.y * a.y, red, xi, q);
    const float s1 = n1 > 0.f ? rsqrtf(n1) : 0.f;
    a = make_float2(a.x * s1, a.y * s1);
    const float pr = pixel_sum<QP>(a.x * b.x + a.y * b.y, red, xi, q);   // Re(conj(a) b)
    const float pi = pixel_sum<QP>(a.x * b.y - a.y * b.x, red, xi, q);   // Im(conj(a) b)
    b = make_float2(b.x - (pr * a.x - pi * a.y), b.y - (pr * a.y + pi * a.x));
    const float n2 = pixel_sum<QP>(b.x * b.x + b.y * b.y, red, xi, q);
    const float s2 = n2 > 0.f ? rsqrtf(n2) : 0.f;
    b = make_float2(b.x * s2, b.y * s2);
  };
  orth(v1, v2);
  vs1[xi * QP + q] = v1;
  vs2[xi * QP + q] = v2;
  __syncthreads();
  float2 g1 = make_float2(0.f, 0.f), g2 = g1;
  for (int it = 0; it <= iters; ++it) {
    g1 = make_float2(0.f, 0.f);
    g2 = g1;
#pragma unroll
    for (int p = 0; p < QP; ++p) {
      cfmac(g1, gcol[p], vs1[xi * QP + p]);
      cfmac(g2, gcol[p], vs2[xi * QP + p]);
    }
    if (it == iters) break;
    v1 = make_float2(v1.x - g1.x * inv_lam, v1.y - g1.y * inv_lam);
    v2 = make_float2(v2.x - g2.x * inv_lam, v2.y - g2.y * inv_lam);
    orth(v1, v2);
    __syncthreads();
    vs1[xi * QP + q] = v1;
    vs2[xi * QP + q] = v2;
    __syncthreads();
  }
  // Rayleigh-Ritz: H = [[a, b], [conj b, c]] = V^H G V, smallest eigenpair in closed form
  const float a = pixel_sum<QP>(v1.x * g1.x + v1.y * g1.y, red, xi, q);
  const float c = pixel_sum<QP>(v2.x * g2.x + v2.y * g2.y, red, xi, q);
  const float br = pixel_sum<QP>(v1.x * g2.x + v1.y * g2.y, red, xi, q);
  const float bi = pixel_sum<QP>(v1.x * g2.y - v1.y * g2.x, red, xi, q);
  const float half = 0.5f * (a - c);
  const float mu = 0.5f * (a + c) - sqrtf(half * half + br * br + bi * bi);
  float2 y1, y2;  // eigenvector of mu from the better-conditioned row
  if (a <= c) {
    y1 = make_float2(c - mu, 0.f);
    y2 = make_float2(-br, bi);  // -conj(b)
  } else {
    y1 = make_float2(-br, -bi);  // -b
    y2 = make_float2(a - mu, 0.f);
  }
  if (y1.x * y1.x + y1.y * y1.y + y2.x * y2.x + y2.y * y2.y == 0.f) y1 = make_float2(1.f, 0.f);
  float2 v = make_float2(y1.x * v1.x - y1.y * v1.y + y2.x * v2.x - y2.y * v2.y,
                         y1.x * v1.y + y1.y * v1.x + y2.x * v2.y + y2.y * v2.x);
  {
    const float n2 = pixel_sum<QP>(v.x * v.x + v.y * v.y, red, xi, q);
    const float s = n2 > 0.f ? rsqrtf(n2) : 0.f;
    v = make_float2(v.x * s, v.y * s);
  }
  const float lam = mu * inv_lam;
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
static cudaError_t launch_block2(const float2* G, const float2* Y, int Q, long long npix, int iters, float lam_size,
                                 unsigned long long seed, float2* V, float* eig, cudaStream_t st) {
  constexpr int PIX = 256 / QP;
  const long long blocks = (npix + PIX - 1) / PIX;
  pi_block2_kernel<QP><<<(unsigned)blocks, 256, 0, st>>>(G, Y, Q, npix, iters, lam_size, seed, V, eig);
  ++g_launches;
  return cudaGetLastError();
}

cudaError_t power_iteration_block2(const float2* G, const float2* Y, int Q, long long npix, int iters,
                                   float lam_size, unsigned long long seed, float2* V, float* eig, cudaStream_t st) {
  if (Q <= 2) return launch_block2<2>(G, Y, Q, npix, iters, lam_size, seed, V, eig, st);
  if (Q <= 4) return launch_block2<4>(G, Y, Q, npix, iters, lam_size, seed, V, eig, st);
  if (Q <= 8) return launch_block2<8>(G, Y, Q, npix, iters, lam_size, seed, V, eig, st);
  if (Q <= 16) return launch_block2<16>(G, Y, Q, npix, iters, lam_size, seed, V, eig, st);
  if (Q <= 32) return launch_block2<32>(G, Y, Q, npix, iters, lam_size, seed, V, eig, st);
  if (Q <= 64) return launch_block2<64>(G, Y, Q, npix, iters, lam_size, seed, V, eig, st);
  return cudaErrorInvalidValue;
}

__global__ void support_mask_kernel(const float* __restrict__ eig, long long n, float thr, unsigned char* __restrict__ mask) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    mask[i] = eig[i] < thr ? 1 : 0;
}

cudaError_t support_mask(const float* eig, long long n, float thr, unsigned char* mask, cudaStream_t st) {
  long long b = (n + 255) / 256;
  if (b > 152 * 8) b = 152 * 8;
  if (b < 1) b = 1;
  support_mask_kernel<<<(unsigned)b, 256, 0, st>>>(eig, n, thr, mask);
  ++g_launches;
  return cudaGetLastError();
}

template <int QP>
static cudaError_t launch_pi(const float2* G, const float2* Y, int Q, long long npix, int iters,
                             float lam_size, unsigned long long seed, float2* V, float* eig,
                             const PiOpts& opt, cudaStream_t st) {
  constexpr int PIX = 256 / QP;
  const long long blocks = (npix + PIX - 1) / PIX;
  pi_kernel<QP><<<dim3((unsigned)blocks, opt.items), 256, 0, st>>>(G, Y, Q, npix, iters, lam_size, seed, V, eig, opt);
  ++g_launches;
  return cudaGetLastError();
}

cudaError_t power_iteration(const float2* G, const float2* Y, int Q, long long npix, int iters,
                            float lam_size, unsigned long long seed, float2* V, float* eig,
                            cudaStream_t st, const PiOpts& opt) {
  if (opt.gate > 0.f && (opt.flags == nullptr || opt.count == nullptr)) return cudaErrorInvalidValue;
  if (Q <= 2) return launch_pi<2>(G, Y, Q, npix, iters, lam_size, seed, V, eig, opt, st);
  if (Q <= 4) return launch_pi<4>(G, Y, Q, npix, iters, lam_size, seed, V, eig, opt, st);
  if (Q <= 8) return launch_pi<8>(G, Y, Q, npix, iters, lam_size, seed, V, eig, opt, st);
  if (Q <= 16) return launch_pi<16>(G, Y, Q, npix, iters, lam_size, seed, V, eig, opt, st);
  if (Q <= 32) return launch_pi<32>(G, Y, Q, npix, iters, lam_size, seed, V, eig, opt, st);
  if (Q <= 64) return launch_pi<64>(G, Y, Q, npix, iters, lam_size, seed, V, eig, opt, st);
  return cudaErrorInvalidValue;
}

}  // namespace pisco
