// C ABI of the warm-start network: a trainable per-pixel MLP held on the device.  Training data,
// initial weights and the learning schedule come from the caller; every forward, backward and
// update step runs in the kernels of kernels_mlp.cu.
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "common.cuh"

using namespace pisco;

struct pisco_mlp_s {
  int n_in = 0, H = 0, n_out = 0;
  long long max_batch = 0;
  size_t nparam = 0;
  cudaStream_t st = nullptr;
  int step = 0;
  int loss_blocks = 0;
  int loss_kind = 0;  // 0 squared error, 1 direction
  std::vector<void*> allocs;
  float *w32 = nullptr, *grad = nullptr, *m1 = nullptr, *m2 = nullptr;
  __half* w16 = nullptr;
  float *H1 = nullptr, *H2 = nullptr, *out = nullptr, *dO = nullptr, *dH2 = nullptr, *dH1 = nullptr;
  float *part = nullptr, *loss_part = nullptr, *h_loss_part = nullptr;
};

namespace pisco {
MlpView mlp_view(const pisco_mlp_s* m) { return MlpView{m->n_in, m->H, m->n_out, m->w32, m->w16}; }
void mlp_dims(const pisco_mlp_s* m, int* n_in, int* H, int* n_out, size_t* nparam) {
  *n_in = m->n_in;
  *H = m->H;
  *n_out = m->n_out;
  *nparam = m->nparam;
}
}  // namespace pisco

namespace {
template <typename T>
bool alloc(pisco_mlp_s* m, T** p, size_t n) {
  void* q = nullptr;
  if (cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) return false;
  m->allocs.push_back(q);
  *p = static_cast<T*>(q);
  return true;
}
}  // namespace

extern "C" {

void pisco_mlp_destroy(pisco_mlp_t m) {
  if (!m) return;
  if (m->st) cudaStreamSynchronize(m->st);
  for (void* p : m->allocs) cudaFree(p);
  if (m->h_loss_part) cudaFreeHost(m->h_loss_part);
  delete m;
}

pisco_status pisco_mlp_create(int n_in, int n_hidden, int n_out, const float* h_params, long long max_batch,
                              void* cuda_stream, pisco_mlp_t* out) {
  if (!out) return PISCO_ERR_ARG;
  *out = nullptr;
  if (n_in < 1 || n_in > 4096 || n_hidden < 1 || n_hidden > 128 || n_out < 1 || n_out > 128) return PISCO_ERR_ARG;
  if (max_batch < 1 || max_batch > 4000000ll || !h_params) return PISCO_ERR_ARG;
  pisco_mlp_s* m = new (std::nothrow) pisco_mlp_s();
  if (!m) return PISCO_ERR_OOM;
  m->n_in = n_in;
  m->H = n_hidden;
  m->n_out = n_out;
  m->max_batch = max_batch;
  m->st = (cudaStream_t)cuda_stream;
  m->nparam = mlp_param_count(n_in, n_hidden, n_out);
  m->loss_blocks = 152;
  if (mlp_prepare() != cudaSuccess) {
    cudaGetLastError();
    delete m;
    return PISCO_ERR_CUDA;
  }
  const size_t P = m->nparam;
  const size_t B = (size_t)max_batch;
  bool ok = alloc(m, &m->w32, P) && alloc(m, &m->w16, P) && alloc(m, &m->grad, P) && alloc(m, &m->m1, P) &&
            alloc(m, &m->m2, P) && alloc(m, &m->H1, B * n_hidden) && alloc(m, &m->H2, B * n_hidden) &&
            alloc(m, &m->out, B * n_out) && alloc(m, &m->dO, B * n_out) && alloc(m, &m->dH2, B * n_hidden) &&
            alloc(m, &m->dH1, B * n_hidden) &&
            alloc(m, &m->part, mlp_part_floats(max_batch, n_in, n_hidden, n_out)) &&
            alloc(m, &m->loss_part, (size_t)m->loss_blocks);
  ok = ok && cudaMallocHost((void**)&m->h_loss_part, sizeof(float) * m->loss_blocks) == cudaSuccess;
  ok = ok && cudaMemcpy(m->w32, h_params, sizeof(float) * P, cudaMemcpyHostToDevice) == cudaSuccess;
  ok = ok && cudaMemset(m->m1, 0, sizeof(float) * P) == cudaSuccess && cudaMemset(m->m2, 0, sizeof(float) * P) == cudaSuccess;
  ok = ok && mlp_to_half(m->w32, m->w16, (long long)P, m->st) == cudaSuccess;
  ok = ok && cudaStreamSynchronize(m->st) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    pisco_mlp_destroy(m);
    return PISCO_ERR_OOM;
  }
  *out = m;
  return PISCO_OK;
}

pisco_status pisco_mlp_write(pisco_mlp_t m, const float* h_params) {
  if (!m || !h_params) return PISCO_ERR_ARG;
  const size_t P = m->nparam;
  if (cudaMemcpyAsync(m->w32, h_params, sizeof(float) * P, cudaMemcpyHostToDevice, m->st) != cudaSuccess ||
      cudaMemsetAsync(m->m1, 0, sizeof(float) * P, m->st) != cudaSuccess ||
      cudaMemsetAsync(m->m2, 0, sizeof(float) * P, m->st) != cudaSuccess ||
      mlp_to_half(m->w32, m->w16, (long long)P, m->st) != cudaSuccess ||
      cudaStreamSynchronize(m->st) != cudaSuccess)
    return PISCO_ERR_CUDA;
  m->step = 0;
  return PISCO_OK;
}

pisco_status pisco_mlp_forward(pisco_mlp_t m, const float* d_x, long long batch, float* d_out) {
  if (!m || !d_x || !d_out || batch < 0 || batch > m->max_batch) return PISCO_ERR_ARG;
  if (batch == 0) return PISCO_OK;
  if (mlp_forward(mlp_view(m), d_x, batch, m->H1, m->H2, d_out, m->st) != cudaSuccess) return PISCO_ERR_CUDA;
  return PISCO_OK;
}

pisco_status pisco_mlp_backward(pisco_mlp_t m, const float* d_x, const float* d_target, long long batch,
                                double* h_loss) {
  if (!m || !d_x || !d_target || batch < 1 || batch > m->max_batch) return PISCO_ERR_ARG;
  if (mlp_backward(mlp_view(m), d_x, d_target, batch, m->H1, m->H2, m->out, m->dO, m->dH2, m->dH1, m->part,
                   m->grad, m->loss_part, m->loss_blocks, m->loss_kind, m->st) != cudaSuccess)
    return PISCO_ERR_CUDA;
  if (h_loss) {
    if (cudaMemcpyAsync(m->h_loss_part, m->loss_part, sizeof(float) * m->loss_blocks, cudaMemcpyDeviceToHost,
                        m->st) != cudaSuccess ||
        cudaStreamSynchronize(m->st) != cudaSuccess)
      return PISCO_ERR_CUDA;
    double s = 0.0;
    for (int i = 0; i < m->loss_blocks; ++i) s += m->h_loss_part[i];
    *h_loss = s / (double)batch;
  }
  return PISCO_OK;
}

pisco_status pisco_mlp_adam(pisco_mlp_t m, float lr, float beta1, float beta2, float eps) {
  if (!m || !(lr > 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
    return PISCO_ERR_ARG;
  m->step += 1;
  if (mlp_adam(m->w32, m->w16, m->grad, m->m1, m->m2, (long long)m->nparam, lr, beta1, beta2, eps, m->step,
               m->st) != cudaSuccess)
    return PISCO_ERR_CUDA;
  return PISCO_OK;
}

pisco_status pisco_mlp_read(pisco_mlp_t m, int which, float* h_out) {
  if (!m || !h_out || (which != 0 && which != 1)) return PISCO_ERR_ARG;
  const float* src = which == 0 ? m->w32 : m->grad;
  if (cudaMemcpyAsync(h_out, src, sizeof(float) * m->nparam, cudaMemcpyDeviceToHost, m->st) != cudaSuccess ||
      cudaStreamSynchronize(m->st) != cudaSuccess)
    return PISCO_ERR_CUDA;
  return PISCO_OK;
}

pisco_status pisco_mlp_set_loss(pisco_mlp_t m, int kind) {
  if (!m || (kind != 0 && kind != 1) || (kind == 1 && (m->n_out % 2) != 0)) return PISCO_ERR_ARG;
  m->loss_kind = kind;
  return PISCO_OK;
}

pisco_status pisco_warm_start_patch_features(const void* d_y, int Q, const int* dims, int ndim, int radius,
                                             float* d_x, void* cuda_stream) {
  if (!d_y || !d_x || !dims || Q < 1 || Q > 64 || (ndim != 2 && ndim != 3) || radius < 0 || radius > 3)
    return PISCO_ERR_ARG;
  const int d3[3] = {ndim == 3 ? dims[0] : 1, dims[ndim == 3 ? 1 : 0], dims[ndim == 3 ? 2 : 1]};
  if (d3[0] < 1 || d3[1] < 1 || d3[2] < 1) return PISCO_ERR_ARG;
  return mlp_patch_features(static_cast<const float2*>(d_y), Q, d3, radius, ndim, d_x, (cudaStream_t)cuda_stream) ==
                 cudaSuccess
             ? PISCO_OK
             : PISCO_ERR_CUDA;
}

pisco_status pisco_warm_start_features(const void* d_y, int Q, long long npix, float* d_x, void* cuda_stream) {
  if (!d_y || !d_x || Q < 1 || Q > 64 || npix < 0) return PISCO_ERR_ARG;
  if (npix == 0) return PISCO_OK;
  return mlp_features(static_cast<const float2*>(d_y), Q, npix, d_x, (cudaStream_t)cuda_stream) == cudaSuccess
             ? PISCO_OK
             : PISCO_ERR_CUDA;
}

}  // extern "C"
