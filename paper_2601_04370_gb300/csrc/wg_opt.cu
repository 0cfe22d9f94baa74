// Optimizer of the coating thicknesses (Results, "Evaluation": gradient-based
// optimization of all PRMA layer thicknesses within 20-200 nm, with layers
// allowed to reach zero thickness through a soft gap between 0 and 20 nm).
//
// The paper does not name its optimizer; this is Adam (Kingma and Ba, 2015)
// on the thicknesses in nm, followed by a projection onto the feasible set:
// clamp to [0, d_max], and a value inside the gap (0, d_min) goes to the
// nearer end (0 below d_min / 2: the layer is eliminated, else d_min). A layer
// at zero thickness stays in its stack as an identity layer, so its gradient
// keeps flowing, and comes back only when a step carries it past d_min / 2.
// Layers the design itself prunes are never updated.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "wg.h"
#include "wg_host.h"

namespace {

// one thread per layer; moments in FP64 (gradients of the CV loss reach ~1e40
// at nearly empty cells, beyond FP32 once squared)
__global__ void k_adam_step(float* theta, double* m, double* v, const double* g, const uint8_t* fixed, int n,
                            double lr, double b1, double b2, double eps, double bc1, double bc2, float d_min,
                            float d_max) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || fixed[i]) return;
  const double gi = g[i];
  if (!isfinite(gi)) return;  // a non-finite gradient entry leaves the layer and its moments as they are
  const double mi = b1 * m[i] + (1.0 - b1) * gi;
  const double vi = b2 * v[i] + (1.0 - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  double x = (double)theta[i] - lr * (mi / bc1) / (sqrt(vi / bc2) + eps);
  x = fmin(fmax(x, 0.0), (double)d_max);
  if (x > 0.0 && x < (double)d_min) x = x < 0.5 * (double)d_min ? 0.0 : (double)d_min;
  theta[i] = (float)x;
}

// the reflection probabilities' step: one thread per mirror, clipped to [lo, hi]
__global__ void k_omega_adam_step(double* w, double* m, double* v, const double* g, float* out, int n, double lr,
                                  double b1, double b2, double eps, double bc1, double bc2, double lo, double hi) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double gk = g[k];
  if (isfinite(gk)) {
    const double mk = b1 * m[k] + (1.0 - b1) * gk;
    const double vk = b2 * v[k] + (1.0 - b2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    w[k] = fmin(fmax(w[k] - lr * (mk / bc1) / (sqrt(vk / bc2) + eps), lo), hi);
  }
  out[k] = (float)w[k];
}

bool is_dev(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

struct wg_adam {
  wg_design* d = nullptr;
  int device = 0;
  int n = 0;
  wg_adam_opts o{};
  long long t = 0;
  float* theta = nullptr;
  double* m = nullptr;
  double* v = nullptr;
  double* g = nullptr;  // staging for host gradients
  uint8_t* fixed = nullptr;
  std::mutex mu;
};

static void adam_free(wg_adam* a) {
  if (!a) return;
  cudaSetDevice(a->device);
  cudaFree(a->theta);
  cudaFree(a->m);
  cudaFree(a->v);
  cudaFree(a->g);
  cudaFree(a->fixed);
  delete a;
}

#define WG_CU(x)                                                                            \
  do {                                                                                      \
    const cudaError_t e_ = (x);                                                             \
    if (e_ != cudaSuccess) {                                                                \
      cudaGetLastError();                                                                   \
      return wgh::set_error(WG_EDEVICE, cudaGetErrorString(e_));                            \
    }                                                                                       \
  } while (0)

extern "C" wg_status wg_adam_create(wg_design* d, const wg_adam_opts* opts, const float* thickness_nm,
                                    wg_adam** out) {
  if (!d || !out) return wgh::set_error(WG_EINVAL, "wg_adam_create: NULL design/out");
  *out = nullptr;
  wg_adam_opts o;
  if (opts) {
    o = *opts;
  } else {
    memset(&o, 0, sizeof(o));
  }
  if (o.lr_nm == 0.0f) o.lr_nm = 2.0f;
  if (o.beta1 == 0.0f) o.beta1 = 0.9f;
  if (o.beta2 == 0.0f) o.beta2 = 0.999f;
  if (o.eps == 0.0f) o.eps = 1e-8f;
  if (o.d_min_nm == 0.0f) o.d_min_nm = 20.0f;
  if (o.d_max_nm == 0.0f) o.d_max_nm = 200.0f;
  if (!(o.lr_nm > 0.0f) || !(o.beta1 >= 0.0f && o.beta1 < 1.0f) || !(o.beta2 >= 0.0f && o.beta2 < 1.0f) ||
      !(o.eps > 0.0f) || !(o.d_min_nm > 0.0f) || !(o.d_max_nm > o.d_min_nm))
    return wgh::set_error(WG_EINVAL, "wg_adam_create: invalid options");
  const int n = (int)wgh::design_params(d);
  wg_ctx* c = wgh::design_ctx(d);
  wg_adam* a = new (std::nothrow) wg_adam();
  if (!a) return wgh::set_error(WG_ENOMEM, "wg_adam_create: out of host memory");
  a->d = d;
  a->device = wgh::ctx_device(c);
  a->n = n;
  a->o = o;
  const size_t nn = (size_t)(n > 0 ? n : 1);
  if (cudaSetDevice(a->device) != cudaSuccess || cudaMalloc(&a->theta, sizeof(float) * nn) != cudaSuccess ||
      cudaMalloc(&a->m, sizeof(double) * nn) != cudaSuccess || cudaMalloc(&a->v, sizeof(double) * nn) != cudaSuccess ||
      cudaMalloc(&a->g, sizeof(double) * nn) != cudaSuccess || cudaMalloc(&a->fixed, nn) != cudaSuccess) {
    cudaGetLastError();
    adam_free(a);
    return wgh::set_error(WG_ENOMEM, "wg_adam_create: device allocation failed");
  }
  const uint8_t* pr = wgh::design_pruned(d);
  if (n > 0) {
    if (cudaMemcpy(a->fixed, pr, (size_t)n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(a->m, 0, sizeof(double) * (size_t)n) != cudaSuccess ||
        cudaMemset(a->v, 0, sizeof(double) * (size_t)n) != cudaSuccess) {
      cudaGetLastError();
      adam_free(a);
      return wgh::set_error(WG_EDEVICE, "wg_adam_create: device copy failed");
    }
    cudaError_t e;
    if (thickness_nm && is_dev(thickness_nm)) {
      e = cudaMemcpy(a->theta, thickness_nm, sizeof(float) * (size_t)n, cudaMemcpyDeviceToDevice);
    } else {
      const float* src = thickness_nm ? thickness_nm : wgh::design_thickness(d);
      for (int i = 0; i < n; ++i)
        if (!std::isfinite(src[i]) || src[i] < 0.0f) {
          adam_free(a);
          return wgh::set_error(WG_EINVAL, "wg_adam_create: invalid thickness");
        }
      e = cudaMemcpy(a->theta, src, sizeof(float) * (size_t)n, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
      cudaGetLastError();
      adam_free(a);
      return wgh::set_error(WG_EDEVICE, "wg_adam_create: device copy failed");
    }
  }
  *out = a;
  return WG_OK;
}

extern "C" wg_status wg_adam_step(wg_adam* a, const double* grad_thickness, void* stream) {
  if (!a || !grad_thickness) return wgh::set_error(WG_EINVAL, "wg_adam_step: NULL optimizer/gradient");
  std::lock_guard<std::mutex> lk(a->mu);
  cudaStream_t s = (cudaStream_t)stream;
  WG_CU(cudaSetDevice(a->device));
  if (a->n == 0) return WG_OK;
  const double* g = grad_thickness;
  if (!is_dev(grad_thickness)) {
    WG_CU(cudaMemcpyAsync(a->g, grad_thickness, sizeof(double) * (size_t)a->n, cudaMemcpyHostToDevice, s));
    g = a->g;
  }
  ++a->t;
  const double b1 = a->o.beta1, b2 = a->o.beta2;
  const double bc1 = 1.0 - std::pow(b1, (double)a->t), bc2 = 1.0 - std::pow(b2, (double)a->t);
  k_adam_step<<<(a->n + 255) / 256, 256, 0, s>>>(a->theta, a->m, a->v, g, a->fixed, a->n, (double)a->o.lr_nm, b1, b2,
                                                 (double)a->o.eps, bc1, bc2, a->o.d_min_nm, a->o.d_max_nm);
  WG_CU(cudaGetLastError());
  // the design takes the new thicknesses (stream-ordered, device to device)
  return wg_set_params(a->d, a->theta, a->n, nullptr, 0, stream);
}

extern "C" wg_status wg_adam_params(wg_adam* a, float* thickness_nm, void* stream) {
  if (!a || !thickness_nm) return wgh::set_error(WG_EINVAL, "wg_adam_params: NULL argument");
  std::lock_guard<std::mutex> lk(a->mu);
  cudaStream_t s = (cudaStream_t)stream;
  WG_CU(cudaSetDevice(a->device));
  if (a->n == 0) return WG_OK;
  WG_CU(cudaMemcpyAsync(thickness_nm, a->theta, sizeof(float) * (size_t)a->n, cudaMemcpyDefault, s));
  if (!is_dev(thickness_nm)) WG_CU(cudaStreamSynchronize(s));
  return WG_OK;
}

extern "C" void wg_adam_destroy(wg_adam* a) { adam_free(a); }

// ---------------------------------------------------------------------------
// Optimizer of the reflection probabilities (the pre-optimization's update,
// Methods, "Learned reflection probabilities"): Adam on omega, clipped.
// ---------------------------------------------------------------------------
struct wg_omega_adam {
  wg_design* d = nullptr;
  int device = 0;
  int n = 0;
  wg_omega_adam_opts o{};
  long long t = 0;
  double* buf = nullptr;  // [4][n]: omega, m, v, gradient staging
  float* out = nullptr;   // [n] FP32 omega of the last step
  std::mutex mu;
};

static void omega_adam_free(wg_omega_adam* a) {
  if (!a) return;
  cudaSetDevice(a->device);
  cudaFree(a->buf);
  cudaFree(a->out);
  delete a;
}

extern "C" wg_status wg_omega_adam_create(wg_design* d, const wg_omega_adam_opts* opts, wg_omega_adam** out) {
  if (!d || !out) return wgh::set_error(WG_EINVAL, "wg_omega_adam_create: NULL design/out");
  *out = nullptr;
  wg_omega_adam_opts o;
  if (opts) {
    o = *opts;
  } else {
    memset(&o, 0, sizeof(o));
  }
  if (o.lr == 0.0f) o.lr = 0.02f;
  if (o.beta1 == 0.0f) o.beta1 = 0.9f;
  if (o.beta2 == 0.0f) o.beta2 = 0.999f;
  if (o.eps == 0.0f) o.eps = 1e-8f;
  if (o.lo == 0.0f && o.hi == 0.0f) {
    o.lo = 0.02f;
    o.hi = 0.98f;
  }
  if (!(o.lr > 0.0f) || !(o.beta1 >= 0.0f && o.beta1 < 1.0f) || !(o.beta2 >= 0.0f && o.beta2 < 1.0f) ||
      !(o.eps > 0.0f) || !(o.lo > 0.0f && o.lo < o.hi && o.hi < 1.0f))
    return wgh::set_error(WG_EINVAL, "wg_omega_adam_create: invalid options");
  int K = 0, n_dev = 0, period = 0, acc = 0;
  wgh::design_shape(d, &K, &n_dev, &period, &acc);
  wg_omega_adam* a = new (std::nothrow) wg_omega_adam();
  if (!a) return wgh::set_error(WG_ENOMEM, "wg_omega_adam_create: out of host memory");
  a->d = d;
  a->device = wgh::ctx_device(wgh::design_ctx(d));
  a->n = K;
  a->o = o;
  if (cudaSetDevice(a->device) != cudaSuccess || cudaMalloc(&a->buf, sizeof(double) * 4 * (size_t)K) != cudaSuccess ||
      cudaMalloc(&a->out, sizeof(float) * (size_t)K) != cudaSuccess) {
    cudaGetLastError();
    omega_adam_free(a);
    return wgh::set_error(WG_ENOMEM, "wg_omega_adam_create: device allocation failed");
  }
  std::vector<double> init(4 * (size_t)K, 0.0);
  const float* om = wgh::design_omega(d);
  for (int k = 0; k < K; ++k) init[k] = (double)om[k];
  if (cudaMemcpy(a->buf, init.data(), sizeof(double) * init.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    omega_adam_free(a);
    return wgh::set_error(WG_EDEVICE, "wg_omega_adam_create: device copy failed");
  }
  *out = a;
  return WG_OK;
}

extern "C" wg_status wg_omega_adam_step(wg_omega_adam* a, const double* grad_omega, float* omega_out, void* stream) {
  if (!a || !grad_omega) return wgh::set_error(WG_EINVAL, "wg_omega_adam_step: NULL optimizer/gradient");
  std::lock_guard<std::mutex> lk(a->mu);
  cudaStream_t s = (cudaStream_t)stream;
  WG_CU(cudaSetDevice(a->device));
  const int n = a->n;
  double* w = a->buf;
  double* m = a->buf + n;
  double* v = a->buf + 2 * n;
  const double* g = grad_omega;
  if (!is_dev(grad_omega)) {
    WG_CU(cudaMemcpyAsync(a->buf + 3 * n, grad_omega, sizeof(double) * (size_t)n, cudaMemcpyHostToDevice, s));
    g = a->buf + 3 * n;
  }
  ++a->t;
  const double b1 = a->o.beta1, b2 = a->o.beta2;
  const double bc1 = 1.0 - std::pow(b1, (double)a->t), bc2 = 1.0 - std::pow(b2, (double)a->t);
  k_omega_adam_step<<<1, 64, 0, s>>>(w, m, v, g, a->out, n, (double)a->o.lr, b1, b2, (double)a->o.eps, bc1, bc2,
                                     (double)a->o.lo, (double)a->o.hi);
  WG_CU(cudaGetLastError());
  std::vector<float> h((size_t)n);
  WG_CU(cudaMemcpyAsync(h.data(), a->out, sizeof(float) * (size_t)n, cudaMemcpyDeviceToHost, s));
  WG_CU(cudaStreamSynchronize(s));
  if (omega_out) memcpy(omega_out, h.data(), sizeof(float) * (size_t)n);
  return wg_set_omega(a->d, h.data(), n, stream);
}

extern "C" void wg_omega_adam_destroy(wg_omega_adam* a) { omega_adam_free(a); }
