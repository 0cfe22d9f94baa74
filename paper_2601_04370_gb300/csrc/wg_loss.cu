// Loss head of Results Eq. 1 on the eyebox tally (FP64):
//   L = -I_mean + w_f U_FoV + w_e U_eyebox
// with pupil images I[cell, p] = sum of the tally over the 4 mm pupil p /
// rays per cell, U = coefficient of variation (population std / mean, the
// paper's choice) or the variance, U_FoV averaged over (lambda, pupil) of the
// spread over fields, U_eyebox averaged over (lambda, field) of the spread
// over pupils; and dL/dtally for the adjoint.
#include <cuda_runtime.h>

#include "wg_internal.h"

namespace wgk {

// pupil membership of a bin; arithmetic without FMA contraction so the
// boundary decisions are the plain FP64 evaluation of the definition
__device__ __forceinline__ bool in_pupil(int dims, int p, int ex, int ey, double cx, double cy, double w, double h,
                                         int nx, int ny) {
  const double D = 4.0, r = 2.0;
  const double xs = __dadd_rn(__dsub_rn(cx, __dmul_rn(0.5, w)), __dmul_rn((double)ex + 0.5, __ddiv_rn(w, (double)nx)));
  const double ox = __dmul_rn(0.5, __dsub_rn(w, D));
  if (dims == 2) {
    const double c = __dadd_rn(cx, (p - 1) * ox);
    return fabs(__dsub_rn(xs, c)) <= r;
  }
  const double ys = __dadd_rn(__dsub_rn(cy, __dmul_rn(0.5, h)), __dmul_rn((double)ey + 0.5, __ddiv_rn(h, (double)ny)));
  const double oy = __dmul_rn(0.5, __dsub_rn(h, D));
  const int px = p % 3, py = p / 3;
  const double ux = __dsub_rn(xs, __dadd_rn(cx, (px - 1) * ox));
  const double uy = __dsub_rn(ys, __dadd_rn(cy, (py - 1) * oy));
  return __dadd_rn(__dmul_rn(ux, ux), __dmul_rn(uy, uy)) <= __dmul_rn(r, r);
}

struct LossGeom {
  int dims, nx, ny, n_pupil;
  double cx, cy, w, h;
};

// pupil membership bitmask of every eyebox bin (the same for all cells)
__global__ void k_pupil_masks(LossGeom g, unsigned short* mask) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= g.nx * g.ny) return;
  const int ex = b % g.nx, ey = b / g.nx;
  unsigned short m = 0;
  for (int p = 0; p < g.n_pupil; ++p)
    if (in_pupil(g.dims, p, ex, ey, g.cx, g.cy, g.w, g.h, g.nx, g.ny)) m |= (unsigned short)(1u << p);
  mask[b] = m;
}

// I[cell, p]
__global__ void k_pupil_sums(const double* tally, LossGeom g, const unsigned short* mask, double inv_ncell,
                             double* I) {
  const long long cell = blockIdx.x;
  const int bins = g.nx * g.ny;
  __shared__ double s_acc[9][32];
  double acc[9];
  for (int p = 0; p < 9; ++p) acc[p] = 0.0;
  const double* t = tally + cell * bins;
  for (int b = threadIdx.x; b < bins; b += blockDim.x) {
    const double v = t[b];
    if (v == 0.0) continue;
    const unsigned m = mask[b];
#pragma unroll
    for (int p = 0; p < 9; ++p)
      if (m & (1u << p)) acc[p] += v;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int p = 0; p < g.n_pupil; ++p) {
    double v = acc[p];
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) s_acc[p][wid] = v;
  }
  __syncthreads();
  if (threadIdx.x < g.n_pupil) {
    double v = 0.0;
    for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) v += s_acc[threadIdx.x][w2];
    I[cell * g.n_pupil + threadIdx.x] = v * inv_ncell;
  }
}

// Spread statistic of x[0..n) with stride: CV (kind 0) or variance (kind 1),
// and its gradient written to dx (scaled by `scale`).
__device__ void spread_grad(const double* x, int n, long long stride, int kind, double scale, double* dx,
                            double& val) {
  double mu = 0.0;
  for (int i = 0; i < n; ++i) mu += x[i * stride];
  mu /= n;
  double var = 0.0;
  for (int i = 0; i < n; ++i) {
    const double d = x[i * stride] - mu;
    var += d * d;
  }
  var /= n;
  if (kind == 1) {
    val = var;
    for (int i = 0; i < n; ++i) dx[i * stride] += scale * 2.0 * (x[i * stride] - mu) / n;
    return;
  }
  const double sd = sqrt(var);
  if (mu == 0.0) {
    val = 0.0;
    return;
  }
  val = sd / mu;
  if (sd <= 0.0) return;
  for (int i = 0; i < n; ++i) {
    const double dsd = (x[i * stride] - mu) / (n * sd);
    dx[i * stride] += scale * (dsd / mu - (val / mu) / n);
  }
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// spread_grad for one group with a whole warp (n values, stride): the sums
// are warp reductions; val is returned in every lane
__device__ void spread_grad_warp(const double* x, int n, long long stride, int kind, double scale, double* dx,
                                 double& val, int lane) {
  double mu = 0.0;
  for (int i = lane; i < n; i += 32) mu += x[i * stride];
  mu = warp_sum_d(mu) / n;
  double var = 0.0;
  for (int i = lane; i < n; i += 32) {
    const double d = x[i * stride] - mu;
    var += d * d;
  }
  var = warp_sum_d(var) / n;
  if (kind == 1) {
    val = var;
    for (int i = lane; i < n; i += 32) dx[i * stride] += scale * 2.0 * (x[i * stride] - mu) / n;
    return;
  }
  const double sd = sqrt(var);
  if (mu == 0.0) {
    val = 0.0;
    return;
  }
  val = sd / mu;
  if (sd <= 0.0) return;
  for (int i = lane; i < n; i += 32) {
    const double dsd = (x[i * stride] - mu) / (n * sd);
    dx[i * stride] += scale * (dsd / mu - (val / mu) / n);
  }
}

// One block: scalars and dL/dI. I is [n_lam][n_f][P]; dI same layout. The
// field-uniformity groups (long: n_f values) take a warp each; the
// eyebox-uniformity groups (P values) a thread each.
__global__ void k_loss_scalar(const double* I, int n_lam, int n_f, int P, int kind, double w_f, double w_e, double* dI,
                              double* out) {
  const long long N = (long long)n_lam * n_f * P;
  __shared__ double s_red[3][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double sum = 0.0, uf = 0.0, ue = 0.0;
  for (long long i = threadIdx.x; i < N; i += blockDim.x) {
    sum += I[i];
    dI[i] = -1.0 / (double)N;
  }
  __syncthreads();
  // U_FoV: over fields for each (lambda, p); gradients touch disjoint entries
  const int nfov = n_lam * P;
  for (int q = wid; q < nfov; q += nw) {
    const int l = q / P, p = q % P;
    double v;
    spread_grad_warp(I + (long long)l * n_f * P + p, n_f, P, kind, w_f / nfov, dI + (long long)l * n_f * P + p, v,
                     lane);
    if (lane == 0) uf += v;
  }
  __syncthreads();
  const int neb = n_lam * n_f;
  for (int q = threadIdx.x; q < neb; q += blockDim.x) {
    double v;
    spread_grad(I + (long long)q * P, P, 1, kind, w_e / neb, dI + (long long)q * P, v);
    ue += v;
  }
  double vals[3] = {sum, uf, ue};
  for (int k = 0; k < 3; ++k) {
    double v = vals[k];
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) s_red[k][wid] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double r[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < 3; ++k)
      for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) r[k] += s_red[k][w2];
    const double mean = r[0] / (double)N, Uf = r[1] / nfov, Ue = r[2] / neb;
    out[0] = -mean + w_f * Uf + w_e * Ue;
    out[1] = mean;
    out[2] = Uf;
    out[3] = Ue;
  }
}

// dL/dtally[cell, bin] = sum_{p containing bin} dL/dI[cell, p] / rays per cell
__global__ void k_loss_scatter(const double* dI, LossGeom g, const unsigned short* mask, double inv_ncell,
                               long long n_cells, double* dL) {
  const long long bins = (long long)g.nx * g.ny;
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n_cells * bins) return;
  const long long cell = i / bins;
  const unsigned m = mask[i % bins];
  double v = 0.0;
  for (int p = 0; p < g.n_pupil; ++p)
    if (m & (1u << p)) v += dI[cell * g.n_pupil + p];
  dL[i] = v * inv_ncell;
}

cudaError_t launch_loss_impl(const double* tally, int dims, int n_lam, int n_f, int nx, int ny, double cx, double cy,
                             double w, double h, double inv_ncell, int kind, double w_f, double w_e, double* ws,
                             double* out_dev, double* dL, cudaStream_t s) {
  LossGeom g{dims, nx, ny, dims == 2 ? 3 : 9, cx, cy, w, h};
  const long long n_cells = (long long)n_lam * n_f;
  double* I = ws;
  double* dI = ws + n_cells * g.n_pupil;
  unsigned short* mask = reinterpret_cast<unsigned short*>(ws + 2 * n_cells * 9 + 8);
  const int bins = nx * ny;
  note_launches(dL ? 4 : 3);
  k_pupil_masks<<<(bins + 255) / 256, 256, 0, s>>>(g, mask);
  k_pupil_sums<<<(unsigned)n_cells, 256, 0, s>>>(tally, g, mask, inv_ncell, I);
  k_loss_scalar<<<1, 512, 0, s>>>(I, n_lam, n_f, g.n_pupil, kind, w_f, w_e, dI, out_dev);
  if (dL) {
    const long long n = n_cells * nx * ny;
    k_loss_scatter<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(dI, g, mask, inv_ncell, n_cells, dL);
  }
  return cudaGetLastError();
}

}  // namespace wgk
