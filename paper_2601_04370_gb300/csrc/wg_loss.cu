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

// I[cell, p]. FP64 adds are scarce on this part: a warp's 32 consecutive
// bins lie in 2-4 pupils, so the add of a pupil that none of them is in is
// skipped for the whole warp (the loop runs in whole warps).
__global__ void k_pupil_sums(const double* tally, LossGeom g, const unsigned short* mask, double inv_ncell,
                             double* I) {
  const long long cell = blockIdx.x;
  const int bins = g.nx * g.ny;
  __shared__ double s_acc[9][32];
  double acc[9];
  for (int p = 0; p < 9; ++p) acc[p] = 0.0;
  const double* t = tally + cell * bins;
  for (int b0 = threadIdx.x & ~31; b0 < bins; b0 += blockDim.x) {
    const int b = b0 + (threadIdx.x & 31);
    const double v = b < bins ? t[b] : 0.0;
    const unsigned m = b < bins ? mask[b] : 0u;
#pragma unroll
    for (int p = 0; p < 9; ++p)
      if (__any_sync(0xffffffffu, m & (1u << p)) && (m & (1u << p))) acc[p] += v;
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

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// The statistic of one group of n values x[i stride] with a whole warp and
// its gradient, scaled, written to dx (every entry: 0 where the statistic has
// none); returns the statistic and the group's sum. The per-group quotients
// are taken once (FP64 divides are slow here) and the entries multiplied.
__device__ void spread_group(const double* x, int n, long long stride, int kind, double scale, double* dx,
                             double& val, double& sum, int lane) {
  double su = 0.0;
  for (int i = lane; i < n; i += 32) su += x[i * stride];
  sum = warp_sum_d(su);
  const double mu = sum / n;
  double var = 0.0;
  for (int i = lane; i < n; i += 32) {
    const double d = x[i * stride] - mu;
    var += d * d;
  }
  var = warp_sum_d(var) / n;
  if (kind == 1) {
    val = var;
    const double c = scale * 2.0 / n;
    for (int i = lane; i < n; i += 32) dx[i * stride] = c * (x[i * stride] - mu);
    return;
  }
  const double sd = sqrt(var);
  val = mu == 0.0 ? 0.0 : sd / mu;
  if (mu == 0.0 || sd <= 0.0) {
    for (int i = lane; i < n; i += 32) dx[i * stride] = 0.0;
    return;
  }
  // d(sd/mu)/dx_i = (x_i - mu)/(n sd mu) - (sd/mu)/(n mu)
  const double a = scale / (n * sd * mu), b = scale * (val / mu) / n;
  for (int i = lane; i < n; i += 32) dx[i * stride] = fma(a, x[i * stride] - mu, -b);
}

// One warp per group: U_FoV groups q < n_lam P ((lambda, pupil): the n_f
// fields at stride P) into dIf, then U_eyebox groups ((lambda, field): its P
// pupils) into dIe; the groups of one kind touch disjoint entries. Each
// group's statistic goes to gval[q] and, for U_FoV (which covers every
// entry once), its sum of I to gsum[q]; k_loss_final adds them up.
__global__ void k_loss_groups(const double* I, int n_lam, int n_f, int P, int kind, double w_f, double w_e,
                              double* dIf, double* dIe, double* gval, double* gsum) {
  const int lane = threadIdx.x & 31;
  const long long q = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;  // the same in a warp
  const long long nfov = (long long)n_lam * P, neb = (long long)n_lam * n_f;
  if (q >= nfov + neb) return;
  double v, sum;
  if (q < nfov) {
    const long long off = (q / P) * n_f * P + q % P;
    spread_group(I + off, n_f, P, kind, w_f / (double)nfov, dIf + off, v, sum, lane);
    if (lane == 0) {
      gval[q] = v;
      gsum[q] = sum;
    }
  } else {
    const long long off = (q - nfov) * P;
    spread_group(I + off, P, 1, kind, w_e / (double)neb, dIe + off, v, sum, lane);
    if (lane == 0) gval[q] = v;
  }
}

// One block: dL/dI = -1/N + the two spread parts, and the scalars
// L = -mean + w_f U_FoV + w_e U_eyebox, sums in a fixed order
__global__ void k_loss_final(int n_lam, int n_f, int P, double w_f, double w_e, const double* dIf, const double* dIe,
                             const double* gval, const double* gsum, double* dI, double* out) {
  const long long N = (long long)n_lam * n_f * P, nfov = (long long)n_lam * P, neb = (long long)n_lam * n_f;
  for (long long i = threadIdx.x; i < N; i += blockDim.x) dI[i] = (-1.0 / (double)N + dIf[i]) + dIe[i];
  __shared__ double s_red[3][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double sum = 0.0, uf = 0.0, ue = 0.0;
  for (long long q = threadIdx.x; q < nfov; q += blockDim.x) {
    sum += gsum[q];
    uf += gval[q];
  }
  for (long long q = threadIdx.x; q < neb; q += blockDim.x) ue += gval[nfov + q];
  double vals[3] = {sum, uf, ue};
  for (int k = 0; k < 3; ++k) {
    const double v = warp_sum_d(vals[k]);
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

// dL/dtally[cell, bin] = sum_{p containing bin} dL/dI[cell, p] / rays per cell.
// The bins take few distinct pupil masks (2-4 pupils overlap at most), so the
// sum is formed once per (cell, mask that occurs) and the bins copy it: no
// FP64 arithmetic per bin (scarce on this part), the same value per bin.
constexpr int kMaskValues = 512;  // 2^9 pupil masks
// one block: the masks that occur, in increasing order, and each bin's index
// among them
__global__ void k_mask_ids(const unsigned short* mask, int bins, int* occ_list, int* n_occ,
                           unsigned short* mid) {
  __shared__ unsigned s_bits[kMaskValues / 32];
  __shared__ unsigned short s_id[kMaskValues];
  for (int i = threadIdx.x; i < kMaskValues / 32; i += blockDim.x) s_bits[i] = 0u;
  __syncthreads();
  for (int b = threadIdx.x; b < bins; b += blockDim.x) atomicOr(&s_bits[mask[b] >> 5], 1u << (mask[b] & 31));
  __syncthreads();
  if (threadIdx.x == 0) {
    int n = 0;
    for (int m = 0; m < kMaskValues; ++m)
      if (s_bits[m >> 5] & (1u << (m & 31))) {
        s_id[m] = (unsigned short)n;
        occ_list[n++] = m;
      }
    *n_occ = n;
  }
  __syncthreads();
  for (int b = threadIdx.x; b < bins; b += blockDim.x) mid[b] = s_id[mask[b]];
}

// table[cell, j] = sum over the pupils p of mask occ_list[j] (increasing p) of
// dL/dI[cell, p], times 1 / rays per cell
__global__ void k_loss_table(const double* dI, int n_pupil, const int* occ_list, const int* n_occ, double inv_ncell,
                             double* table) {
  const long long cell = blockIdx.x;
  const int n = *n_occ;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const unsigned m = (unsigned)occ_list[j];
    double v = 0.0;
    for (int p = 0; p < n_pupil; ++p)
      if (m & (1u << p)) v += dI[cell * n_pupil + p];
    table[cell * kMaskValues + j] = v * inv_ncell;
  }
}

// dL/dtally[cell, bin] (grid: bins in x, cells in y)
__global__ void k_loss_scatter(const double* table, const unsigned short* mid, int bins, double* dL) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  const long long cell = blockIdx.y;
  if (b < bins) dL[cell * bins + b] = table[cell * kMaskValues + mid[b]];
}

cudaError_t launch_loss_impl(const double* tally, int dims, int n_lam, int n_f, int nx, int ny, double cx, double cy,
                             double w, double h, double inv_ncell, int kind, double w_f, double w_e, double* ws,
                             double* out_dev, double* dL, cudaStream_t s) {
  LossGeom g{dims, nx, ny, dims == 2 ? 3 : 9, cx, cy, w, h};
  const long long n_cells = (long long)n_lam * n_f;
  const int bins = nx * ny;
  double* I = ws;
  double* dI = ws + n_cells * g.n_pupil;
  unsigned short* mask = reinterpret_cast<unsigned short*>(ws + 2 * n_cells * 9 + 8);
  double* dIf = ws + loss_ws_extra(n_cells, bins);
  double* dIe = dIf + n_cells * 9;
  double* gval = dIe + n_cells * 9;
  double* gsum = gval + n_cells + 9 * (long long)n_lam;
  double* table = gsum + n_cells + 9 * (long long)n_lam;
  int* occ_list = reinterpret_cast<int*>(table + n_cells * kMaskValues);
  int* n_occ = occ_list + kMaskValues;
  unsigned short* mid = reinterpret_cast<unsigned short*>(n_occ + 4);
  const long long n_groups = (long long)n_lam * g.n_pupil + n_cells;
  note_launches(dL ? 7 : 4);
  k_pupil_masks<<<(bins + 255) / 256, 256, 0, s>>>(g, mask);
  k_pupil_sums<<<(unsigned)n_cells, 256, 0, s>>>(tally, g, mask, inv_ncell, I);
  k_loss_groups<<<(unsigned)((n_groups * 32 + 255) / 256), 256, 0, s>>>(I, n_lam, n_f, g.n_pupil, kind, w_f, w_e, dIf,
                                                                         dIe, gval, gsum);
  k_loss_final<<<1, 256, 0, s>>>(n_lam, n_f, g.n_pupil, w_f, w_e, dIf, dIe, gval, gsum, dI, out_dev);
  if (dL) {
    k_mask_ids<<<1, 1024, 0, s>>>(mask, bins, occ_list, n_occ, mid);
    k_loss_table<<<(unsigned)n_cells, 64, 0, s>>>(dI, g.n_pupil, occ_list, n_occ, inv_ncell, table);
    k_loss_scatter<<<dim3((unsigned)((bins + 255) / 256), (unsigned)n_cells), 256, 0, s>>>(table, mid, bins, dL);
  }
  return cudaGetLastError();
}

}  // namespace wgk
