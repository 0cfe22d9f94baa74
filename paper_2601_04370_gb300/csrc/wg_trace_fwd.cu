// Instances of the forward trace kernel (fast layer evaluation) and the
// forward launchers; the accurate instances are in wg_trace_fwd_acc.cu.
#include "wg_kernels.cuh"

namespace wgk {

using FwdKernel = void (*)(const TraceArgs, const TraceArgs*, const int*);
FwdKernel pick_fwd_accurate(int F, int P, int gm);
FwdKernel pick_fwd_table(int F, int gm, bool acc);

template <int GM>
static FwdKernel pick_fwd_gm(int F, int P) {
  return F == 2 ? (P == 3 ? k_trace_fwd<2, 3, GM, false> : P == 2 ? k_trace_fwd<2, 2, GM, false> : k_trace_fwd<2, 0, GM, false>)
                : (P == 3 ? k_trace_fwd<1, 3, GM, false> : P == 2 ? k_trace_fwd<1, 2, GM, false> : k_trace_fwd<1, 0, GM, false>);
}
// kernel instance for (fields F, material period P, geometry mode gm, accuracy mode acc)
static FwdKernel pick_fwd(int F, int P, int gm, bool acc) {
  if (acc) return pick_fwd_accurate(F, P, gm);
  return gm == 1 ? pick_fwd_gm<1>(F, P) : gm == 2 ? pick_fwd_gm<2>(F, P) : pick_fwd_gm<0>(F, P);
}

cudaError_t preload_field_kernel();

cudaError_t preload_forward_kernels() {
  for (int acc = 0; acc < 2; ++acc)
    for (int gm = 0; gm < 3; ++gm)
      for (int F = 1; F <= 2; ++F) {
        for (int P : {0, 2, 3}) {
          cudaFuncAttributes fa;
          const cudaError_t e = cudaFuncGetAttributes(&fa, pick_fwd(F, P, gm, acc != 0));
          if (e != cudaSuccess) return e;
        }
        cudaFuncAttributes fa;
        const cudaError_t e = cudaFuncGetAttributes(&fa, pick_fwd_table(F, gm, acc != 0));
        if (e != cudaSuccess) return e;
      }
  return preload_field_kernel();
}

int trace_fwd_blocks_per_sm(int F, int P, int gm, bool acc, size_t smem) {
  return occupancy(pick_fwd(F, P, gm, acc), smem);
}

cudaError_t launch_trace_fwd(const TraceArgs& a, int F, int P, int gm, bool acc, int grid, size_t smem,
                             cudaStream_t s) {
  // the coating table's instance when the call interpolates coefficients
  auto k = a.lut ? pick_fwd_table(F, gm, acc) : pick_fwd(F, P, gm, acc);
  raise_smem_limit(k);
  note_launches(1);
  TraceArgs a1 = a;
  a1.n_cta = grid;
  k<<<grid, kBlock, smem, s>>>(a1, nullptr, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_trace_fwd_fused(const TraceArgs* jobs_dev, const int* cta_job_dev, int F, int P, bool acc,
                                   int grid, size_t smem, cudaStream_t s) {
  auto k = pick_fwd(F, P, 2, acc);  // the jobs of a fused launch may mix PRMA and general designs
  raise_smem_limit(k);
  note_launches(1);
  TraceArgs unused;
  memset(&unused, 0, sizeof(unused));
  k<<<grid, kBlock, smem, s>>>(unused, jobs_dev, cta_job_dev);
  return cudaGetLastError();
}

}  // namespace wgk
