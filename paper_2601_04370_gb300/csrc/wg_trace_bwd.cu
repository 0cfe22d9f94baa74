// Instances of the replay and tilt-tangent kernels (fast layer evaluation)
// and their launchers; the accurate instances are in wg_trace_bwd_acc.cu.
#include "wg_kernels.cuh"

namespace wgk {

using TraceKernel = void (*)(const TraceArgs);
TraceKernel pick_replay_accurate(int F, int P, bool tilt, int gm);
TraceKernel pick_tilt_accurate(int F, int gm);

template <bool T, int GM>
static TraceKernel pick_replay_gm(int F, int P) {
  return F == 2 ? (P == 3 ? k_bwd_replay<2, 3, T, GM, false> : P == 2 ? k_bwd_replay<2, 2, T, GM, false>
                                                                     : k_bwd_replay<2, 0, T, GM, false>)
                : (P == 3 ? k_bwd_replay<1, 3, T, GM, false> : P == 2 ? k_bwd_replay<1, 2, T, GM, false>
                                                                     : k_bwd_replay<1, 0, T, GM, false>);
}
static TraceKernel pick_replay(int F, int P, bool tilt, int gm, bool acc) {
  if (acc) return pick_replay_accurate(F, P, tilt, gm);
  return tilt ? (gm == 1 ? pick_replay_gm<true, 1>(F, P) : pick_replay_gm<true, 0>(F, P))
              : (gm == 1 ? pick_replay_gm<false, 1>(F, P) : pick_replay_gm<false, 0>(F, P));
}
static TraceKernel pick_tilt(int F, int gm, bool acc) {
  if (acc) return pick_tilt_accurate(F, gm);
  return gm == 1 ? (F == 2 ? k_tilt_grad<2, 1, false> : k_tilt_grad<1, 1, false>)
                 : (F == 2 ? k_tilt_grad<2, 0, false> : k_tilt_grad<1, 0, false>);
}

int bwd_replay_blocks_per_sm(int F, int P, bool tilt, int gm, bool acc, size_t smem) {
  return occupancy(pick_replay(F, P, tilt, gm, acc), smem);
}

cudaError_t launch_bwd_replay(const TraceArgs& a, int F, int P, bool tilt, int gm, bool acc, int grid, size_t smem,
                              cudaStream_t s) {
  auto k = pick_replay(F, P, tilt, gm, acc);
  raise_smem_limit(k);
  note_launches(1);
  k<<<grid, kBlock, smem, s>>>(a);
  return cudaGetLastError();
}

int tilt_blocks_per_sm(int F, int P, int gm, bool acc, size_t smem) {
  (void)P;
  auto k = pick_tilt(F, gm, acc);
  int n = 0;
  raise_smem_limit(k);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kTiltBlock, smem);
  return n;
}

cudaError_t launch_tilt_grad(const TraceArgs& a, int F, int P, int gm, bool acc, int grid, size_t smem,
                             cudaStream_t s) {
  (void)P;
  auto k = pick_tilt(F, gm, acc);
  raise_smem_limit(k);
  note_launches(1);
  k<<<grid, kTiltBlock, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace wgk
