// Instances of the replay and tilt-tangent kernels with the accurate layer
// evaluation and direction (designs with stacks longer than kAccLayers).
#include "wg_kernels.cuh"

namespace wgk {

using TraceKernel = void (*)(const TraceArgs);

template <bool T, int GM>
static TraceKernel pick_gm(int F, int P) {
  return F == 2 ? (P == 3 ? k_bwd_replay<2, 3, T, GM, true> : P == 2 ? k_bwd_replay<2, 2, T, GM, true>
                                                                    : k_bwd_replay<2, 0, T, GM, true>)
                : (P == 3 ? k_bwd_replay<1, 3, T, GM, true> : P == 2 ? k_bwd_replay<1, 2, T, GM, true>
                                                                    : k_bwd_replay<1, 0, T, GM, true>);
}
TraceKernel pick_replay_accurate(int F, int P, bool tilt, int gm) {
  return tilt ? (gm == 1 ? pick_gm<true, 1>(F, P) : pick_gm<true, 0>(F, P))
              : (gm == 1 ? pick_gm<false, 1>(F, P) : pick_gm<false, 0>(F, P));
}
TraceKernel pick_tilt_accurate(int F, int gm) {
  return gm == 1 ? (F == 2 ? k_tilt_grad<2, 1, true> : k_tilt_grad<1, 1, true>)
                 : (F == 2 ? k_tilt_grad<2, 0, true> : k_tilt_grad<1, 0, true>);
}

}  // namespace wgk
