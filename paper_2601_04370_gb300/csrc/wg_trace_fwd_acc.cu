// Instances of the forward trace kernel with the accurate layer evaluation
// (designs with stacks longer than kAccLayers), and the coating table's
// instances (no layer chain: one per fields, geometry and accuracy mode).
#include "wg_kernels.cuh"

namespace wgk {

using FwdKernel = void (*)(const TraceArgs, const TraceArgs*, const int*);

template <int GM>
static FwdKernel pick_gm(int F, int P) {
  return F == 2 ? (P == 3 ? k_trace_fwd<2, 3, GM, true> : P == 2 ? k_trace_fwd<2, 2, GM, true> : k_trace_fwd<2, 0, GM, true>)
                : (P == 3 ? k_trace_fwd<1, 3, GM, true> : P == 2 ? k_trace_fwd<1, 2, GM, true> : k_trace_fwd<1, 0, GM, true>);
}
FwdKernel pick_fwd_accurate(int F, int P, int gm) {
  return gm == 1 ? pick_gm<1>(F, P) : gm == 2 ? pick_gm<2>(F, P) : pick_gm<0>(F, P);
}

template <int GM, bool ACC>
static FwdKernel pick_table_gm(int F) {
  return F == 2 ? k_trace_fwd<2, 0, GM, ACC, true> : k_trace_fwd<1, 0, GM, ACC, true>;
}
FwdKernel pick_fwd_table(int F, int gm, bool acc) {
  if (acc) return gm == 1 ? pick_table_gm<1, true>(F) : gm == 2 ? pick_table_gm<2, true>(F) : pick_table_gm<0, true>(F);
  return gm == 1 ? pick_table_gm<1, false>(F) : gm == 2 ? pick_table_gm<2, false>(F) : pick_table_gm<0, false>(F);
}

}  // namespace wgk
