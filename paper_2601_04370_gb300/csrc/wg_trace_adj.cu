// Instances of the thin-film adjoint over hit records, the coating table
// build and the coating test hooks (both accuracy modes), with their launchers.
#include "wg_kernels.cuh"

namespace wgk {

template <bool T, bool ACC>
static void (*pick_adjoint_acc(int P))(const AdjArgs) {
  return P == 3 ? k_bwd_adjoint<3, T, ACC> : P == 2 ? k_bwd_adjoint<2, T, ACC> : k_bwd_adjoint<0, T, ACC>;
}
static void (*pick_adjoint(int P, bool tilt, bool acc))(const AdjArgs) {
  return tilt ? (acc ? pick_adjoint_acc<true, true>(P) : pick_adjoint_acc<true, false>(P))
              : (acc ? pick_adjoint_acc<false, true>(P) : pick_adjoint_acc<false, false>(P));
}
int bwd_adjoint_blocks_per_sm(int P, bool acc, size_t smem) { return occupancy(pick_adjoint(P, false, acc), smem); }

cudaError_t launch_bwd_adjoint(const AdjArgs& a, int P, bool acc, int grid, size_t smem, cudaStream_t s) {
  auto k = pick_adjoint(P, a.tilt_aux != nullptr, acc);
  raise_smem_limit(k);
  note_launches(1);
  k<<<grid, kBlock, smem, s>>>(a);
  return cudaGetLastError();
}

#define WG_PICK_PA(K, P, A)                                             \
  ((A) ? ((P) == 3 ? K<3, true> : (P) == 2 ? K<2, true> : K<0, true>)   \
       : ((P) == 3 ? K<3, false> : (P) == 2 ? K<2, false> : K<0, false>))

cudaError_t launch_coating_eval(const uint8_t* blob, int P, bool acc, int mirror, int side, long long n,
                                const float* cos0, const float* lam, float* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  note_launches(1);
  WG_PICK_PA(k_coating_eval, P, acc)<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(blob, mirror, side, n, cos0, lam,
                                                                                 out);
  return cudaGetLastError();
}

cudaError_t launch_lut_build(const uint8_t* blob, int P, bool acc, int n_mir, int n_lam, const float* lam, int n,
                             float c0, float dc, float4* out, cudaStream_t s) {
  const long long total = (long long)n_mir * 2 * n_lam * n;
  if (total <= 0) return cudaSuccess;
  note_launches(1);
  WG_PICK_PA(k_lut_build, P, acc)<<<(unsigned)((total + 127) / 128), 128, 0, s>>>(blob, n_mir, n_lam, lam, n, c0,
                                                                                  dc, out);
  return cudaGetLastError();
}

cudaError_t launch_coating_grad(const uint8_t* blob, int P, bool acc, int mirror, int side, long long n,
                                const float* cos0, const float* lam, const float* w, int which, float* grad,
                                cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  note_launches(1);
  WG_PICK_PA(k_coating_grad, P, acc)<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(blob, mirror, side, n, cos0, lam,
                                                                                 w, which, grad);
  return cudaGetLastError();
}

cudaError_t launch_coating_dcos(const uint8_t* blob, int P, bool acc, int mirror, int side, long long n,
                                const float* cos0, const float* lam, const float* w, int which, float* out,
                                cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  note_launches(1);
  WG_PICK_PA(k_coating_dcos, P, acc)<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(blob, mirror, side, n, cos0, lam,
                                                                                 w, which, out);
  return cudaGetLastError();
}

}  // namespace wgk
