// Host-side declarations shared by the CUDA translation units of libwg.so.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace wgk {

struct FieldRec;
struct HitRec;

// A ray that ended in the eyebox: its id and flat tally index. The forward
// trace lists them; the adjoint replays only listed rays whose bin has a
// non-zero dL/dtally (every other ray contributes no gradient).
struct ExitRec {
  long long id;
  int flat;  // flat tally index; -1: an unused slot (hole)
  int pad;   // the ray's mirror hits (the backward groups rays by it)
};

// Per hit record of a replay that also serves the tilt gradient: the applied
// coefficients of the hit (incl. the 1/sqrt(omega) rescale) and dL/d(cos t0)
// of the hit through its coating, 2 Re(A_s dc_s + A_p dc_p) with G folded in.
struct TiltAux {
  float2 cs, cp;
  double g_cos;
};
// A replayed ray with records: the tilt pass re-traces it and reads its hits'
// TiltAux entries [first, first + emit).
struct RayHead {
  long long id;
  int cell;
  int first;
  int emit;
  int events;  // surface events of the replayed path (the tangent pass groups its rays by it)
};

// Arguments of the trace kernels (passed by value).
struct TraceArgs {
  const uint8_t* blob;        // design blob (global), staged into smem
  int blob_bytes;             // multiple of 16
  const FieldRec* fields;     // [n_f]
  const float* lambda;        // [n_lam]
  int n_f, pol, max_events, bins;  // bins per cell = eb_nx * eb_ny
  long long n_cell;           // rays per cell
  long long ray_begin, ray_end;
  long long cell_lo;          // first cell touched by [ray_begin, ray_end)
  long long chunk_rays;       // rays per chunk
  long long chunks_per_cell;
  long long n_chunks;
  uint32_t key0, key1;
  int eb_nx, eb_ny;
  float eb_x0, eb_y0, eb_sx, eb_sy;  // bin = floor((q - x0) * s)
  float pupil_y;
  // outputs
  double* tally;              // forward: FP64 tally (full layout)
  const double* G;            // backward: dL/dtally
  double* ledger;             // [6]
  unsigned long long* counters;  // [10]: rays, hits, events, tir, layer steps, overflow, tallied,
                                 // adjoint layer steps, non-finite gradient terms, reserved
  void* records;              // wg_ray_record* or null
  unsigned long long* work;   // chunk queue counter (zeroed before launch)
  unsigned int* error;        // device error word (bounded waits)
  // backward replay
  HitRec* hit_buf;            // [hit_cap] hit records
  long long hit_cap;
  unsigned long long* hit_count;  // records reserved (may exceed hit_cap: overflow)
  int n_layers;               // device layers
  // forward: list of eyebox rays (null: not recorded)
  ExitRec* exit_list;
  long long exit_cap;
  unsigned long long* exit_count;
  // backward: replay the list entries [list_begin, list_end) instead of a ray range (null: ray range)
  const ExitRec* replay_list;
  long long list_begin, list_end;
  int n_cta;                  // CTAs of the launch working on this job
  int n_slots;                // forward: tally slots per CTA (1..kFwdSlots)
  // tilt gradient: FP64 per-degree sums for mirrors [tilt_k0, tilt_k0 + 8)
  double* grad_tilt;
  int tilt_k0;
  // replay with the tilt gradient: per-record TiltAux [hit_cap], one RayHead
  // per ray with records (head_count counts them); the tilt pass reads n_heads
  TiltAux* tilt_aux;
  RayHead* ray_heads;
  long long head_cap;
  unsigned long long* head_count;
  long long n_heads;
  // coating look-up table (null: exact transfer-matrix chain per hit):
  // per (mirror, side (0: ray on the +normal side), wavelength, cos bin j)
  // the raw coefficients at cos_j = lut_c0 + j / lut_inv_dc and their
  // derivatives d/d(cos t0), as float4 {r_s, r_p}, {t_s, t_p}, {dr_s, dr_p},
  // {dt_s, dt_p}; hits interpolate both linearly in cos(theta_0)
  const float4* lut;
  int lut_n, n_lam;
  float lut_c0, lut_inv_dc;
  // backward with the table: FP64 dL/d(coefficient) per entry, {r_s, r_p, t_s, t_p} x {re, im}
  double* lut_grad;
  // Applied coefficients (c_s, c_p as a float4) of the first coef_slots
  // mirror hits of every ray of a listing forward, at
  // (ray - coef_base) * coef_slots + hit (a ray's hits share a line for the
  // replay, which reads them in order): written by the forward (coef_mode 1)
  // and read back by the replay (coef_mode 2), which then skips those hits'
  // layer chains; 0: not used.
  float4* coef;
  long long coef_base, coef_rays;
  int coef_slots, coef_mode;
  unsigned long long wait_ns;  // limit of the bounded waits (device clock)
};

// Arguments of the thin-film adjoint over sorted hit records.
struct AdjArgs {
  const uint8_t* blob;
  int blob_bytes;
  const HitRec* recs;         // sorted by stack
  const float* lambda;        // [n_lam]: the records carry wavelength indices
  long long n_rec;
  int rec_chunk;              // records per CTA work item
  int n_layers;
  double* grad_acc;           // [n_layers] FP64 sums (device layer order)
  unsigned long long* work;
  unsigned long long* counters;
  unsigned int* error;
  // tilt gradient (null: none): dL/d(cos t0) of each record, written to
  // tilt_aux[perm[i]].g_cos (the record's slot before the sort)
  TiltAux* tilt_aux;
  const unsigned int* perm;
  unsigned long long wait_ns;  // limit of the bounded waits (device clock)
};

constexpr int kBlock = 256;
// sort keys of the adjoint's hit records: stack (mirror, side; 2 x 64) x
// evanescence class (how many of the design's materials are evanescent at
// the hit's incidence angle, 0..7)
constexpr int kStackKeys = 128, kClsPerStack = 8, kSortKeys = kStackKeys * kClsPerStack;
// the forward kernel keeps up to this many chunks (cells) in flight per CTA,
// each with its own FP32 shared tally. Large chunks take two: a CTA then
// draws its rays from fewer cells at a time (same wavelength and field, so
// its warps diverge less); small chunks take three, so a CTA does not wait
// for a slot while a chunk's last slow rays finish.
constexpr int kFwdSlots = 3;
inline int fwd_slots(long long chunk_rays) { return chunk_rays >= 1536 ? 2 : 3; }
// rays a warp of the forward kernel owns at a time (its lanes plus its two
// shared-memory queues), and the slots of each queue's ring (a power of two,
// so that a ring index is a mask; at least kFwdQCap); a queued ray takes
// 9 + 4 F words (+ 3 in accurate mode)
constexpr int kFwdQCap = 64;
constexpr int kFwdQRing = 64;
static_assert(kFwdQRing >= kFwdQCap && (kFwdQRing & (kFwdQRing - 1)) == 0, "queue ring");
// a warp of the forward kernel reserves eyebox-ray list slots this many at a
// time (one global atomic per chunk); slots it leaves unused are holes
// (flat = -1). The list holds at most rays + 64 warps per SM x one chunk.
constexpr int kExitChunk = 64;
inline long long exit_list_cap(long long rays, int sm_count) {
  return rays + (long long)sm_count * 64 * kExitChunk;
}
inline size_t fwd_smem_bytes(int blob_bytes, long long bins, int F, int n_slots, bool acc) {
  return (size_t)blob_bytes + sizeof(float) * (size_t)n_slots * (size_t)bins +
         sizeof(uint32_t) * (size_t)(kBlock / 32) * 2 * (size_t)kFwdQRing * (size_t)(9 + 4 * F + (acc ? 3 : 0));
}
// Accurate layer evaluation (direction, incidence cosine, material constants
// and layer phases carried as hi + lo; sin/cos on the FMA pipe) for designs
// whose longest stack has more than this many layers: the FP32 evaluation's
// error grows with the stack length and passes 1e-4 on long stacks.
constexpr int kAccLayers = 48;

// loads every instance of the forward trace kernel and the field preparation
// kernel onto the current device (under lazy loading a kernel is otherwise
// loaded, and its code placed in device memory, at its first launch)
cudaError_t preload_forward_kernels();

// number of kernels this library has launched (all launchers add to it)
void note_launches(unsigned long long n);
unsigned long long launches();

// launchers (return cudaError_t of the launch). P: material period of the
// design's stacks (0 = any, 2, 3); F: fields per ray (2 = s+p pair); acc:
// the accurate layer evaluation (designs with stacks longer than kAccLayers).
cudaError_t launch_prep_design(uint8_t* blob, const float* mir_x, const float* mir_tilt, const float* mir_omega,
                               const float* geo, int n_mir, float ic_tilt_deg, float thick, cudaStream_t s);
cudaError_t launch_prep_fields(FieldRec* out, const float* fx, const float* fy, int n_fx, int n_fy,
                               float n_slab, float ic_tilt_deg, int dims, cudaStream_t s);
cudaError_t launch_trace_fwd(const TraceArgs& a, int F, int P, int gm, bool acc, int grid, size_t smem,
                             cudaStream_t s);
// several jobs (designs / configurations with the same F and P) in one
// launch: CTA b works on job cta_job[b] (device arrays; each job's n_cta set)
// clears, for each of the n jobs of a fused launch (device table), its
// tally over the cells its ray range touches and its eyebox-ray counter
cudaError_t launch_zero_jobs(const TraceArgs* jobs_dev, int n, long long max_doubles, cudaStream_t s);
cudaError_t launch_trace_fwd_fused(const TraceArgs* jobs_dev, const int* cta_job_dev, int F, int P, bool acc,
                                   int grid, size_t smem, cudaStream_t s);
// tilt: also record TiltAux per hit and a RayHead per ray (a.tilt_aux, a.ray_heads)
cudaError_t launch_bwd_replay(const TraceArgs& a, int F, int P, bool tilt, int gm, bool acc, int grid, size_t smem,
                              cudaStream_t s);
// perm (may be null): perm[sorted position] = index of the record in `in`
cudaError_t launch_wait_flag(const unsigned* flag, unsigned* err, unsigned long long limit_ns, cudaStream_t s);
cudaError_t launch_bwd_sort(const HitRec* in, long long n, const uint8_t* blob, unsigned int* key_count, unsigned int* key_off,
                            unsigned int* key_cursor, HitRec* out, unsigned int* perm, cudaStream_t s);
cudaError_t launch_bwd_adjoint(const AdjArgs& a, int P, bool acc, int grid, size_t smem,
                               cudaStream_t s);  // a.tilt_aux picks the variant
cudaError_t launch_scatter_grad(const double* acc, int n_layers, const int* dev_to_orig, double* out,
                                cudaStream_t s);
cudaError_t launch_coating_eval(const uint8_t* blob, int P, bool acc, int mirror, int side, long long n,
                                const float* cos0, const float* lam, float* out, cudaStream_t s);
cudaError_t launch_coating_grad(const uint8_t* blob, int P, bool acc, int mirror, int side, long long n,
                                const float* cos0, const float* lam, const float* w, int which, float* grad,
                                cudaStream_t s);
cudaError_t launch_thickness_update(uint8_t* blob, const float* d_orig, const int* orig_to_store, int n_orig,
                                    cudaStream_t s);
// coating look-up table: entries for every (mirror, side, wavelength, bin)
// of the design (lam: device [n_lam]); records: one hit record per (entry,
// r or t) carrying the entry's accumulated FP64 weights, in stack order
// d f / d(cos theta_0) per sample through the coating (the adjoint's dual reverse sweep)
cudaError_t launch_coating_dcos(const uint8_t* blob, int P, bool acc, int mirror, int side, long long n,
                                const float* cos0, const float* lam, const float* w, int which, float* out,
                                cudaStream_t s);
cudaError_t launch_lut_build(const uint8_t* blob, int P, bool acc, int n_mir, int n_lam, const float* lam, int n,
                             float c0, float dc, float4* out, cudaStream_t s);
cudaError_t launch_lut_records(const double* grad, int n_mir, int n_lam, const float* lam, int n, float c0, float dc,
                               HitRec* out, cudaStream_t s);
// ray heads / listed eyebox rays grouped by their mirror-hit count (cnt: device
// scratch of kHitSortScratch bytes)
// bytes of the hit-count sort's counters (one per hit count 0..TAPE_HITS)
constexpr size_t kHitSortScratch = 1024;
cudaError_t launch_heads_sort(const RayHead* in, long long n, unsigned int* cnt, RayHead* out, cudaStream_t s);
cudaError_t launch_exits_sort(const ExitRec* in, long long n, unsigned int* cnt, ExitRec* out, cudaStream_t s);
// reflection-probability pre-optimization: geometric trace of the rays of a
// (a.tally, a.G; grad_omega [n_mir] FP64 sums, may be null)
cudaError_t launch_omega_trace(const TraceArgs& a, double* grad_omega, int gm, int sm_count, cudaStream_t s);
// mirror-tilt gradient of the a.n_heads rays a tilt replay recorded, one
// pass per group of 8 mirrors starting at a.tilt_k0
cudaError_t launch_tilt_grad(const TraceArgs& a, int F, int P, int gm, bool acc, int grid, size_t smem,
                             cudaStream_t s);
size_t tilt_smem_bytes(int blob_bytes, int F);
int tilt_blocks_per_sm(int F, int P, int gm, bool acc, size_t smem);
int trace_fwd_blocks_per_sm(int F, int P, int gm, bool acc, size_t smem);
int bwd_replay_blocks_per_sm(int F, int P, bool tilt, int gm, bool acc, size_t smem);
int bwd_adjoint_blocks_per_sm(int P, bool acc, size_t smem);
// dynamic shared memory of the adjoint kernel (blob, per-layer sums, segment buffers)
size_t adj_smem_bytes(int blob_bytes, int n_layers, int P);
size_t hit_rec_bytes();

// loss (workspace: 2 * cells * 9 + 8 doubles, then one u16 pupil mask per eyebox bin)
// loss workspace (doubles): I and dL/dI (9 per cell each), 8 result words,
// the pupil masks of the bins (u16), then the two spread parts of dL/dI, the
// statistic of every group and the sums of the field groups, the per-cell
// table over the 512 possible pupil masks, the masks that occur (512 ints and
// their count) and each bin's index among them (u16)
inline long long loss_ws_extra(long long n_cells, long long bins) {
  return 2 * n_cells * 9 + 8 + (bins * 2 + 7) / 8;
}
inline long long loss_ws_doubles(long long n_cells, long long bins, int n_lam) {
  return loss_ws_extra(n_cells, bins) + 2 * n_cells * 9 + 2 * (n_cells + 9 * (long long)n_lam) + n_cells * 512 +
         (512 * 4 + 16 + bins * 2 + 7) / 8;
}
cudaError_t launch_loss_impl(const double* tally, int dims, int n_lam, int n_f, int nx, int ny, double cx, double cy,
                             double w, double h, double inv_ncell, int kind, double w_f, double w_e, double* ws,
                             double* out_dev, double* dL, cudaStream_t s);

}  // namespace wgk
