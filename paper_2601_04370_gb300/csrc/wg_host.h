// Internal host interfaces between the C-ABI translation units of libwg.so
// (wg_api.cu: contexts, designs, trace calls; wg_serve.cu: the serving
// runtime behind wg_submit / wg_poll / wg_cancel).
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "wg.h"

namespace wgh {

// One design evaluation of a fused forward launch.
struct FusedJob {
  const wg_design* design;
  const wg_trace_cfg* cfg;  // stream and ray_records are ignored
  double* tally;            // device [tally size], zeroed by the call
  long long chunk_rays;     // rays per chunk (0: the default split of a cell into chunks of <= 4096)
  wg_stats stats;           // out: this job's statistics
  wg_status status;         // out
  unsigned error_word;      // out: the job's device error bits (0 = none)
  int n_cta;                // out: CTAs the launch gave the job
  long long n_chunks;       // out: chunks of the job
};

// All jobs in as few kernel launches as possible: one persistent launch per
// (fields per ray, material period) group, each job on its own range of the
// launch's CTAs (in proportion to its estimated work). Stream-ordered on s;
// returns after the launches completed and the statistics were read.
// blocks_per_sm <= 0: the occupancy limit.
wg_status fused_forward(wg_ctx* c, FusedJob* jobs, int n, int blocks_per_sm, cudaStream_t s);

// The same in three steps, for CUDA graph capture of the device work:
// fused_prepare (host only: plans, allocations, pinned job tables),
// fused_enqueue (stream operations only: copies from pinned memory, memsets,
// kernel launches, event records; capturable), fused_finish (after the
// stream completed: statistics). The context's fused workspace must not be
// reallocated between a capture and its replays (fused_dev_base tells).
struct FusedBatch {
  struct Impl;
  Impl* impl;
  FusedBatch();
  ~FusedBatch();
  FusedBatch(const FusedBatch&) = delete;
  FusedBatch& operator=(const FusedBatch&) = delete;
};
wg_status fused_prepare(wg_ctx* c, FusedJob* jobs, int n, int blocks_per_sm, FusedBatch& fb);
wg_status fused_enqueue(wg_ctx* c, FusedJob* jobs, FusedBatch& fb, cudaStream_t s);
wg_status fused_finish(wg_ctx* c, FusedJob* jobs, FusedBatch& fb);
const void* fused_dev_base(const wg_ctx* c);
// Hash of what a captured fused_enqueue depends on besides the pinned
// contents; a graph is replayed only for a batch with the same signature.
uint64_t fused_signature(const wg_ctx* c, const FusedJob* jobs, const FusedBatch& fb);

// Size of a configuration's tally (doubles) and of a design's gradient, or -1
// if the configuration is invalid for the design.
long long tally_doubles(const wg_design* d, const wg_trace_cfg* cfg);
long long design_params(const wg_design* d);
// mirrors, device (non-pruned) layers, material period of the stacks
void design_shape(const wg_design* d, int* K, int* n_dev, int* period, int* acc);
// the design's context; its thicknesses as last set from the host (nm, 0 for
// layers the design prunes) and its pruned mask, both [design_params]
wg_ctx* design_ctx(const wg_design* d);
const float* design_thickness(const wg_design* d);
const uint8_t* design_pruned(const wg_design* d);
// the mirrors' reflection probabilities as last set [K]
const float* design_omega(const wg_design* d);
// Device bytes a forward (and a backward) evaluation of cfg holds while it
// runs, for admission against the HBM budget.
size_t eval_device_bytes(const wg_design* d, const wg_trace_cfg* cfg, bool backward);

// Context accessors for the serving runtime.
int ctx_device(const wg_ctx* c);
int ctx_sm_count(const wg_ctx* c);
int ctx_max_slots(const wg_ctx* c);
int ctx_max_queue(const wg_ctx* c);
long long ctx_max_batch_rays(const wg_ctx* c);
unsigned long long ctx_wait_limit(const wg_ctx* c);
size_t ctx_hbm_budget(const wg_ctx* c);
const char* ctx_autotune_cache(const wg_ctx* c);
void** ctx_serve_slot(wg_ctx* c);  // opaque serving state owned by wg_serve.cu

// Serving runtime teardown (wg_serve.cu), called by wg_shutdown before the
// context's resources are released.
void serve_shutdown(wg_ctx* c);

// Sets the calling thread's wg_last_error message and returns st.
wg_status set_error(wg_status st, const char* msg);

}  // namespace wgh
