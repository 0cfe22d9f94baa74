/*
 * wg.h - C ABI of the GB300 waveguide ray-trace library (libwg.so).
 *
 * The library evaluates the hot path of "End-to-end differentiable design of
 * geometric waveguide displays" (arXiv 2601.04370): Monte Carlo
 * non-sequential polarization ray tracing through a slab waveguide with a
 * partially reflective mirror array (PRMA), a multilayer thin-film
 * transfer-matrix evaluation at every ray-mirror hit, the eyebox tally, the
 * loss of Eq. 1 and the adjoint of the whole chain with respect to the layer
 * thicknesses. All arithmetic runs in hand-written CUDA kernels for sm_103a.
 *
 * Conventions (every entry point):
 *  - Every call returns a wg_status (0 = WG_OK, negative = error) and never
 *    aborts the process; wg_last_error() returns a message for the calling
 *    thread's last failure.
 *  - Lengths are mm, layer thicknesses and wavelengths nm, angles degrees.
 *  - A `stream` argument is a cudaStream_t passed as void*; NULL means the
 *    legacy default stream. Calls are stream-ordered unless stated otherwise.
 *  - Pointers documented as "host or device" are inspected with
 *    cudaPointerGetAttributes: device pointers are used in place; host
 *    pointers are staged through device memory inside the call (the call then
 *    synchronizes its stream before returning).
 *  - Tally layout: row-major [lambda][field_y][field_x][eyebox_y][eyebox_x],
 *    FP64. Thickness-gradient layout: the design's layers, mirror by mirror,
 *    layer 1 first (the order of wg_design_desc.layer_thickness_nm).
 *  - Inputs are FP32 at the boundary except tallies and gradients (FP64);
 *    the kernels compute in FP32 and accumulate tallies/gradients in FP64.
 */
#ifndef WG_H_
#define WG_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t wg_status;
#define WG_OK 0
#define WG_EINVAL (-1)      /* invalid argument or design */
#define WG_ENOMEM (-2)      /* device allocation failed / admission refused */
#define WG_EBUSY (-3)       /* request queue full */
#define WG_ENOTREADY (-4)   /* poll timed out; request still running */
#define WG_ETIMEOUT (-5)    /* a bounded device wait ran out */
#define WG_ECANCELED (-6)   /* request was cancelled */
#define WG_EDEVICE (-7)     /* CUDA runtime error */
#define WG_ENOTFOUND (-8)   /* unknown ticket */

#define WG_MAX_MIRRORS 64
#define WG_MAX_MATERIALS 4
#define WG_MAX_EVENTS 128   /* upper bound of wg_trace_cfg.max_events */

/* polarization of the launched light */
#define WG_POL_PAIR 0          /* unpolarized: s and p Jones pair, I = (I_s+I_p)/2 */
#define WG_POL_RANDOM_LINEAR 1 /* linear at angle pi*u per ray */
#define WG_POL_S 2
#define WG_POL_P 3

/* wg_trace_cfg.flags. By default wg_trace_forward also lists, in device
 * memory owned by the design (16 bytes per traced ray), the rays that ended
 * in the eyebox with their tally bin, tagged with the configuration and the
 * mirror geometry it traced. Ray paths do not depend on layer thicknesses
 * (Methods, Monte Carlo sampling: decisions depend only on the keys and the
 * geometry), so a later wg_trace_backward with the same configuration and
 * geometry, whatever the thicknesses, replays only the listed rays whose bin
 * has a non-zero dL/dtally; every other ray contributes no gradient. Any
 * other backward call replays every ray. The list holds up to 16 bytes x
 * (rays + 4096 x the GPU's SM count); unused slots are marked with bin -1.
 * A forward with WG_TRACE_NO_EXIT_LIST leaves an earlier list as it was. */
#define WG_TRACE_NO_EXIT_LIST 1  /* forward: do not record the list */

/* energy ledger slots (wg_stats.ledger) */
#define WG_LEDGER_EYEBOX 0     /* tallied intensity */
#define WG_LEDGER_MISSED 1     /* left through the eye-side face outside the eyebox */
#define WG_LEDGER_EXIT_REFL 2  /* Fresnel-reflected remainder at eye-side exits */
#define WG_LEDGER_LEAKED 3     /* left through the back face */
#define WG_LEDGER_ABSORBED 4   /* hit the input mirror side, the far end or a lateral side */
#define WG_LEDGER_TRUNCATED 5  /* still alive after max_events surface events */

typedef struct wg_ctx wg_ctx;
typedef struct wg_design wg_design;

typedef struct wg_init_opts {
  int32_t device;              /* CUDA device ordinal */
  int32_t max_slots;           /* serving: requests admitted at once (0 = 64) */
  size_t hbm_budget_bytes;     /* serving: admission budget (0 = 80% of free HBM) */
  const char* autotune_cache;  /* serving: file for autotuned launch shapes, or NULL */
  /* limit of every bounded wait inside the kernels (design staging, a warp
   * waiting for its CTA's next chunk), by the device clock; a kernel whose
   * wait runs out sets its error word, finishes what it holds and returns,
   * and the call returns WG_ETIMEOUT (0 = 0.5 s) */
  uint64_t wait_limit_ns;
  int32_t max_queue;           /* serving: queued requests before wg_submit returns WG_EBUSY (0 = 4096) */
  int32_t reserved;
  int64_t max_batch_rays;      /* serving: rays a batch admits beyond its first request (0 = 2^25) */
} wg_init_opts;

/*
 * Waveguide design (Results, "System Architecture"): a glass slab
 * 0 <= z <= thickness with TIR faces, an input mirror (plane through the
 * origin tilted by ic_tilt_deg about y) that couples the panel's rays in, and
 * K partially reflective mirrors, mirror k a plane through
 * (mirror_x_mm[k], 0, thickness/2) with normal (-sin a, 0, cos a),
 * a = mirror_tilt_deg[k]. Each mirror carries a lossless multilayer stack;
 * layer 1 faces the +normal side. A pruned layer has zero thickness and is
 * skipped. mirror_omega[k] is the Monte Carlo reflection probability
 * (Methods, "Differentiable Monte Carlo ...", Eq. 5), 0 < omega < 1.
 * mirror_geometry (NULL: the planes above) makes every mirror a general
 * plane, for fold-and-output layouts such as the paper's two-dimensional
 * pupil expansion (30 folding and 16 output mirrors, Results, "System
 * Architecture"). Row k holds 14 floats: a unit normal N0, a pivot point on
 * the plane (mm), a unit tilt axis perpendicular to N0, the rectangle x0, x1,
 * y0, y1 (mm, +-inf allowed) of the slab's (x, y) where the mirror acts (a ray
 * that crosses the plane outside it passes unchanged), and t0 (deg), the
 * tilt at which the normal is N0. At the tilt t = mirror_tilt_deg[k] (or
 * wg_set_params) the normal is cos(t - t0) N0 + sin(t - t0) axis x N0, the
 * plane through the pivot; the tilt gradient is per degree of that rotation.
 * mirror_x_mm is then only a label. WG_EINVAL for a non-unit normal or axis, an axis not
 * perpendicular to the normal, or an empty rectangle.
 * All arrays are host memory owned by the caller; wg_create_design copies
 * them.
 */
typedef struct wg_design_desc {
  int32_t dims;         /* 2 (x-z plane) or 3 */
  int32_t n_materials;  /* <= WG_MAX_MATERIALS */
  int32_t n_mirrors;    /* 1..WG_MAX_MIRRORS */
  int32_t reserved;
  float n_slab, thickness_mm, width_mm, x_end_mm, eye_relief_mm, ic_tilt_deg;
  const float* material_n;          /* [n_materials] refractive index */
  const float* mirror_x_mm;         /* [n_mirrors] */
  const float* mirror_tilt_deg;     /* [n_mirrors] */
  const float* mirror_omega;        /* [n_mirrors] */
  const int32_t* n_layers;          /* [n_mirrors] */
  const int32_t* layer_material;    /* [sum n_layers] material index */
  const float* layer_thickness_nm;  /* [sum n_layers] */
  const uint8_t* layer_pruned;      /* [sum n_layers] 1 = pruned, or NULL */
  const float* mirror_geometry;     /* [n_mirrors][14] general mirrors (above), or NULL */
} wg_design_desc;

/*
 * Trace configuration (Results, "System Architecture": parallel rays per
 * field-of-view sample from the panel, several wavelengths, an eyebox grid at
 * the eye relief). Ray r belongs to cell r / N_cell, N_cell =
 * ceil(n_rays / (n_lambda * n_fx * n_fy)); cell = (lambda * n_fy + fy) * n_fx
 * + fx. Its random numbers are Philox4x32-10 with key = seed and counter
 * (r_lo, r_hi, 0, "GEN0") for the launch, (r_lo, r_hi, m >> 2, "EVT0") word
 * m & 3 for the decision at its m-th mirror hit.
 */
typedef struct wg_trace_cfg {
  int32_t n_lambda, n_fx, n_fy, pol;
  const float* lambda_nm;     /* host [n_lambda] */
  const float* field_x_deg;   /* host [n_fx] field angle about y, in air */
  const float* field_y_deg;   /* host [n_fy] field angle about x, in air (2D: one value, 0) */
  int64_t n_rays;             /* requested rays (rounded up to whole cells) */
  uint64_t seed;
  int32_t max_events;         /* surface events per ray, <= WG_MAX_EVENTS */
  int32_t eb_nx, eb_ny;       /* eyebox bins (2D: eb_ny = 1) */
  int32_t flags;              /* WG_TRACE_* bits, 0 = defaults */
  float pupil_y_mm;           /* 3D: lateral extent of the launch region */
  float eb_cx_mm, eb_cy_mm, eb_w_mm, eb_h_mm;  /* eyebox centre and size */
  int32_t lut_bins;           /* 0: each hit runs its stack's transfer-matrix chain. N in
                                 [16, 65536]: the coating look-up table of the paper's
                                 memory-saving variant (Fig. 3c, Results): per mirror,
                                 side and wavelength the coefficients at cos(theta_0) =
                                 (j + 1/2) / N are computed once per call, every hit
                                 interpolates linearly in cos(theta_0), and the adjoint
                                 scatters dL/dc into the table's entries and runs the
                                 thin-film adjoint once per entry. wg_trace_forward and
                                 wg_trace_backward only (not served, not no-alloc). */
  void* stream;               /* cudaStream_t or NULL */
  int64_t ray_begin, ray_end; /* traced ray ids [begin, end); end <= 0: all */
  void* ray_records;          /* NULL or device wg_ray_record[end - begin]; a host pointer: WG_EINVAL */
} wg_trace_cfg;

/* per-ray record written when wg_trace_cfg.ray_records != NULL */
typedef struct wg_ray_record {
  uint32_t hash;     /* FNV-1a over (surface id | 0x80 if reflected at a mirror) per event */
  int32_t n_events;  /* surface events */
  int32_t n_hits;    /* ray-mirror (PRMA) interactions */
  int32_t cat;       /* WG_LEDGER_* category of the ray's end */
  int32_t bin;       /* flat tally index, -1 if not tallied */
  float intensity;   /* tallied intensity (0 if not tallied) */
  float weight;      /* |E|^2 at the ray's end (pair-averaged) */
  int32_t pad;
} wg_ray_record;

typedef struct wg_stats {
  int64_t n_rays;         /* rays traced */
  int64_t n_hits;         /* ray-mirror (PRMA) interactions: the throughput unit */
  int64_t n_events;       /* all surface events */
  int64_t n_tir;          /* total internal reflections */
  int64_t n_layer_steps;  /* transfer-matrix layer steps (sum of layers over hits) */
  double ledger[6];       /* energy by WG_LEDGER_* slot, in units of launched power */
  float kernel_ms;        /* device time of the main kernel (CUDA events) */
  int32_t overflow;       /* backward: rays with more than 64 mirror hits (gradient skipped) */
  int64_t n_tallied;      /* backward: rays that ended in the eyebox */
  int64_t n_adjoint_steps;/* backward: layer steps of the thin-film adjoint */
  int64_t n_nonfinite;    /* backward: non-finite per-layer terms dropped (expected 0) */
  float replay_ms;        /* backward: device time of the replay launches (CUDA events) */
  float adjoint_ms;       /* backward: device time of the thin-film adjoint launches */
  float tilt_ms;          /* backward: device time of the tilt tangent passes (0 without grad_tilt) */
  int32_t n_adjoint_launches; /* backward: thin-film adjoint launches (one per replay batch with records) */
} wg_stats;

/* ---- context ---------------------------------------------------------- */

/* Creates a context on opts->device (NULL opts: device 0, defaults).
 * Errors: WG_EINVAL (bad device), WG_EDEVICE. Owns no caller memory. */
wg_status wg_init(wg_ctx** ctx, const wg_init_opts* opts);

/* Stops the serving thread, frees every device buffer of the context and of
 * designs still alive. Safe on NULL. */
void wg_shutdown(wg_ctx* ctx);

/* Message of the calling thread's last failed call (static storage). */
const char* wg_last_error(void);

/* Library version string. */
const char* wg_version(void);

/* Number of CUDA kernels this library has launched in this process (all
 * entry points, all contexts). Lets a caller count the kernels of a timed
 * region. */
uint64_t wg_kernel_launches(void);

/* ---- designs ---------------------------------------------------------- */

/* Validates and uploads a design (deep copy; the caller keeps its arrays).
 * Errors: WG_EINVAL (dims, counts, NaN or negative thickness, omega outside
 * (0,1), index out of range), WG_ENOMEM. */
wg_status wg_create_design(wg_ctx* ctx, const wg_design_desc* desc, wg_design** out);

/* Optimizer step: replaces thicknesses ([sum n_layers], host or device, FP32;
 * NULL keeps them) and tilts ([n_mirrors], host, degrees; NULL keeps them).
 * Pruned layers keep zero thickness. Stream-ordered on `stream`.
 * Errors: WG_EINVAL on size mismatch or invalid values. */
wg_status wg_set_params(wg_design* d, const float* thickness_nm, int64_t n_thickness,
                        const float* tilt_deg, int32_t n_tilt, void* stream);

/* Frees the design's device memory (after its stream work completes). */
void wg_destroy_design(wg_design* d);

/* ---- thin-film coating (Methods, "Multilayer thin-film solver") ------- */

/*
 * Effective coefficients of mirror `mirror`'s stack between two half-spaces
 * of slab glass, by the characteristic-matrix method (Heavens): per layer
 * delta = 2 pi n d cos(theta)/lambda and M = [[cos d, i sin d/eta],
 * [i eta sin d, cos d]], eta_s = n cos, eta_p = n / cos. Results use the
 * paper's Fresnel sign convention (r_p = -r_s at normal incidence).
 * side = 0: light arrives on the +normal side (layer 1 first); 1: reversed.
 * cos_theta, lambda_nm: device [n]; out_rt: device [n][8] =
 * Re/Im of r_s, r_p, t_s, t_p. Errors: WG_EINVAL.
 */
wg_status wg_eval_coating(wg_ctx* ctx, const wg_design* d, int32_t mirror, int32_t side, int64_t n,
                          const float* cos_theta, const float* lambda_nm, float* out_rt, void* stream);

/*
 * Gradient of f = 2 Re(A_s c_s + A_p c_p) (c = r if which == 0, t if 1) with
 * respect to each non-pruned layer thickness of the mirror's stack, in
 * traversal order, by the checkpointed reverse sweep the adjoint kernel uses.
 * weights: device [n][4] = Re A_s, Im A_s, Re A_p, Im A_p. grad: device
 * [n][L] (L = non-pruned layers of the mirror, per nm, FP32).
 */
wg_status wg_eval_coating_grad(wg_ctx* ctx, const wg_design* d, int32_t mirror, int32_t side, int64_t n,
                               const float* cos_theta, const float* lambda_nm, const float* weights,
                               int32_t which, float* grad, void* stream);
/*
 * d f / d(cos theta_0) of the same f through the coating (the coating term of
 * the mirror-tilt gradient), from the same reverse sweep: grad_cos device [n]
 * FP32. Errors: WG_EINVAL.
 */
wg_status wg_eval_coating_dcos(wg_ctx* ctx, const wg_design* d, int32_t mirror, int32_t side, int64_t n,
                               const float* cos_theta, const float* lambda_nm, const float* weights, int32_t which,
                               float* grad_cos, void* stream);

/* ---- trace, loss, adjoint --------------------------------------------- */

/*
 * Forward Monte Carlo trace (Methods, "Polarization ray tracing" Eq. 4 and
 * "Differentiable Monte Carlo ..." Eq. 5; intensity I = sum |E|^2).
 * Per ray: launch on the input mirror, TIR at the slab faces (Fresnel with an
 * evanescent transmitted wave), at every mirror hit the stack's (r_s, r_p,
 * t_s, t_p), projection onto the local s/p basis, reflect with probability
 * omega and rescale the field by 1/sqrt(omega) or 1/sqrt(1-omega); at the
 * eye-side face the Fresnel power transmission into air, propagation to the
 * eye plane and an FP64 tally.
 * tally: host or device, FP64, tally layout, overwritten for the traced cells
 * (zeroed first). stats: host, optional (NULL: no synchronization).
 * Errors: WG_EINVAL, WG_ENOMEM, WG_EDEVICE.
 */
wg_status wg_trace_forward(wg_ctx* ctx, const wg_design* d, const wg_trace_cfg* cfg, double* tally,
                           wg_stats* stats);

/*
 * Loss of Results Eq. 1 on a tally: L = -I_mean + w_f U_FoV + w_e U_eyebox,
 * with pupil images I[lambda, field, pupil] = sum of the tally over 3x3
 * discs of 4 mm diameter spanning the eyebox (3 intervals in 2D), divided by
 * rays per cell; U = coefficient of variation (kind 0, paper) or variance
 * (kind 1), averaged over the other axes. tally: device FP64. out: host
 * double[4] = L, I_mean, U_FoV, U_eyebox (the call synchronizes). dL_dtally:
 * device FP64, tally layout, or NULL.
 */
wg_status wg_loss(wg_ctx* ctx, const wg_design* d, const wg_trace_cfg* cfg, int32_t kind, double w_f,
                  double w_e, const double* tally, double* out, double* dL_dtally);

/*
 * Adjoint of the trace with respect to layer thicknesses and mirror tilts
 * (Fig. 3b/c): replays the rays from their Philox keys (only the forward's
 * listed eyebox rays whose bins carry gradient when the list matches, see
 * WG_TRACE_NO_EXIT_LIST; every ray otherwise), propagates G[bin] dI/dE
 * backwards through each ray's Jones maps and back-propagates each hit's
 * coefficient sensitivity through the characteristic-matrix chain
 * (checkpointed forward products; a stack whose layers all propagate is
 * walked back by inverse layer steps between checkpoints). The sampled path
 * (keys, surfaces, decisions, TIR counts, bin) is held fixed: exact for the
 * thicknesses, which the sampling does not depend on; for the tilts it is
 * the derivative along the fixed path (a ray whose path or bin would change
 * contributes only that). dL_dtally: host or device FP64 in tally layout.
 * grad_thickness: host or device FP64 [sum n_layers] (pruned layers get 0),
 * overwritten. grad_tilt: NULL, or host or device FP64 [n_mirrors],
 * overwritten with dL/d(tilt) per degree (forward-mode tangents of every
 * ray's directions and fields, 8 mirrors per replay pass).
 * Errors: WG_EINVAL, WG_ENOMEM, WG_EDEVICE, WG_ETIMEOUT.
 */
wg_status wg_trace_backward(wg_ctx* ctx, const wg_design* d, const wg_trace_cfg* cfg,
                            const double* dL_dtally, double* grad_thickness, double* grad_tilt,
                            wg_stats* stats);

/*
 * Allocation-free forward trace. The paper has no counterpart to this entry
 * point: it is for callers that cannot allocate device memory while they
 * trace, for example a host application whose own allocator owns all of the
 * GPU's memory, or a loop with a fixed memory budget where an allocation
 * could fail or stall. It computes what wg_trace_forward computes with the
 * same kernels, but its per-call scratch (counters, energy ledger, chunk
 * queue, wavelength and field tables) lives in one static device array of
 * WG_NOALLOC_SCRATCH_BYTES bytes compiled into libwg.so instead of the
 * context's workspace; every GPU that loads the library holds that array
 * until the process exits. The call makes no device allocation.
 *  - tally: device memory only (FP64, tally layout), overwritten for the
 *    traced cells; a host pointer is rejected with WG_EINVAL (staging it
 *    would allocate).
 *  - The scratch needed is 256 B + the wavelength and field-angle arrays +
 *    48 B per field (up to ~2700 fields); a configuration that needs more
 *    than WG_NOALLOC_SCRATCH_BYTES is rejected with WG_EINVAL.
 *  - wg_init places the array on its device and looks up its device address
 *    (cudaGetSymbolAddress, with that device current), and loads the forward
 *    kernels there, so no call of this entry point, the first included,
 *    loads or allocates anything on the device.
 *  - Every call shares the array and clears the parts that must start at
 *    zero; the array keeps the last call's contents. Calls whose work
 *    overlaps on the GPU (other streams, other threads) race on the array:
 *    serialize them.
 * stats: host, optional (non-NULL synchronizes the stream).
 */
#define WG_NOALLOC_SCRATCH_BYTES (128 * 1024)
wg_status wg_trace_forward_noalloc(wg_ctx* ctx, const wg_design* d, const wg_trace_cfg* cfg, double* tally,
                                   wg_stats* stats);

/* ------------------------------------------------------------------------
 * Serving: design evaluations (the inner step of the paper's design
 * optimisation, Methods) submitted as they arrive.
 *
 * wg_submit copies the request and returns at once. A scheduler thread of
 * the context (started by the first submit, stopped by wg_shutdown) forms a
 * batch from whatever is queued whenever the GPU is free: FIFO, at most
 * wg_init_opts.max_slots requests, admitted while the batch's device memory
 * fits the HBM budget (wg_init_opts.hbm_budget_bytes, 0 = 80% of free HBM).
 * It traces the batch's forward passes in fused persistent launches (one per
 * kernel variant, each design on its own range of CTAs, chunk sizes and CTAs
 * per SM from the autotuned table); a batch whose launches were captured
 * before replays the captured CUDA graph. Then it runs the loss and adjoint
 * of loss+gradient requests and completes the tickets. With max_slots > 1
 * loss+gradient requests run instead on a second lane (its own thread,
 * internal context and lower-priority stream, FIFO, one at a time) that
 * overlaps the forward lane on the GPU, so forward requests do not wait for
 * adjoints; forward requests then record no eyebox-ray list. max_slots = 1
 * serves every request FIFO, one design per launch. Designs stay resident
 * on the device; the caller must not change or destroy a design while a
 * request that uses it is pending.
 * ------------------------------------------------------------------------ */
typedef uint64_t wg_ticket;
#define WG_REQ_FORWARD 0    /* forward trace: tally and statistics */
#define WG_REQ_LOSS_GRAD 1  /* forward + loss (Eq. 1) + adjoint: loss terms and thickness gradient */

typedef struct wg_request {
  int32_t kind;             /* WG_REQ_* */
  int32_t loss_kind;        /* LOSS_GRAD: 0 = coefficient of variation (the paper's), 1 = variance */
  double w_f, w_e;          /* LOSS_GRAD: weights of U_FoV and U_eyebox */
  const wg_design* design;
  wg_trace_cfg cfg;         /* copied with its arrays; stream, ray_records are ignored */
  double* tally;            /* NULL or host/device [tally size]: the forward tally */
  double* grad_thickness;   /* LOSS_GRAD: NULL or host/device [sum of layers] */
  double* loss;             /* LOSS_GRAD: NULL or host [4]: L, I_mean, U_FoV, U_eyebox */
} wg_request;

typedef struct wg_result {
  wg_status status;         /* of the evaluation: WG_OK, WG_ECANCELED or its error */
  int32_t batch_size;       /* requests in the batch that served it */
  int32_t graph_replayed;   /* 1 if the batch's forward replayed a captured CUDA graph */
  int32_t pad;
  double queue_ms;          /* submit -> start of its batch (host clock) */
  double run_ms;            /* start of its batch -> completion */
  wg_stats stats;           /* forward statistics of this request (kernel_ms: its fused launches) */
} wg_result;

/* WG_EINVAL (bad request), WG_ENOMEM (needs more device memory than the
 * budget: can never be admitted), WG_EBUSY (queue full: 4096 pending). The
 * output buffers must stay valid until the ticket is done. */
wg_status wg_submit(wg_ctx* ctx, const wg_request* req, wg_ticket* ticket);
/* Waits up to timeout_us (0: no wait, < 0: forever) for the ticket. WG_OK:
 * done, *out filled and the ticket released; WG_ENOTREADY: still pending;
 * WG_ENOTFOUND: unknown or already released ticket. */
wg_status wg_poll(wg_ctx* ctx, wg_ticket ticket, int64_t timeout_us, wg_result* out);
/* A queued request is dropped; a running one completes with its outputs
 * unspecified. Its wg_poll then reports status WG_ECANCELED. */
wg_status wg_cancel(wg_ctx* ctx, wg_ticket ticket);
/* Times the forward kernel's chunk size and CTAs per SM on (a bounded sample
 * of) this evaluation and stores the fastest for its class (fields per ray,
 * material period, accuracy mode, layers per mirror, rays per cell) in the
 * context's table, and in wg_init_opts.autotune_cache when given. The
 * scheduler tunes classes it has not seen on their first batch. */
wg_status wg_autotune(wg_ctx* ctx, const wg_design* d, const wg_trace_cfg* cfg);
/* Forward traces of n designs (the batching workload: many designs of
 * uneven mirror and layer counts and ray budgets) in one fused persistent
 * launch per kernel variant (fields per ray, material period, accuracy mode;
 * each design on its own CTAs, a design whose chunks run out hands its SMs
 * to the others), with the autotuned launch shape of each design's class; a
 * composition met before replays its captured CUDA graph. cfgs[i] and
 * tallies[i] (device FP64 in cfgs[i]'s tally layout, overwritten) belong to
 * designs[i]; stats: NULL or host [n]. Runs on the context's serving stream
 * and returns when done (cfgs[i].stream is ignored). graph_replayed: NULL or
 * host, set to 1 when the launches were a graph replay. Errors: WG_EINVAL,
 * WG_ENOMEM, WG_EDEVICE, WG_ETIMEOUT (then the stats tell which design). */
wg_status wg_trace_forward_batch(wg_ctx* ctx, int32_t n, const wg_design* const* designs, const wg_trace_cfg* cfgs,
                                 double* const* tallies, wg_stats* stats, int32_t* graph_replayed);
/* The table's entry for the class of (d, cfg): the launch shape the runtime
 * uses for it and, when this context timed it (wg_autotune or a first
 * batch), every candidate it timed. An entry read from the cache file has
 * n_tried = 0. Errors: WG_EINVAL, WG_ENOTFOUND (no entry for the class). */
#define WG_TUNE_MAX_TRIED 8
typedef struct wg_tune_info {
  int32_t chunk_rays;    /* rays per chunk of the forward kernel */
  int32_t ctas_per_sm;   /* CTAs per SM (0: the occupancy limit) */
  float best_ms;         /* the chosen shape's time on the sample (0: from the cache file) */
  int32_t n_tried;       /* candidates timed */
  int32_t tried_chunk_rays[WG_TUNE_MAX_TRIED];
  int32_t tried_ctas_per_sm[WG_TUNE_MAX_TRIED];
  float tried_ms[WG_TUNE_MAX_TRIED];
} wg_tune_info;
wg_status wg_autotune_info(wg_ctx* ctx, const wg_design* d, const wg_trace_cfg* cfg, wg_tune_info* out);

/* ------------------------------------------------------------------------
 * Reflection-probability pre-optimization (Methods, "Learned reflection
 * probabilities"): before the thicknesses are optimized, each mirror's
 * omega is chosen to bring throughput to the pupils, with each coating
 * idealized as a scalar reflectance (here equal to its omega, so every
 * sampled path has weight one) and geometric tracing without polarization.
 * ------------------------------------------------------------------------ */
/* The model's trace of cfg's rays: tally (host or device FP64, tally layout,
 * overwritten) gets each eyebox ray's unpolarized exit transmittance
 * (T_s + T_p) / 2; with dL_dtally (host or device, may be NULL)
 * grad_omega (host or device FP64 [n_mirrors], may be NULL, overwritten)
 * gets dL/d omega, the score-function estimator: the sum over tallied rays of
 * dL/dtally[bin] I (n_r,k / omega_k - n_t,k / (1 - omega_k)). Same Philox
 * decisions as wg_trace_forward. Errors: WG_EINVAL, WG_ENOMEM, WG_EDEVICE. */
wg_status wg_omega_trace(wg_ctx* ctx, const wg_design* d, const wg_trace_cfg* cfg, const double* dL_dtally,
                         double* tally, double* grad_omega);
/* Replaces the mirrors' reflection probabilities ([n_mirrors], host, each in
 * (0, 1)); the sampled paths change, so an earlier eyebox-ray list no longer
 * applies. Returns once the device copy is done. Errors: WG_EINVAL. */
wg_status wg_set_omega(wg_design* d, const float* omega, int32_t n, void* stream);

/* Optimizer of the reflection probabilities (the pre-optimization's update):
 * Adam on the n_mirrors values of omega with the gradient of a loss to
 * minimize (wg_omega_trace's grad_omega of L = -I_mean maximizes the mean
 * pupil throughput), each value then clipped to [lo, hi]. The paper names no
 * optimizer for this step. */
typedef struct wg_omega_adam_opts {
  float lr;        /* step size (0 = 0.02) */
  float beta1;     /* (0 = 0.9) */
  float beta2;     /* (0 = 0.999) */
  float eps;       /* (0 = 1e-8) */
  float lo, hi;    /* clip range, 0 < lo < hi < 1 (both 0: [0.02, 0.98]) */
} wg_omega_adam_opts;
typedef struct wg_omega_adam wg_omega_adam;
/* State (FP64 values and moments on the design's device) starting from the
 * design's current omega. NULL opts: the defaults. Errors: WG_EINVAL, WG_ENOMEM. */
wg_status wg_omega_adam_create(wg_design* d, const wg_omega_adam_opts* opts, wg_omega_adam** out);
/* One step with dL/d omega ([n_mirrors] FP64, host or device); the clipped
 * values go to the design (as wg_set_omega; returns once they are there).
 * omega_out: NULL or host FP32 [n_mirrors], the new values. Non-finite
 * gradient entries leave their mirror unchanged. Errors: WG_EINVAL, WG_EDEVICE. */
wg_status wg_omega_adam_step(wg_omega_adam* a, const double* grad_omega, float* omega_out, void* stream);
void wg_omega_adam_destroy(wg_omega_adam* a);

/* A counter that every change of the design's parameters (wg_set_params,
 * wg_set_omega, the optimizers' steps) increases: a caller that pairs a
 * forward trace with a later backward can check that both saw the same
 * parameters. Errors: WG_EINVAL. */
wg_status wg_design_version(const wg_design* d, uint64_t* version);

/* Failure-path test hook (no counterpart in the paper): one device thread
 * waits for a flag that nothing sets, with the bounded wait the trace kernels
 * use (device clock); after limit_ns (0 < limit_ns <= 1e9) it gives up, sets
 * the error word and returns, and the call returns WG_ETIMEOUT with the
 * context still usable. It allocates and frees 8 bytes of device memory and
 * synchronizes the context's stream. Errors: WG_EINVAL, WG_EDEVICE. */
wg_status wg_test_bounded_wait(wg_ctx* ctx, uint64_t limit_ns);

/* ------------------------------------------------------------------------
 * Optimizer of the layer thicknesses (Results, "Evaluation": all PRMA
 * thicknesses optimized jointly within 20-200 nm; a soft gap between 0 and
 * 20 nm lets layers be eliminated, which prunes an over-parameterized stack).
 * The paper does not name its optimizer: this is Adam on the thicknesses in
 * nm, followed by a projection: clamp to [0, d_max]; a value inside the gap
 * (0, d_min) goes to 0 below d_min / 2, else to d_min. A layer at zero
 * thickness stays in its stack as an identity layer (its gradient keeps
 * flowing); layers the design prunes are never updated. One optimization
 * step is wg_trace_forward, wg_loss, wg_trace_backward, wg_adam_step.
 * ------------------------------------------------------------------------ */
typedef struct wg_adam_opts {
  float lr_nm;     /* step size in nm (0 = 2) */
  float beta1;     /* first-moment decay (0 = 0.9) */
  float beta2;     /* second-moment decay (0 = 0.999) */
  float eps;       /* (0 = 1e-8) */
  float d_min_nm;  /* smallest manufacturable thickness, upper end of the gap (0 = 20) */
  float d_max_nm;  /* upper bound (0 = 200) */
} wg_adam_opts;
typedef struct wg_adam wg_adam;

/* Optimizer state (FP32 thicknesses, FP64 moments, on the design's device)
 * for design d. thickness_nm: the starting thicknesses ([sum n_layers],
 * host or device; NULL: the design's as last set from the host). NULL opts:
 * the defaults. Does not change the design. Errors: WG_EINVAL, WG_ENOMEM. */
wg_status wg_adam_create(wg_design* d, const wg_adam_opts* opts, const float* thickness_nm, wg_adam** out);
/* One step with dL/dthickness ([sum n_layers] FP64, host or device, as
 * wg_trace_backward writes it); the projected thicknesses go to the design
 * (wg_set_params, stream-ordered on `stream`). Non-finite gradient entries
 * leave their layer unchanged. Errors: WG_EINVAL, WG_EDEVICE. */
wg_status wg_adam_step(wg_adam* a, const double* grad_thickness, void* stream);
/* Copies the current thicknesses ([sum n_layers] FP32, host or device). */
wg_status wg_adam_params(wg_adam* a, float* thickness_nm, void* stream);
void wg_adam_destroy(wg_adam* a);

#ifdef __cplusplus
}
#endif

#endif /* WG_H_ */
