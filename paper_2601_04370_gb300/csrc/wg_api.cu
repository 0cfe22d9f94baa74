// C ABI of libwg.so: contexts, designs, and the trace / loss / adjoint entry
// points declared in include/wg.h. Host code here validates arguments, lays
// out device buffers and launches the kernels; every step of the hot path's
// arithmetic runs in the kernels of wg_trace.cu and wg_loss.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "wg.h"
#include "wg_device.cuh"
#include "wg_host.h"
#include "wg_internal.h"

using namespace wgk;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_err;

static wg_status fail(wg_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

#define CU(call)                                                                                       \
  do {                                                                                                 \
    cudaError_t e_ = (call);                                                                           \
    if (e_ != cudaSuccess) return fail(WG_EDEVICE, "%s failed: %s", #call, cudaGetErrorString(e_));    \
  } while (0)

extern "C" const char* wg_last_error(void) { return g_err.c_str(); }
extern "C" const char* wg_version(void) { return "wg 0.1 (sm_103a)"; }
extern "C" uint64_t wg_kernel_launches(void) { return (uint64_t)launches(); }

// ---------------------------------------------------------------------------
// objects
// ---------------------------------------------------------------------------
// gen counts the reallocations: a captured CUDA graph that refers to the
// buffer must not be replayed after one, even when the new allocation lands
// at the old address (the graph's nodes still refer to the freed one)
struct DevBuf {
  void* p = nullptr;
  size_t n = 0;
  unsigned long long gen = 0;
  cudaError_t ensure(size_t bytes) {
    if (bytes <= n) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
    ++gen;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e == cudaSuccess) n = bytes;
    return e;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
};

struct wg_ctx {
  int device = 0;
  int sm_count = 0;
  std::mutex mu;
  DevBuf ws;      // small per-call workspace (counters, cfg arrays, fields)
  DevBuf bwd;     // adjoint scratch (hit records, per-CTA rows)
  DevBuf loss;    // loss workspace
  cudaEvent_t ws_free = nullptr;  // last use of the workspaces
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  cudaEvent_t kev[6] = {};  // backward with stats: around the replay, adjoint and tilt launches
  int max_slots = 64;
  size_t hbm_budget = 0;
  std::string autotune_cache;
  std::vector<wg_design*> designs;
  DevBuf fws;     // fused-forward workspace (per-job heads, configuration arrays, job table)
  DevBuf lut;     // coating look-up table of the last call that asked for one
  DevBuf lsort;   // the eyebox-ray list grouped by hit count, for the replay
  void* serve = nullptr;  // serving runtime state (wg_serve.cu)
  void* noalloc_scratch = nullptr;  // device address of the no-allocation trace's static array
  unsigned long long wait_limit_ns = 0;  // bounded waits in the kernels (0: the default 0.5 s)
  int max_queue = 4096;                  // serving queue length
  // serving: rays one batch admits beyond its first request (every request
  // of a batch completes when the batch does, so a bounded batch keeps
  // latency short)
  long long max_batch_rays = 1ll << 25;
};

struct wg_design {
  wg_ctx* ctx = nullptr;
  int dims = 3, n_mat = 0, K = 0, n_orig = 0, n_dev = 0;
  float n_slab = 0, thick = 0, width = 0, x_end = 0, eye_relief = 0, ic_tilt = 0;
  std::vector<float> mat_n, mir_x, mir_tilt, omega, layer_d;
  std::vector<int> n_layers, layer_mat, orig_to_store, dev_to_orig;
  std::vector<uint8_t> pruned;
  uint8_t* blob = nullptr;
  int blob_bytes = 0;
  float* d_mir = nullptr;      // [3][K]: x, tilt, omega
  std::vector<float> geo;      // general mirrors: [K][14] as in the descriptor; empty: PRMA
  float* d_geo = nullptr;      // device copy of geo, or NULL
  int* d_orig_to_store = nullptr;  // original layer -> index in the blob's padded layer arrays (-1 pruned)
  int* d_dev_to_orig = nullptr;
  float* d_stage = nullptr;    // [n_orig] thickness staging for set_params
  int period = 0;              // material period shared by all stacks (0, 2 or 3)
  bool acc = false;            // accurate layer evaluation (a stack longer than kAccLayers)
  int geom_version = 0;        // bumped whenever the mirror geometry (tilts) changes
  // eyebox rays of the last listing forward trace: count (u64) | ExitRec[],
  // valid for the configuration and geometry with fingerprint exit_fp (0: none)
  DevBuf exits;
  uint64_t exit_fp = 0;
  long long exit_cap = 0;  // entries of the list (rays + hole allowance)
  // applied coefficients of the first coef_slots hits of every ray of the
  // last listing forward (TraceArgs::coef), valid for the paths with
  // fingerprint coef_fp, the thicknesses of version coef_thick and the
  // coating table size coef_lut
  DevBuf coefs;
  uint64_t coef_fp = 0;
  int coef_thick = -1, coef_lut = 0, coef_slots = 0;
  long long coef_base = 0, coef_rays = 0;
  int thick_version = 0;  // bumped whenever the thicknesses change
  uint64_t param_version = 0;  // bumped by every parameter change (wg_design_version)
};

// hits per ray whose coefficients the listing forward keeps for the replay:
// 8 (a PRMA ray meets ~4 mirrors), 32 for designs of more than 8 mirrors,
// fewer when the store would pass 8 GB
static int coef_slots_for(int n_mirrors, long long rays) {
  const int want = n_mirrors > 8 ? 32 : 8;
  const long long fit = (8ll << 30) / (16ll * std::max(1ll, rays));
  return (int)std::min<long long>(want, fit);
}

// instantiation of the trace kernels: 0 for the PRMA's slab planes, 1 for
// general mirrors (the plane-family search compiled inline)
static int geo_mode(const wg_design* d) { return d->geo.empty() ? 0 : 1; }

static size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

static bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// ---------------------------------------------------------------------------
// Scratch of the allocation-free forward trace (wg_trace_forward_noalloc),
// for callers that cannot allocate device memory: the per-call scratch lives
// in this static device array instead of the context's workspace. Host code
// must not pass the array's name to a kernel (on the host it is only a
// stand-in); wg_init looks up its device address with the context's device
// current and keeps it in the context.
// ---------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_noalloc_scratch[WG_NOALLOC_SCRATCH_BYTES];

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
extern "C" wg_status wg_init(wg_ctx** out, const wg_init_opts* opts) {
  if (!out) return fail(WG_EINVAL, "wg_init: out is NULL");
  *out = nullptr;
  int dev = opts ? opts->device : 0;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) {
    cudaGetLastError();
    return fail(WG_EDEVICE, "wg_init: no CUDA device");
  }
  if (dev < 0 || dev >= n) return fail(WG_EINVAL, "wg_init: device %d out of range [0,%d)", dev, n);
  CU(cudaSetDevice(dev));
  cudaDeviceProp prop;
  CU(cudaGetDeviceProperties(&prop, dev));
  wg_ctx* c = new wg_ctx();
  c->device = dev;
  c->sm_count = prop.multiProcessorCount;
  if (opts && opts->max_slots > 0) c->max_slots = opts->max_slots;
  if (opts) c->hbm_budget = opts->hbm_budget_bytes;
  if (opts && opts->autotune_cache) c->autotune_cache = opts->autotune_cache;
  if (opts) c->wait_limit_ns = opts->wait_limit_ns;
  if (opts && opts->max_queue > 0) c->max_queue = opts->max_queue;
  if (opts && opts->max_batch_rays > 0) c->max_batch_rays = opts->max_batch_rays;
  // the allocation-free trace's array: looking up its address places it on
  // this device now, and loading the forward kernels now keeps a first
  // wg_trace_forward_noalloc call from loading (allocating) anything
  {
    const cudaError_t e = cudaGetSymbolAddress(&c->noalloc_scratch, g_noalloc_scratch);
    if (e != cudaSuccess || !c->noalloc_scratch) {
      delete c;
      return fail(WG_EDEVICE, "wg_init: cudaGetSymbolAddress of the no-allocation scratch failed: %s",
                  cudaGetErrorString(e));
    }
    const cudaError_t e2 = preload_forward_kernels();
    if (e2 != cudaSuccess) {
      delete c;
      return fail(WG_EDEVICE, "wg_init: loading the forward kernels failed: %s", cudaGetErrorString(e2));
    }
  }
  if (cudaEventCreateWithFlags(&c->ws_free, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreate(&c->t0) != cudaSuccess || cudaEventCreate(&c->t1) != cudaSuccess ||
      cudaEventCreate(&c->kev[0]) != cudaSuccess || cudaEventCreate(&c->kev[1]) != cudaSuccess ||
      cudaEventCreate(&c->kev[2]) != cudaSuccess || cudaEventCreate(&c->kev[3]) != cudaSuccess ||
      cudaEventCreate(&c->kev[4]) != cudaSuccess || cudaEventCreate(&c->kev[5]) != cudaSuccess) {
    delete c;
    return fail(WG_EDEVICE, "wg_init: event creation failed");
  }
  *out = c;
  return WG_OK;
}

static void destroy_design_dev(wg_design* d) {
  if (d->blob) cudaFree(d->blob);
  if (d->d_mir) cudaFree(d->d_mir);
  if (d->d_geo) cudaFree(d->d_geo);
  if (d->d_orig_to_store) cudaFree(d->d_orig_to_store);
  if (d->d_dev_to_orig) cudaFree(d->d_dev_to_orig);
  if (d->d_stage) cudaFree(d->d_stage);
  d->exits.release();
  d->exit_fp = 0;
  d->coefs.release();
  d->coef_fp = 0;
  d->blob = nullptr;
}

extern "C" void wg_shutdown(wg_ctx* c) {
  if (!c) return;
  wgh::serve_shutdown(c);  // stops the scheduler thread first: it uses the context
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  for (wg_design* d : c->designs) {
    destroy_design_dev(d);
    delete d;
  }
  c->ws.release();
  c->bwd.release();
  c->loss.release();
  c->fws.release();
  if (c->ws_free) cudaEventDestroy(c->ws_free);
  if (c->t0) cudaEventDestroy(c->t0);
  if (c->t1) cudaEventDestroy(c->t1);
  for (cudaEvent_t e : c->kev)
    if (e) cudaEventDestroy(e);
  delete c;
}

// ---------------------------------------------------------------------------
// designs
// ---------------------------------------------------------------------------
static wg_status validate_desc(const wg_design_desc* s) {
  if (!s) return fail(WG_EINVAL, "design: desc is NULL");
  if (s->dims != 2 && s->dims != 3) return fail(WG_EINVAL, "design: dims must be 2 or 3 (got %d)", s->dims);
  if (s->n_materials < 1 || s->n_materials > WG_MAX_MATERIALS)
    return fail(WG_EINVAL, "design: n_materials must be in [1,%d]", WG_MAX_MATERIALS);
  if (s->n_mirrors < 1 || s->n_mirrors > WG_MAX_MIRRORS)
    return fail(WG_EINVAL, "design: n_mirrors must be in [1,%d]", WG_MAX_MIRRORS);
  if (!s->material_n || !s->mirror_x_mm || !s->mirror_tilt_deg || !s->mirror_omega || !s->n_layers ||
      !s->layer_material || !s->layer_thickness_nm)
    return fail(WG_EINVAL, "design: NULL array");
  if (!(s->n_slab > 1.0f) || !(s->thickness_mm > 0.0f) || !(s->eye_relief_mm > 0.0f) || !(s->width_mm > 0.0f))
    return fail(WG_EINVAL, "design: n_slab > 1, thickness, width and eye relief > 0 required");
  if (!(s->ic_tilt_deg > 0.0f && s->ic_tilt_deg < 90.0f)) return fail(WG_EINVAL, "design: ic_tilt_deg in (0,90)");
  for (int i = 0; i < s->n_materials; ++i)
    if (!(s->material_n[i] >= 1.0f) || !std::isfinite(s->material_n[i]))
      return fail(WG_EINVAL, "design: material %d index must be finite and >= 1", i);
  long long total = 0;
  for (int k = 0; k < s->n_mirrors; ++k) {
    if (s->n_layers[k] < 0 || s->n_layers[k] > MAX_LAYERS_MIRROR)
      return fail(WG_EINVAL, "design: mirror %d layer count must be in [0,%d]", k, MAX_LAYERS_MIRROR);
    if (!(s->mirror_omega[k] > 0.0f && s->mirror_omega[k] < 1.0f))
      return fail(WG_EINVAL, "design: mirror %d omega must be in (0,1)", k);
    if (!std::isfinite(s->mirror_x_mm[k]) || !std::isfinite(s->mirror_tilt_deg[k]) ||
        !(std::fabs(s->mirror_tilt_deg[k]) < 89.0f))
      return fail(WG_EINVAL, "design: mirror %d position/tilt invalid", k);
    if (s->mirror_geometry) {
      const float* g = s->mirror_geometry + 14 * k;
      for (int i = 0; i < 14; ++i)
        if (!std::isfinite(g[i]) && (i < 9 || i == 13))
          return fail(WG_EINVAL, "design: mirror %d geometry value %d not finite", k, i);
      const double nn = (double)g[0] * g[0] + (double)g[1] * g[1] + (double)g[2] * g[2];
      const double aa = (double)g[6] * g[6] + (double)g[7] * g[7] + (double)g[8] * g[8];
      const double an = (double)g[0] * g[6] + (double)g[1] * g[7] + (double)g[2] * g[8];
      if (std::fabs(nn - 1.0) > 1e-4 || std::fabs(aa - 1.0) > 1e-4 || std::fabs(an) > 1e-4)
        return fail(WG_EINVAL, "design: mirror %d normal and tilt axis must be unit and perpendicular", k);
      if (!(g[9] <= g[10]) || !(g[11] <= g[12]))
        return fail(WG_EINVAL, "design: mirror %d rectangle must have x0 <= x1 and y0 <= y1", k);
    }
    total += s->n_layers[k];
  }
  for (long long i = 0; i < total; ++i) {
    if (s->layer_material[i] < 0 || s->layer_material[i] >= s->n_materials)
      return fail(WG_EINVAL, "design: layer %lld material out of range", i);
    const float d = s->layer_thickness_nm[i];
    if (!std::isfinite(d) || d < 0.0f) return fail(WG_EINVAL, "design: layer %lld thickness must be finite and >= 0", i);
  }
  return WG_OK;
}

// host layout of the blob; geometry-derived fields are filled by k_prep_design
static std::vector<uint8_t> build_blob(const wg_design& d) {
  const size_t off_mir = sizeof(BlobHeader);
  // general designs: the plane-family table follows the mirror records
  const size_t fam_bytes = d.geo.empty() ? 0 : sizeof(FamRec) * d.K;
  // layer arrays: kStackPad zero-thickness layers (material 0) before each
  // stack and after the last
  const size_t n_store = (size_t)d.n_dev + (size_t)kStackPad * (d.K + 1);
  const size_t off_d = align16(off_mir + sizeof(MirrorRec) * d.K + fam_bytes);
  const size_t off_m = align16(off_d + sizeof(float) * n_store);
  const size_t bytes = align16(off_m + n_store + 1);
  std::vector<uint8_t> b(bytes, 0);
  BlobHeader h;
  memset(&h, 0, sizeof(h));
  h.dims = d.dims;
  h.n_mat = d.n_mat;
  h.n_mir = d.K;
  h.n_layers = d.n_dev;
  h.n_slab = d.n_slab;
  h.thick = d.thick;
  h.half_w = 0.5f * d.width;
  h.x_end = d.x_end;
  h.eye_relief = d.eye_relief;
  for (int i = 0; i < d.n_mat; ++i) {
    h.mat_n[i] = d.mat_n[i];
    h.mat_inv_n[i] = (float)(1.0 / (double)d.mat_n[i]);
    const double r = (double)d.n_slab / (double)d.mat_n[i];
    h.mat_r2[i] = (float)(r * r);
    h.mat_r2_lo[i] = (float)(r * r - (double)h.mat_r2[i]);
  }
  h.off_mir = (int)off_mir;
  h.off_d = (int)off_d;
  h.off_m = (int)off_m;
  h.bytes = (int)bytes;
  memcpy(b.data(), &h, sizeof(h));
  MirrorRec* mir = reinterpret_cast<MirrorRec*>(b.data() + off_mir);
  float* dd = reinterpret_cast<float*>(b.data() + off_d);
  uint8_t* mm = b.data() + off_m;
  int orig = 0, dev = 0;
  for (int k = 0; k < d.K; ++k) {
    MirrorRec r;
    memset(&r, 0, sizeof(r));
    r.layer_off = dev;
    r.store_off = dev + kStackPad * (k + 1);
    for (int l = 0; l < d.n_layers[k]; ++l, ++orig) {
      if (d.pruned[orig]) continue;
      dd[dev + kStackPad * (k + 1)] = d.layer_d[orig];
      mm[dev + kStackPad * (k + 1)] = (uint8_t)d.layer_mat[orig];
      ++dev;
    }
    r.n_layers = dev - r.layer_off;
    mir[k] = r;
  }
  return b;
}

// Smallest P in {2, 3} such that every mirror's (non-pruned) layer i has the
// material of its layer i mod P; 0 if there is none. The kernels unroll the
// layer loop by P with the material constants of each slot in registers.
static int design_period(const wg_design& d) {
  for (int P : {2, 3}) {
    bool ok = true;
    int orig = 0;
    for (int k = 0; k < d.K && ok; ++k) {
      std::vector<int> m;
      for (int l = 0; l < d.n_layers[k]; ++l, ++orig)
        if (!d.pruned[orig]) m.push_back(d.layer_mat[orig]);
      for (size_t i = 0; i < m.size() && ok; ++i) ok = m[i] == m[i % P];
    }
    if (ok) return P;
  }
  return 0;
}

// the accurate layer evaluation for designs with a stack of more than
// kAccLayers (non-pruned) layers
static bool design_acc(const wg_design& d) {
  int orig = 0;
  for (int k = 0; k < d.K; ++k) {
    int n = 0;
    for (int l = 0; l < d.n_layers[k]; ++l, ++orig) n += d.pruned[orig] ? 0 : 1;
    if (n > kAccLayers) return true;
  }
  return false;
}

static wg_status upload_design(wg_design* d, cudaStream_t s) {
  d->period = design_period(*d);
  d->acc = design_acc(*d);
  std::vector<uint8_t> b = build_blob(*d);
  d->blob_bytes = (int)b.size();
  CU(cudaMalloc(&d->blob, b.size()));
  CU(cudaMemcpyAsync(d->blob, b.data(), b.size(), cudaMemcpyHostToDevice, s));
  CU(cudaMalloc(&d->d_mir, sizeof(float) * 3 * d->K));
  std::vector<float> m(3 * d->K);
  for (int k = 0; k < d->K; ++k) {
    m[k] = d->mir_x[k];
    m[d->K + k] = d->mir_tilt[k];
    m[2 * d->K + k] = d->omega[k];
  }
  CU(cudaMemcpyAsync(d->d_mir, m.data(), sizeof(float) * m.size(), cudaMemcpyHostToDevice, s));
  if (!d->geo.empty()) {
    CU(cudaMalloc(&d->d_geo, sizeof(float) * d->geo.size()));
    CU(cudaMemcpyAsync(d->d_geo, d->geo.data(), sizeof(float) * d->geo.size(), cudaMemcpyHostToDevice, s));
  }
  CU(cudaMalloc(&d->d_orig_to_store, sizeof(int) * std::max(1, d->n_orig)));
  CU(cudaMalloc(&d->d_dev_to_orig, sizeof(int) * std::max(1, d->n_dev)));
  CU(cudaMalloc(&d->d_stage, sizeof(float) * std::max(1, d->n_orig)));
  if (d->n_orig)
    CU(cudaMemcpyAsync(d->d_orig_to_store, d->orig_to_store.data(), sizeof(int) * d->n_orig, cudaMemcpyHostToDevice,
                       s));
  if (d->n_dev)
    CU(cudaMemcpyAsync(d->d_dev_to_orig, d->dev_to_orig.data(), sizeof(int) * d->n_dev, cudaMemcpyHostToDevice, s));
  CU(launch_prep_design(d->blob, d->d_mir, d->d_mir + d->K, d->d_mir + 2 * d->K, d->d_geo, d->K, d->ic_tilt, d->thick, s));
  CU(cudaStreamSynchronize(s));
  return WG_OK;
}

extern "C" wg_status wg_create_design(wg_ctx* c, const wg_design_desc* s, wg_design** out) {
  if (!c || !out) return fail(WG_EINVAL, "wg_create_design: NULL ctx/out");
  *out = nullptr;
  wg_status st = validate_desc(s);
  if (st != WG_OK) return st;
  std::lock_guard<std::mutex> lk(c->mu);
  CU(cudaSetDevice(c->device));
  wg_design* d = new wg_design();
  d->ctx = c;
  d->dims = s->dims;
  d->n_mat = s->n_materials;
  d->K = s->n_mirrors;
  d->n_slab = s->n_slab;
  d->thick = s->thickness_mm;
  d->width = s->width_mm;
  d->x_end = s->x_end_mm;
  d->eye_relief = s->eye_relief_mm;
  d->ic_tilt = s->ic_tilt_deg;
  d->mat_n.assign(s->material_n, s->material_n + d->n_mat);
  d->mir_x.assign(s->mirror_x_mm, s->mirror_x_mm + d->K);
  d->mir_tilt.assign(s->mirror_tilt_deg, s->mirror_tilt_deg + d->K);
  d->omega.assign(s->mirror_omega, s->mirror_omega + d->K);
  if (s->mirror_geometry) d->geo.assign(s->mirror_geometry, s->mirror_geometry + 14 * (size_t)d->K);
  d->n_layers.assign(s->n_layers, s->n_layers + d->K);
  int total = 0;
  for (int k = 0; k < d->K; ++k) total += d->n_layers[k];
  d->n_orig = total;
  d->layer_mat.assign(s->layer_material, s->layer_material + total);
  d->layer_d.assign(s->layer_thickness_nm, s->layer_thickness_nm + total);
  d->pruned.assign(total, 0);
  if (s->layer_pruned)
    for (int i = 0; i < total; ++i) d->pruned[i] = s->layer_pruned[i] ? 1 : 0;
  // device layers: the non-pruned ones in order; mirror k's stack sits in the
  // blob's layer arrays after k + 1 pads of kStackPad
  d->orig_to_store.assign(total, -1);
  for (int k = 0, i = 0; k < d->K; ++k) {
    for (int l = 0; l < d->n_layers[k]; ++l, ++i) {
      if (d->pruned[i]) {
        d->layer_d[i] = 0.0f;
        continue;
      }
      d->orig_to_store[i] = (int)d->dev_to_orig.size() + kStackPad * (k + 1);
      d->dev_to_orig.push_back(i);
    }
  }
  d->n_dev = (int)d->dev_to_orig.size();
  st = upload_design(d, 0);
  if (st != WG_OK) {
    destroy_design_dev(d);
    delete d;
    return st;
  }
  c->designs.push_back(d);
  *out = d;
  return WG_OK;
}

extern "C" void wg_destroy_design(wg_design* d) {
  if (!d) return;
  wg_ctx* c = d->ctx;
  std::lock_guard<std::mutex> lk(c->mu);
  cudaSetDevice(c->device);
  cudaEventSynchronize(c->ws_free);
  cudaDeviceSynchronize();
  c->designs.erase(std::remove(c->designs.begin(), c->designs.end(), d), c->designs.end());
  destroy_design_dev(d);
  delete d;
}

extern "C" wg_status wg_set_params(wg_design* d, const float* thickness_nm, int64_t n_thickness,
                                   const float* tilt_deg, int32_t n_tilt, void* stream) {
  if (!d) return fail(WG_EINVAL, "wg_set_params: NULL design");
  wg_ctx* c = d->ctx;
  cudaStream_t s = (cudaStream_t)stream;
  std::lock_guard<std::mutex> lk(c->mu);
  CU(cudaSetDevice(c->device));
  if (thickness_nm) {
    if (n_thickness != d->n_orig) return fail(WG_EINVAL, "wg_set_params: %lld thicknesses for %d layers",
                                              (long long)n_thickness, d->n_orig);
    if (is_device_ptr(thickness_nm)) {
      CU(cudaMemcpyAsync(d->d_stage, thickness_nm, sizeof(float) * d->n_orig, cudaMemcpyDeviceToDevice, s));
    } else {
      for (int i = 0; i < d->n_orig; ++i)
        if (!std::isfinite(thickness_nm[i]) || thickness_nm[i] < 0.0f)
          return fail(WG_EINVAL, "wg_set_params: thickness %d invalid", i);
      for (int i = 0; i < d->n_orig; ++i) d->layer_d[i] = d->pruned[i] ? 0.0f : thickness_nm[i];
      CU(cudaMemcpyAsync(d->d_stage, thickness_nm, sizeof(float) * d->n_orig, cudaMemcpyHostToDevice, s));
    }
    CU(launch_thickness_update(d->blob, d->d_stage, d->d_orig_to_store, d->n_orig, s));
    ++d->thick_version;  // the coefficients kept by the last listing forward are stale
    ++d->param_version;
  }
  if (tilt_deg) {
    if (n_tilt != d->K) return fail(WG_EINVAL, "wg_set_params: %d tilts for %d mirrors", n_tilt, d->K);
    for (int k = 0; k < d->K; ++k)
      if (!std::isfinite(tilt_deg[k]) || !(std::fabs(tilt_deg[k]) < 89.0f))
        return fail(WG_EINVAL, "wg_set_params: tilt %d invalid", k);
    d->mir_tilt.assign(tilt_deg, tilt_deg + d->K);
    ++d->geom_version;  // ray paths change with the geometry: the eyebox-ray list is stale
    ++d->param_version;
    d->exit_fp = 0;
    CU(cudaMemcpyAsync(d->d_mir + d->K, tilt_deg, sizeof(float) * d->K, cudaMemcpyHostToDevice, s));
    CU(launch_prep_design(d->blob, d->d_mir, d->d_mir + d->K, d->d_mir + 2 * d->K, d->d_geo, d->K, d->ic_tilt, d->thick, s));
  }
  return WG_OK;
}

extern "C" wg_status wg_design_version(const wg_design* d, uint64_t* version) {
  if (!d || !version) return fail(WG_EINVAL, "wg_design_version: NULL design/version");
  std::lock_guard<std::mutex> lk(d->ctx->mu);
  *version = d->param_version;
  return WG_OK;
}

extern "C" wg_status wg_set_omega(wg_design* d, const float* omega, int32_t n, void* stream) {
  if (!d || !omega) return fail(WG_EINVAL, "wg_set_omega: NULL design/omega");
  if (n != d->K) return fail(WG_EINVAL, "wg_set_omega: %d values for %d mirrors", n, d->K);
  for (int k = 0; k < n; ++k)
    if (!(omega[k] > 0.0f && omega[k] < 1.0f)) return fail(WG_EINVAL, "wg_set_omega: omega %d outside (0, 1)", k);
  wg_ctx* c = d->ctx;
  cudaStream_t s = (cudaStream_t)stream;
  std::lock_guard<std::mutex> lk(c->mu);
  CU(cudaSetDevice(c->device));
  d->omega.assign(omega, omega + n);
  ++d->geom_version;  // the sampled paths change with omega: the eyebox-ray list is stale
  ++d->param_version;
  d->exit_fp = 0;
  CU(cudaMemcpyAsync(d->d_mir + 2 * d->K, omega, sizeof(float) * d->K, cudaMemcpyHostToDevice, s));
  CU(launch_prep_design(d->blob, d->d_mir, d->d_mir + d->K, d->d_mir + 2 * d->K, d->d_geo, d->K, d->ic_tilt, d->thick, s));
  CU(cudaStreamSynchronize(s));  // the caller's omega array may go once this returns
  return WG_OK;
}

// ---------------------------------------------------------------------------
// coating hooks
// ---------------------------------------------------------------------------
extern "C" wg_status wg_eval_coating(wg_ctx* c, const wg_design* d, int32_t mirror, int32_t side, int64_t n,
                                     const float* cos_theta, const float* lambda_nm, float* out_rt, void* stream) {
  if (!c || !d) return fail(WG_EINVAL, "wg_eval_coating: NULL ctx/design");
  if (mirror < 0 || mirror >= d->K || (side != 0 && side != 1) || n < 0)
    return fail(WG_EINVAL, "wg_eval_coating: bad mirror/side/n");
  if (n == 0) return WG_OK;
  if (!is_device_ptr(cos_theta) || !is_device_ptr(lambda_nm) || !is_device_ptr(out_rt))
    return fail(WG_EINVAL, "wg_eval_coating: arrays must be device memory");
  std::lock_guard<std::mutex> lk(c->mu);
  CU(cudaSetDevice(c->device));
  CU(launch_coating_eval(d->blob, d->period, d->acc, mirror, side, n, cos_theta, lambda_nm, out_rt, (cudaStream_t)stream));
  return WG_OK;
}

extern "C" wg_status wg_eval_coating_grad(wg_ctx* c, const wg_design* d, int32_t mirror, int32_t side, int64_t n,
                                          const float* cos_theta, const float* lambda_nm, const float* weights,
                                          int32_t which, float* grad, void* stream) {
  if (!c || !d) return fail(WG_EINVAL, "wg_eval_coating_grad: NULL ctx/design");
  if (mirror < 0 || mirror >= d->K || (side != 0 && side != 1) || n < 0 || (which != 0 && which != 1))
    return fail(WG_EINVAL, "wg_eval_coating_grad: bad mirror/side/which/n");
  if (n == 0) return WG_OK;
  if (!is_device_ptr(cos_theta) || !is_device_ptr(lambda_nm) || !is_device_ptr(weights) || !is_device_ptr(grad))
    return fail(WG_EINVAL, "wg_eval_coating_grad: arrays must be device memory");
  std::lock_guard<std::mutex> lk(c->mu);
  CU(cudaSetDevice(c->device));
  CU(launch_coating_grad(d->blob, d->period, d->acc, mirror, side, n, cos_theta, lambda_nm, weights, which, grad,
                          (cudaStream_t)stream));
  return WG_OK;
}

extern "C" wg_status wg_eval_coating_dcos(wg_ctx* c, const wg_design* d, int32_t mirror, int32_t side, int64_t n,
                                          const float* cos_theta, const float* lambda_nm, const float* weights,
                                          int32_t which, float* grad_cos, void* stream) {
  if (!c || !d) return fail(WG_EINVAL, "wg_eval_coating_dcos: NULL ctx/design");
  if (mirror < 0 || mirror >= d->K || (side != 0 && side != 1) || n < 0 || (which != 0 && which != 1))
    return fail(WG_EINVAL, "wg_eval_coating_dcos: bad mirror/side/which/n");
  if (n == 0) return WG_OK;
  if (!is_device_ptr(cos_theta) || !is_device_ptr(lambda_nm) || !is_device_ptr(weights) || !is_device_ptr(grad_cos))
    return fail(WG_EINVAL, "wg_eval_coating_dcos: arrays must be device memory");
  std::lock_guard<std::mutex> lk(c->mu);
  CU(cudaSetDevice(c->device));
  CU(launch_coating_dcos(d->blob, d->period, d->acc, mirror, side, n, cos_theta, lambda_nm, weights, which, grad_cos,
                         (cudaStream_t)stream));
  return WG_OK;
}

extern "C" wg_status wg_test_bounded_wait(wg_ctx* c, uint64_t limit_ns) {
  if (!c) return fail(WG_EINVAL, "wg_test_bounded_wait: NULL ctx");
  if (limit_ns == 0 || limit_ns > 1000000000ull) return fail(WG_EINVAL, "wg_test_bounded_wait: limit_ns must be in (0, 1e9]");
  std::lock_guard<std::mutex> lk(c->mu);
  CU(cudaSetDevice(c->device));
  const cudaStream_t s = 0;  // the legacy default stream of the device
  unsigned* dw = nullptr;
  CU(cudaMalloc(&dw, 2 * sizeof(unsigned)));
  unsigned h[2] = {0u, 0u};
  cudaError_t e = cudaMemsetAsync(dw, 0, 2 * sizeof(unsigned), s);
  if (e == cudaSuccess) e = launch_wait_flag(dw, dw + 1, (unsigned long long)limit_ns, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, dw, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(dw);
  if (e != cudaSuccess) return fail(WG_EDEVICE, "wg_test_bounded_wait: %s", cudaGetErrorString(e));
  if (h[1]) return fail(WG_ETIMEOUT, "a bounded device wait ran out (error word %u)", h[1]);
  return WG_OK;
}

// ---------------------------------------------------------------------------
// trace plumbing
// ---------------------------------------------------------------------------
struct Plan {
  long long n_cells, n_cell, total, rb, re, cell_lo, cell_hi, chunk_rays, chunks_per_cell, n_chunks;
  int n_f, bins, F;
  long long tally_size;
};

static wg_status validate_cfg(const wg_design* d, const wg_trace_cfg* cfg) {
  if (!cfg) return fail(WG_EINVAL, "cfg is NULL");
  if (cfg->n_lambda < 1 || cfg->n_fx < 1 || cfg->n_fy < 1 || !cfg->lambda_nm || !cfg->field_x_deg || !cfg->field_y_deg)
    return fail(WG_EINVAL, "cfg: need n_lambda, n_fx, n_fy >= 1 and their arrays");
  if ((long long)cfg->n_fx * cfg->n_fy > 65536) return fail(WG_EINVAL, "cfg: at most 65536 fields");
  if (d->dims == 2 && (cfg->n_fy != 1 || cfg->field_y_deg[0] != 0.0f || cfg->eb_ny != 1))
    return fail(WG_EINVAL, "cfg: 2D designs take one field_y of 0 and eb_ny = 1");
  if (cfg->pol < 0 || cfg->pol > 3) return fail(WG_EINVAL, "cfg: pol must be 0..3");
  if (cfg->n_lambda > 65536) return fail(WG_EINVAL, "cfg: at most 65536 wavelengths");
  if (cfg->n_rays < 1) return fail(WG_EINVAL, "cfg: n_rays must be >= 1");
  // the kernels write the per-ray records directly: a host pointer would fault
  if (cfg->ray_records && !is_device_ptr(cfg->ray_records))
    return fail(WG_EINVAL, "cfg: ray_records must be device memory");
  if (cfg->max_events < 1 || cfg->max_events > WG_MAX_EVENTS)
    return fail(WG_EINVAL, "cfg: max_events must be in [1,%d]", WG_MAX_EVENTS);
  if (cfg->eb_nx < 1 || cfg->eb_ny < 1 || (long long)cfg->eb_nx * cfg->eb_ny > 16384)
    return fail(WG_EINVAL, "cfg: eyebox bins must be >= 1 and at most 16384 per cell");
  if (!(cfg->eb_w_mm > 0.0f) || !(cfg->eb_h_mm > 0.0f)) return fail(WG_EINVAL, "cfg: eyebox size must be > 0");
  for (int i = 0; i < cfg->n_lambda; ++i)
    if (!(cfg->lambda_nm[i] > 0.0f) || !std::isfinite(cfg->lambda_nm[i]))
      return fail(WG_EINVAL, "cfg: wavelength %d invalid", i);
  for (int i = 0; i < cfg->n_fx; ++i)
    if (!(std::fabs(cfg->field_x_deg[i]) < 80.0f)) return fail(WG_EINVAL, "cfg: field_x %d invalid", i);
  for (int i = 0; i < cfg->n_fy; ++i)
    if (!(std::fabs(cfg->field_y_deg[i]) < 80.0f)) return fail(WG_EINVAL, "cfg: field_y %d invalid", i);
  if (cfg->flags & ~WG_TRACE_NO_EXIT_LIST) return fail(WG_EINVAL, "cfg: unknown flags 0x%x", cfg->flags);
  if (cfg->lut_bins != 0 && (cfg->lut_bins < 16 || cfg->lut_bins > 65536))
    return fail(WG_EINVAL, "cfg: lut_bins must be 0 or in [16, 65536]");
  return WG_OK;
}

static wg_status make_plan(const wg_design* d, const wg_trace_cfg* cfg, long long chunk_rays, Plan& p) {
  wg_status st = validate_cfg(d, cfg);
  if (st != WG_OK) return st;
  p.n_f = cfg->n_fx * cfg->n_fy;
  p.n_cells = (long long)cfg->n_lambda * p.n_f;
  p.n_cell = (cfg->n_rays + p.n_cells - 1) / p.n_cells;
  p.total = p.n_cell * p.n_cells;
  p.rb = std::max<long long>(0, cfg->ray_begin);
  p.re = cfg->ray_end > 0 ? std::min<long long>(cfg->ray_end, p.total) : p.total;
  if (p.rb >= p.re) return fail(WG_EINVAL, "cfg: empty ray range [%lld, %lld)", p.rb, p.re);
  if (p.re - p.rb >= (1ll << 32))
    return fail(WG_EINVAL, "cfg: %lld rays in one call; at most 2^32 - 1 (split the range with ray_begin/ray_end)",
                p.re - p.rb);
  p.cell_lo = p.rb / p.n_cell;
  p.cell_hi = (p.re - 1) / p.n_cell;
  p.chunk_rays = std::max<long long>(32, chunk_rays);
  p.chunks_per_cell = (p.n_cell + p.chunk_rays - 1) / p.chunk_rays;
  p.n_chunks = (p.cell_hi - p.cell_lo + 1) * p.chunks_per_cell;
  p.bins = cfg->eb_nx * cfg->eb_ny;
  p.F = cfg->pol == WG_POL_PAIR ? 2 : 1;
  p.tally_size = p.n_cells * p.bins;
  return WG_OK;
}

// workspace head: counters[10] u64 | ledger[6] f64 | work u64 | error u32 | pad -> 256 B
struct WsHead {
  unsigned long long counters[10];
  double ledger[6];
  unsigned long long work;
  unsigned int error;
  unsigned int pad[19];
};
static_assert(sizeof(WsHead) <= 256, "workspace head");

struct WsLayout {
  WsHead* head;
  float* lam;
  float* fx;
  float* fy;
  FieldRec* fields;
  size_t bytes;
};

static WsLayout ws_layout(void* base, const wg_trace_cfg* cfg, int n_f) {
  WsLayout w;
  uint8_t* b = (uint8_t*)base;
  size_t off = 0;
  w.head = (WsHead*)(b + off);
  off += 256;
  w.lam = (float*)(b + off);
  off = align16(off + sizeof(float) * cfg->n_lambda);
  w.fx = (float*)(b + off);
  off = align16(off + sizeof(float) * cfg->n_fx);
  w.fy = (float*)(b + off);
  off = align16(off + sizeof(float) * cfg->n_fy);
  w.fields = (FieldRec*)(b + off);
  off = align16(off + sizeof(FieldRec) * n_f);
  w.bytes = off;
  return w;
}

static wg_status prepare_ws(wg_ctx* c, const wg_design* d, const wg_trace_cfg* cfg, const Plan& p, cudaStream_t s,
                            WsLayout& w) {
  w = ws_layout(nullptr, cfg, p.n_f);
  CU(cudaStreamWaitEvent(s, c->ws_free, 0));
  if (w.bytes > c->ws.n) {
    CU(cudaEventSynchronize(c->ws_free));
    CU(c->ws.ensure(w.bytes + 4096));
  }
  w = ws_layout(c->ws.p, cfg, p.n_f);
  CU(cudaMemsetAsync(w.head, 0, 256, s));
  CU(cudaMemcpyAsync(w.lam, cfg->lambda_nm, sizeof(float) * cfg->n_lambda, cudaMemcpyHostToDevice, s));
  CU(cudaMemcpyAsync(w.fx, cfg->field_x_deg, sizeof(float) * cfg->n_fx, cudaMemcpyHostToDevice, s));
  CU(cudaMemcpyAsync(w.fy, cfg->field_y_deg, sizeof(float) * cfg->n_fy, cudaMemcpyHostToDevice, s));
  CU(launch_prep_fields(w.fields, w.fx, w.fy, cfg->n_fx, cfg->n_fy, d->n_slab, d->ic_tilt, d->dims, s));
  return WG_OK;
}

static TraceArgs base_args(const wg_design* d, const wg_trace_cfg* cfg, const Plan& p, const WsLayout& w) {
  TraceArgs a;
  memset(&a, 0, sizeof(a));
  a.wait_ns = d->ctx->wait_limit_ns;
  a.blob = d->blob;
  a.blob_bytes = d->blob_bytes;
  a.fields = w.fields;
  a.lambda = w.lam;
  a.n_f = p.n_f;
  a.pol = cfg->pol;
  a.max_events = cfg->max_events;
  a.bins = p.bins;
  a.n_cell = p.n_cell;
  a.ray_begin = p.rb;
  a.ray_end = p.re;
  a.cell_lo = p.cell_lo;
  a.chunk_rays = p.chunk_rays;
  a.n_slots = fwd_slots(p.chunk_rays);
  a.chunks_per_cell = p.chunks_per_cell;
  a.n_chunks = p.n_chunks;
  a.key0 = (uint32_t)cfg->seed;
  a.key1 = (uint32_t)(cfg->seed >> 32);
  a.eb_nx = cfg->eb_nx;
  a.eb_ny = cfg->eb_ny;
  a.eb_x0 = cfg->eb_cx_mm - 0.5f * cfg->eb_w_mm;
  a.eb_y0 = cfg->eb_cy_mm - 0.5f * cfg->eb_h_mm;
  a.eb_sx = (float)cfg->eb_nx / cfg->eb_w_mm;
  a.eb_sy = (float)cfg->eb_ny / cfg->eb_h_mm;
  a.pupil_y = cfg->pupil_y_mm;
  a.ledger = w.head->ledger;
  a.counters = w.head->counters;
  a.work = &w.head->work;
  a.error = &w.head->error;
  a.records = cfg->ray_records;
  a.n_layers = d->n_dev;
  return a;
}

// Fingerprint of everything a ray's path and tally bin depend on: the
// configuration's rays, keys, fields, wavelengths, eyebox and event cap, and
// the design's geometry version (not its layer thicknesses). Never 0.
static uint64_t path_fingerprint(const wg_design* d, const wg_trace_cfg* cfg, const Plan& p) {
  uint64_t h = 1469598103934665603ull;
  auto mix = [&](const void* x, size_t n) {
    const uint8_t* b = static_cast<const uint8_t*>(x);
    for (size_t i = 0; i < n; ++i) {
      h ^= b[i];
      h *= 1099511628211ull;
    }
  };
  mix(&d->geom_version, sizeof(d->geom_version));
  mix(&cfg->n_lambda, 4 * sizeof(int32_t));  // n_lambda, n_fx, n_fy, pol
  mix(cfg->lambda_nm, sizeof(float) * cfg->n_lambda);
  mix(cfg->field_x_deg, sizeof(float) * cfg->n_fx);
  mix(cfg->field_y_deg, sizeof(float) * cfg->n_fy);
  mix(&p.n_cell, sizeof(p.n_cell));
  mix(&p.rb, sizeof(p.rb));
  mix(&p.re, sizeof(p.re));
  mix(&cfg->seed, sizeof(cfg->seed));
  mix(&cfg->max_events, 3 * sizeof(int32_t));  // max_events, eb_nx, eb_ny
  mix(&cfg->pupil_y_mm, 5 * sizeof(float));    // pupil_y, eyebox centre and size
  return h | 1ull;
}

// Device list of eyebox rays for a forward trace of p (null when not recorded).
static const size_t kExitHead = 64;  // count word, padded
static wg_status prepare_exit_list(wg_design* d, const wg_trace_cfg* cfg, const Plan& p, int sm_count,
                                   cudaStream_t s, TraceArgs& a) {
  // a forward without the list leaves the design's list (and the
  // configuration and geometry it is valid for) as it is
  if (cfg->flags & WG_TRACE_NO_EXIT_LIST) return WG_OK;
  d->exit_fp = 0;
  const long long n = exit_list_cap(p.re - p.rb, sm_count);
  const size_t bytes = kExitHead + sizeof(ExitRec) * (size_t)n;
  if (bytes > ((size_t)8 << 30)) return WG_OK;  // not worth 8 GB: the backward replays every ray
  if (bytes > d->exits.n) CU(d->exits.ensure(bytes));
  CU(cudaMemsetAsync(d->exits.p, 0, sizeof(unsigned long long), s));
  a.exit_count = static_cast<unsigned long long*>(d->exits.p);
  a.exit_list = reinterpret_cast<ExitRec*>(static_cast<uint8_t*>(d->exits.p) + kExitHead);
  a.exit_cap = n;
  d->exit_cap = n;
  return WG_OK;
}

// Coating look-up table (cfg->lut_bins > 0): built on s for the design's
// current thicknesses and the call's wavelengths; bin centres cos_j = (j + 1/2) / N.
static long long lut_entries(const wg_design* d, const wg_trace_cfg* cfg) {
  return (long long)d->K * 2 * cfg->n_lambda * cfg->lut_bins;
}
static wg_status prepare_lut(wg_ctx* c, const wg_design* d, const wg_trace_cfg* cfg, const WsLayout& w, cudaStream_t s,
                             TraceArgs& a) {
  if (cfg->lut_bins <= 0) return WG_OK;
  const int N = cfg->lut_bins;
  const long long ne = lut_entries(d, cfg);
  const size_t bytes = sizeof(float4) * 4 * (size_t)ne;
  if (bytes > c->lut.n) {
    CU(cudaEventSynchronize(c->ws_free));
    CU(c->lut.ensure(bytes));
  }
  const float c0 = 0.5f / (float)N, dc = 1.0f / (float)N;
  CU(launch_lut_build(d->blob, d->period, d->acc, d->K, cfg->n_lambda, w.lam, N, c0, dc, static_cast<float4*>(c->lut.p), s));
  a.lut = static_cast<const float4*>(c->lut.p);
  a.lut_n = N;
  a.n_lam = cfg->n_lambda;
  a.lut_c0 = c0;
  a.lut_inv_dc = (float)N;
  return WG_OK;
}

static wg_status finish_stats(wg_ctx* c, const WsLayout& w, cudaStream_t s, wg_stats* stats, bool timed) {
  WsHead h;
  CU(cudaMemcpyAsync(&h, w.head, sizeof(WsHead), cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  if (h.error) return fail(WG_ETIMEOUT, "a bounded device wait ran out (error word %u)", h.error);
  if (stats) {
    stats->n_rays = (int64_t)h.counters[0];
    stats->n_hits = (int64_t)h.counters[1];
    stats->n_events = (int64_t)h.counters[2];
    stats->n_tir = (int64_t)h.counters[3];
    stats->n_layer_steps = (int64_t)h.counters[4];
    stats->overflow = (int32_t)h.counters[5];
    stats->n_tallied = (int64_t)h.counters[6];
    stats->n_adjoint_steps = (int64_t)h.counters[7];
    stats->n_nonfinite = (int64_t)h.counters[8];
    stats->replay_ms = stats->adjoint_ms = stats->tilt_ms = 0.f;
    stats->n_adjoint_launches = 0;
    for (int i = 0; i < 6; ++i) stats->ledger[i] = h.ledger[i];
    stats->kernel_ms = 0.f;
    if (timed) cudaEventElapsedTime(&stats->kernel_ms, c->t0, c->t1);
  }
  return WG_OK;
}

// rays per chunk: a cell split into equal chunks of at most 4096 rays
static long long default_chunk(const Plan& p) {
  const long long parts = (p.n_cell + 4095) / 4096;
  return (p.n_cell + parts - 1) / parts;
}

extern "C" wg_status wg_omega_trace(wg_ctx* c, const wg_design* d, const wg_trace_cfg* cfg, const double* dL_dtally,
                                    double* tally, double* grad_omega) {
  if (!c || !d || !tally) return fail(WG_EINVAL, "wg_omega_trace: NULL ctx/design/tally");
  if (cfg && (cfg->lut_bins || cfg->ray_records)) return fail(WG_EINVAL, "wg_omega_trace: no coating table or records");
  Plan p;
  wg_status st = make_plan(d, cfg, 2048, p);
  if (st != WG_OK) return st;
  cudaStream_t s = (cudaStream_t)cfg->stream;
  std::lock_guard<std::mutex> lk(c->mu);
  CU(cudaSetDevice(c->device));
  WsLayout w;
  st = prepare_ws(c, d, cfg, p, s, w);
  if (st != WG_OK) return st;
  double* t = tally;
  const bool dev_t = is_device_ptr(tally);
  if (!dev_t) CU(cudaMallocAsync((void**)&t, sizeof(double) * p.tally_size, s));
  CU(cudaMemsetAsync(t, 0, sizeof(double) * p.tally_size, s));
  const double* G = dL_dtally;
  if (G && !is_device_ptr(G)) {
    double* tmp;
    CU(cudaMallocAsync((void**)&tmp, sizeof(double) * p.tally_size, s));
    CU(cudaMemcpyAsync(tmp, dL_dtally, sizeof(double) * p.tally_size, cudaMemcpyHostToDevice, s));
    G = tmp;
  }
  double* g = grad_omega;
  const bool dev_g = grad_omega && is_device_ptr(grad_omega);
  if (grad_omega && !dev_g) CU(cudaMallocAsync((void**)&g, sizeof(double) * d->K, s));
  if (g) CU(cudaMemsetAsync(g, 0, sizeof(double) * d->K, s));
  TraceArgs a = base_args(d, cfg, p, w);
  a.tally = t;
  a.G = G;
  CU(launch_omega_trace(a, G ? g : nullptr, geo_mode(d), c->sm_count, s));
  CU(cudaEventRecord(c->ws_free, s));
  if (!dev_t) {
    CU(cudaMemcpyAsync(tally, t, sizeof(double) * p.tally_size, cudaMemcpyDeviceToHost, s));
    CU(cudaFreeAsync(t, s));
  }
  if (G && G != dL_dtally) CU(cudaFreeAsync((void*)G, s));
  if (grad_omega && !dev_g) {
    CU(cudaMemcpyAsync(grad_omega, g, sizeof(double) * d->K, cudaMemcpyDeviceToHost, s));
    CU(cudaFreeAsync(g, s));
  }
  return finish_stats(c, w, s, nullptr, false);
}

extern "C" wg_status wg_trace_forward(wg_ctx* c, const wg_design* d, const wg_trace_cfg* cfg, double* tally,
                                      wg_stats* stats) {
  if (!c || !d || !tally) return fail(WG_EINVAL, "wg_trace_forward: NULL ctx/design/tally");
  Plan p;
  wg_status st = make_plan(d, cfg, 2048, p);
  if (st != WG_OK) return st;
  p.chunk_rays = default_chunk(p);
  p.chunks_per_cell = (p.n_cell + p.chunk_rays - 1) / p.chunk_rays;
  p.n_chunks = (p.cell_hi - p.cell_lo + 1) * p.chunks_per_cell;
  const size_t smem = fwd_smem_bytes(d->blob_bytes, p.bins, p.F, fwd_slots(p.chunk_rays), d->acc);
  if (smem > 200 * 1024) return fail(WG_EINVAL, "wg_trace_forward: design + eyebox too large for shared memory");
  cudaStream_t s = (cudaStream_t)cfg->stream;
  std::lock_guard<std::mutex> lk(c->mu);
  CU(cudaSetDevice(c->device));
  WsLayout w;
  st = prepare_ws(c, d, cfg, p, s, w);
  if (st != WG_OK) return st;
  const bool dev_tally = is_device_ptr(tally);
  double* t = tally;
  if (!dev_tally) CU(cudaMallocAsync((void**)&t, sizeof(double) * p.tally_size, s));
  CU(cudaMemsetAsync(t + p.cell_lo * p.bins, 0, sizeof(double) * (p.cell_hi - p.cell_lo + 1) * p.bins, s));
  TraceArgs a = base_args(d, cfg, p, w);
  a.tally = t;
  wg_design* dm = const_cast<wg_design*>(d);  // the eyebox-ray list is a cache owned by the design
  st = prepare_exit_list(dm, cfg, p, c->sm_count, s, a);
  if (st != WG_OK) return st;
  st = prepare_lut(c, d, cfg, w, s, a);
  if (st != WG_OK) return st;
  // a listing forward keeps each hit's applied coefficients for the replay
  // (a forward without the list leaves the kept ones as they are); not with
  // the coating table, whose coefficients cost the replay two loads per hit
  if (!(cfg->flags & WG_TRACE_NO_EXIT_LIST)) dm->coef_fp = 0;
  if (a.exit_list && cfg->lut_bins <= 0) {
    const int slots = coef_slots_for(d->K, p.re - p.rb);
    if (slots > 0) {
      const size_t cb = sizeof(float4) * (size_t)slots * (size_t)(p.re - p.rb);
      if (cb > dm->coefs.n) CU(dm->coefs.ensure(cb));
      a.coef = static_cast<float4*>(dm->coefs.p);
      a.coef_base = p.rb;
      a.coef_rays = p.re - p.rb;
      a.coef_slots = slots;
      a.coef_mode = 1;
    }
  }
  const int bps = std::max(1, trace_fwd_blocks_per_sm(p.F, d->period, geo_mode(d), d->acc, smem));
  const int grid = (int)std::min<long long>(p.n_chunks, (long long)c->sm_count * bps);
  if (stats) CU(cudaEventRecord(c->t0, s));
  CU(launch_trace_fwd(a, p.F, d->period, geo_mode(d), d->acc, grid, smem, s));
  if (a.exit_list) dm->exit_fp = path_fingerprint(d, cfg, p);
  if (a.coef_mode == 1) {
    dm->coef_fp = dm->exit_fp;
    dm->coef_thick = d->thick_version;
    dm->coef_lut = cfg->lut_bins;
    dm->coef_base = p.rb;
    dm->coef_rays = p.re - p.rb;
    dm->coef_slots = a.coef_slots;
  }
  if (stats) CU(cudaEventRecord(c->t1, s));
  CU(cudaEventRecord(c->ws_free, s));
  if (!dev_tally) {
    CU(cudaMemcpyAsync(tally, t, sizeof(double) * p.tally_size, cudaMemcpyDeviceToHost, s));
    CU(cudaFreeAsync(t, s));
    CU(cudaStreamSynchronize(s));
  }
  if (stats || !dev_tally) {
    const wg_status fs = finish_stats(c, w, s, stats, stats != nullptr);
    if (fs != WG_OK) {  // an incomplete trace: its eyebox-ray list and kept coefficients do not apply
      dm->exit_fp = 0;
      dm->coef_fp = 0;
    }
    return fs;
  }
  return WG_OK;
}

// ---------------------------------------------------------------------------
// fused multi-design forward (serving runtime)
// ---------------------------------------------------------------------------
namespace wgh {

wg_status set_error(wg_status st, const char* msg) { return fail(st, "%s", msg); }
int ctx_device(const wg_ctx* c) { return c->device; }
int ctx_sm_count(const wg_ctx* c) { return c->sm_count; }
int ctx_max_slots(const wg_ctx* c) { return c->max_slots; }
int ctx_max_queue(const wg_ctx* c) { return c->max_queue; }
long long ctx_max_batch_rays(const wg_ctx* c) { return c->max_batch_rays; }
unsigned long long ctx_wait_limit(const wg_ctx* c) { return c->wait_limit_ns; }
size_t ctx_hbm_budget(const wg_ctx* c) { return c->hbm_budget; }
const char* ctx_autotune_cache(const wg_ctx* c) { return c->autotune_cache.empty() ? nullptr : c->autotune_cache.c_str(); }
void** ctx_serve_slot(wg_ctx* c) { return &c->serve; }
const void* fused_dev_base(const wg_ctx* c) { return c->fws.p; }
long long design_params(const wg_design* d) { return d->n_orig; }
wg_ctx* design_ctx(const wg_design* d) { return d->ctx; }
const float* design_thickness(const wg_design* d) { return d->layer_d.data(); }
const uint8_t* design_pruned(const wg_design* d) { return d->pruned.data(); }
const float* design_omega(const wg_design* d) { return d->omega.data(); }
void design_shape(const wg_design* d, int* K, int* n_dev, int* period, int* acc) {
  *K = d->K;
  *n_dev = d->n_dev;
  *period = d->period;
  *acc = d->acc ? 1 : 0;
}

long long tally_doubles(const wg_design* d, const wg_trace_cfg* cfg) {
  Plan p;
  if (make_plan(d, cfg, 2048, p) != WG_OK) return -1;
  return p.tally_size;
}

size_t eval_device_bytes(const wg_design* d, const wg_trace_cfg* cfg, bool backward) {
  Plan p;
  if (make_plan(d, cfg, 2048, p) != WG_OK) return 0;
  const long long rays = p.re - p.rb;
  size_t b = sizeof(double) * (size_t)p.tally_size;      // tally
  b += 64 + sizeof(ExitRec) * (size_t)exit_list_cap(rays, d->ctx->sm_count);  // eyebox-ray list (with holes)
  if (backward) {
    b += sizeof(double) * (size_t)p.tally_size;          // dL/dtally
    const long long batch = std::min<long long>(rays, 1ll << 22);
    b += 2 * (size_t)batch * 16 * hit_rec_bytes();       // hit records of one replay batch (and sorted copy)
  }
  return b;
}

// Pinned host staging of a fused launch: per-job configuration arrays, the
// job table and the CTA-to-job map (copied to the device by stream-ordered
// copies that a CUDA graph can capture), and the per-job heads read back.
struct FusedPinned {
  void* p = nullptr;
  size_t n = 0;
  unsigned long long gen = 0;  // reallocations (as DevBuf::gen)
  cudaError_t ensure(size_t bytes) {
    if (bytes <= n) return cudaSuccess;
    if (p) cudaFreeHost(p);
    p = nullptr;
    n = 0;
    ++gen;
    cudaError_t e = cudaMallocHost(&p, bytes);
    if (e == cudaSuccess) n = bytes;
    return e;
  }
  ~FusedPinned() {
    if (p) cudaFreeHost(p);
  }
};

// per-job workspace heads of a fused launch, contiguous at this stride
static const size_t kHeadStride = 256;

struct FusedBatch::Impl {
  FusedPinned pin;
  cudaEvent_t e0 = nullptr, e1 = nullptr;  // around the fused launches (recorded by graph replays too)
  size_t dev_bytes = 0;
  struct Copy {
    size_t src, dst, bytes;  // pinned offset -> device offset
  };
  std::vector<Copy> copies;
  struct Group {
    int F, P, acc, grid, first, cta0;
    size_t smem;
  };
  std::vector<Group> groups;
  std::vector<Plan> plans;
  std::vector<WsLayout> lay;
  std::vector<TraceArgs> args;
  size_t heads_pin = 0;  // pinned offset of the heads read back
  size_t tab_dev = 0, cta_dev = 0;
  int n = 0;
};

FusedBatch::FusedBatch() : impl(new Impl) {}
FusedBatch::~FusedBatch() {
  if (impl->e0) cudaEventDestroy(impl->e0);
  if (impl->e1) cudaEventDestroy(impl->e1);
  delete impl;
}

wg_status fused_prepare(wg_ctx* c, FusedJob* jobs, int n, int blocks_per_sm, FusedBatch& fb) {
  if (!c || !jobs || n < 1) return fail(WG_EINVAL, "fused forward: no jobs");
  FusedBatch::Impl& B = *fb.impl;
  B.n = n;
  B.plans.assign(n, Plan());
  B.lay.assign(n, WsLayout());
  B.args.assign(n, TraceArgs());
  B.copies.clear();
  B.groups.clear();
  std::vector<size_t> smem(n);
  for (int j = 0; j < n; ++j) {
    FusedJob& J = jobs[j];
    J.status = WG_OK;
    memset(&J.stats, 0, sizeof(J.stats));
    if (!J.design || !J.cfg || !J.tally) return fail(WG_EINVAL, "fused forward: job %d incomplete", j);
    if (J.cfg->lut_bins) return fail(WG_EINVAL, "fused forward: job %d asks for the coating table (not fused)", j);
    Plan& p = B.plans[j];
    wg_status st = make_plan(J.design, J.cfg, 2048, p);
    if (st != WG_OK) return st;
    p.chunk_rays = J.chunk_rays > 0 ? std::min<long long>(J.chunk_rays, p.n_cell) : default_chunk(p);
    p.chunks_per_cell = (p.n_cell + p.chunk_rays - 1) / p.chunk_rays;
    p.n_chunks = (p.cell_hi - p.cell_lo + 1) * p.chunks_per_cell;
    smem[j] = fwd_smem_bytes(J.design->blob_bytes, p.bins, p.F, fwd_slots(p.chunk_rays), J.design->acc);
    if (smem[j] > 200 * 1024) return fail(WG_EINVAL, "fused forward: job %d design + eyebox too large", j);
  }
  // device arena: heads (contiguous) | per-job arrays | job table | CTA map;
  // the pinned buffer mirrors the same offsets for what is copied in
  const int max_grid = c->sm_count * 2;
  // every job <= G CTAs (G <= max_grid)
  const size_t max_ctas = (size_t)n * (size_t)max_grid;
  size_t off = align16((size_t)n * kHeadStride);
  std::vector<size_t> job_off(n);
  for (int j = 0; j < n; ++j) {
    job_off[j] = off;
    off += align16(ws_layout(nullptr, jobs[j].cfg, B.plans[j].n_f).bytes - 256);
  }
  B.tab_dev = off;
  off += align16(sizeof(TraceArgs) * (size_t)n);
  B.cta_dev = off;
  off += align16(sizeof(int) * max_ctas);
  B.dev_bytes = off;
  B.heads_pin = off;  // pinned: same layout plus the heads read back at the end
  {
    std::lock_guard<std::mutex> lk(c->mu);
    CU(cudaSetDevice(c->device));
    if (off > c->fws.n) {
      CU(cudaEventSynchronize(c->ws_free));
      CU(c->fws.ensure(off + 4096));
    }
  }
  CU(B.pin.ensure(off + (size_t)kHeadStride * (size_t)n));
  if (!B.e0) CU(cudaEventCreate(&B.e0));
  if (!B.e1) CU(cudaEventCreate(&B.e1));
  uint8_t* dev = static_cast<uint8_t*>(c->fws.p);
  uint8_t* pin = static_cast<uint8_t*>(B.pin.p);
  // a design evaluated twice in one batch keeps no eyebox-ray list (one list per design)
  std::vector<int> dup(n, 0);
  for (int j = 0; j < n; ++j)
    for (int k = 0; k < n; ++k)
      if (k != j && jobs[k].design == jobs[j].design) dup[j] = 1;
  for (int j = 0; j < n; ++j) {
    FusedJob& J = jobs[j];
    const Plan& p = B.plans[j];
    WsLayout w = ws_layout(dev + job_off[j] - 256, J.cfg, p.n_f);
    w.head = reinterpret_cast<WsHead*>(dev + kHeadStride * (size_t)j);
    B.lay[j] = w;
    const size_t o_lam = (size_t)((uint8_t*)w.lam - dev), o_fx = (size_t)((uint8_t*)w.fx - dev),
                 o_fy = (size_t)((uint8_t*)w.fy - dev);
    memcpy(pin + o_lam, J.cfg->lambda_nm, sizeof(float) * J.cfg->n_lambda);
    memcpy(pin + o_fx, J.cfg->field_x_deg, sizeof(float) * J.cfg->n_fx);
    memcpy(pin + o_fy, J.cfg->field_y_deg, sizeof(float) * J.cfg->n_fy);
    B.copies.push_back({o_lam, o_lam, (size_t)((uint8_t*)w.fields - (uint8_t*)w.lam)});  // lam, fx, fy together
    TraceArgs a = base_args(J.design, J.cfg, p, w);
    a.tally = J.tally;
    a.records = nullptr;
    if (J.cfg->flags & WG_TRACE_NO_EXIT_LIST) {
      // no list: the design's list stays valid for what it was made for
    } else if (dup[j]) {
      const_cast<wg_design*>(J.design)->exit_fp = 0;
    } else {
      wg_design* dm = const_cast<wg_design*>(J.design);
      dm->exit_fp = 0;
      const long long nr = exit_list_cap(p.re - p.rb, c->sm_count);
      const size_t bytes = kExitHead + sizeof(ExitRec) * (size_t)nr;
      if (bytes <= ((size_t)8 << 30)) {
        std::lock_guard<std::mutex> lk(c->mu);
        if (bytes > dm->exits.n) CU(dm->exits.ensure(bytes));
        a.exit_count = static_cast<unsigned long long*>(dm->exits.p);
        a.exit_list = reinterpret_cast<ExitRec*>(static_cast<uint8_t*>(dm->exits.p) + kExitHead);
        a.exit_cap = nr;
        dm->exit_cap = nr;
      }
    }
    B.args[j] = a;
  }
  // groups of jobs sharing the kernel variant (fields per ray, material period, accuracy mode)
  std::vector<int> order(n);
  for (int j = 0; j < n; ++j) order[j] = j;
  auto variant = [&](int j) { return B.plans[j].F * 8 + jobs[j].design->period * 2 + (jobs[j].design->acc ? 1 : 0); };
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return variant(x) < variant(y); });
  TraceArgs* tab_h = reinterpret_cast<TraceArgs*>(pin + B.tab_dev);
  int* cta_h = reinterpret_cast<int*>(pin + B.cta_dev);
  size_t n_cta = 0;
  for (size_t g0 = 0; g0 < order.size();) {
    size_t g1 = g0;
    const int F = B.plans[order[g0]].F, P = jobs[order[g0]].design->period;
    const bool acc = jobs[order[g0]].design->acc;
    size_t sm_max = 0;
    double cost = 0.0;
    auto job_cost = [&](int j) {
      const double layers = (double)jobs[j].design->n_dev / std::max(1, jobs[j].design->K);
      return (double)(B.plans[j].re - B.plans[j].rb) * (10.0 + layers);
    };
    while (g1 < order.size() && variant(order[g1]) == variant(order[g0])) {
      sm_max = std::max(sm_max, smem[order[g1]]);
      cost += job_cost(order[g1]);
      ++g1;
    }
    int bps = std::max(1, trace_fwd_blocks_per_sm(F, P, 2, acc, sm_max));
    if (blocks_per_sm > 0) bps = std::min(bps, blocks_per_sm);
    const int G = c->sm_count * bps;
    FusedBatch::Impl::Group gr{F, P, acc ? 1 : 0, 0, (int)g0, (int)n_cta, sm_max};
    // CTAs per job: as many as the GPU holds at once (at most its chunks),
    // in an order that interleaves the jobs in proportion to their estimated
    // work. The first G CTAs to start share the GPU between the jobs; a CTA
    // exits when its job's chunks are gone, and the hardware then starts
    // pending CTAs, whichever job they belong to (one with no chunks left
    // exits at once). So a job that runs longer than estimated still gets
    // every freed SM for its tail, where a proportional split of CTAs would
    // leave it with its own share only.
    std::vector<std::pair<double, int>> seq;
    for (size_t q = g0; q < g1; ++q) {
      const int j = order[q];
      const double share = job_cost(j) / std::max(cost, 1.0);
      const long long k = std::max<long long>(1, std::min<long long>(G, B.plans[j].n_chunks));
      B.args[j].n_cta = (int)k;
      tab_h[q] = B.args[j];
      // start times ~ b / (share * G): a job's first CTAs come early in
      // proportion to its work, the rest of its G behind everyone's share
      for (long long b = 0; b < k; ++b) seq.push_back({((double)b + 0.5) / (std::max(share, 1e-6) * G), (int)q});
    }
    std::stable_sort(seq.begin(), seq.end());
    for (const auto& e : seq)
      if (n_cta < max_ctas) cta_h[n_cta++] = e.second;
    gr.grid = (int)(n_cta - (size_t)gr.cta0);
    B.groups.push_back(gr);
    g0 = g1;
  }
  B.copies.push_back({B.tab_dev, B.tab_dev, sizeof(TraceArgs) * (size_t)n});
  B.copies.push_back({B.cta_dev, B.cta_dev, sizeof(int) * n_cta});
  return WG_OK;
}

wg_status fused_enqueue(wg_ctx* c, FusedJob* jobs, FusedBatch& fb, cudaStream_t s) {
  FusedBatch::Impl& B = *fb.impl;
  uint8_t* dev = static_cast<uint8_t*>(c->fws.p);
  const uint8_t* pin = static_cast<const uint8_t*>(B.pin.p);
  std::lock_guard<std::mutex> lk(c->mu);
  CU(cudaSetDevice(c->device));
  // What this enqueues (and a captured graph of it bakes in) refers only to
  // the context's workspace and the batch's pinned staging; the jobs' tallies
  // and eyebox-ray counters are cleared by a kernel that reads them from the
  // job table copied in here, so a replay never touches a caller's buffer
  // through a stale address.
  CU(cudaMemsetAsync(dev, 0, (size_t)B.n * kHeadStride, s));
  for (const auto& cp : B.copies) CU(cudaMemcpyAsync(dev + cp.dst, pin + cp.src, cp.bytes, cudaMemcpyHostToDevice, s));
  long long max_doubles = 0;
  for (int j = 0; j < B.n; ++j) {
    const FusedJob& J = jobs[j];
    const Plan& p = B.plans[j];
    const WsLayout& w = B.lay[j];
    CU(launch_prep_fields(w.fields, w.fx, w.fy, J.cfg->n_fx, J.cfg->n_fy, J.design->n_slab, J.design->ic_tilt,
                          J.design->dims, s));
    max_doubles = std::max<long long>(max_doubles, (p.cell_hi - p.cell_lo + 1) * p.bins);
  }
  const TraceArgs* tab = reinterpret_cast<const TraceArgs*>(dev + B.tab_dev);
  const int* cta = reinterpret_cast<const int*>(dev + B.cta_dev);
  CU(launch_zero_jobs(tab, B.n, max_doubles, s));
  CU(cudaEventRecord(B.e0, s));
  for (const auto& g : B.groups)
    CU(launch_trace_fwd_fused(tab, cta + g.cta0, g.F, g.P, g.acc != 0, g.grid, g.smem, s));
  CU(cudaEventRecord(B.e1, s));
  CU(cudaMemcpyAsync(static_cast<uint8_t*>(B.pin.p) + B.heads_pin, dev, (size_t)kHeadStride * (size_t)B.n,
                     cudaMemcpyDeviceToHost, s));
  return WG_OK;
}

wg_status fused_finish(wg_ctx* c, FusedJob* jobs, FusedBatch& fb) {
  FusedBatch::Impl& B = *fb.impl;
  const uint8_t* heads = static_cast<const uint8_t*>(B.pin.p) + B.heads_pin;
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, B.e0, B.e1) != cudaSuccess) cudaGetLastError();
  for (int j = 0; j < B.n; ++j) {
    const WsHead& h = *reinterpret_cast<const WsHead*>(heads + (size_t)kHeadStride * (size_t)j);
    wg_stats& st = jobs[j].stats;
    jobs[j].status = h.error ? WG_ETIMEOUT : WG_OK;
    jobs[j].error_word = h.error;
    jobs[j].n_cta = B.args[j].n_cta;
    jobs[j].n_chunks = B.plans[j].n_chunks;
    st.n_rays = (int64_t)h.counters[0];
    st.n_hits = (int64_t)h.counters[1];
    st.n_events = (int64_t)h.counters[2];
    st.n_tir = (int64_t)h.counters[3];
    st.n_layer_steps = (int64_t)h.counters[4];
    for (int i = 0; i < 6; ++i) st.ledger[i] = h.ledger[i];
    st.kernel_ms = ms;
    if (B.args[j].exit_list)
      const_cast<wg_design*>(jobs[j].design)->exit_fp = path_fingerprint(jobs[j].design, jobs[j].cfg, B.plans[j]);
  }
  return WG_OK;
}

// Everything fused_enqueue bakes into a captured graph besides what it copies
// from the pinned buffer: device and pinned addresses, copy and memset
// extents, kernel launch shapes and the per-job preparation arguments.
uint64_t fused_signature(const wg_ctx* c, const FusedJob* jobs, const FusedBatch& fb) {
  const FusedBatch::Impl& B = *fb.impl;
  uint64_t h = 1469598103934665603ull;
  auto mix = [&](const void* x, size_t n) {
    const uint8_t* b = static_cast<const uint8_t*>(x);
    for (size_t i = 0; i < n; ++i) {
      h ^= b[i];
      h *= 1099511628211ull;
    }
  };
  auto mixv = [&](auto v) { mix(&v, sizeof(v)); };
  mixv(c->fws.p);
  mixv(c->fws.gen);
  mixv(B.pin.p);
  mixv(B.pin.gen);
  mixv(B.n);
  for (const auto& cp : B.copies) mix(&cp, sizeof(cp));
  for (const auto& g : B.groups) {
    mixv(g.F), mixv(g.P), mixv(g.acc), mixv(g.grid), mixv(g.first), mixv(g.cta0), mixv(g.smem);
  }
  for (int j = 0; j < B.n; ++j) {
    const Plan& p = B.plans[j];
    mixv(jobs[j].tally), mixv(p.cell_lo), mixv(p.cell_hi), mixv(p.bins);
    mixv(B.args[j].exit_count);
    mixv(B.lay[j].fields), mixv(jobs[j].cfg->n_fx), mixv(jobs[j].cfg->n_fy);
    mixv(jobs[j].design->n_slab), mixv(jobs[j].design->ic_tilt), mixv(jobs[j].design->dims);
  }
  return h;
}

wg_status fused_forward(wg_ctx* c, FusedJob* jobs, int n, int blocks_per_sm, cudaStream_t s) {
  FusedBatch fb;
  wg_status st = fused_prepare(c, jobs, n, blocks_per_sm, fb);
  if (st != WG_OK) return st;
  {
    std::lock_guard<std::mutex> lk(c->mu);
    CU(cudaStreamWaitEvent(s, c->ws_free, 0));
  }
  st = fused_enqueue(c, jobs, fb, s);
  if (st != WG_OK) return st;
  {
    std::lock_guard<std::mutex> lk(c->mu);
    CU(cudaEventRecord(c->ws_free, s));
  }
  CU(cudaStreamSynchronize(s));
  return fused_finish(c, jobs, fb);
}

}  // namespace wgh

// chunk layout of the ray range [rb, re) (cells touched, chunks per cell)
static void plan_range(Plan& p, long long rb, long long re) {
  p.rb = rb;
  p.re = re;
  p.cell_lo = rb / p.n_cell;
  p.cell_hi = (re - 1) / p.n_cell;
  p.chunks_per_cell = (p.n_cell + p.chunk_rays - 1) / p.chunk_rays;
  p.n_chunks = (p.cell_hi - p.cell_lo + 1) * p.chunks_per_cell;
}

// Adjoint scratch: hit records of one batch of rays (unsorted and sorted),
// per-stack counts and offsets, FP64 per-layer sums.
struct BwdScratch {
  HitRec* rec;
  HitRec* sorted;
  unsigned int* keys;   // [3][kSortKeys]: counts, offsets, cursors
  unsigned long long* hit_count;
  double* grad_acc;
  long long cap;
};

static const long long kRecordsPerRay = 16;  // record capacity per ray of a batch without the list (the list gives exact counts)
static const long long kReplayUnit = 32;     // rays per work unit of the replay kernel (32: shorter tails than 64)

extern "C" wg_status wg_trace_backward(wg_ctx* c, const wg_design* d, const wg_trace_cfg* cfg, const double* dL_dtally,
                                       double* grad_thickness, double* grad_tilt, wg_stats* stats) {
  if (!c || !d || !dL_dtally || !grad_thickness) return fail(WG_EINVAL, "wg_trace_backward: NULL argument");
  Plan p;
  wg_status st = make_plan(d, cfg, 2048, p);
  if (st != WG_OK) return st;
  p.chunk_rays = kReplayUnit;  // the replay's warps claim ranges of this many rays
  const size_t smem_r = (size_t)d->blob_bytes;
  const size_t smem_a = adj_smem_bytes(d->blob_bytes, d->n_dev, d->period);
  if (smem_a > 200 * 1024) return fail(WG_EINVAL, "wg_trace_backward: design too large for shared memory");
  cudaStream_t s = (cudaStream_t)cfg->stream;
  std::lock_guard<std::mutex> lk(c->mu);
  CU(cudaSetDevice(c->device));
  WsLayout w;
  st = prepare_ws(c, d, cfg, p, s, w);
  if (st != WG_OK) return st;
  std::vector<unsigned int> hit_end(TAPE_HITS + 1, 0u);
  // rays to replay: the eyebox rays listed by the forward trace of this
  // configuration and geometry if there is such a list, else the ray range
  bool use_list = d->exit_fp != 0 && d->exit_fp == path_fingerprint(d, cfg, p);
  long long n_list = 0;
  if (use_list) {
    unsigned long long cnt = 0;
    CU(cudaMemcpyAsync(&cnt, d->exits.p, sizeof(cnt), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    use_list = (long long)cnt <= d->exit_cap;  // more would mean the list overflowed
    n_list = (long long)cnt;
  }
  const ExitRec* list =
      use_list ? reinterpret_cast<const ExitRec*>(static_cast<const uint8_t*>(d->exits.p) + kExitHead) : nullptr;
  if (use_list && n_list > 0) {
    // rays grouped by their hit count: a replay warp then gets rays of equal length
    const size_t lb = kHitSortScratch + sizeof(ExitRec) * (size_t)n_list;
    if (lb > c->lsort.n) {
      CU(cudaEventSynchronize(c->ws_free));
      CU(c->lsort.ensure(lb));
    }
    ExitRec* sorted = reinterpret_cast<ExitRec*>(static_cast<uint8_t*>(c->lsort.p) + kHitSortScratch);
    CU(launch_exits_sort(list, n_list, static_cast<unsigned int*>(c->lsort.p), sorted, s));
    list = sorted;
    // the sort's counters end as the end offset of each hit count in the
    // sorted list: the records of any range of listed rays are known exactly
    CU(cudaMemcpyAsync(hit_end.data(), c->lsort.p, sizeof(unsigned int) * hit_end.size(), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
  }
  // batches of rays large enough to fill the GPU many times over; with the
  // list the record capacity is the largest batch's exact record count (from
  // the hit counts the list carries), so no record of a listed ray is dropped.
  // (One batch for all listed rays made the replay slower: 5.5 ms against
  // 4.3 ms at 1e7 rays.)
  const bool tilt = grad_tilt != nullptr;
  const long long total = p.re - p.rb;
  const long long dflt = std::min<long long>(total, std::max<long long>(4096ll * c->sm_count * 4, 1ll << 21));
  long long batch = dflt, cap = dflt * kRecordsPerRay;
  if (use_list && n_list > 0) {
    auto records_in = [&](long long b0, long long b1) {
      long long r = 0, start = 0;
      for (size_t h = 0; h < hit_end.size(); ++h) {
        const long long end = hit_end[h];
        const long long lo = std::max(start, b0), hi = std::min(end, b1);
        if (hi > lo) r += (long long)h * (hi - lo);
        start = end;
      }
      return r;
    };
    batch = std::min<long long>(dflt, n_list);
    cap = 1;
    for (long long b0 = 0; b0 < n_list; b0 += batch) cap = std::max(cap, records_in(b0, std::min(n_list, b0 + batch)));
  }
  // the scratch arrays follow one another: a multiple of 64 records keeps
  // every one of them (TiltAux, ray heads, permutation, sums) aligned
  cap = (cap + 63) & ~63ll;
  const size_t rec_bytes = (size_t)cap * hit_rec_bytes();
  const size_t acc_bytes = (sizeof(double) * std::max(1, d->n_dev) + 15) & ~(size_t)15;
  const size_t aux_bytes =
      tilt ? (size_t)cap * (sizeof(TiltAux) + sizeof(unsigned int)) + 2 * (size_t)batch * sizeof(RayHead) + kHitSortScratch
           : 0;
  // coating table: FP64 dL/dc per entry and the second stage's records
  const bool use_lut = cfg->lut_bins > 0;
  const long long n_lut = use_lut ? lut_entries(d, cfg) : 0;
  const size_t lut_bytes = use_lut ? (size_t)n_lut * (8 * sizeof(double) + 2 * hit_rec_bytes()) : 0;
  const size_t need = 2 * rec_bytes + 3 * kSortKeys * sizeof(unsigned int) + 64 + acc_bytes + aux_bytes + lut_bytes;
  if (need > c->bwd.n) {
    CU(cudaEventSynchronize(c->ws_free));
    CU(c->bwd.ensure(need));
  }
  uint8_t* bw = (uint8_t*)c->bwd.p;
  BwdScratch sc;
  sc.rec = (HitRec*)bw;
  sc.sorted = (HitRec*)(bw + rec_bytes);
  sc.keys = (unsigned int*)(bw + 2 * rec_bytes);
  sc.hit_count = (unsigned long long*)(bw + 2 * rec_bytes + 3 * kSortKeys * sizeof(unsigned int));
  sc.grad_acc = (double*)(bw + 2 * rec_bytes + 3 * kSortKeys * sizeof(unsigned int) + 64);
  sc.cap = cap;
  TiltAux* tilt_aux = nullptr;
  RayHead* heads = nullptr;
  unsigned int* perm = nullptr;  // sorted record -> its slot in tilt_aux
  if (tilt) {
    tilt_aux = (TiltAux*)(bw + 2 * rec_bytes + 3 * kSortKeys * sizeof(unsigned int) + 64 + acc_bytes);
    heads = (RayHead*)((uint8_t*)tilt_aux + (size_t)cap * sizeof(TiltAux));
    perm = (unsigned int*)((uint8_t*)heads + (size_t)batch * sizeof(RayHead));
  }
  // the heads sorted by hit count for the tangent pass, and the sort's counters
  RayHead* heads_sorted = nullptr;
  unsigned int* head_keys = nullptr;
  if (tilt) {
    heads_sorted = (RayHead*)((uint8_t*)perm + (size_t)cap * sizeof(unsigned int));
    head_keys = (unsigned int*)((uint8_t*)heads_sorted + (size_t)batch * sizeof(RayHead));
  }
  double* lut_grad = nullptr;
  HitRec* lut_recs = nullptr;
  if (use_lut) {
    lut_grad = (double*)(bw + 2 * rec_bytes + 3 * kSortKeys * sizeof(unsigned int) + 64 + acc_bytes + aux_bytes);
    lut_recs = (HitRec*)((uint8_t*)lut_grad + (size_t)n_lut * 8 * sizeof(double));
  }
  const bool dev_G = is_device_ptr(dL_dtally);
  const bool dev_g = is_device_ptr(grad_thickness);
  const double* G = dL_dtally;
  double* gout = grad_thickness;
  if (!dev_G) {
    double* tmp;
    CU(cudaMallocAsync((void**)&tmp, sizeof(double) * p.tally_size, s));
    CU(cudaMemcpyAsync(tmp, dL_dtally, sizeof(double) * p.tally_size, cudaMemcpyHostToDevice, s));
    G = tmp;
  }
  if (!dev_g) CU(cudaMallocAsync((void**)&gout, sizeof(double) * std::max(1, d->n_orig), s));
  CU(cudaMemsetAsync(gout, 0, sizeof(double) * std::max(1, d->n_orig), s));
  CU(cudaMemsetAsync(sc.grad_acc, 0, sizeof(double) * std::max(1, d->n_dev), s));
  const int bps_r = std::max(1, bwd_replay_blocks_per_sm(p.F, d->period, tilt, geo_mode(d), d->acc, smem_r));
  // mirror tilts: the replay records each hit's coefficients, the adjoint kernel its dL/d(cos t0);
  // after each batch a tangent pass per 8 mirrors re-traces its rays
  double* gt = grad_tilt;
  const bool dev_t = tilt && is_device_ptr(grad_tilt);
  const size_t smem_t = tilt_smem_bytes(d->blob_bytes, p.F);
  const int bps_t = tilt ? std::max(1, tilt_blocks_per_sm(p.F, d->period, geo_mode(d), d->acc, smem_t)) : 0;
  if (tilt) {
    if (!dev_t) CU(cudaMallocAsync((void**)&gt, sizeof(double) * d->K, s));
    CU(cudaMemsetAsync(gt, 0, sizeof(double) * d->K, s));
  }
  const int bps_a = std::max(1, bwd_adjoint_blocks_per_sm(d->period, d->acc, smem_a));
  // coating table: the same table as the forward's (same thicknesses), and
  // the FP64 sums of dL/dc per entry that the replay scatters into
  TraceArgs lut_a;
  memset(&lut_a, 0, sizeof(lut_a));
  if (use_lut) {
    st = prepare_lut(c, d, cfg, w, s, lut_a);
    if (st != WG_OK) return st;
    CU(cudaMemsetAsync(lut_grad, 0, (size_t)n_lut * 8 * sizeof(double), s));
    lut_a.lut_grad = lut_grad;
  }
  const long long w_begin = use_list ? 0 : p.rb, w_end = use_list ? n_list : p.re;
  // the listing forward's coefficients, if they are those of these paths,
  // thicknesses and coating table
  const bool use_coef = d->coef_fp != 0 && d->coef_fp == path_fingerprint(d, cfg, p) &&
                        d->coef_thick == d->thick_version && d->coef_lut == cfg->lut_bins;
  float ms_total = 0.f, ms_replay = 0.f, ms_adjoint = 0.f, ms_tilt = 0.f;
  int n_adj_launches = 0;
  for (long long b0 = w_begin; b0 < w_end;) {
    const long long b1 = std::min(w_end, b0 + batch);
    Plan q = p;
    if (!use_list) plan_range(q, b0, b1);
    TraceArgs a = base_args(d, cfg, q, w);
    if (use_coef) {
      a.coef = static_cast<float4*>(d->coefs.p);
      a.coef_base = d->coef_base;
      a.coef_rays = d->coef_rays;
      a.coef_slots = d->coef_slots;
      a.coef_mode = 2;
    }
    if (use_list) {
      a.replay_list = list;
      a.list_begin = b0;
      a.list_end = b1;
      a.n_chunks = (b1 - b0 + kReplayUnit - 1) / kReplayUnit;
    }
    a.G = G;
    a.hit_buf = sc.rec;
    a.hit_cap = cap;
    a.hit_count = sc.hit_count;
    a.tilt_aux = tilt_aux;
    a.ray_heads = heads;
    a.head_cap = b1 - b0;
    a.head_count = sc.hit_count + 1;
    a.lut = lut_a.lut;
    a.lut_n = lut_a.lut_n;
    a.n_lam = lut_a.n_lam;
    a.lut_c0 = lut_a.lut_c0;
    a.lut_inv_dc = lut_a.lut_inv_dc;
    a.lut_grad = lut_a.lut_grad;
    CU(cudaMemsetAsync(&w.head->work, 0, sizeof(unsigned long long), s));
    CU(cudaMemsetAsync(sc.keys, 0, kSortKeys * sizeof(unsigned int), s));
    CU(cudaMemsetAsync(sc.hit_count, 0, 2 * sizeof(unsigned long long), s));
    const int grid_r = (int)std::max<long long>(1, std::min<long long>(a.n_chunks, (long long)c->sm_count * bps_r));
    if (stats) CU(cudaEventRecord(c->t0, s));
    CU(launch_bwd_replay(a, p.F, d->period, tilt, geo_mode(d), d->acc, grid_r, smem_r, s));
    if (stats) CU(cudaEventRecord(c->kev[1], s));
    unsigned long long counts[2] = {0, 0};  // records, ray heads
    CU(cudaMemcpyAsync(counts, sc.hit_count, sizeof(counts), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    const unsigned long long n_rec = counts[0];
    if ((long long)n_rec > cap) {
      // more records than the batch holds (never seen: ~2 records per ray against 16):
      // redo this batch with half the rays
      if (b1 - b0 <= 1) return fail(WG_ENOMEM, "wg_trace_backward: one ray needs more than %lld hit records", cap);
      // (the dropped attempt's replay counters stay in the statistics)
      batch = std::max<long long>(1, (b1 - b0) / 2);
      continue;
    }
    if (!use_lut) CU(launch_bwd_sort(sc.rec, (long long)n_rec, d->blob, sc.keys, sc.keys + kSortKeys, sc.keys + 2 * kSortKeys,
                                         sc.sorted, perm, s));
    AdjArgs aa;
    memset(&aa, 0, sizeof(aa));
    aa.wait_ns = c->wait_limit_ns;
    aa.tilt_aux = tilt_aux;
    aa.perm = perm;
    aa.blob = d->blob;
    aa.blob_bytes = d->blob_bytes;
    aa.recs = sc.sorted;
    aa.lambda = w.lam;
    aa.n_rec = (long long)n_rec;
    aa.rec_chunk = 1024;
    aa.n_layers = d->n_dev;
    aa.grad_acc = sc.grad_acc;
    aa.work = &w.head->work;
    aa.counters = w.head->counters;
    aa.error = &w.head->error;
    CU(cudaMemsetAsync(&w.head->work, 0, sizeof(unsigned long long), s));
    if (stats) CU(cudaEventRecord(c->kev[2], s));
    if (n_rec > 0 && !use_lut) {  // (table mode: one adjoint over the table's entries after the last batch)
      const long long chunks = ((long long)n_rec + aa.rec_chunk - 1) / aa.rec_chunk;
      const int grid_a = (int)std::min<long long>(chunks, (long long)c->sm_count * bps_a);
      CU(launch_bwd_adjoint(aa, d->period, d->acc, grid_a, smem_a, s));
      ++n_adj_launches;
    }
    if (stats) CU(cudaEventRecord(c->kev[3], s));
    const long long n_heads = std::min<long long>((long long)counts[1], b1 - b0);
    if (tilt && n_heads > 0) CU(launch_heads_sort(heads, n_heads, head_keys, heads_sorted, s));
    for (int k0 = 0; tilt && n_heads > 0 && k0 < d->K; k0 += 8) {
      TraceArgs at = a;
      at.ray_heads = heads_sorted;
      at.n_heads = n_heads;
      at.grad_tilt = gt;
      at.tilt_k0 = k0;
      const int grid_t =
          (int)std::max<long long>(1, std::min<long long>((n_heads + 127) / 128, (long long)c->sm_count * bps_t));
      CU(launch_tilt_grad(at, p.F, d->period, geo_mode(d), d->acc, grid_t, smem_t, s));
    }
    if (stats) {
      CU(cudaEventRecord(c->t1, s));
      CU(cudaEventSynchronize(c->t1));
      float ms = 0.f, mr = 0.f, ma = 0.f, mt = 0.f;
      cudaEventElapsedTime(&ms, c->t0, c->t1);
      cudaEventElapsedTime(&mr, c->t0, c->kev[1]);
      cudaEventElapsedTime(&ma, c->kev[2], c->kev[3]);
      cudaEventElapsedTime(&mt, c->kev[3], c->t1);
      ms_total += ms;
      ms_replay += mr;
      ms_adjoint += ma;
      ms_tilt += mt;
    }
    b0 = b1;
  }
  if (use_lut) {
    // second stage: the thin-film adjoint once per (table entry, r or t) with
    // the entry's accumulated dL/dc as its weights
    CU(launch_lut_records(lut_grad, d->K, cfg->n_lambda, w.lam, lut_a.lut_n, lut_a.lut_c0, 1.0f / lut_a.lut_inv_dc,
                          lut_recs, s));
    AdjArgs aa;
    memset(&aa, 0, sizeof(aa));
    aa.wait_ns = c->wait_limit_ns;
    aa.blob = d->blob;
    aa.blob_bytes = d->blob_bytes;
    aa.recs = lut_recs;
    aa.lambda = w.lam;
    aa.n_rec = 2 * n_lut;
    aa.rec_chunk = 1024;
    aa.n_layers = d->n_dev;
    aa.grad_acc = sc.grad_acc;
    aa.work = &w.head->work;
    aa.counters = w.head->counters;
    aa.error = &w.head->error;
    CU(cudaMemsetAsync(&w.head->work, 0, sizeof(unsigned long long), s));
    if (stats) CU(cudaEventRecord(c->kev[2], s));
    const long long chunks = (aa.n_rec + aa.rec_chunk - 1) / aa.rec_chunk;
    const int grid_a = (int)std::min<long long>(chunks, (long long)c->sm_count * bps_a);
    CU(launch_bwd_adjoint(aa, d->period, d->acc, grid_a, smem_a, s));
    ++n_adj_launches;
    if (stats) {
      CU(cudaEventRecord(c->kev[3], s));
      CU(cudaEventSynchronize(c->kev[3]));
      float ma = 0.f;
      cudaEventElapsedTime(&ma, c->kev[2], c->kev[3]);
      ms_adjoint += ma;
      ms_total += ma;
    }
  }
  CU(launch_scatter_grad(sc.grad_acc, d->n_dev, d->d_dev_to_orig, gout, s));
  if (tilt && !dev_t) {
    CU(cudaMemcpyAsync(grad_tilt, gt, sizeof(double) * d->K, cudaMemcpyDeviceToHost, s));
    CU(cudaFreeAsync(gt, s));
    CU(cudaStreamSynchronize(s));
  }
  CU(cudaEventRecord(c->ws_free, s));
  if (!dev_G) CU(cudaFreeAsync((void*)G, s));
  if (!dev_g) {
    CU(cudaMemcpyAsync(grad_thickness, gout, sizeof(double) * d->n_orig, cudaMemcpyDeviceToHost, s));
    CU(cudaFreeAsync(gout, s));
    CU(cudaStreamSynchronize(s));
  }
  if (stats || !dev_g) {
    st = finish_stats(c, w, s, stats, false);
    if (stats) {
      stats->kernel_ms = ms_total;
      stats->replay_ms = ms_replay;
      stats->adjoint_ms = ms_adjoint;
      stats->tilt_ms = ms_tilt;
      stats->n_adjoint_launches = n_adj_launches;
    }
    return st;
  }
  return WG_OK;
}

extern "C" wg_status wg_loss(wg_ctx* c, const wg_design* d, const wg_trace_cfg* cfg, int32_t kind, double w_f,
                             double w_e, const double* tally, double* out, double* dL_dtally) {
  if (!c || !d || !tally || !out) return fail(WG_EINVAL, "wg_loss: NULL argument");
  if (kind != 0 && kind != 1) return fail(WG_EINVAL, "wg_loss: kind must be 0 (CV) or 1 (variance)");
  Plan p;
  wg_status st = make_plan(d, cfg, 2048, p);
  if (st != WG_OK) return st;
  if (!is_device_ptr(tally) || (dL_dtally && !is_device_ptr(dL_dtally)))
    return fail(WG_EINVAL, "wg_loss: tally and dL_dtally must be device memory");
  cudaStream_t s = (cudaStream_t)cfg->stream;
  std::lock_guard<std::mutex> lk(c->mu);
  CU(cudaSetDevice(c->device));
  const size_t need = sizeof(double) * (size_t)loss_ws_doubles(p.n_cells, p.bins, cfg->n_lambda) + 16;
  CU(cudaStreamWaitEvent(s, c->ws_free, 0));
  if (need > c->loss.n) {
    CU(cudaEventSynchronize(c->ws_free));
    CU(c->loss.ensure(need));
  }
  double* ws = (double*)c->loss.p;
  double* odev = ws + 2 * p.n_cells * 9;  // 8 doubles; pupil masks follow
  CU(launch_loss_impl(tally, d->dims, cfg->n_lambda, p.n_f, cfg->eb_nx, cfg->eb_ny, cfg->eb_cx_mm, cfg->eb_cy_mm,
                      cfg->eb_w_mm, cfg->eb_h_mm, 1.0 / (double)p.n_cell, kind, w_f, w_e, ws, odev, dL_dtally, s));
  CU(cudaMemcpyAsync(out, odev, sizeof(double) * 4, cudaMemcpyDeviceToHost, s));
  CU(cudaEventRecord(c->ws_free, s));
  CU(cudaStreamSynchronize(s));
  return WG_OK;
}

extern "C" wg_status wg_trace_forward_noalloc(wg_ctx* c, const wg_design* d, const wg_trace_cfg* cfg, double* tally,
                                              wg_stats* stats) {
  if (!c || !d || !tally) return fail(WG_EINVAL, "wg_trace_forward_noalloc: NULL ctx/design/tally");
  if (cfg && cfg->lut_bins) return fail(WG_EINVAL, "wg_trace_forward_noalloc: the coating table needs allocations");
  Plan p;
  wg_status st = make_plan(d, cfg, 2048, p);
  if (st != WG_OK) return st;
  p.chunk_rays = default_chunk(p);
  p.chunks_per_cell = (p.n_cell + p.chunk_rays - 1) / p.chunk_rays;
  p.n_chunks = (p.cell_hi - p.cell_lo + 1) * p.chunks_per_cell;
  const size_t smem = fwd_smem_bytes(d->blob_bytes, p.bins, p.F, fwd_slots(p.chunk_rays), d->acc);
  if (smem > 200 * 1024) return fail(WG_EINVAL, "wg_trace_forward_noalloc: design + eyebox too large for shared memory");
  const WsLayout need = ws_layout(nullptr, cfg, p.n_f);
  if (need.bytes > (size_t)WG_NOALLOC_SCRATCH_BYTES)
    return fail(WG_EINVAL,
                "wg_trace_forward_noalloc: this configuration needs %zu bytes of scratch, the static array holds %d "
                "(%d fields x 48 B + wavelength/angle arrays + 256 B); use fewer fields or wg_trace_forward",
                need.bytes, WG_NOALLOC_SCRATCH_BYTES, p.n_f);
  cudaStream_t s = (cudaStream_t)cfg->stream;
  std::lock_guard<std::mutex> lk(c->mu);
  CU(cudaSetDevice(c->device));
  if (!is_device_ptr(tally))
    return fail(WG_EINVAL, "wg_trace_forward_noalloc: tally must be device memory (host buffers would need staging)");
  const WsLayout w = ws_layout(c->noalloc_scratch, cfg, p.n_f);
  // clear what must start at zero: counters, ledger, chunk queue, error word
  CU(cudaMemsetAsync(w.head, 0, 256, s));
  CU(cudaMemcpyAsync(w.lam, cfg->lambda_nm, sizeof(float) * cfg->n_lambda, cudaMemcpyHostToDevice, s));
  CU(cudaMemcpyAsync(w.fx, cfg->field_x_deg, sizeof(float) * cfg->n_fx, cudaMemcpyHostToDevice, s));
  CU(cudaMemcpyAsync(w.fy, cfg->field_y_deg, sizeof(float) * cfg->n_fy, cudaMemcpyHostToDevice, s));
  CU(launch_prep_fields(w.fields, w.fx, w.fy, cfg->n_fx, cfg->n_fy, d->n_slab, d->ic_tilt, d->dims, s));
  CU(cudaMemsetAsync(tally + p.cell_lo * p.bins, 0, sizeof(double) * (p.cell_hi - p.cell_lo + 1) * p.bins, s));
  TraceArgs a = base_args(d, cfg, p, w);
  a.tally = tally;
  const int bps = std::max(1, trace_fwd_blocks_per_sm(p.F, d->period, geo_mode(d), d->acc, smem));
  const int grid = (int)std::min<long long>(p.n_chunks, (long long)c->sm_count * bps);
  if (stats) CU(cudaEventRecord(c->t0, s));
  CU(launch_trace_fwd(a, p.F, d->period, geo_mode(d), d->acc, grid, smem, s));
  if (stats) {
    CU(cudaEventRecord(c->t1, s));
    return finish_stats(c, w, s, stats, true);
  }
  return WG_OK;
}
