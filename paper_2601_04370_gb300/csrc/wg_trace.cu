// Small kernels of the waveguide trace and their launchers: design and field
// preparation (FP64), thickness updates, the reflection-probability trace, the
// hit-count and stack sorts, the gradient scatter and the coating table's
// second-stage records. The large trace kernels are instantiated in
// wg_trace_fwd*.cu, wg_trace_bwd*.cu and wg_trace_adj.cu.
#include <atomic>

#include "wg_kernels.cuh"

namespace wgk {

size_t hit_rec_bytes() { return sizeof(HitRec); }

static std::atomic<unsigned long long> g_launches{0};
void note_launches(unsigned long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
unsigned long long launches() { return g_launches.load(std::memory_order_relaxed); }

// ---------------------------------------------------------------------------
// Preparation (FP64, tiny): mirror planes from tilts, input-mirror normal,
// per-field launch directions and transverse bases.
// ---------------------------------------------------------------------------
// geo (general designs, else NULL): per mirror 14 floats, the normal N0 at
// the nominal tilt, the pivot, the tilt axis a, the rectangle x0 x1 y0 y1 and
// the nominal tilt (deg); the normal at tilt t is N0 rotated about a by
// t - t0, cos(t - t0) N0 + sin(t - t0) a x N0, through the pivot.
__global__ void k_prep_design(uint8_t* blob, const float* mir_x, const float* mir_tilt, const float* mir_omega,
                              const float* geo, int n_mir, float ic_tilt_deg, float thick) {
  BlobHeader* h = reinterpret_cast<BlobHeader*>(blob);
  MirrorRec* mir = reinterpret_cast<MirrorRec*>(blob + h->off_mir);
  const double deg = 3.14159265358979323846 / 180.0;
  for (int k = threadIdx.x; k < n_mir; k += blockDim.x) {
    const double a = (double)mir_tilt[k] * deg;
    if (!geo) {
      const double nx = -sin(a), nz = cos(a);
      mir[k].nx = (float)nx;
      mir[k].ny = 0.0f;
      mir[k].nz = (float)nz;
      mir[k].nlx = (float)(nx - (double)mir[k].nx);
      mir[k].nly = 0.0f;
      mir[k].nlz = (float)(nz - (double)mir[k].nz);
      mir[k].c = (float)(nx * (double)mir_x[k] + nz * 0.5 * (double)thick);
      mir[k].ax = 0.0f;
      mir[k].ay = -1.0f;
      mir[k].az = 0.0f;
      mir[k].x0 = mir[k].y0 = -__int_as_float(0x7f800000);
      mir[k].x1 = mir[k].y1 = __int_as_float(0x7f800000);
    } else {
      const float* g = geo + 14 * k;
      const double del = a - (double)g[13] * deg;
      const double c = cos(del), sn = sin(del);
      const double n0x = g[0], n0y = g[1], n0z = g[2], ax = g[6], ay = g[7], az = g[8];
      double nx = c * n0x + sn * (ay * n0z - az * n0y);
      double ny = c * n0y + sn * (az * n0x - ax * n0z);
      double nz = c * n0z + sn * (ax * n0y - ay * n0x);
      const double inv = 1.0 / sqrt(nx * nx + ny * ny + nz * nz);  // unit in FP64 (float32 inputs)
      nx *= inv;
      ny *= inv;
      nz *= inv;
      mir[k].nx = (float)nx;
      mir[k].ny = (float)ny;
      mir[k].nz = (float)nz;
      mir[k].nlx = (float)(nx - (double)mir[k].nx);
      mir[k].nly = (float)(ny - (double)mir[k].ny);
      mir[k].nlz = (float)(nz - (double)mir[k].nz);
      mir[k].c = (float)(nx * (double)g[3] + ny * (double)g[4] + nz * (double)g[5]);
      mir[k].ax = g[6];
      mir[k].ay = g[7];
      mir[k].az = g[8];
      mir[k].x0 = g[9];
      mir[k].x1 = g[10];
      mir[k].y0 = g[11];
      mir[k].y1 = g[12];
    }
    const double w = (double)mir_omega[k];
    mir[k].omega = mir_omega[k];
    mir[k].isw = (float)(1.0 / sqrt(w));
    mir[k].is1w = (float)(1.0 / sqrt(1.0 - w));
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double a = (double)ic_tilt_deg * deg;
    h->ic_nx = (float)(-sin(a));
    h->ic_nz = (float)cos(a);
    h->ic_cot = (float)(cos(a) / sin(a));
    h->general = geo != nullptr;
    h->n_fam = 0;
    if (geo) {
      // families: runs of consecutive mirrors with the same normal (bitwise)
      // and strictly monotone offsets
      FamRec* fam = reinterpret_cast<FamRec*>(blob + h->off_mir + sizeof(MirrorRec) * n_mir);
      int nf = 0;
      for (int k = 0; k < n_mir;) {
        int j = k + 1, dir = 0;
        while (j < n_mir && mir[j].nx == mir[k].nx && mir[j].ny == mir[k].ny && mir[j].nz == mir[k].nz) {
          const int sd = mir[j].c > mir[j - 1].c ? 1 : (mir[j].c < mir[j - 1].c ? -1 : 0);
          if (sd == 0 || (dir != 0 && sd != dir)) break;
          dir = sd;
          ++j;
        }
        fam[nf].k0 = k;
        fam[nf].n = j - k;
        fam[nf].dir = dir == 0 ? 1 : dir;
        fam[nf].pad = 0;
        ++nf;
        k = j;
      }
      h->n_fam = nf;
    }
    // ordering of the planes along x on both faces (planes that are ordered
    // on both faces do not cross inside the slab), with a 0.1 um margin;
    // general designs test every plane
    const double margin = 1e-4;
    int ok = fabs((double)h->ic_nx) > 1e-3 && geo == nullptr;
    for (int f = 0; f < 2 && ok; ++f) {
      const double z = f ? (double)thick : 0.0;
      double prev = ok ? -(double)h->ic_nz * z / (double)h->ic_nx : 0.0;
      for (int k = 0; k < n_mir && ok; ++k) {
        const double nx = mir[k].nx, nz = mir[k].nz, c = mir[k].c;
        if (fabs(nx) < 1e-3) {
          ok = 0;
          break;
        }
        const double x = (c - nz * z) / nx;
        ok = x > prev + margin;
        prev = x;
      }
      ok = ok && (double)h->x_end > prev + margin;
    }
    h->ordered = ok;
  }
}

__global__ void k_prep_fields(FieldRec* out, const float* fx, const float* fy, int n_fx, int n_fy, float n_slab,
                              float ic_tilt_deg, int dims) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= n_fx * n_fy) return;
  const double deg = 3.14159265358979323846 / 180.0;
  const int ix = f % n_fx, iy = f / n_fx;
  const double tx = tan((double)fx[ix] * deg);
  const double ty = dims == 3 ? tan((double)fy[iy] * deg) : 0.0;
  const double an = sqrt(tx * tx + ty * ty + 1.0);
  const double ax = tx / an, ay = ty / an, n = (double)n_slab;
  const double gx = ax / n, gy = ay / n, gz = sqrt(1.0 - (ax * ax + ay * ay) / (n * n));
  const double a = (double)ic_tilt_deg * deg;
  const double Nx = -sin(a), Nz = cos(a);
  const double dn = gx * Nx + gz * Nz;
  const double dx = gx - 2.0 * dn * Nx, dy = gy, dz = gz - 2.0 * dn * Nz;
  // e1 = normalize(y - (y.d) d), e2 = d x e1
  double e1x = -dy * dx, e1y = 1.0 - dy * dy, e1z = -dy * dz;
  const double e1n = sqrt(e1x * e1x + e1y * e1y + e1z * e1z);
  e1x /= e1n;
  e1y /= e1n;
  e1z /= e1n;
  const double e2x = dy * e1z - dz * e1y, e2y = dz * e1x - dx * e1z, e2z = dx * e1y - dy * e1x;
  FieldRec r;
  r.dx = (float)dx;
  r.dy = (float)dy;
  r.dz = (float)dz;
  r.e1x = (float)e1x;
  r.e1y = (float)e1y;
  r.e1z = (float)e1z;
  r.e2x = (float)e2x;
  r.e2y = (float)e2y;
  r.e2z = (float)e2z;
  r.dlx = (float)(dx - (double)r.dx);
  r.dly = (float)(dy - (double)r.dy);
  r.dlz = (float)(dz - (double)r.dz);
  out[f] = r;
}

__global__ void k_thickness_update(uint8_t* blob, const float* d_orig, const int* orig_to_store, int n_orig) {
  const BlobHeader* h = reinterpret_cast<const BlobHeader*>(blob);
  float* d = reinterpret_cast<float*>(blob + h->off_d);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_orig) {
    const int j = orig_to_store[i];
    if (j >= 0) d[j] = d_orig[i];
  }
}

// ---------------------------------------------------------------------------
// Reflection-probability pre-optimization (Methods, "Learned reflection
// probabilities"): each coating a scalar reflectance equal to its mirror's
// omega, geometric tracing without polarization. With the sampling
// probability equal to the reflectance every path has weight one: a ray that
// reaches the eyebox adds the unpolarized exit transmittance (T_s + T_p) / 2
// to the tally (a two-field ray with unit s and p amplitudes through
// face_event), and with G = dL/dtally its score to dL/d omega:
//   G[bin] I sum over its hits (reflected ? 1/omega_k : -1/(1 - omega_k)).
// One ray per thread; the gradient is summed per CTA in shared memory.
// ---------------------------------------------------------------------------
constexpr int kOmegaBlock = 256;
template <int GM>
__global__ void __launch_bounds__(kOmegaBlock) k_omega_trace(const TraceArgs A, double* grad_omega) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ __align__(8) uint64_t s_mbar;
  __shared__ double s_grad[MAX_MIR];
  __shared__ unsigned long long s_cnt[3];
  for (int k = threadIdx.x; k < MAX_MIR; k += blockDim.x) s_grad[k] = 0.0;
  if (threadIdx.x < 3) s_cnt[threadIdx.x] = 0ull;
  if (!stage_blob(smem, A.blob, A.blob_bytes, &s_mbar, A.error, wait_limit(A.wait_ns))) return;
  Blob B;
  B.bind(smem);
  const BlobHeader& H = *B.h;
  unsigned long long c_rays = 0, c_hits = 0, c_over = 0;
  for (long long id = A.ray_begin + blockIdx.x * (long long)blockDim.x + threadIdx.x; id < A.ray_end;
       id += (long long)gridDim.x * blockDim.x) {
    const long long cell = id / A.n_cell;
    const ChunkConst cc = chunk_const(A, cell);
    Ray<2> R;
    gen_ray(R, id, cc, H, A);
    R.a[0] = make_float2(1.f, 0.f);
    R.b[0] = make_float2(0.f, 0.f);
    R.a[1] = make_float2(0.f, 0.f);
    R.b[1] = make_float2(1.f, 0.f);
    uint8_t hk[TAPE_HITS];  // mirror | 0x80 if reflected, per hit
    int nh = 0;
    ++c_rays;
    for (;;) {
      float t;
      const int sid = next_surface<GM>(B, R.p, R.d, R.last, R.reg, t);
      ++R.ev;
      if (sid < 0) break;
      R.p = v3(fmaf(t, R.d.x, R.p.x), fmaf(t, R.d.y, R.p.y), fmaf(t, R.d.z, R.p.z));
      R.last = sid;
      if (sid >= S_MIR) {
        const int k = sid - S_MIR;
        const MirrorRec& M = B.mir[k];
        const float cd = fmaf(R.d.x, M.nx, fmaf(R.d.y, M.ny, R.d.z * M.nz));
        const int m = R.hits;
        const uint4 rnd = philox10(
            make_uint4((uint32_t)R.id, (uint32_t)((unsigned long long)R.id >> 32), (uint32_t)(m >> 2), TAG_EVT),
            A.key0, A.key1);
        const uint32_t word = (m & 3) == 0 ? rnd.x : (m & 3) == 1 ? rnd.y : (m & 3) == 2 ? rnd.z : rnd.w;
        const bool refl = u24(word) < M.omega;
        if (refl) R.d = v3(fmaf(-2.0f * cd, M.nx, R.d.x), fmaf(-2.0f * cd, M.ny, R.d.y), fmaf(-2.0f * cd, M.nz, R.d.z));
        R.reg = region_after(B, R.reg, k, R.d);
        R.hits = m + 1;
        if (nh < TAPE_HITS) hk[nh] = (uint8_t)(k | (refl ? 0x80 : 0));
        ++nh;
        if (R.ev >= A.max_events) break;
        continue;
      }
      int dummy = 0;
      const Outcome o = face_event<2>(R, sid, H, A, nullptr, nullptr, dummy);
      if (!o.term) {
        if (R.ev >= A.max_events) break;
        continue;
      }
      if (o.cat == L_EYEBOX) {
        const long long flat = cell * A.bins + o.bin;
        atomicAdd(A.tally + flat, (double)o.I);
        if (grad_omega && A.G) {
          const double g = A.G[flat] * (double)o.I;
          if (nh > TAPE_HITS) {
            ++c_over;  // more hits than the list holds: no gradient from this ray
          } else if (g != 0.0) {
            for (int h = 0; h < nh; ++h) {
              const int k = hk[h] & 0x7f;
              const double w = (double)B.mir[k].omega;
              atomicAdd(&s_grad[k], (hk[h] & 0x80) ? g / w : -g / (1.0 - w));
            }
          }
        }
      }
      break;
    }
    c_hits += R.hits;
  }
  const unsigned long long cv[3] = {c_rays, c_hits, c_over};
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const unsigned long long v = warp_sum_u(cv[i]);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(&s_cnt[i], v);
  }
  __syncthreads();
  if (grad_omega)
    for (int k = threadIdx.x; k < H.n_mir; k += blockDim.x)
      if (s_grad[k] != 0.0) atomicAdd(grad_omega + k, s_grad[k]);
  if (threadIdx.x == 0 && s_cnt[0]) atomicAdd(A.counters + 0, s_cnt[0]);
  if (threadIdx.x == 1 && s_cnt[1]) atomicAdd(A.counters + 1, s_cnt[1]);
  if (threadIdx.x == 2 && s_cnt[2]) atomicAdd(A.counters + 5, s_cnt[2]);
}

cudaError_t launch_omega_trace(const TraceArgs& a, double* grad_omega, int gm, int sm_count, cudaStream_t s) {
  const long long n = a.ray_end - a.ray_begin;
  if (n <= 0) return cudaSuccess;
  const int grid = (int)std::max<long long>(1, std::min<long long>((n + kOmegaBlock - 1) / kOmegaBlock, 8ll * sm_count));
  auto k = gm == 1 ? k_omega_trace<1> : k_omega_trace<0>;
  raise_smem_limit(k);
  note_launches(1);
  k<<<grid, kOmegaBlock, a.blob_bytes, s>>>(a, grad_omega);
  return cudaGetLastError();
}

// Rays grouped by their length (a counting sort over 0..TAPE_HITS): the
// replay and the tangent pass then give each warp rays of equal length
// instead of waiting for its longest one. Keys: a listed eyebox ray's hit
// count (ExitRec::pad; holes go first: the replay's record capacity comes
// from these counts), a ray head's surface events (the tangent pass re-traces
// every event of the path; grouped by events it ran 2.40 -> 1.93 ms against
// grouping by hits at 1e7 rays).
constexpr int kHitKeys = TAPE_HITS + 1;
static_assert(sizeof(unsigned int) * kHitKeys <= kHitSortScratch, "hit-count sort scratch");
__device__ __forceinline__ int hit_key(const RayHead& r) { return min(max(r.events, 0), TAPE_HITS); }
__device__ __forceinline__ int hit_key(const ExitRec& r) { return r.flat < 0 ? 0 : min(max(r.pad, 0), TAPE_HITS); }

template <class R>
__global__ void k_hits_count(const R* in, long long n, unsigned int* cnt) {
  __shared__ unsigned int s[kHitKeys];
  for (int i = threadIdx.x; i < kHitKeys; i += blockDim.x) s[i] = 0u;
  __syncthreads();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    atomicAdd(&s[hit_key(in[i])], 1u);
  __syncthreads();
  for (int i = threadIdx.x; i < kHitKeys; i += blockDim.x)
    if (s[i]) atomicAdd(cnt + i, s[i]);
}
// counts -> exclusive offsets, in place (one thread)
__global__ void k_hits_offsets(unsigned int* cnt) {
  unsigned int run = 0;
  for (int i = 0; i < kHitKeys; ++i) {
    const unsigned int c = cnt[i];
    cnt[i] = run;
    run += c;
  }
}
// each block ranks its records per key in shared memory and reserves one
// range per key from the global cursors
template <class R>
__global__ void k_hits_scatter(const R* in, long long n, unsigned int* cursor, R* out) {
  __shared__ unsigned int s_cnt[kHitKeys], s_base[kHitKeys];
  for (int i = threadIdx.x; i < kHitKeys; i += blockDim.x) s_cnt[i] = 0u;
  __syncthreads();
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  R r;
  int key = -1;
  unsigned int rank = 0;
  if (i < n) {
    r = in[i];
    key = hit_key(r);
    rank = atomicAdd(&s_cnt[key], 1u);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < kHitKeys; k += blockDim.x)
    if (s_cnt[k]) s_base[k] = atomicAdd(cursor + k, s_cnt[k]);
  __syncthreads();
  if (key >= 0) out[s_base[key] + rank] = r;
}

template <class R>
static cudaError_t hits_sort(const R* in, long long n, unsigned int* cnt, R* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(unsigned int) * kHitKeys, s);
  if (e != cudaSuccess) return e;
  note_launches(3);
  k_hits_count<R><<<(unsigned)std::min<long long>((n + 255) / 256, 1024), 256, 0, s>>>(in, n, cnt);
  k_hits_offsets<<<1, 1, 0, s>>>(cnt);
  k_hits_scatter<R><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in, n, cnt, out);
  return cudaGetLastError();
}
cudaError_t launch_heads_sort(const RayHead* in, long long n, unsigned int* cnt, RayHead* out, cudaStream_t s) {
  return hits_sort(in, n, cnt, out, s);
}
cudaError_t launch_exits_sort(const ExitRec* in, long long n, unsigned int* cnt, ExitRec* out, cudaStream_t s) {
  return hits_sort(in, n, cnt, out, s);
}

size_t tilt_smem_bytes(int blob_bytes, int F) {
  return (size_t)blob_bytes + sizeof(double) * (size_t)(kTiltBlock / 32) * kTiltPass * 32 +
         sizeof(float) * (size_t)(kTiltBlock / 32) * kTiltPass * (3 + 4 * F) * 32;
}

// exclusive prefix of the per-key record counts (one block of kSortKeys
// threads: warp-level inclusive scans, then the scan of the warp totals)
__global__ void k_bwd_scan(const unsigned int* key_count, unsigned int* key_off, unsigned int* key_cursor) {
  constexpr int NW = kSortKeys / 32;
  __shared__ unsigned int s_w[NW];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const unsigned int c = key_count[t];
  unsigned int x = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned int y = __shfl_up_sync(FULL, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_w[w] = x;
  __syncthreads();
  if (w == 0) {
    unsigned int v = lane < NW ? s_w[lane] : 0u;
    const unsigned int own = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int y = __shfl_up_sync(FULL, v, o);
      if (lane >= o) v += y;
    }
    if (lane < NW) s_w[lane] = v - own;  // exclusive prefix of the warp totals
  }
  __syncthreads();
  const unsigned int off = s_w[w] + x - c;
  key_off[t] = off;
  key_cursor[t] = off;
}

// Records per sort key (stack, then evanescence class), counted per block in
// shared memory (warp-aggregated) and added to the global counts.
constexpr int kScatterItems = 8;
__global__ void k_bwd_count(const HitRec* in, long long n, const uint8_t* blob, unsigned int* key_count) {
  __shared__ unsigned int s_cnt[kSortKeys];
  const BlobHeader& H = *reinterpret_cast<const BlobHeader*>(blob);
  const int tid = threadIdx.x, lane = tid & 31;
  for (int k = tid; k < kSortKeys; k += blockDim.x) s_cnt[k] = 0u;
  __syncthreads();
  const long long tile = (long long)blockIdx.x * blockDim.x * kScatterItems;
#pragma unroll
  for (int t = 0; t < kScatterItems; ++t) {
    const long long i = tile + (long long)t * blockDim.x + tid;
    int key = -1;
    if (i < n) {
      const HitRec r = in[i];
      if (r.kfw >= 0) key = sort_key(r, H);
    }
    const unsigned peers = __match_any_sync(FULL, key);
    if (key >= 0 && lane == __ffs(peers) - 1) atomicAdd(&s_cnt[key], (unsigned)__popc(peers));
  }
  __syncthreads();
  for (int k = tid; k < kSortKeys; k += blockDim.x)
    if (s_cnt[k]) atomicAdd(key_count + k, s_cnt[k]);
}

// Scatter into key order. A block takes a tile of kScatterItems records per
// thread, ranks them per key in shared memory (warp-aggregated), reserves
// one range per key with a single global atomic, then writes.
// perm (optional): perm[sorted position] = record index before the sort
__global__ void k_bwd_scatter(const HitRec* in, long long n, const uint8_t* blob, unsigned int* key_cursor,
                              HitRec* out, unsigned int* perm) {
  const BlobHeader& H = *reinterpret_cast<const BlobHeader*>(blob);
  __shared__ unsigned int s_cnt[kSortKeys], s_base[kSortKeys];
  const int tid = threadIdx.x, lane = tid & 31;
  for (int k = tid; k < kSortKeys; k += blockDim.x) s_cnt[k] = 0u;
  __syncthreads();
  const long long tile = (long long)blockIdx.x * blockDim.x * kScatterItems;
  HitRec r[kScatterItems];
  int key[kScatterItems];
  unsigned int rank[kScatterItems];
#pragma unroll
  for (int t = 0; t < kScatterItems; ++t) {
    const long long i = tile + (long long)t * blockDim.x + tid;
    key[t] = -1;
    if (i < n) {
      r[t] = in[i];
      if (r[t].kfw >= 0) key[t] = sort_key(r[t], H);
    }
    const unsigned peers = __match_any_sync(FULL, key[t]);
    const int leader = __ffs(peers) - 1;
    unsigned int base = 0;
    if (key[t] >= 0 && lane == leader) base = atomicAdd(&s_cnt[key[t]], (unsigned)__popc(peers));
    base = __shfl_sync(FULL, base, leader);
    rank[t] = base + __popc(peers & ((1u << lane) - 1u));
  }
  __syncthreads();
  for (int k = tid; k < kSortKeys; k += blockDim.x)
    if (s_cnt[k]) s_base[k] = atomicAdd(key_cursor + k, s_cnt[k]);
  __syncthreads();
#pragma unroll
  for (int t = 0; t < kScatterItems; ++t)
    if (key[t] >= 0) {
      const unsigned int pos = s_base[key[t]] + rank[t];
      out[pos] = r[t];
      if (perm) perm[pos] = (unsigned int)(tile + (long long)t * blockDim.x + tid);
    }
}

size_t adj_smem_bytes(int blob_bytes, int n_layers, int P) {
  if (P == 3) return adj_smem_bytes_p<3>(blob_bytes, n_layers);
  if (P == 2) return adj_smem_bytes_p<2>(blob_bytes, n_layers);
  return adj_smem_bytes_p<0>(blob_bytes, n_layers);
}

// FP64 per-layer sums -> the caller's gradient in design order
__global__ void k_scatter_grad(const double* acc, int n_layers, const int* dev_to_orig, double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_layers) out[dev_to_orig[i]] = acc[i];
}

// Hit records of the table's second stage: one per (entry, r or t), in
// stack order, with the entry's accumulated dL/dc as weights (a common
// power of two split off into eA, as for the per-hit records)
__global__ void k_lut_records(const double* grad, int n_mir, int n_lam, const float* lam, int n, float c0, float dc,
                              HitRec* out) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long total = (long long)n_mir * 2 * n_lam * 2 * n;
  if (i >= total) return;
  const int j = (int)(i % n);
  long long q = i / n;
  const int which = (int)(q % 2);
  q /= 2;
  const int li = (int)(q % n_lam);
  q /= n_lam;
  const int side = (int)(q % 2);
  const int k = (int)(q / 2);
  const long long e = (((long long)k * 2 + side) * n_lam + li) * n + j;
  const double* g = grad + 8 * e + 4 * which;
  const double m = fmax(fmax(fabs(g[0]), fabs(g[1])), fmax(fabs(g[2]), fabs(g[3])));
  int eA = 0;
  if (m > 0.0) frexp(m, &eA);
  HitRec r;
  r.kfw = k | ((side == 0 ? 1 : 0) << 8) | (which << 9) | (li << 10);
  r.cos0 = fmaf((float)j, dc, c0);
  r.cos0l = 0.0f;
  r.eA = eA;
  r.As = make_float2((float)ldexp(g[0], -eA), (float)ldexp(g[1], -eA));
  r.Ap = make_float2((float)ldexp(g[2], -eA), (float)ldexp(g[3], -eA));
  out[i] = r;
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t launch_prep_design(uint8_t* blob, const float* mir_x, const float* mir_tilt, const float* mir_omega,
                               const float* geo, int n_mir, float ic_tilt_deg, float thick, cudaStream_t s) {
  note_launches(1);
  k_prep_design<<<1, 64, 0, s>>>(blob, mir_x, mir_tilt, mir_omega, geo, n_mir, ic_tilt_deg, thick);
  return cudaGetLastError();
}

// job j = blockIdx.y of a fused launch: its tally cells [cell_lo, cell_hi]
// and its eyebox-ray counter to zero
__global__ void k_zero_jobs(const TraceArgs* __restrict__ jobs) {
  const TraceArgs& A = jobs[blockIdx.y];
  const long long cell_hi = (A.ray_end - 1) / A.n_cell;
  const long long lo = A.cell_lo * A.bins, hi = (cell_hi + 1) * A.bins;
  for (long long i = lo + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < hi;
       i += (long long)gridDim.x * blockDim.x)
    A.tally[i] = 0.0;
  if (blockIdx.x == 0 && threadIdx.x == 0 && A.exit_count) *A.exit_count = 0ull;
}

cudaError_t launch_zero_jobs(const TraceArgs* jobs_dev, int n, long long max_doubles, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const long long bx = std::max<long long>(1, std::min<long long>((max_doubles + 255) / 256, 256));
  note_launches(1);
  k_zero_jobs<<<dim3((unsigned)bx, (unsigned)n), 256, 0, s>>>(jobs_dev);
  return cudaGetLastError();
}

cudaError_t preload_field_kernel() {
  cudaFuncAttributes fa;
  return cudaFuncGetAttributes(&fa, k_prep_fields);
}

cudaError_t launch_prep_fields(FieldRec* out, const float* fx, const float* fy, int n_fx, int n_fy, float n_slab,
                               float ic_tilt_deg, int dims, cudaStream_t s) {
  const int n = n_fx * n_fy;
  note_launches(1);
  k_prep_fields<<<(n + 127) / 128, 128, 0, s>>>(out, fx, fy, n_fx, n_fy, n_slab, ic_tilt_deg, dims);
  return cudaGetLastError();
}

cudaError_t launch_thickness_update(uint8_t* blob, const float* d_orig, const int* orig_to_store, int n_orig,
                                    cudaStream_t s) {
  note_launches(1);
  k_thickness_update<<<(n_orig + 255) / 256, 256, 0, s>>>(blob, d_orig, orig_to_store, n_orig);
  return cudaGetLastError();
}

// Failure-path test hook: one thread waits, with the trace kernels' bounded
// wait (device clock, at most 2^24 polls), for a flag that nothing sets; when
// the limit runs out it sets bit 2 of the error word (as an idle wait of the
// forward trace does) and returns.
__global__ void k_wait_flag(const unsigned* flag, unsigned* err, unsigned long long limit_ns) {
  if (threadIdx.x != 0) return;
  const unsigned long long t0 = gtimer_ns();
  for (int it = 0; it < (1 << 24); ++it) {
    if (*reinterpret_cast<const volatile unsigned*>(flag)) return;
    if (gtimer_ns() - t0 > limit_ns) break;
    __nanosleep(64);
  }
  atomicOr(err, 2u);
}
cudaError_t launch_wait_flag(const unsigned* flag, unsigned* err, unsigned long long limit_ns, cudaStream_t s) {
  note_launches(1);
  k_wait_flag<<<1, 32, 0, s>>>(flag, err, limit_ns);
  return cudaGetLastError();
}

// counting sort of the records by key: key_count must be zero on entry
cudaError_t launch_bwd_sort(const HitRec* in, long long n, const uint8_t* blob, unsigned int* key_count,
                            unsigned int* key_off, unsigned int* key_cursor, HitRec* out, unsigned int* perm,
                            cudaStream_t s) {
  const long long per_block = 256ll * kScatterItems;
  const unsigned grid = (unsigned)((n + per_block - 1) / per_block);
  if (n > 0) {
    note_launches(1);
    k_bwd_count<<<grid, 256, 0, s>>>(in, n, blob, key_count);
  }
  note_launches(1);
  static_assert(kSortKeys % 32 == 0 && kSortKeys / 32 <= 32 && kSortKeys <= 1024, "one scan block");
  k_bwd_scan<<<1, kSortKeys, 0, s>>>(key_count, key_off, key_cursor);
  if (n > 0) {
    note_launches(1);
    k_bwd_scatter<<<grid, 256, 0, s>>>(in, n, blob, key_cursor, out, perm);
  }
  return cudaGetLastError();
}

cudaError_t launch_scatter_grad(const double* acc, int n_layers, const int* dev_to_orig, double* out,
                                cudaStream_t s) {
  if (n_layers == 0) return cudaSuccess;
  note_launches(1);
  k_scatter_grad<<<(n_layers + 127) / 128, 128, 0, s>>>(acc, n_layers, dev_to_orig, out);
  return cudaGetLastError();
}

cudaError_t launch_lut_records(const double* grad, int n_mir, int n_lam, const float* lam, int n, float c0, float dc,
                               HitRec* out, cudaStream_t s) {
  const long long total = (long long)n_mir * 2 * n_lam * 2 * n;
  if (total <= 0) return cudaSuccess;
  note_launches(1);
  k_lut_records<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(grad, n_mir, n_lam, lam, n, c0, dc, out);
  return cudaGetLastError();
}

}  // namespace wgk
