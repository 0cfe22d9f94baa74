// Kernel templates and device code of the waveguide trace, shared by the
// translation units that instantiate them (wg_trace*.cu): design/field preparation, the persistent
// forward Monte Carlo trace (K2), the adjoint (K3: replay -> hit records ->
// counting sort by stack -> per-hit thin-film adjoint), coating test hooks
// (K1) and the gradient scatter.
//
// Paper: "End-to-end differentiable design of geometric waveguide displays"
// (arXiv 2601.04370), Methods: "Multilayer thin-film solver" (Eq. 2, Eq. 3,
// transfer matrices), "Polarization ray tracing" (Eq. 4), "Differentiable
// Monte Carlo non-sequential ray tracing" (Eq. 5, I = sum |E|^2); Fig. 3b/c
// (two-pass intersection, gradient checkpoint between trace and thin film):
// here the backward pass replays each ray from its Philox key and hands the
// per-hit coefficient sensitivities to a checkpointed thin-film adjoint.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "wg_device.cuh"
#include "wg_internal.h"

namespace wgk {

constexpr unsigned FULL = 0xffffffffu;
constexpr float HALF_ULP24 = 2.98023223876953125e-08f;  // 2^-25

struct alignas(16) HitRec {
  int kfw;     // mirror | front << 8 | which << 9 (0 = r, 1 = t) | wavelength index << 10; -1 = slot of a dropped ray
  float cos0;
  float cos0l; // low part of cos(theta_0) (accurate mode), else 0
  int eA;      // weights are (As, Ap) * 2^eA (dL/dtally spans the FP64 range)
  float2 As, Ap;
};
__device__ __forceinline__ int kfw_lam(int kfw) { return (kfw >> 10) & 0xffff; }
static_assert(kStackKeys == 2 * MAX_MIR, "stack keys");
// stack of a hit record: (mirror, side)
__device__ __forceinline__ int stack_key(int kfw) { return ((kfw & 0xff) << 1) | ((kfw >> 8) & 1); }
// evanescence class of an incidence cosine: the number of the design's
// materials with (n0/n)^2 sin^2 t0 > 1. The adjoint's records are sorted by
// it within their stack, so that the lanes of a warp agree on which layers
// are evanescent (a divergent branch in the layer loop otherwise runs both
// of its sides); it decides nothing else.
__device__ __forceinline__ int evan_class(const BlobHeader& H, float cos0) {
  const float sin2 = fmaf(-cos0, cos0, 1.0f);
  int n = 0;
#pragma unroll
  for (int i = 0; i < MAX_MAT; ++i) n += (i < H.n_mat && H.mat_r2[i] * sin2 > 1.0f) ? 1 : 0;
  return min(n, kClsPerStack - 1);
}
// sort key of a record: its stack, then its evanescence class
__device__ __forceinline__ int sort_key(const HitRec& r, const BlobHeader& H) {
  return stack_key(r.kfw) * kClsPerStack + evan_class(H, r.cos0);
}
static_assert(sizeof(HitRec) == 32, "hit record");
// per-ray record (layout of wg_ray_record)
struct RayRec {
  uint32_t hash;
  int n_events, n_hits, cat, bin;
  float I, w;
  int pad;
};

// device clock in ns (%globaltimer) and the limit of every bounded wait
__device__ __forceinline__ unsigned long long gtimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
constexpr unsigned long long kWaitLimitNs = 500ull * 1000ull * 1000ull;  // 0.5 s, the default limit
__host__ __device__ __forceinline__ unsigned long long wait_limit(unsigned long long ns) {
  return ns ? ns : kWaitLimitNs;
}

// ---------------------------------------------------------------------------
// Bulk (TMA) staging of the design blob into shared memory, mbarrier
// completion with a bounded wait. Returns false (uniformly across the CTA)
// if the wait ran out; the caller then exits after flagging the error.
// ---------------------------------------------------------------------------
static __device__ bool stage_blob(uint8_t* s_dst, const uint8_t* g_src, int bytes, uint64_t* mbar, unsigned* err,
                                  unsigned long long limit_ns) {
  const uint32_t bar = (uint32_t)__cvta_generic_to_shared(mbar);
  const uint32_t dst = (uint32_t)__cvta_generic_to_shared(s_dst);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    for (int off = 0; off < bytes; off += 16384) {
      const int n = min(16384, bytes - off);
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst + off),
          "l"(g_src + off), "r"(n), "r"(bar)
          : "memory");
    }
  }
  uint32_t done = 0;
  const unsigned long long t_start = gtimer_ns();
  for (int it = 0; it < (1 << 22) && !done; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(0)
        : "memory");
    if (!done && gtimer_ns() - t_start > limit_ns) break;
  }
  const int ok = __syncthreads_and(done != 0);
  if (!ok && threadIdx.x == 0) atomicOr(err, 1u);
  return ok != 0;
}

// ---------------------------------------------------------------------------
// Ray state and events shared by the forward and backward kernels.
// ---------------------------------------------------------------------------
template <int F>
struct Ray {
  V3 p, d;
  V3 dl;              // accurate mode: the low parts of d (d + dl), else unused
  float2 a[F], b[F];  // field in the face s/p basis of d
  long long id;
  int ev, hits, last;
  int reg;            // region between mirror planes (ordered designs), else -1
  uint32_t hash;
};

struct ChunkConst {
  V3 fd;                  // guided launch direction
  V3 fdl;                 // its low parts (accurate mode)
  float a1, b1, a2, b2;   // e1, e2 in the face basis of fd
  float lam, inv_lam;     // the cell's wavelength and 1/lambda
  int li;                 // its wavelength index
  long long cell;
};

template <int F>
__device__ __forceinline__ void gen_ray(Ray<F>& R, long long id, const ChunkConst& cc, const BlobHeader& H,
                                        const TraceArgs& A) {
  const uint4 r0 = philox10(make_uint4((uint32_t)id, (uint32_t)((unsigned long long)id >> 32), 0u, TAG_GEN),
                            A.key0, A.key1);
  const float z0 = H.thick * (u24(r0.x) + HALF_ULP24);
  R.p = v3(z0 * H.ic_cot, H.dims == 3 ? (u24(r0.y) + HALF_ULP24 - 0.5f) * A.pupil_y : 0.0f, z0);
  R.d = cc.fd;
  R.dl = cc.fdl;
  if (F == 2) {
    R.a[0] = make_float2(cc.a1, 0.f);
    R.b[0] = make_float2(cc.b1, 0.f);
    R.a[F - 1] = make_float2(cc.a2, 0.f);
    R.b[F - 1] = make_float2(cc.b2, 0.f);
  } else {
    float c = 1.0f, s = 0.0f;
    if (A.pol == 1) {
      sincospif(u24(r0.z), &s, &c);
    } else if (A.pol == 3) {
      c = 0.0f;
      s = 1.0f;
    }
    R.a[0] = make_float2(fmaf(c, cc.a1, s * cc.a2), 0.f);
    R.b[0] = make_float2(fmaf(c, cc.b1, s * cc.b2), 0.f);
  }
  R.id = id;
  R.ev = 0;
  R.hits = 0;
  R.last = S_LEFT;
  R.reg = H.ordered ? 0 : -1;  // rays start on the input mirror, left of mirror 0
  R.hash = 2166136261u;
}

template <int F>
__device__ __forceinline__ float ray_weight(const Ray<F>& R) {
  float w = 0.f;
#pragma unroll
  for (int f = 0; f < F; ++f) w += cabs2(R.a[f]) + cabs2(R.b[f]);
  return w * (1.0f / F);
}

// outcome of a non-mirror event
struct Outcome {
  int term;   // 0 alive, 1 terminated
  int cat;
  int bin;    // flat tally bin within the cell (eyebox exits), -1 otherwise
  float I, w;
  float Ts, Tp;
};

// Face / end event at surface sid (position already advanced).
template <int F>
__device__ __forceinline__ Outcome face_event(Ray<F>& R, int sid, const BlobHeader& H, const TraceArgs& A,
                                              float2* seg_s, float2* seg_p, int& n_tir) {
  Outcome o;
  o.term = 0;
  o.bin = -1;
  o.I = 0.f;
  o.Ts = o.Tp = 0.f;
  R.hash = fnv(R.hash, (uint32_t)sid);
  if (sid <= S_TOP) {
    const float n = H.n_slab;
    const float cz = R.d.z;
    const float ci = fabsf(cz);
    const float sin2 = fmaf(-cz, cz, 1.0f);
    const float x = n * n * sin2;
    if (x > 1.0f) {
      float2 rs, rp;
      tir_coef(n, ci, sin2, rs, rp);
#pragma unroll
      for (int f = 0; f < F; ++f) {
        R.a[f] = cmul(rs, R.a[f]);
        R.b[f] = cmul(rp, R.b[f]);
      }
      if (seg_s) {
        *seg_s = cmul(*seg_s, rs);
        *seg_p = cmul(*seg_p, rp);
      }
      R.d.z = -cz;
      R.dl.z = -R.dl.z;
      ++n_tir;
      return o;
    }
    o.term = 1;
    o.w = ray_weight(R);
    if (sid == S_BOT) {
      o.cat = L_LEAKED;
      return o;
    }
    // eye-side exit: Fresnel power transmission glass -> air
    const float ct = sqrtf(fmaxf(1.0f - x, 0.0f));
    const float u = n * ci;
    // the Fresnel factors only scale the intensity: fast quotients (the
    // eye-plane distance below, which decides the bin, keeps the IEEE one)
    const float ts = __fdividef(2.0f * u, u + ct);
    const float tp = __fdividef(2.0f * u, fmaf(n, ct, ci));
    const float tf = __fdividef(ct, u);
    o.Ts = tf * ts * ts;
    o.Tp = tf * tp * tp;
    float I = 0.f;
#pragma unroll
    for (int f = 0; f < F; ++f) I += fmaf(o.Ts, cabs2(R.a[f]), o.Tp * cabs2(R.b[f]));
    o.I = I * (1.0f / F);
    const float sfac = H.eye_relief / ct;
    const float qx = fmaf(sfac * n, R.d.x, R.p.x);
    const float qy = fmaf(sfac * n, R.d.y, R.p.y);
    const float fxb = floorf((qx - A.eb_x0) * A.eb_sx);
    bool inside = fxb >= 0.0f && fxb < (float)A.eb_nx;
    int ey = 0;
    if (H.dims == 3) {
      const float fyb = floorf((qy - A.eb_y0) * A.eb_sy);
      inside = inside && fyb >= 0.0f && fyb < (float)A.eb_ny;
      ey = inside ? (int)fyb : 0;
    }
    if (inside) {
      o.cat = L_EYEBOX;
      o.bin = ey * A.eb_nx + (int)fxb;
    } else {
      o.cat = L_MISSED;
    }
    return o;
  }
  o.term = 1;
  o.cat = L_ABSORBED;
  o.w = ray_weight(R);
  return o;
}

// Mirror event: coefficients, basis rotation, MC decision and rescaling.
// Fills the tape entry fields when `te` is non-null.
struct MirrorStep {
  float2 cs, cp;   // applied coefficients (incl. 1/sqrt scaling)
  float cphi, sphi, cpsi, spsi;
  float cos0, cos0l;  // cos(theta_0) = cos0 + cos0l (cos0l = 0 in fast mode)
  int front, refl;
};

// Entry and weight of the coating table for cos(theta_0) = c: the hit's
// coefficients are (1 - f) entry(j) + f entry(j + 1); f is clamped to [0, 1]
// (constant beyond the grid's end points).
__device__ __forceinline__ void lut_locate(const TraceArgs& A, float c, int& j, float& f) {
  const float x = (c - A.lut_c0) * A.lut_inv_dc;
  j = min(max((int)floorf(x), 0), A.lut_n - 2);
  f = fminf(fmaxf(x - (float)j, 0.0f), 1.0f);
}
__device__ __forceinline__ long long lut_entry(const TraceArgs& A, int k, bool front, int li, int j) {
  return (((long long)k * 2 + (front ? 0 : 1)) * A.n_lam + li) * A.lut_n + j;
}
__device__ __forceinline__ float2 lerp2(float2 a, float2 b, float f) {
  return make_float2(fmaf(f, b.x - a.x, a.x), fmaf(f, b.y - a.y, a.y));
}

// lam, inv_lam, li: the hit's wavelength, 1/lambda and wavelength index (the
// coating table's, when A.lut is set), computed once per cell
// CM: 1 in the forward (may keep the applied coefficients, TraceArgs::coef),
// 2 in the replay (may read them back); the other direction is compiled out.
// ACC: accurate mode (direction and incidence cosine as hi + lo, the
// accurate layer evaluation), for long stacks.
// LM: where the coefficients come from: 0 the layer chain (the coating
// table's branch compiled out), 1 the coating table, 2 the table when A.lut
// is set, else the chain.
template <int F, int P, int CM, bool ACC, int LM = 2>
__device__ __forceinline__ MirrorStep mirror_event(Ray<F>& R, int k, const Blob& B, float lam, float inv_lam, int li,
                                                   const TraceArgs& A, int& layer_steps, float2* Es_out,
                                                   float2* Ep_out) {
  const BlobHeader& H = *B.h;
  const MirrorRec& M = B.mir[k];
  const V3 N = v3(M.nx, M.ny, M.nz);
  F2 cdf{0.0f, 0.0f};
  if constexpr (ACC) cdf = dot3_df(R.d, R.dl, N, v3(M.nlx, M.nly, M.nlz));
  const float cd = ACC ? cdf.h : dot3(R.d, N);
  MirrorStep st;
  st.front = cd < 0.0f;
  st.cos0 = fabsf(cd);
  st.cos0l = cd < 0.0f ? -cdf.l : cdf.l;
  // the listing forward's applied coefficients of this hit, when kept
  const int m = R.hits;
  const bool kept = CM == 2 && A.coef_mode == 2 && m < A.coef_slots;
  Coef cf;
  float4 kv;
  if (kept) {
    kv = A.coef[(R.id - A.coef_base) * A.coef_slots + m];
  } else if (LM == 1 || (LM == 2 && A.lut)) {
    int j;
    float f;
    lut_locate(A, st.cos0, j, f);
    const float4* e = A.lut + 4 * lut_entry(A, k, st.front, li, j);
    const float4 a0 = __ldg(e), a1 = __ldg(e + 1), b0 = __ldg(e + 4), b1 = __ldg(e + 5);
    cf.rs = lerp2(make_float2(a0.x, a0.y), make_float2(b0.x, b0.y), f);
    cf.rp = lerp2(make_float2(a0.z, a0.w), make_float2(b0.z, b0.w), f);
    cf.ts = lerp2(make_float2(a1.x, a1.y), make_float2(b1.x, b1.y), f);
    cf.tp = lerp2(make_float2(a1.z, a1.w), make_float2(b1.z, b1.w), f);
  } else {
    const StackView sv{B.d, B.m, M.store_off, M.n_layers, M.store_off - M.layer_off};
    if constexpr (P > 0) {
      // a periodic stack: each slot's material evaluated directly
      MatK kb[P];
      slot_consts<P, ACC>(H, sv, st.front, st.cos0, st.cos0l, lam, inv_lam, kb);
      MatTable unused;
      cf = tmm_forward_k<P, ACC>(sv, st.front, unused, kb, H.n_slab, st.cos0, layer_steps);
    } else {
      MatTable mt;
      if constexpr (ACC) {
        mt.init_acc(H, st.cos0, st.cos0l, lam);
      } else {
        mt.init_inv(H, st.cos0, inv_lam);
      }
      cf = tmm_forward<P, ACC>(sv, st.front, mt, H.n_slab, st.cos0, layer_steps);
    }
  }
  // hit m draws word m & 3 of the block for counter (ray, m >> 2); the block
  // is recomputed per hit so the ray state needs no RNG words
  const uint4 rnd = philox10(
      make_uint4((uint32_t)R.id, (uint32_t)((unsigned long long)R.id >> 32), (uint32_t)(m >> 2), TAG_EVT), A.key0,
      A.key1);
  const uint32_t word = (m & 3) == 0 ? rnd.x : (m & 3) == 1 ? rnd.y : (m & 3) == 2 ? rnd.z : rnd.w;
  st.refl = u24(word) < M.omega;
  if (kept) {
    st.cs = make_float2(kv.x, kv.y);
    st.cp = make_float2(kv.z, kv.w);
  } else {
    if (st.refl) {
      st.cs = cscale(cf.rs, M.isw);
      st.cp = cscale(cf.rp, M.isw);
    } else {
      st.cs = cscale(cf.ts, M.is1w);
      st.cp = cscale(cf.tp, M.is1w);
    }
    if (CM == 1 && A.coef_mode == 1 && m < A.coef_slots)
      A.coef[(R.id - A.coef_base) * A.coef_slots + m] = make_float4(st.cs.x, st.cs.y, st.cp.x, st.cp.y);
  }
  V3 sf, pf;
  face_basis(R.d, sf, pf);
  V3 sm = cross3(R.d, N);
  const float sm2 = dot3(sm, sm);
  if (sm2 > 1e-24f) {
    const float r = rsqrtf(sm2);
    sm = v3(sm.x * r, sm.y * r, sm.z * r);
  } else {
    sm = sf;
  }
  st.cphi = dot3(sf, sm);
  st.sphi = dot3(pf, sm);
  V3 d2 = R.d, dl2 = R.dl;
  if (st.refl) {
    if constexpr (ACC) {
      reflect_df(d2, dl2, N, v3(M.nlx, M.nly, M.nlz), cdf);
    } else {
      d2 = v3(fmaf(-2.0f * cd, N.x, R.d.x), fmaf(-2.0f * cd, N.y, R.d.y), fmaf(-2.0f * cd, N.z, R.d.z));
    }
  }
  const V3 pm2 = cross3(sm, d2);
  V3 sf2, pf2;
  face_basis(d2, sf2, pf2);
  st.cpsi = dot3(sf2, sm);
  st.spsi = dot3(sf2, pm2);
#pragma unroll
  for (int f = 0; f < F; ++f) {
    const float2 Es = make_float2(fmaf(st.cphi, R.a[f].x, st.sphi * R.b[f].x), fmaf(st.cphi, R.a[f].y, st.sphi * R.b[f].y));
    const float2 Ep = make_float2(fmaf(-st.sphi, R.a[f].x, st.cphi * R.b[f].x), fmaf(-st.sphi, R.a[f].y, st.cphi * R.b[f].y));
    if (Es_out) {
      Es_out[f] = Es;
      Ep_out[f] = Ep;
    }
    const float2 Os = cmul(st.cs, Es), Op = cmul(st.cp, Ep);
    R.a[f] = make_float2(fmaf(st.cpsi, Os.x, st.spsi * Op.x), fmaf(st.cpsi, Os.y, st.spsi * Op.y));
    R.b[f] = make_float2(fmaf(-st.spsi, Os.x, st.cpsi * Op.x), fmaf(-st.spsi, Os.y, st.cpsi * Op.y));
  }
  R.d = d2;
  R.dl = dl2;
  R.reg = region_after(B, R.reg, k, d2);
  R.hash = fnv(R.hash, (uint32_t)(S_MIR + k) | (st.refl ? 0x80u : 0u));
  R.hits = m + 1;
  return st;
}

__device__ __forceinline__ ChunkConst chunk_const(const TraceArgs& A, long long cell) {
  ChunkConst cc;
  cc.cell = cell;
  const int li = (int)(cell / A.n_f), f = (int)(cell % A.n_f);
  cc.lam = __ldg(A.lambda + li);
  cc.inv_lam = 1.0f / cc.lam;
  cc.li = li;
  const FieldRec fr = A.fields[f];
  cc.fd = v3(fr.dx, fr.dy, fr.dz);
  cc.fdl = v3(fr.dlx, fr.dly, fr.dlz);
  V3 sf, pf;
  face_basis(cc.fd, sf, pf);
  const V3 e1 = v3(fr.e1x, fr.e1y, fr.e1z), e2 = v3(fr.e2x, fr.e2y, fr.e2z);
  cc.a1 = dot3(e1, sf);
  cc.b1 = dot3(e1, pf);
  cc.a2 = dot3(e2, sf);
  cc.b2 = dot3(e2, pf);
  return cc;
}

// chunk -> cell and ray range; false for an empty chunk
__device__ __forceinline__ bool chunk_range(const TraceArgs& A, long long chunk, long long& cell, long long& r0,
                                            long long& r1) {
  cell = A.cell_lo + chunk / A.chunks_per_cell;
  const long long j = chunk % A.chunks_per_cell;
  r0 = cell * A.n_cell + j * A.chunk_rays;
  r1 = min(r0 + A.chunk_rays, (cell + 1) * A.n_cell);
  r0 = max(r0, A.ray_begin);
  r1 = min(r1, A.ray_end);
  return r0 < r1;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_down_sync(FULL, v, o);
  return v;
}
__device__ __forceinline__ unsigned long long warp_sum_u(unsigned long long v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_down_sync(FULL, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// K2: forward Monte Carlo trace. Persistent CTAs; lanes pull rays from a
// CTA-wide sequence that runs over the chunks (one cell, a range of rays)
// the CTA has bound to its tally slots (A.n_slots <= kSlots). A warp advances its rays
// through face events until every live ray sits on a mirror, then runs the
// per-hit transfer-matrix chain together. Exits are added into the slot's
// FP32 shared tally; the lane whose ray completes a chunk has its warp flush
// the slot to the FP64 global
// tally and frees it for the CTA's next chunk. No CTA barrier separates
// chunks, so lanes never idle at a chunk's tail while rays remain.
// ---------------------------------------------------------------------------
constexpr int kSlots = kFwdSlots;
constexpr int kSizeBits = 20;  // chunk size field of SlotState::range

struct SlotState {
  unsigned long long range;  // (first virtual ray << kSizeBits) | rays: one word, read whole
  long long cell, r0;
  int j;                     // CTA-local chunk number bound to the slot
  unsigned int done;         // rays of the chunk finished
  ChunkConst cc;
};

struct FwdRing {
  SlotState slot[kSlots];
  int ns;                    // slots in use (the launch's n_slots)
  unsigned long long vnext;  // next virtual ray handed out
  unsigned long long ready;  // virtual rays of the chunks bound so far
  int free_for[kSlots];      // the chunk number slot s takes next (set when its previous chunk is flushed)
  int jready;                // chunks bound so far (under lock)
  int lock, no_more;
};

template <class T>
__device__ __forceinline__ T vload(const T& x) {
  return *const_cast<const volatile T*>(&x);
}
template <class T>
__device__ __forceinline__ void vstore(T& x, T v) {
  *const_cast<volatile T*>(&x) = v;
}

// Bind the global queue's next chunks to free slots (one thread; returns
// false at once if another thread holds the lock).
static __device__ bool ring_bind(FwdRing& S, const TraceArgs& A) {
  if (atomicCAS(&S.lock, 0, 1) != 0) return false;
  __threadfence_block();
  bool made = false;
  const int ns = S.ns;
  for (int it = 0; it < 2 * ns; ++it) {
    const int j = S.jready;
    const int s = j % ns;
    // slot s takes chunk j only after chunk j - ns was flushed from it
    if (vload(S.no_more) || vload(S.free_for[s]) != j) break;
    const long long c = (long long)atomicAdd(A.work, 1ull);
    if (c >= A.n_chunks) {
      __threadfence_block();  // every bound chunk's `ready` before `no_more`
      vstore(S.no_more, 1);
      break;
    }
    long long cell, r0, r1;
    const bool ne = chunk_range(A, c, cell, r0, r1);
    S.jready = j + 1;
    if (!ne) {  // nothing to trace: the slot stays free for the next chunk
      vstore(S.free_for[s], j + ns);
      continue;
    }
    SlotState& st = S.slot[s];
    st.cell = cell;
    st.r0 = r0;
    st.j = j;
    st.done = 0u;
    st.cc = chunk_const(A, cell);
    const unsigned long long v0 = S.ready;
    __threadfence_block();
    vstore(st.range, (v0 << kSizeBits) | (unsigned long long)(r1 - r0));
    __threadfence_block();
    vstore(S.ready, v0 + (unsigned long long)(r1 - r0));
    made = true;
  }
  __threadfence_block();
  atomicExch(&S.lock, 0);
  return made;
}

// per-ray record of ray index i of the launch range (bounds-checked)
__device__ __forceinline__ void put_rec(RayRec* recs, long long i, const TraceArgs& A, const RayRec& rr) {
  if (i >= 0 && i < A.ray_end - A.ray_begin) {
    recs[i] = rr;
  } else {
    atomicOr(A.error, 8u);
  }
}

// true once the global queue is exhausted and every bound ray handed out.
// Evaluated by lane 0 and broadcast: the shared words can change between two
// lanes' reads, and a loop exit taken by only part of a warp would leave the
// rest at a different full-warp intrinsic.
__device__ __forceinline__ bool ring_drained(const FwdRing& S, int lane) {
  int d = 0;
  if (lane == 0 && vload(S.no_more)) {
    __threadfence_block();
    d = vload(S.vnext) >= vload(S.ready);
  }
  return __shfl_sync(FULL, d, 0) != 0;
}
// device clock read by lane 0, the same value in every lane
__device__ __forceinline__ unsigned long long warp_time_ns() { return __shfl_sync(FULL, gtimer_ns(), 0); }

// Up to n consecutive virtual rays for one warp (called by its leader).
static __device__ unsigned long long ring_fetch(FwdRing& S, const TraceArgs& A, int n, int& got) {
  got = 0;
  for (int tries = 0; tries < 8; ++tries) {
    const unsigned long long old = vload(S.vnext);
    const unsigned long long re = vload(S.ready);
    if (re - old < 2ull * kBlock) ring_bind(S, A);  // keep a chunk bound ahead
    if (old >= re) {
      if (vload(S.ready) == re) return 0;
      continue;
    }
    const int take = (int)min((unsigned long long)n, re - old);
    if (atomicCAS(&S.vnext, old, old + (unsigned long long)take) == old) {
      got = take;
      return old;
    }
  }
  return 0;
}

// Flush slot s (whole warp) and free it.
static __device__ void ring_flush(FwdRing& S, int s, float* s_tally, const TraceArgs& A, int lane) {
  const SlotState& st = S.slot[s];
  float* tl = s_tally + (long long)s * A.bins;
  double* gt = A.tally + st.cell * (long long)A.bins;
  for (int i = lane; i < A.bins; i += 32) {
    const float v = tl[i];
    if (v != 0.f) {
      atomicAdd(gt + i, (double)v);
      tl[i] = 0.f;
    }
  }
  __syncwarp();
  __threadfence_block();
  if (lane == 0) vstore(S.free_for[s], st.j + S.ns);
}

// Count the warp's finished rays into their chunks; the warp that finishes
// a chunk's last ray flushes its slot. The fence orders each warp's tally
// adds before its counts, so a slot is flushed only after every add to it.
__device__ __forceinline__ void ring_finish(FwdRing& S, bool fin, int slot, float* s_tally, const TraceArgs& A,
                                            int lane) {
  if (!__any_sync(FULL, fin)) return;
  __threadfence_block();
  __syncwarp();  // every lane's tally adds ordered before the counts below
  // one count per finished ray: the lane whose count completes the chunk flushes it
  bool complete = false;
  if (fin) {
    const unsigned old = atomicAdd(&S.slot[slot].done, 1u);
    complete = old + 1u == (unsigned)(vload(S.slot[slot].range) & ((1ull << kSizeBits) - 1ull));
  }
  unsigned cm = __ballot_sync(FULL, complete);
  while (cm) {
    const int src = __ffs(cm) - 1;
    cm &= cm - 1;
    const int s = __shfl_sync(FULL, slot, src);
    __syncwarp();
    __threadfence_block();
    ring_flush(S, s, s_tally, A, lane);
  }
}

// Per-warp ray queues of the forward kernel, in shared memory (structure of
// arrays, one 32-bit word per field and slot): rays waiting at a mirror for
// the warp's next transfer-matrix round, and rays waiting for a geometry
// lane. A warp owns at most kFwdQCap rays (lanes + both queues), so neither
// queue can overflow.
constexpr int kQCap = kFwdQCap;    // rays a warp owns at a time
constexpr int kQRing = kFwdQRing;  // slots of a queue's ring
constexpr int kGenBatch = 24;      // fewest new rays a warp generates at once

// words of a queued ray (accurate mode: also the direction's low parts)
template <int F, bool ACC>
__host__ __device__ constexpr int q_words() { return 9 + 4 * F + (ACC ? 3 : 0); }

template <int F, bool ACC>
__device__ __forceinline__ void q_put(uint32_t* q, unsigned i, const Ray<F>& R, long long ray_begin, int slot) {
  uint32_t* w = q + i;
  constexpr int C = kQRing;
  w[0 * C] = __float_as_uint(R.p.x);
  w[1 * C] = __float_as_uint(R.p.y);
  w[2 * C] = __float_as_uint(R.p.z);
  w[3 * C] = __float_as_uint(R.d.x);
  w[4 * C] = __float_as_uint(R.d.y);
  w[5 * C] = __float_as_uint(R.d.z);
#pragma unroll
  for (int f = 0; f < F; ++f) {
    w[(6 + 4 * f) * C] = __float_as_uint(R.a[f].x);
    w[(7 + 4 * f) * C] = __float_as_uint(R.a[f].y);
    w[(8 + 4 * f) * C] = __float_as_uint(R.b[f].x);
    w[(9 + 4 * f) * C] = __float_as_uint(R.b[f].y);
  }
  // counters: events (8 bits), hits (8), last surface (7), region + 1 (7), tally slot (2)
  w[(6 + 4 * F) * C] = (uint32_t)(R.id - ray_begin);
  w[(7 + 4 * F) * C] = (uint32_t)R.ev | ((uint32_t)R.hits << 8) | ((uint32_t)R.last << 16) |
                       ((uint32_t)(R.reg + 1) << 23) | ((uint32_t)slot << 30);
  w[(8 + 4 * F) * C] = R.hash;
  if constexpr (ACC) {
    w[(9 + 4 * F) * C] = __float_as_uint(R.dl.x);
    w[(10 + 4 * F) * C] = __float_as_uint(R.dl.y);
    w[(11 + 4 * F) * C] = __float_as_uint(R.dl.z);
  }
}

template <int F, bool ACC>
__device__ __forceinline__ int q_get(const uint32_t* q, unsigned i, Ray<F>& R, long long ray_begin) {
  const uint32_t* w = q + i;
  constexpr int C = kQRing;
  R.p = v3(__uint_as_float(w[0 * C]), __uint_as_float(w[1 * C]), __uint_as_float(w[2 * C]));
  R.d = v3(__uint_as_float(w[3 * C]), __uint_as_float(w[4 * C]), __uint_as_float(w[5 * C]));
#pragma unroll
  for (int f = 0; f < F; ++f) {
    R.a[f] = make_float2(__uint_as_float(w[(6 + 4 * f) * C]), __uint_as_float(w[(7 + 4 * f) * C]));
    R.b[f] = make_float2(__uint_as_float(w[(8 + 4 * f) * C]), __uint_as_float(w[(9 + 4 * f) * C]));
  }
  R.id = ray_begin + (long long)w[(6 + 4 * F) * C];
  const uint32_t c = w[(7 + 4 * F) * C];
  R.ev = (int)(c & 0xffu);
  R.hits = (int)((c >> 8) & 0xffu);
  R.last = (int)((c >> 16) & 0x7fu);
  R.reg = (int)((c >> 23) & 0x7fu) - 1;
  R.hash = w[(8 + 4 * F) * C];
  if constexpr (ACC) {
    R.dl = v3(__uint_as_float(w[(9 + 4 * F) * C]), __uint_as_float(w[(10 + 4 * F) * C]),
              __uint_as_float(w[(11 + 4 * F) * C]));
  } else {
    R.dl = v3(0.0f, 0.0f, 0.0f);
  }
  return (int)(c >> 30);
}

// GM: geometry mode of next_surface (0 PRMA, 1 general, 2 either: fused launches)
// LUT: the coating table's instance (coefficients interpolated, no layer
// chain); the exact instances carry no table code
template <int F, int P, int GM, bool ACC, bool LUT = false>
__global__ void __launch_bounds__(kBlock, 2)
    k_trace_fwd(const TraceArgs A0, const TraceArgs* __restrict__ jobs, const int* __restrict__ cta_job) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ __align__(8) uint64_t s_mbar;
  __shared__ FwdRing S;
  __shared__ float s_led[6];
  __shared__ unsigned long long s_cnt[8];
  // this CTA's job: one design + configuration for the whole launch (a fused
  // launch gives each job its own range of CTAs; jobs == null: the one job A0)
  __shared__ TraceArgs A;
  if (threadIdx.x == 0) A = jobs ? jobs[cta_job[blockIdx.x]] : A0;
  __syncthreads();
  constexpr int NW = q_words<F, ACC>();
  float* s_tally = reinterpret_cast<float*>(smem + A.blob_bytes);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int n_slots = min(max(A.n_slots, 1), kSlots);
  uint32_t* mq = reinterpret_cast<uint32_t*>(smem + A.blob_bytes + sizeof(float) * n_slots * A.bins) +
                 wid * 2 * NW * kQRing;
  uint32_t* gq = mq + NW * kQRing;
  if (tid < 6) s_led[tid] = 0.f;
  if (tid < 8) s_cnt[tid] = 0ull;
  if (tid < kSlots) {
    S.free_for[tid] = tid;
    S.slot[tid].range = 0ull;
  }
  if (tid == 0) {
    S.ns = n_slots;
    S.vnext = 0ull;
    S.ready = 0ull;
    S.jready = 0;
    S.lock = 0;
    S.no_more = 0;
  }
  for (int i = tid; i < n_slots * A.bins; i += blockDim.x) s_tally[i] = 0.f;
  if (!stage_blob(smem, A.blob, A.blob_bytes, &s_mbar, A.error, wait_limit(A.wait_ns))) return;  // includes a CTA barrier
  Blob B;
  B.bind(smem);
  const BlobHeader& H = *B.h;
  const unsigned lt_mask = (1u << lane) - 1u;

  float led[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  int c_rays = 0, c_hits = 0, c_events = 0, c_tir = 0, c_steps = 0;
  RayRec* recs = reinterpret_cast<RayRec*>(A.records);

  Ray<F> R;
  bool has = false;
  int slot = 0;
  unsigned mh = 0, mt = 0, gh = 0, gt = 0;  // queue heads / tails (warp-uniform)
  int n_fly = 0;                            // rays this warp owns (warp-uniform)
  unsigned long long idle_t0 = 0;
  bool idling = false;
  // safety net: a warp needs at most ~2 loop passes per event of each ray it
  // traces (plus bounded idle waits); past this cap it flags and stops
  const unsigned long long it_cap =
      4ull * (unsigned long long)A.max_events *
          (unsigned long long)((A.ray_end - A.ray_begin) / ((long long)max(1, A.n_cta) * (kBlock / 32)) + 256) +
      (1ull << 24);
  unsigned long long iters = 0;
  unsigned long long x_next = 0, x_end = 0;  // this warp's unused eyebox-list slots (warp-uniform)
  for (;;) {
    if (++iters > it_cap) {
      if (lane == 0) atomicOr(A.error, 16u);
      break;
    }
    // ---- free lanes take rays waiting for geometry, then new rays ----
    unsigned need = __ballot_sync(FULL, !has);
    if (need && gt != gh) {
      const unsigned avail = gt - gh;
      const unsigned rank = __popc(need & lt_mask);
      if (!has && rank < avail) {
        slot = q_get<F, ACC>(gq, (gh + rank) & (kQRing - 1), R, A.ray_begin);
        has = true;
      }
      gh += min((unsigned)__popc(need), avail);
      need = __ballot_sync(FULL, !has);
    }
    // New rays in batches: with no parked ray left, and room for at least
    // kGenBatch, every lane generates one ray (the generation runs once for
    // up to 32 rays instead of once per pass for the few lanes that freed
    // up); a free lane keeps its own, a busy lane parks its in the geometry
    // queue, from which lanes take them as they free up
    if (need && gt == gh && n_fly <= kQCap - kGenBatch) {
      unsigned long long base = 0;
      int got = 0;
      if (lane == 0) base = ring_fetch(S, A, min(32, kQCap - n_fly), got);
      base = __shfl_sync(FULL, base, 0);
      got = __shfl_sync(FULL, got, 0);
      __threadfence_block();
      bool mapped = false;
      int tsl = 0;
      Ray<F> T;
      if (lane < got) {
        const unsigned long long v = base + (unsigned long long)lane;
        int sl = -1;
#pragma unroll
        for (int s = 0; s < kSlots; ++s) {
          const unsigned long long r = vload(S.slot[s].range);
          const unsigned long long v0 = r >> kSizeBits;
          if (v >= v0 && v < v0 + (r & ((1ull << kSizeBits) - 1ull))) sl = s;
        }
        if (sl < 0) {
          atomicOr(A.error, 4u);  // a handed-out ray outside every bound chunk: never traced
        } else {
          tsl = sl;
          const SlotState& st = S.slot[sl];
          gen_ray(T, st.r0 + (long long)(v - (st.range >> kSizeBits)), st.cc, H, A);
          mapped = true;
          ++c_rays;
        }
      }
      const bool park = mapped && has;
      const unsigned pk = __ballot_sync(FULL, park);
      if (park) q_put<F, ACC>(gq, (gt + __popc(pk & lt_mask)) & (kQRing - 1), T, A.ray_begin, tsl);
      gt += __popc(pk);
      if (mapped && !has) {
        R = T;
        slot = tsl;
        has = true;
      }
      n_fly += __popc(__ballot_sync(FULL, mapped));
    }
    // ---- one event per lane ----
    if (__any_sync(FULL, has)) {
      int pend_bin = -1;
      float pend_I = 0.f;
      bool fin = false, to_mir = false;
      if (has) {
        float t;
        const int sid = next_surface<GM>(B, R.p, R.d, R.last, R.reg, t);
        ++R.ev;
        Outcome o;
        o.term = 0;
        if (sid < 0) {
          o.term = 1;
          o.cat = L_ABSORBED;
          o.bin = -1;
          o.I = 0.f;
          o.w = ray_weight(R);
        } else {
          R.p = v3(fmaf(t, R.d.x, R.p.x), fmaf(t, R.d.y, R.p.y), fmaf(t, R.d.z, R.p.z));
          R.last = sid;
          if (sid >= S_MIR) {
            to_mir = true;
          } else {
            o = face_event<F>(R, sid, H, A, nullptr, nullptr, c_tir);
          }
        }
        if (!o.term && !to_mir && R.ev >= A.max_events) {
          o.term = 1;
          o.cat = L_TRUNCATED;
          o.bin = -1;
          o.I = 0.f;
          o.w = ray_weight(R);
        }
        if (o.term) {
          fin = true;
          c_events += R.ev;
          c_hits += R.hits;
          if (o.cat == L_EYEBOX) {
            led[L_EYEBOX] += o.I;
            led[L_EXIT_REFL] += o.w - o.I;
            pend_bin = o.bin;
            pend_I = o.I;
          } else if (o.cat == L_MISSED) {
            led[L_MISSED] += o.I;
            led[L_EXIT_REFL] += o.w - o.I;
          } else {
            // (a static index per category keeps the ledger in registers)
#pragma unroll
            for (int c = 0; c < 6; ++c)
              if (c == o.cat) led[c] += o.w;
          }
          if (recs) {
            RayRec rr;
            rr.hash = R.hash;
            rr.n_events = R.ev;
            rr.n_hits = R.hits;
            rr.cat = o.cat;
            rr.bin = o.cat == L_EYEBOX ? (int)(S.slot[slot].cell * A.bins + o.bin) : -1;
            rr.I = o.cat == L_EYEBOX ? o.I : 0.f;
            rr.w = o.w;
            rr.pad = 0;
            put_rec(recs, R.id - A.ray_begin, A, rr);
          }
        }
        if (fin || to_mir) has = false;
      }
      // rays that reached a mirror wait in the mirror queue
      const unsigned pmask = __ballot_sync(FULL, to_mir);
      if (to_mir) q_put<F, ACC>(mq, (mt + __popc(pmask & lt_mask)) & (kQRing - 1), R, A.ray_begin, slot);
      mt += __popc(pmask);
      // exits into the slot tallies: a few lanes per pass over thousands of
      // bins rarely meet, so each adds its own (a warp-level aggregation by
      // bin cost more than the collisions it saved)
      const unsigned pm = __ballot_sync(FULL, pend_bin >= 0);
      if (pm) {
        if (pend_bin >= 0) atomicAdd(&s_tally[slot * A.bins + pend_bin], pend_I);
        // list of eyebox rays for the adjoint: slots from the warp's reserved
        // chunk, a new chunk of kExitChunk when it runs out
        if (A.exit_list) {
          const unsigned cnt = __popc(pm), rank = __popc(pm & lt_mask);
          const unsigned left = (unsigned)(x_end - x_next);
          unsigned long long nb = 0;
          if (cnt > left) {
            if (lane == 0) nb = atomicAdd(A.exit_count, (unsigned long long)kExitChunk);
            nb = __shfl_sync(FULL, nb, 0);
          }
          if (pend_bin >= 0) {
            const unsigned long long i = rank < left ? x_next + rank : nb + (rank - left);
            if (i < (unsigned long long)A.exit_cap) {
              ExitRec e;
              e.id = R.id;
              e.flat = (int)(S.slot[slot].cell * A.bins + pend_bin);
              e.pad = R.hits;  // the backward sorts the list by it
              A.exit_list[i] = e;
            }
          }
          if (cnt > left) {
            x_next = nb + (cnt - left);
            x_end = nb + kExitChunk;
          } else {
            x_next += cnt;
          }
        }
      }
      ring_finish(S, fin, slot, s_tally, A, lane);
      n_fly -= __popc(__ballot_sync(FULL, fin));
    }
    // ---- transfer-matrix round: 32 queued hits (fewer when nothing else can run) ----
    const unsigned nm = mt - mh;
    if (nm >= 32u || (nm > 0u && !__any_sync(FULL, has) && gt == gh)) {
      // the geometry rays wait in the geometry queue meanwhile
      const unsigned hm = __ballot_sync(FULL, has);
      if (has) q_put<F, ACC>(gq, (gt + __popc(hm & lt_mask)) & (kQRing - 1), R, A.ray_begin, slot);
      gt += __popc(hm);
      has = false;
      const unsigned n = min(nm, 32u);
      bool fin = false, keep = false;
      if ((unsigned)lane < n) {
        slot = q_get<F, ACC>(mq, (mh + lane) & (kQRing - 1), R, A.ray_begin);
        const ChunkConst& scc = S.slot[slot].cc;
        mirror_event<F, P, 1, ACC, LUT ? 1 : 0>(R, R.last - S_MIR, B, scc.lam, scc.inv_lam, scc.li, A, c_steps,
                           nullptr, nullptr);
        if (R.ev >= A.max_events) {
          fin = true;
          c_events += R.ev;
          c_hits += R.hits;
          const float w = ray_weight(R);
          led[L_TRUNCATED] += w;
          if (recs) {
            RayRec rr;
            rr.hash = R.hash;
            rr.n_events = R.ev;
            rr.n_hits = R.hits;
            rr.cat = L_TRUNCATED;
            rr.bin = -1;
            rr.I = 0.f;
            rr.w = w;
            rr.pad = 0;
            put_rec(recs, R.id - A.ray_begin, A, rr);
          }
        } else {
          keep = true;
        }
      }
      mh += n;
      // a lane keeps the ray it took on through the mirror (its next event
      // comes in the next pass); the rays parked in the geometry queue return
      // to lanes as they free up (the order of the warp's work, not any ray's
      // result, depends on this)
      has = keep;
      ring_finish(S, fin, slot, s_tally, A, lane);
      n_fly -= __popc(__ballot_sync(FULL, fin));
      continue;
    }
    // ---- no ray in this warp: finished, or wait for the CTA's next chunk ----
    if (n_fly == 0) {
      if (ring_drained(S, lane)) break;
      __nanosleep(256);
      const unsigned long long now = warp_time_ns();
      if (!idling) idle_t0 = now;
      idling = true;
      if (now - idle_t0 > wait_limit(A.wait_ns)) {  // no work within the wait limit: give up and flag
        if (lane == 0) atomicOr(A.error, 2u);
        break;
      }
    } else {
      idling = false;
    }
  }
  // the rest of the warp's last chunk: holes
  for (unsigned long long i = x_next + lane; i < x_end; i += 32) {
    if (i < (unsigned long long)A.exit_cap) {
      ExitRec e;
      e.id = -1;
      e.flat = -1;
      e.pad = 0;
      A.exit_list[i] = e;
    }
  }
  // ---- statistics ----
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const float v = warp_sum(led[i]);
    if (lane == 0 && v != 0.f) atomicAdd(&s_led[i], v);
  }
  const unsigned long long cv[5] = {(unsigned long long)c_rays, (unsigned long long)c_hits,
                                    (unsigned long long)c_events, (unsigned long long)c_tir,
                                    (unsigned long long)c_steps};
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const unsigned long long v = warp_sum_u(cv[i]);
    if (lane == 0 && v) atomicAdd(&s_cnt[i], v);
  }
  __syncthreads();
  if (tid < 6 && s_led[tid] != 0.f) atomicAdd(A.ledger + tid, (double)s_led[tid]);
  if (tid < 5 && s_cnt[tid]) atomicAdd(A.counters + tid, s_cnt[tid]);
}

// ---------------------------------------------------------------------------
// K3: adjoint, in three kernels with their own register budgets.
//
// k_bwd_replay: the forward trace again from the same keys (the applied
//   coefficients of a ray's first hits read back from the listing forward,
//   TraceArgs::coef, instead of re-running their layer chains), with a per-ray
//   tape of mirror hits in local memory (incoming field, applied
//   coefficients, basis rotations, TIR products since the previous hit). A
//   ray that ends in the eyebox seeds dL/dE* = G[bin]/F (T_s a, T_p b),
//   walks its tape backwards and emits one record per hit: the weights A of
//   f = 2 Re(A_s c_s + A_p c_p) (dL/dc of that hit's raw coefficients).
//   Each warp claims short ray ranges of one cell from the global queue and
//   its lanes keep their own cell, so no CTA barrier separates ranges.
// k_bwd_scan + k_bwd_scatter: counting sort of the records by stack
//   (mirror, side), so a warp's 32 records share one stack.
// k_bwd_adjoint: one record per lane, checkpointed thin-film adjoint; when
//   the warp's 32 records share a stack every layer step touches the same
//   gradient entry in all lanes, which is reduced with shuffles and added
//   once; partial FP32 sums in shared memory go to FP64 after each chunk.
//   With the tilt gradient the reverse sweep also forms each record's
//   dL/d(cos theta_0) (tmm_adjoint<..., DUAL>).
// ---------------------------------------------------------------------------
// the low part of a hit's incidence cosine: kept in the tape in accurate
// mode only (the fast mode's tape stays as small as before)
template <bool ACC>
struct TapeLo {
  float cos0l_;
  __device__ __forceinline__ float cos0l() const { return cos0l_; }
  __device__ __forceinline__ void set_cos0l(float v) { cos0l_ = v; }
};
template <>
struct TapeLo<false> {
  __device__ __forceinline__ float cos0l() const { return 0.0f; }
  __device__ __forceinline__ void set_cos0l(float) {}
};
template <int F, bool ACC>
struct TapeE : TapeLo<ACC> {
  float2 cs, cp;
  float2 Es[F], Ep[F];
  float cphi, sphi, cpsi, spsi;
  float2 seg_s, seg_p;
  float cos0;
  int kfw;
};

// fewest eyebox rays whose reverse sweeps a warp of the replay runs together
// (fewer when the warp has no live ray left)
constexpr int kSweepMin = 16;

// T: the replay also serves the tilt gradient: each emitted record gets its
// TiltAux (the applied coefficients; the adjoint kernel adds dL/d(cos t0))
// and its ray a RayHead.
template <int F, int P, bool T, int GM, bool ACC>
__global__ void __launch_bounds__(kBlock, 2) k_bwd_replay(const TraceArgs A) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ __align__(8) uint64_t s_mbar;
  __shared__ unsigned long long s_cnt[8];
  const int tid = threadIdx.x, lane = tid & 31;
  if (tid < 8) s_cnt[tid] = 0ull;
  if (!stage_blob(smem, A.blob, A.blob_bytes, &s_mbar, A.error, wait_limit(A.wait_ns))) return;
  Blob B;
  B.bind(smem);
  const BlobHeader& H = *B.h;
  const unsigned lt_mask = (1u << lane) - 1u;
  HitRec* hb = A.hit_buf;
  const long long cap = A.hit_cap;

  int c_rays = 0, c_hits = 0, c_overflow = 0, c_tallied = 0, c_steps = 0;
  TapeE<F, ACC> tape[TAPE_HITS];

  // warp-private work unit (a short ray range of one cell, warp-uniform)
  long long u_cell = 0, u_next = 0, u_end = 0;
  bool u_more = true;
  ChunkConst ucc;
  ucc.lam = 0.f;
  ucc.inv_lam = 0.f;
  ucc.li = 0;
  Ray<F> R;
  bool has = false, at_mir = false;
  int hit_k = 0;
  long long cell_l = 0;  // cell and wavelength of this lane's ray
  float lam_l = 0.f, inv_lam_l = 0.f;
  int li_l = 0;
  float2 seg_s = make_float2(1.f, 0.f), seg_p = make_float2(1.f, 0.f);
  // a ray that ended in the eyebox waits in its lane (which takes no new ray
  // meanwhile) for the warp's next reverse sweep: emit hits, dL/dtally as
  // g0 2^eG, its exit transmittances
  int emit = 0, eG = 0;
  float g0 = 0.f, x_Ts = 0.f, x_Tp = 0.f;
  for (;;) {
        for (;;) {
          // lanes without a ray take the next rays of the warp's unit; the
          // warp claims units from the global queue as they run out
          unsigned fm = __ballot_sync(FULL, !has && emit == 0);
          while (fm && u_more) {
            if (u_next >= u_end) {
              long long c = 0;
              if (lane == 0) c = (long long)atomicAdd(A.work, 1ull);
              c = __shfl_sync(FULL, c, 0);
              if (c >= A.n_chunks) {
                u_more = false;
                break;
              }
              if (A.replay_list) {  // a range of the forward's eyebox-ray list
                u_next = A.list_begin + c * A.chunk_rays;
                u_end = min(u_next + A.chunk_rays, A.list_end);
              } else {
                long long cell, r0, r1;
                if (!chunk_range(A, c, cell, r0, r1)) continue;
                u_cell = cell;
                u_next = r0;
                u_end = r1;
                ucc = chunk_const(A, cell);
              }
            }
            const int take = (int)min((long long)__popc(fm), u_end - u_next);
            const int rank = __popc(fm & lt_mask);
            if (!has && emit == 0 && rank < take) {  // a waiting lane keeps its ray until its sweep
              if (A.replay_list) {
                // listed ray: replayed only if its bin carries gradient
                const ExitRec e = A.replay_list[u_next + rank];
                if (e.flat >= 0 && A.G[e.flat] != 0.0) {  // flat < 0: a hole of the list
                  cell_l = e.flat / A.bins;
                  const ChunkConst cc = chunk_const(A, cell_l);
                  gen_ray(R, e.id, cc, H, A);
                  lam_l = cc.lam;
                  inv_lam_l = cc.inv_lam;
                  li_l = cc.li;
                  has = true;
                }
              } else {
                gen_ray(R, u_next + rank, ucc, H, A);
                cell_l = u_cell;
                lam_l = ucc.lam;
                inv_lam_l = ucc.inv_lam;
                li_l = ucc.li;
                has = true;
              }
              if (has) {
                seg_s = make_float2(1.f, 0.f);
                seg_p = make_float2(1.f, 0.f);
                ++c_rays;
              }
            }
            u_next += take;
            fm = __ballot_sync(FULL, !has && emit == 0);
          }
          const bool adv = has && !at_mir;
          // leave for the mirror step when no lane can advance, unless
          // waiting lanes are left with no live ray in the warp: their sweep
          // runs first (below; every pass either advances a ray or empties
          // the waiting lanes)
          if (!__any_sync(FULL, adv) && !(__any_sync(FULL, emit > 0) && !__any_sync(FULL, has))) break;
          Outcome o;
          o.term = 0;
          if (adv) {
            float t;
            const int sid = next_surface<GM>(B, R.p, R.d, R.last, R.reg, t);
            ++R.ev;
            if (sid < 0) {
              o.term = 1;
              o.cat = L_ABSORBED;
            } else {
              R.p = v3(fmaf(t, R.d.x, R.p.x), fmaf(t, R.d.y, R.p.y), fmaf(t, R.d.z, R.p.z));
              R.last = sid;
              if (sid >= S_MIR) {
                at_mir = true;
                hit_k = sid - S_MIR;
              } else {
                int dummy = 0;
                o = face_event<F>(R, sid, H, A, &seg_s, &seg_p, dummy);
              }
            }
            if (!o.term && !at_mir && R.ev >= A.max_events) {
              o.term = 1;
              o.cat = L_TRUNCATED;
            }
            if (o.term) {
              has = false;
              c_hits += R.hits;
              if (o.cat == L_EYEBOX) {
                const double g = A.G[cell_l * A.bins + o.bin];
                if (g != 0.0) {
                  if (R.hits <= TAPE_HITS) {
                    emit = R.hits;
                    g0 = (float)frexp(g, &eG);  // mantissa in [0.5, 1), exponent eG
                    x_Ts = o.Ts;
                    x_Tp = o.Tp;
                  } else {
                    ++c_overflow;
                  }
                }
                ++c_tallied;
              }
            }
          }
          // the reverse sweeps run for the waiting lanes together: once
          // kSweepMin wait, or when no live ray is left in the warp (the
          // sweep of one or two lanes at a time left the rest of the warp idle)
          const unsigned wm = __ballot_sync(FULL, emit > 0);
          if (!wm || (__popc(wm) < kSweepMin && __any_sync(FULL, has))) continue;
          // warp-aggregated reservation of record slots in the global buffer
          int incl = emit;
#pragma unroll
          for (int off = 1; off < 32; off <<= 1) {
            const int v = __shfl_up_sync(FULL, incl, off);
            if (lane >= off) incl += v;
          }
          const int total = __shfl_sync(FULL, incl, 31);
          if (total) {
            unsigned long long base = 0;
            if (lane == 31) base = atomicAdd(A.hit_count, (unsigned long long)total);
            base = __shfl_sync(FULL, base, 31);
            if constexpr (T) {
              // one head per ray whose records fit (warp-aggregated slot)
              const long long f0 = (long long)base + incl - emit;
              const bool ok = emit > 0 && f0 + emit <= cap;
              const unsigned hm = __ballot_sync(FULL, ok);
              unsigned long long hb0 = 0;
              if (lane == 0) hb0 = atomicAdd(A.head_count, (unsigned long long)__popc(hm));
              hb0 = __shfl_sync(FULL, hb0, 0);
              if (ok) {
                const long long hi = (long long)hb0 + __popc(hm & lt_mask);
                if (hi < A.head_cap) {
                  RayHead rh;
                  rh.id = R.id;
                  rh.cell = (int)cell_l;
                  rh.first = (int)f0;
                  rh.emit = emit;
                  rh.events = R.ev;
                  A.ray_heads[hi] = rh;
                }
              }
            }
            if (emit) {
              const long long first = (long long)base + incl - emit;
              if (first + emit > cap) {
                // no room: drop this ray's gradient and mark its slots inside the buffer
                for (long long h = first; h < first + emit && h < cap; ++h) hb[h].kfw = -1;
                ++c_overflow;
              } else {
                // reverse Jones sweep over the tape
                const float sc = g0 * (1.0f / F);
                float2 ga[F], gb[F];
#pragma unroll
                for (int f = 0; f < F; ++f) {
                  ga[f] = cmulc(seg_s, cscale(R.a[f], sc * x_Ts));
                  gb[f] = cmulc(seg_p, cscale(R.b[f], sc * x_Tp));
                }
                for (int h = emit - 1; h >= 0; --h) {
                  const TapeE<F, ACC>& E = tape[h];
                  float2 gs[F], gp[F];
                  float2 As = make_float2(0.f, 0.f), Ap = make_float2(0.f, 0.f);
                  const int k = E.kfw & 0xff;
                  const bool refl = ((E.kfw >> 9) & 1) == 0;  // bit 9: 0 = reflected (r), 1 = transmitted (t)
                  const float scl = refl ? B.mir[k].isw : B.mir[k].is1w;
#pragma unroll
                  for (int f = 0; f < F; ++f) {
                    gs[f] = make_float2(fmaf(E.cpsi, ga[f].x, -E.spsi * gb[f].x), fmaf(E.cpsi, ga[f].y, -E.spsi * gb[f].y));
                    gp[f] = make_float2(fmaf(E.spsi, ga[f].x, E.cpsi * gb[f].x), fmaf(E.spsi, ga[f].y, E.cpsi * gb[f].y));
                    As = cadd(As, cmulc(gs[f], E.Es[f]));
                    Ap = cadd(Ap, cmulc(gp[f], E.Ep[f]));
                  }
                  double g_cos = 0.0;  // dL/d(cos t0) of the hit through its coating (table mode)
                  if (A.lut) {
                    // two-stage adjoint: dL/dc of the hit goes to the two table
                    // entries it interpolated, with the interpolation weights
                    int j;
                    float f;
                    lut_locate(A, E.cos0, j, f);
                    const bool front = (E.kfw >> 8) & 1;
                    const long long e = lut_entry(A, k, front, li_l, j);
                    // FP32 relative to the ray's exponent of dL/dtally; one exact
                    // power of two turns each value into FP64 for the sums
                    const double p2 = pow2d(eG);
                    const float2 gs_ = cscale(As, scl), gp_ = cscale(Ap, scl);
                    const float gq[4] = {gs_.x, gs_.y, gp_.x, gp_.y};
                    double* g0 = A.lut_grad + 8 * e + (refl ? 0 : 4);
                    const float w0 = 1.0f - f, w1 = f;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                      if (gq[q] != 0.0f) {
                        if (w0 != 0.0f) atomicAdd(g0 + q, (double)(w0 * gq[q]) * p2);
                        if (w1 != 0.0f) atomicAdd(g0 + 8 + q, (double)(w1 * gq[q]) * p2);
                      }
                    }
                    if constexpr (T) {
                      // d/d(cos t0) of the coefficients: the tabulated exact
                      // derivatives, interpolated like the values
                      const float4* t4 = A.lut + 4 * e + 2 + (refl ? 0 : 1);
                      const float4 a = __ldg(t4), b = __ldg(t4 + 4);
                      const float2 ds = make_float2(fmaf(f, b.x - a.x, a.x), fmaf(f, b.y - a.y, a.y));
                      const float2 dp = make_float2(fmaf(f, b.z - a.z, a.z), fmaf(f, b.w - a.w, a.w));
                      g_cos = (double)(2.0f * (cmul(gs_, ds).x + cmul(gp_, dp).x)) * p2;
                    }
                  } else {
                    HitRec rec;
                    rec.kfw = E.kfw | (li_l << 10);
                    rec.cos0 = E.cos0;
                    rec.cos0l = E.cos0l();
                    rec.eA = eG;
                    rec.As = cscale(As, scl);
                    rec.Ap = cscale(Ap, scl);
                    hb[first + h] = rec;
                  }
                  if constexpr (T) {
                    TiltAux ta;
                    ta.cs = E.cs;
                    ta.cp = E.cp;
                    ta.g_cos = g_cos;  // exact mode: set by the adjoint kernel
                    A.tilt_aux[first + h] = ta;
                  }
#pragma unroll
                  for (int f = 0; f < F; ++f) {
                    const float2 xs = cmulc(E.cs, gs[f]), xp = cmulc(E.cp, gp[f]);
                    const float2 ya = make_float2(fmaf(E.cphi, xs.x, -E.sphi * xp.x), fmaf(E.cphi, xs.y, -E.sphi * xp.y));
                    const float2 yb = make_float2(fmaf(E.sphi, xs.x, E.cphi * xp.x), fmaf(E.sphi, xs.y, E.cphi * xp.y));
                    ga[f] = cmulc(E.seg_s, ya);
                    gb[f] = cmulc(E.seg_p, yb);
                  }
                }
              }
            }
          }
          emit = 0;  // swept: the lane takes a new ray
        }
        if (!__any_sync(FULL, at_mir)) break;  // no ray left in this warp and no unit to claim
        if (at_mir) {
          const int h = R.hits;
          float2 Es[F], Ep[F];
          const MirrorStep ms = mirror_event<F, P, 2, ACC>(R, hit_k, B, lam_l, inv_lam_l, li_l, A, c_steps, Es, Ep);
          if (h < TAPE_HITS) {
            TapeE<F, ACC>& E = tape[h];
            E.cs = ms.cs;
            E.cp = ms.cp;
#pragma unroll
            for (int f = 0; f < F; ++f) {
              E.Es[f] = Es[f];
              E.Ep[f] = Ep[f];
            }
            E.cphi = ms.cphi;
            E.sphi = ms.sphi;
            E.cpsi = ms.cpsi;
            E.spsi = ms.spsi;
            E.seg_s = seg_s;
            E.seg_p = seg_p;
            E.cos0 = ms.cos0;
            E.set_cos0l(ms.cos0l);
            E.kfw = hit_k | (ms.front << 8) | ((ms.refl ? 0 : 1) << 9);
          }
          seg_s = make_float2(1.f, 0.f);
          seg_p = make_float2(1.f, 0.f);
          at_mir = false;
          if (R.ev >= A.max_events) {
            has = false;
            c_hits += R.hits;
          }
        }
  }
  __syncthreads();
  const unsigned long long cv[5] = {(unsigned long long)c_rays, (unsigned long long)c_hits, 0ull, 0ull,
                                    (unsigned long long)c_steps};
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const unsigned long long v = warp_sum_u(cv[i]);
    if (lane == 0 && v) atomicAdd(&s_cnt[i], v);
  }
  const unsigned long long ov = warp_sum_u((unsigned long long)c_overflow);
  const unsigned long long tl = warp_sum_u((unsigned long long)c_tallied);
  if (lane == 0) {
    if (ov) atomicAdd(&s_cnt[5], ov);
    if (tl) atomicAdd(&s_cnt[6], tl);
  }
  __syncthreads();
  if (tid < 7 && s_cnt[tid]) atomicAdd(A.counters + tid, s_cnt[tid]);
}

// ---------------------------------------------------------------------------
// K3b: mirror-tilt gradient, split in two parts along the sampled path.
// (1) Through the coatings: the thin-film adjoint kernel, whose first sweep
//     also runs the dual layer chain, forms g = dL/d(cos theta_0) of every
//     hit record from its weights A (TiltAux); here g times the tangent of
//     cos(theta_0) of that hit.
// (2) Everything else with the coefficients held at their values: the
//     reflected directions, the mirror and face s/p bases, the TIR phases and
//     the exit transmittances. k_tilt_grad re-traces each ray that produced
//     records (RayHead) with the forward's geometry, reads the applied
//     coefficients of its hits from TiltAux (no layer chain), and carries
//     tangents of its direction and field with respect to the tilts of up to
//     kTiltPass mirrors (per lane in shared memory, word w of tangent t at
//     col[(t * W + w) * 32]). At the eyebox exit G[bin] dI/d(tilt) is added.
// Sums are FP64 per lane in shared memory, reported per degree.
// ---------------------------------------------------------------------------
constexpr int kTiltPass = 8;
constexpr int kTiltBlock = 128;

template <int F>
__device__ __forceinline__ float& tan_w(float* col, int t, int w) {
  return col[(t * (3 + 4 * F) + w) * 32];
}

// mirror_event with tangents: the same geometry and decision as the
// forward, the coefficients as the replay applied them
// live: bit t set once the ray has hit mirror k0 + t (every other tangent is
// still zero, and its column is not touched)
template <int F, bool ACC>
__device__ void mirror_event_tilt(Ray<F>& R, int k, const Blob& B, const TraceArgs& A, int k0, int nk, float* col,
                                  double* acc, const TiltAux& X, unsigned& live) {
  const MirrorRec& M = B.mir[k];
  const V3 N = v3(M.nx, M.ny, M.nz);
  const V3 dN = cross3(v3(M.ax, M.ay, M.az), N);  // dN/d(tilt) per radian
  F2 cdf{0.0f, 0.0f};
  if constexpr (ACC) cdf = dot3_df(R.d, R.dl, N, v3(M.nlx, M.nly, M.nlz));
  const float cd = ACC ? cdf.h : dot3(R.d, N);
  const bool front = cd < 0.0f;
  const float2 cs = X.cs, cp = X.cp;
  V3 sf, pf;
  face_basis(R.d, sf, pf);
  const V3 w = cross3(R.d, N);
  const float sm2 = dot3(w, w);
  const bool degen = !(sm2 > 1e-24f);
  V3 sm = sf;
  if (!degen) {
    const float r = rsqrtf(sm2);
    sm = v3(w.x * r, w.y * r, w.z * r);
  }
  const float cphi = dot3(sf, sm), sphi = dot3(pf, sm);
  const int m = R.hits;
  const uint4 rnd = philox10(
      make_uint4((uint32_t)R.id, (uint32_t)((unsigned long long)R.id >> 32), (uint32_t)(m >> 2), TAG_EVT), A.key0,
      A.key1);
  const uint32_t word = (m & 3) == 0 ? rnd.x : (m & 3) == 1 ? rnd.y : (m & 3) == 2 ? rnd.z : rnd.w;
  const bool refl = u24(word) < M.omega;
  V3 d2 = R.d, dl2 = R.dl;  // the same direction update as mirror_event (same path)
  if (refl) {
    if constexpr (ACC) {
      reflect_df(d2, dl2, N, v3(M.nlx, M.nly, M.nlz), cdf);
    } else {
      d2 = v3(fmaf(-2.0f * cd, N.x, R.d.x), fmaf(-2.0f * cd, N.y, R.d.y), fmaf(-2.0f * cd, N.z, R.d.z));
    }
  }
  const V3 pm2 = cross3(sm, d2);
  V3 sf2, pf2;
  face_basis(d2, sf2, pf2);
  const float cpsi = dot3(sf2, sm), spsi = dot3(sf2, pm2);
  const int to = k - k0;
  if (to >= 0 && to < nk && !((live >> to) & 1u)) {
    for (int w = 0; w < 3 + 4 * F; ++w) tan_w<F>(col, to, w) = 0.0f;
    live |= 1u << to;
  }
  // tangents (the field before the hit is still in R). The field tangent is
  // carried as the projections of dE on the current face basis,
  // (dE.s, dE.p): then only the mirror basis is differentiated here, never
  // the face basis, whose azimuth turns at a rate ~1/h for a direction near
  // the face normal (the out-coupled ray of the 0 deg field).
  for (unsigned lm = live; lm; lm &= lm - 1) {
    const int t = __ffs(lm) - 1;
    const bool own = t == to;
    const V3 dd = v3(tan_w<F>(col, t, 0), tan_w<F>(col, t, 1), tan_w<F>(col, t, 2));
    const V3 dNt = own ? dN : v3(0.0f, 0.0f, 0.0f);
    const float dcd = dot3(dd, N) + dot3(R.d, dNt);
    acc[t * 32] += X.g_cos * (double)(front ? -dcd : dcd);  // part (1)
    V3 dsm;
    if (!degen) {
      const V3 a = cross3(dd, N), b = cross3(R.d, dNt);
      dsm = normalize_d(w, v3(a.x + b.x, a.y + b.y, a.z + b.z));
    } else {
      V3 dpf;
      face_basis_d(R.d, dd, sf, dsm, dpf);  // normal incidence: the mirror basis is the face basis
    }
    const V3 u1 = cross3(dsm, R.d), u2 = cross3(sm, dd);
    const V3 dpm = v3(u1.x + u2.x, u1.y + u2.y, u1.z + u2.z);
    V3 dd2 = dd;
    if (refl)
      dd2 = v3(dd.x - 2.0f * fmaf(dcd, N.x, cd * dNt.x), dd.y - 2.0f * fmaf(dcd, N.y, cd * dNt.y),
               dd.z - 2.0f * fmaf(dcd, N.z, cd * dNt.z));
    const V3 e1 = cross3(dsm, d2), e2 = cross3(sm, dd2);
    const V3 dpm2 = v3(e1.x + e2.x, e1.y + e2.y, e1.z + e2.z);
    const float qs = dot3(sf, dsm), qp = dot3(pf, dsm), rs_ = dot3(sf, dpm), rp_ = dot3(pf, dpm);
    const float us = dot3(dsm, sf2), up = dot3(dsm, pf2), vs = dot3(dpm2, sf2), vp = dot3(dpm2, pf2);
#pragma unroll
    for (int f = 0; f < F; ++f) {
      const float2 a = R.a[f], b = R.b[f];
      const float2 xa = make_float2(tan_w<F>(col, t, 3 + 4 * f), tan_w<F>(col, t, 4 + 4 * f));
      const float2 xb = make_float2(tan_w<F>(col, t, 5 + 4 * f), tan_w<F>(col, t, 6 + 4 * f));
      const float2 Es = make_float2(fmaf(cphi, a.x, sphi * b.x), fmaf(cphi, a.y, sphi * b.y));
      const float2 Ep = make_float2(fmaf(-sphi, a.x, cphi * b.x), fmaf(-sphi, a.y, cphi * b.y));
      // d(E.sm) and d(E.pm) of the incoming field
      const float2 dEs = make_float2(cphi * xa.x + sphi * xb.x + qs * a.x + qp * b.x,
                                     cphi * xa.y + sphi * xb.y + qs * a.y + qp * b.y);
      const float2 dEp = make_float2(-sphi * xa.x + cphi * xb.x + rs_ * a.x + rp_ * b.x,
                                     -sphi * xa.y + cphi * xb.y + rs_ * a.y + rp_ * b.y);
      const float2 Os = cmul(cs, Es), Op = cmul(cp, Ep);
      const float2 dOs = cmul(cs, dEs), dOp = cmul(cp, dEp);  // part (2): coefficients held
      // dE' = dOs sm + dOp pm2 + Os dsm + Op dpm2, projected on (sf2, pf2)
      tan_w<F>(col, t, 3 + 4 * f) = cpsi * dOs.x + spsi * dOp.x + us * Os.x + vs * Op.x;
      tan_w<F>(col, t, 4 + 4 * f) = cpsi * dOs.y + spsi * dOp.y + us * Os.y + vs * Op.y;
      tan_w<F>(col, t, 5 + 4 * f) = -spsi * dOs.x + cpsi * dOp.x + up * Os.x + vp * Op.x;
      tan_w<F>(col, t, 6 + 4 * f) = -spsi * dOs.y + cpsi * dOp.y + up * Os.y + vp * Op.y;
    }
    tan_w<F>(col, t, 0) = dd2.x;
    tan_w<F>(col, t, 1) = dd2.y;
    tan_w<F>(col, t, 2) = dd2.z;
  }
  // values (as mirror_event)
#pragma unroll
  for (int f = 0; f < F; ++f) {
    const float2 Es = make_float2(fmaf(cphi, R.a[f].x, sphi * R.b[f].x), fmaf(cphi, R.a[f].y, sphi * R.b[f].y));
    const float2 Ep = make_float2(fmaf(-sphi, R.a[f].x, cphi * R.b[f].x), fmaf(-sphi, R.a[f].y, cphi * R.b[f].y));
    const float2 Os = cmul(cs, Es), Op = cmul(cp, Ep);
    R.a[f] = make_float2(fmaf(cpsi, Os.x, spsi * Op.x), fmaf(cpsi, Os.y, spsi * Op.y));
    R.b[f] = make_float2(fmaf(-spsi, Os.x, cpsi * Op.x), fmaf(-spsi, Os.y, cpsi * Op.y));
  }
  R.d = d2;
  R.dl = dl2;
  R.reg = region_after(B, R.reg, k, d2);
  R.hash = fnv(R.hash, (uint32_t)(S_MIR + k) | (refl ? 0x80u : 0u));
  R.hits = m + 1;
}

template <int F, int GM, bool ACC>
__global__ void __launch_bounds__(kTiltBlock) k_tilt_grad(const TraceArgs A) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ __align__(8) uint64_t s_mbar;
  constexpr int W = 3 + 4 * F;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* acc = reinterpret_cast<double*>(smem + A.blob_bytes) + warp * (kTiltPass * 32) + lane;
  float* col = reinterpret_cast<float*>(smem + A.blob_bytes + sizeof(double) * (kTiltBlock / 32) * kTiltPass * 32) +
               warp * (kTiltPass * W * 32) + lane;
  if (!stage_blob(smem, A.blob, A.blob_bytes, &s_mbar, A.error, wait_limit(A.wait_ns))) return;
  Blob B;
  B.bind(smem);
  const BlobHeader& H = *B.h;
  const int k0 = A.tilt_k0, nk = min(kTiltPass, H.n_mir - k0);
  for (int t = 0; t < kTiltPass; ++t) acc[t * 32] = 0.0;
  const float n = H.n_slab;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < A.n_heads;
       i += (long long)gridDim.x * blockDim.x) {
    const RayHead rh = A.ray_heads[i];
    const long long cell = rh.cell;
    const ChunkConst cc = chunk_const(A, cell);
    Ray<F> R;
    gen_ray(R, rh.id, cc, H, A);
    unsigned live = 0u;
    for (;;) {
      float tt;
      const int sid = next_surface<GM>(B, R.p, R.d, R.last, R.reg, tt);
      ++R.ev;
      if (sid < 0) break;
      R.p = v3(fmaf(tt, R.d.x, R.p.x), fmaf(tt, R.d.y, R.p.y), fmaf(tt, R.d.z, R.p.z));
      R.last = sid;
      if (sid >= S_MIR) {
        if (R.hits >= rh.emit) {  // more hits than the replay recorded: not the replayed path
          atomicOr(A.error, 8u);
          break;
        }
        const TiltAux X = A.tilt_aux[rh.first + R.hits];
        mirror_event_tilt<F, ACC>(R, sid - S_MIR, B, A, k0, nk, col, acc, X, live);
        if (R.ev >= A.max_events) break;
        continue;
      }
      const float dz0 = R.d.z;
      const V3 d0 = R.d;
      float2 a0[F], b0[F];
#pragma unroll
      for (int f = 0; f < F; ++f) {
        a0[f] = R.a[f];
        b0[f] = R.b[f];
      }
      int dummy = 0;
      const Outcome o = face_event<F>(R, sid, H, A, nullptr, nullptr, dummy);
      const float ci = fabsf(dz0), sg = dz0 < 0.0f ? -1.0f : 1.0f;
      if (!o.term) {  // TIR: d_z flipped, field times (r_s, r_p)(cos i)
        if (!live) {
          if (R.ev >= A.max_events) break;
          continue;
        }
        float2 rs, rp, drs, drp;
        tir_coef(n, ci, fmaf(-ci, ci, 1.0f), rs, rp);
        tir_coef_d(n, ci, rs, rp, drs, drp);
        const float2 rsp = cadd(rs, rp);
        // TIR needs sin(i) > 1/n: the face basis is well conditioned here
        const float ih2 = 1.0f / fmaf(d0.x, d0.x, d0.y * d0.y);
        for (unsigned lm = live; lm; lm &= lm - 1) {
          const int t = __ffs(lm) - 1;
          const float ddx = tan_w<F>(col, t, 0), ddy = tan_w<F>(col, t, 1), ddz = tan_w<F>(col, t, 2);
          const float dci = sg * ddz;
          // the face basis turns about d at om = p . ds = -d_z dpsi; in
          // projections the TIR map gains (r_s + r_p) om terms
          const float om = -dz0 * fmaf(d0.x, ddy, -d0.y * ddx) * ih2;
          tan_w<F>(col, t, 2) = -ddz;
#pragma unroll
          for (int f = 0; f < F; ++f) {
            const float2 da = make_float2(tan_w<F>(col, t, 3 + 4 * f), tan_w<F>(col, t, 4 + 4 * f));
            const float2 db = make_float2(tan_w<F>(col, t, 5 + 4 * f), tan_w<F>(col, t, 6 + 4 * f));
            const float2 na =
                cadd(cadd(cmul(rs, da), cscale(cmul(drs, a0[f]), dci)), cscale(cmul(rsp, b0[f]), om));
            const float2 nb =
                csub(cadd(cmul(rp, db), cscale(cmul(drp, b0[f]), dci)), cscale(cmul(rsp, a0[f]), om));
            tan_w<F>(col, t, 3 + 4 * f) = na.x;
            tan_w<F>(col, t, 4 + 4 * f) = na.y;
            tan_w<F>(col, t, 5 + 4 * f) = nb.x;
            tan_w<F>(col, t, 6 + 4 * f) = nb.y;
          }
        }
        if (R.ev >= A.max_events) break;
        continue;
      }
      if (o.cat == L_EYEBOX) {  // dI = (dT_s |a|^2 + 2 T_s Re(a* da) + ...) / F
        if (R.hits != rh.emit) {
          atomicOr(A.error, 8u);
          break;
        }
        const double g = A.G[cell * A.bins + o.bin];
        float dTs, dTp;
        exit_T_d(n, ci, dTs, dTp);
        // om (T_s - T_p), the turn of the face basis times the s/p contrast:
        // T_s - T_p = -4 n c_i c_t (n^2 - 1)^2 h^2 / ((n c_i + c_t)^2 (c_i + n c_t)^2)
        // and om = -d_z (d_x dd_y - d_y dd_x) / h^2, so h^2 cancels and the
        // term stays exact for a ray leaving along the normal
        const float ct = sqrtf(fmaxf(1.0f - n * n * fmaf(-ci, ci, 1.0f), 0.0f));
        const float q1 = fmaf(n, ci, ct), q2 = fmaf(n, ct, ci), nn1 = fmaf(n, n, -1.0f);
        const float kx = 4.0f * n * ci * ct * nn1 * nn1 / (q1 * q1 * q2 * q2);
        for (unsigned lm = live; lm; lm &= lm - 1) {
          const int t = __ffs(lm) - 1;
          const float ddx = tan_w<F>(col, t, 0), ddy = tan_w<F>(col, t, 1);
          const float dci = sg * tan_w<F>(col, t, 2);
          const float wdt = dz0 * fmaf(d0.x, ddy, -d0.y * ddx) * kx;
          float dI = 0.0f;
#pragma unroll
          for (int f = 0; f < F; ++f) {
            const float2 da = make_float2(tan_w<F>(col, t, 3 + 4 * f), tan_w<F>(col, t, 4 + 4 * f));
            const float2 db = make_float2(tan_w<F>(col, t, 5 + 4 * f), tan_w<F>(col, t, 6 + 4 * f));
            dI += dTs * dci * cabs2(R.a[f]) + 2.0f * o.Ts * fmaf(R.a[f].x, da.x, R.a[f].y * da.y);
            dI += dTp * dci * cabs2(R.b[f]) + 2.0f * o.Tp * fmaf(R.b[f].x, db.x, R.b[f].y * db.y);
            dI += 2.0f * wdt * fmaf(R.a[f].x, R.b[f].x, R.a[f].y * R.b[f].y);
          }
          acc[t * 32] += g * (double)(dI * (1.0f / F));
        }
      }
      break;
    }
  }
  const double per_degree = 3.14159265358979323846 / 180.0;
  for (int t = 0; t < nk; ++t) {
    double v = acc[t * 32];
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    if (lane == 0 && v != 0.0) atomicAdd(A.grad_tilt + k0 + t, v * per_degree);
  }
}

// Gradient terms of one record per lane, a segment (up to 8 layers) at a
// time. When all 32 lanes hold records of the same stack (uniform, a
// warp-uniform flag) their terms go to the same layers: summed across the
// warp with one transposing reduction per segment and added once per layer;
// else added per lane. Non-finite sums are counted (wg_stats) and not added.
struct GradSink {
  float* s_grad;
  int* bad;
  int lane;
  bool uniform;
  __device__ __forceinline__ void segment(const float (&t)[8], int n, int i0, int di) const {
    if (uniform) {
      const float r = warp_transpose_sum8(t, lane);
      const int u = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
      if ((lane & 3) == 0 && u < n) {
        if (isfinite(r)) {
          atomicAdd(s_grad + i0 + u * di, r);
        } else {
          ++*bad;
        }
      }
    } else {
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (u < n) {
          if (!isfinite(t[u])) {
            ++*bad;
          } else if (t[u] != 0.f) {
            atomicAdd(s_grad + i0 + u * di, t[u]);
          }
        }
    }
  }
};

// shared memory of the adjoint kernel: blob | per-layer FP32 sums (padded
// to 32 floats) | per-warp segment buffers
template <int P>
static size_t adj_smem_bytes_p(int blob_bytes, int n_layers) {
  return (size_t)blob_bytes + sizeof(float) * (size_t)((std::max(1, n_layers) + 31) & ~31) +
         sizeof(float) * (size_t)(kBlock / 32) * (size_t)seg_floats_per_warp<P>();
}
// T: also dL/d(cos t0) of every record through its coating (the tilt
// gradient's coating term), written to A.tilt_aux[A.perm[i]].g_cos
template <int P, bool T, bool ACC>
__global__ void __launch_bounds__(kBlock, 2) k_bwd_adjoint(const AdjArgs A) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ __align__(8) uint64_t s_mbar;
  __shared__ long long s_chunk;
  __shared__ unsigned long long s_cnt[2];
  float* s_grad = reinterpret_cast<float*>(smem + A.blob_bytes);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  // (8-byte aligned: the blob's size is a multiple of 16 bytes, the other offsets even)
  float2* seg = reinterpret_cast<float2*>(s_grad + ((max(1, A.n_layers) + 31) & ~31) + warp * seg_floats_per_warp<P>()) +
                lane;
  if (tid < 2) s_cnt[tid] = 0ull;
  if (!stage_blob(smem, A.blob, A.blob_bytes, &s_mbar, A.error, wait_limit(A.wait_ns))) return;
  Blob B;
  B.bind(smem);
  const BlobHeader& H = *B.h;
  for (int i = tid; i < A.n_layers; i += blockDim.x) s_grad[i] = 0.f;
  long long c_steps = 0;
  int bad = 0;
  for (;;) {
    if (tid == 0) s_chunk = (long long)atomicAdd(A.work, 1ull);
    __syncthreads();
    const long long base = s_chunk * (long long)A.rec_chunk;
    if (base >= A.n_rec) break;
    const long long end = min(base + (long long)A.rec_chunk, A.n_rec);
    for (long long r0 = base + 32ll * warp; r0 < end; r0 += 32ll * nwarp) {
      const long long i = r0 + lane;
      const bool valid = i < end;
      HitRec rec;
      rec.kfw = -1;
      if (valid) rec = A.recs[i];
      const int key = valid ? stack_key(rec.kfw) : -1 - lane;
      const int key0 = __shfl_sync(FULL, key, 0);
      const bool uniform = __all_sync(FULL, key == key0);
      if (valid) {
        const int k = rec.kfw & 0xff;
        const bool front = (rec.kfw >> 8) & 1;
        const int which = (rec.kfw >> 9) & 1;
        const MirrorRec& M = B.mir[k];
        const StackView sv{B.d, B.m, M.store_off, M.n_layers, M.store_off - M.layer_off};
        const float lam = __ldg(A.lambda + kfw_lam(rec.kfw));
        // a periodic stack's slots evaluated directly; a general stack's table
        MatTable mt;
        MatK kb[P > 0 ? P : 1];
        if constexpr (P > 0) {
          slot_consts<P, ACC>(H, sv, front, rec.cos0, rec.cos0l, lam, 1.0f / lam, kb);
        } else {
          mt.init_sel<ACC>(H, rec.cos0, rec.cos0l, lam);
        }
        const MatK* slots = P > 0 ? kb : nullptr;
        GradSink sink{s_grad, &bad, lane, uniform};
        if constexpr (T) {
          TiltTable tt;
          tt.init(H, rec.cos0);
          float g = 0.f;
          tmm_adjoint<P, GradSink, true, ACC>(sv, front, mt, H.n_slab, rec.cos0, rec.As, rec.Ap, which, sink, seg,
                                              rec.eA, &tt, &g, slots);
          A.tilt_aux[A.perm[i]].g_cos = (double)g * pow2d(rec.eA);
        } else {
          tmm_adjoint<P, GradSink, false, ACC>(sv, front, mt, H.n_slab, rec.cos0, rec.As, rec.Ap, which, sink, seg,
                                               rec.eA, nullptr, nullptr, slots);
        }
        c_steps += M.n_layers;
      }
    }
    __syncthreads();
    for (int i = tid; i < A.n_layers; i += blockDim.x) {
      const float v = s_grad[i];
      if (v != 0.f) {
        atomicAdd(A.grad_acc + i, (double)v);
        s_grad[i] = 0.f;
      }
    }
    __syncthreads();
  }
  const unsigned long long st = warp_sum_u((unsigned long long)c_steps);
  const unsigned long long bd = warp_sum_u((unsigned long long)bad);
  if (lane == 0) {
    if (st) atomicAdd(&s_cnt[0], st);
    if (bd) atomicAdd(&s_cnt[1], bd);
  }
  __syncthreads();
  if (tid == 0 && s_cnt[0]) atomicAdd(A.counters + 7, s_cnt[0]);
  if (tid == 1 && s_cnt[1]) atomicAdd(A.counters + 8, s_cnt[1]);
}

// ---------------------------------------------------------------------------
// K1: coating evaluation and its adjoint (test hooks, global-memory stack)
// ---------------------------------------------------------------------------
// Coating look-up table: one thread per (mirror, side, wavelength, bin j),
// the raw coefficients at cos_j = c0 + j dc and their derivatives d/d(cos t0)
// from the dual layer chain (entry layout as TraceArgs::lut)
template <int P, bool ACC>
__global__ void k_lut_build(const uint8_t* blob, int n_mir, int n_lam, const float* lam, int n, float c0, float dc,
                            float4* out) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long total = (long long)n_mir * 2 * n_lam * n;
  if (i >= total) return;
  const int j = (int)(i % n);
  const long long q = i / n;
  const int li = (int)(q % n_lam);
  const int side = (int)((q / n_lam) % 2);
  const int k = (int)(q / (2ll * n_lam));
  Blob B;
  B.bind(blob);
  const BlobHeader& H = *B.h;
  const MirrorRec& M = B.mir[k];
  const float c = fmaf((float)j, dc, c0);
  MatTable mt;
  mt.init_sel<ACC>(H, c, 0.0f, lam[li]);
  MatTableD mtd;
  mtd.init(H, c, lam[li], mt);
  const StackView sv{B.d, B.m, M.store_off, M.n_layers, M.store_off - M.layer_off};
  Coef cf, dcf;
  tmm_forward_dual<P, ACC>(sv, side == 0, mt, mtd, H.n_slab, c, cf, dcf);
  out[4 * i] = make_float4(cf.rs.x, cf.rs.y, cf.rp.x, cf.rp.y);
  out[4 * i + 1] = make_float4(cf.ts.x, cf.ts.y, cf.tp.x, cf.tp.y);
  out[4 * i + 2] = make_float4(dcf.rs.x, dcf.rs.y, dcf.rp.x, dcf.rp.y);
  out[4 * i + 3] = make_float4(dcf.ts.x, dcf.ts.y, dcf.tp.x, dcf.tp.y);
}

template <int P, bool ACC>
__global__ void k_coating_eval(const uint8_t* blob, int mirror, int side, long long n, const float* cos0,
                               const float* lam, float* out) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  Blob B;
  B.bind(blob);
  const BlobHeader& H = *B.h;
  const MirrorRec& M = B.mir[mirror];
  MatTable mt;
  mt.init_sel<ACC>(H, cos0[i], 0.0f, lam[i]);
  const StackView sv{B.d, B.m, M.store_off, M.n_layers, M.store_off - M.layer_off};
  int steps = 0;
  const Coef c = tmm_forward<P, ACC>(sv, side == 0, mt, H.n_slab, cos0[i], steps);
  float* o = out + i * 8;
  o[0] = c.rs.x;
  o[1] = c.rs.y;
  o[2] = c.rp.x;
  o[3] = c.rp.y;
  o[4] = c.ts.x;
  o[5] = c.ts.y;
  o[6] = c.tp.x;
  o[7] = c.tp.y;
}

struct RowSink {
  float* row;
  int off, L;
  bool front;
  __device__ __forceinline__ void segment(const float (&t)[8], int n, int i0, int di) const {
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (u < n) {
        const int idx = i0 + u * di;
        row[front ? idx - off : off + L - 1 - idx] = t[u];
      }
  }
};

template <int P, bool ACC>
__global__ void __launch_bounds__(128) k_coating_grad(const uint8_t* blob, int mirror, int side, long long n,
                                                       const float* cos0, const float* lam, const float* w, int which,
                                                       float* grad) {
  __shared__ __align__(16) float s_seg[4 * seg_floats_per_warp<P>()];
  float2* seg = reinterpret_cast<float2*>(s_seg + (threadIdx.x >> 5) * seg_floats_per_warp<P>()) + (threadIdx.x & 31);
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  Blob B;
  B.bind(blob);
  const BlobHeader& H = *B.h;
  const MirrorRec& M = B.mir[mirror];
  MatTable mt;
  mt.init_sel<ACC>(H, cos0[i], 0.0f, lam[i]);
  const StackView sv{B.d, B.m, M.store_off, M.n_layers, M.store_off - M.layer_off};
  RowSink sink{grad + i * M.n_layers, M.layer_off, M.n_layers, side == 0};
  tmm_adjoint<P, RowSink, false, ACC>(sv, side == 0, mt, H.n_slab, cos0[i], make_float2(w[4 * i], w[4 * i + 1]),
                 make_float2(w[4 * i + 2], w[4 * i + 3]), which, sink, seg);
}

struct NullSink {
  __device__ __forceinline__ void segment(const float (&)[8], int, int, int) const {}
};

// d f / d(cos theta_0) of single coatings (test hook of the adjoint's dual sweep)
template <int P, bool ACC>
__global__ void __launch_bounds__(128) k_coating_dcos(const uint8_t* blob, int mirror, int side, long long n,
                                                       const float* cos0, const float* lam, const float* w, int which,
                                                       float* out) {
  __shared__ __align__(16) float s_seg[4 * seg_floats_per_warp<P>()];
  float2* seg = reinterpret_cast<float2*>(s_seg + (threadIdx.x >> 5) * seg_floats_per_warp<P>()) + (threadIdx.x & 31);
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  Blob B;
  B.bind(blob);
  const BlobHeader& H = *B.h;
  const MirrorRec& M = B.mir[mirror];
  MatTable mt;
  mt.init_sel<ACC>(H, cos0[i], 0.0f, lam[i]);
  TiltTable tt;
  tt.init(H, cos0[i]);
  const StackView sv{B.d, B.m, M.store_off, M.n_layers, M.store_off - M.layer_off};
  NullSink sink;
  float g = 0.f;
  tmm_adjoint<P, NullSink, true, ACC>(sv, side == 0, mt, H.n_slab, cos0[i], make_float2(w[4 * i], w[4 * i + 1]),
                                       make_float2(w[4 * i + 2], w[4 * i + 3]), which, sink, seg, 0, &tt, &g);
  out[i] = g;
}

// Every kernel's dynamic shared memory limit is raised once to the device's
// opt-in maximum and never lowered: a limit set per launch to that launch's
// size would drop below what a CUDA graph captured earlier needs for the same
// kernel, and replaying that graph then crashed inside the driver's launch.
static inline int max_dyn_smem() {
  static int v[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return 227 * 1024;
  if (!v[dev]) {
    int x = 0;
    if (cudaDeviceGetAttribute(&x, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess || x <= 0) {
      cudaGetLastError();
      x = 227 * 1024;
    }
    v[dev] = x;
  }
  return v[dev];
}
// raises the kernel's limit to the opt-in maximum less its static shared
// memory (once: later calls find it there); errors are cleared, so they never
// reach the launch's status
template <class K>
static void raise_smem_limit(K kernel) {
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  const int want = max_dyn_smem() - (int)fa.sharedSizeBytes;
  if (fa.maxDynamicSharedSizeBytes < want &&
      cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, want) != cudaSuccess)
    cudaGetLastError();
}
template <class K>
static int occupancy(K kernel, size_t smem) {
  int n = 0;
  raise_smem_limit(kernel);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, kBlock, smem);
  return n;
}

}  // namespace wgk
