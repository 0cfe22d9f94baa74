// Device-side building blocks of the waveguide trace (sm_103a, FP32).
//
// Paper: "End-to-end differentiable design of geometric waveguide displays"
// (arXiv 2601.04370), Methods: Fresnel coefficients (Eq. 2), Airy / transfer
// matrices (Eq. 3 and Heavens' method), polarization ray tracing (Eq. 4),
// Monte Carlo reflect/transmit sampling with amplitude rescaling (Eq. 5).
//
// GB300 design choices (not the paper's):
//  * every layer's characteristic matrix is real-structured ([[c, i m12],
//    [i m21, c]] with real entries, also for evanescent layers); the stack
//    is applied to the substrate-side vector [1, eta]^T from the substrate
//    outwards (8 FMA-pipe ops per layer and polarization), which keeps FP32
//    accurate behind evanescent barriers where a left-to-right matrix
//    product loses the subdominant part;
//  * each layer's phase is reduced exactly to [-1/2, 1/2) turn before the
//    fast sin/cos;
//  * the field is kept as two complex coefficients in the slab-face s/p basis
//    of the current direction (s = d x z / |d x z|): a TIR bounce is then a
//    diagonal multiply; mirror hits rotate into the mirror's s/p basis and
//    back (same physics as Eq. 4's 3-vector form);
//  * the product is rescaled by exact powers of two every 8 layers (evanescent
//    layers grow like cosh), with the exponent tracked separately;
//  * the adjoint never inverts a layer matrix: it recomputes substrate-side
//    vectors from checkpoints taken every 8 layers.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace wgk {

constexpr int MAX_MAT = 4;
constexpr int MAX_MIR = 64;
constexpr int MAX_EVENTS = 128;
constexpr int TAPE_HITS = 128;  // = WG_MAX_EVENTS: a ray's mirror hits always fit
constexpr int CK = 8;                 // checkpoint stride (layers)
constexpr int MAX_LAYERS_MIRROR = 512;
constexpr int MAX_CK = MAX_LAYERS_MIRROR / 6 + 2;  // checkpoints at the shortest segment (6 layers)
// Zero-thickness layers stored before every stack and after the last one in
// the blob's thickness and material arrays (material 0): at least the longest
// segment minus one, so the steps of a stack's last segment that lie past its
// end read thickness 0, an exact identity step, with no test of the index.
constexpr int kStackPad = 8;
constexpr float TWO_PI = 6.283185307179586f;

enum { S_BOT = 0, S_TOP = 1, S_LEFT = 2, S_RIGHT = 3, S_YNEG = 4, S_YPOS = 5, S_MIR = 8 };
enum { L_EYEBOX = 0, L_MISSED = 1, L_EXIT_REFL = 2, L_LEAKED = 3, L_ABSORBED = 4, L_TRUNCATED = 5 };

// Philox counter tags ("GEN0", "EVT0")
constexpr uint32_t TAG_GEN = 0x47454E30u;
constexpr uint32_t TAG_EVT = 0x45565430u;

// ---------------------------------------------------------------------------
// Design blob: header | mirrors | layer thickness (FP32) | layer material (u8);
// the two layer arrays hold kStackPad zero-thickness layers before each
// mirror's stack and after the last
// Staged into shared memory per CTA with a bulk (TMA) copy.
// ---------------------------------------------------------------------------
struct alignas(16) BlobHeader {
  int dims, n_mat, n_mir, n_layers;      // n_layers: device (non-pruned) layers
  float n_slab, thick, half_w, x_end;
  float eye_relief, ic_nx, ic_nz, ic_cot; // input mirror normal (-sin a, cos a), cot a
  float mat_n[MAX_MAT];
  int off_mir, off_d, off_m, bytes;       // byte offsets, total size (multiple of 16)
  // 1: inside the slab the input mirror, the mirror planes in index order and
  // the end face are disjoint and ordered along x, so a ray between plane k-1
  // and plane k can only meet one of those two next (set by k_prep_design)
  int ordered;
  // 1: general mirrors (any normal, a tilt axis, an (x, y) rectangle where
  // the plane acts); 0: PRMA planes nx x + nz z = c across the whole slab
  int general;
  int n_fam;  // general designs: plane families (FamRec table after the mirror records)
  int pad_;
  float mat_inv_n[MAX_MAT];               // 1 / n
  float mat_r2[MAX_MAT];                  // (n_slab / n)^2, rounded from FP64
  float mat_r2_lo[MAX_MAT];               // (n_slab / n)^2 - mat_r2 (accurate layer evaluation)
};
static_assert(sizeof(BlobHeader) == 144, "header layout");

struct alignas(16) MirrorRec {
  float nx, ny, nz, c;       // plane n . p = c (PRMA: ny = 0)
  float omega, isw, is1w;    // reflection probability, 1/sqrt(omega), 1/sqrt(1-omega)
  int layer_off;             // first device layer; traversal order = layer 1 first
  int n_layers;              // device layers of this mirror
  float ax, ay, az;          // tilt axis: dn/d(tilt) = a x n per radian (PRMA: a = -y)
  float x0, x1, y0, y1;      // (x, y) rectangle where a general mirror acts
  float nlx, nly, nlz;       // FP64 normal minus (nx, ny, nz): the low part (accurate mode)
  int store_off;             // first layer in the blob's padded layer arrays
};
static_assert(sizeof(MirrorRec) == 80, "mirror layout");

// A family of a general design: mirrors k0 .. k0 + n - 1 with the same normal
// (bitwise) and offsets c monotone in the index (dir = +1 increasing, -1
// decreasing), searched by offset instead of plane by plane. Every mirror is
// in exactly one family (a single mirror is a family of one).
struct alignas(16) FamRec {
  int k0, n, dir, pad;
};

struct Blob {
  const BlobHeader* h;
  const MirrorRec* mir;
  const FamRec* fam;  // general designs: right after the mirror records
  const float* d;
  const uint8_t* m;
  __device__ __forceinline__ void bind(const uint8_t* base) {
    h = reinterpret_cast<const BlobHeader*>(base);
    mir = reinterpret_cast<const MirrorRec*>(base + h->off_mir);
    fam = reinterpret_cast<const FamRec*>(base + h->off_mir + sizeof(MirrorRec) * h->n_mir);
    d = reinterpret_cast<const float*>(base + h->off_d);
    m = base + h->off_m;
  }
};

// per-field launch constants: guided direction after the input mirror and
// the transverse basis e1 (y projected off d), e2 = d x e1; dlx, dly, dlz:
// the FP64 direction minus (dx, dy, dz) (accurate mode)
struct alignas(16) FieldRec {
  float dx, dy, dz, dlx;
  float e1x, e1y, e1z, dly;
  float e2x, e2y, e2z, dlz;
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}
// 24-bit uniform in [0, 1), exact in FP32
__device__ __forceinline__ float u24(uint32_t x) { return (float)(x >> 8) * 5.9604644775390625e-08f; }

// ---------------------------------------------------------------------------
// small complex helpers (float2 = re, im)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // conj(a) * b
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -a.y * b.x));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cdiv(float2 a, float2 b) {
  const float inv = 1.0f / fmaf(b.x, b.x, b.y * b.y);
  return make_float2(fmaf(a.x, b.x, a.y * b.y) * inv, fmaf(a.y, b.x, -a.x * b.y) * inv);
}
__device__ __forceinline__ float cabs2(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }
// a / b for |b| anywhere in the FP32 range: both are scaled by 1/max|b_i|
// first, so |b|^2 cannot overflow (the transfer-matrix vectors reach ~2^70)
__device__ __forceinline__ float2 cdiv_s(float2 a, float2 b) {
  const float k = 1.0f / fmaxf(fabsf(b.x), fabsf(b.y));
  return cdiv(cscale(a, k), cscale(b, k));
}

// ---------------------------------------------------------------------------
// Per-hit material constants for the characteristic matrices.
// Propagating layer (real cos t): x = kappa d, c = cos x, s = sin x,
//   s-pol m12 = s / eta, m21 = s eta (eta = n cos t); p-pol eta = n / cos t.
// Evanescent layer (cos t = -i a): x = beta d, c = cosh x, s = sinh x,
//   s-pol m12 = s/(n a), m21 = -s n a; p-pol m12 = -s a/n, m21 = s n / a.
// In both cases M = [[c, i m12], [i m21, c]].
// ---------------------------------------------------------------------------
// kap: d(phase)/d(thickness) in rad/nm (2 pi n cos / lambda, or beta = 2 pi n a / lambda);
// kt: the rate the layer loop multiplies by: turns/nm for a propagating layer
// (the phase is reduced exactly to [-1/2, 1/2) turn before the fast sin/cos),
// beta for an evanescent one.
// ktl: the low part of kt in the accurate evaluation (kt + ktl), unused otherwise.
struct MatK {
  float kap, kt, ktl, q12s, q21s, q12p, q21p;
  int evan;
};

// rad = 1 - (n0/n)^2 sin^2 t0 = cos^2 t with (n0/n)^2 rounded once from FP64;
// c = sqrt|rad| is cos t (propagating) or a (evanescent, cos t = -i a).
// c sets every layer's phase rate, and a long stack multiplies the phase
// error by its length, so it is taken to within about half an ulp: the
// hardware reciprocal square root r, one Newton step on r (Newton-Raphson for
// 1/sqrt), then c = rad r with one Newton correction of the square. The
// quotients 1/(n c) and n/c start from r / n and n r and take one Newton
// correction each (residual of the product, times the reciprocal), which
// brings them to about half an ulp as well.
// No divide and no branch: each hit evaluates this for every material.
__device__ __forceinline__ MatK mat_const(float sin2_0, float n, float inv_n, float r2, float inv_lam) {
  MatK k;
  const float rad = fmaf(-r2, sin2_0, 1.0f);
  const bool ev = !(rad >= 0.0f);
  const float x = fmaxf(fabsf(rad), 1e-30f);
  float r = rsqrtf(x);
  r = fmaf(0.5f * r, fmaf(-x * r, r, 1.0f), r);
  float c = x * r;
  c = fmaf(0.5f * r, fmaf(-c, c, x), c);
  const float nc = n * c;
  const float kt = nc * inv_lam;
  float q12 = r * inv_n;
  q12 = fmaf(q12, fmaf(-nc, q12, 1.0f), q12);  // 1 / (n c)
  float q21p = n * r;
  q21p = fmaf(fmaf(-c, q21p, n), r, q21p);     // n / c
  k.kap = TWO_PI * kt;
  k.kt = ev ? k.kap : kt;
  k.q12s = q12;
  k.q21s = ev ? -nc : nc;
  k.q12p = (ev ? -c : c) * inv_n;
  k.q21p = q21p;
  k.ktl = 0.0f;
  k.evan = ev;
  return k;
}

// ---------------------------------------------------------------------------
// Double-float arithmetic (a value carried as an unevaluated sum hi + lo of
// two floats) for the accurate layer evaluation. A 200-layer stack turns a
// phase-rate error e into a coherent phase error of ~70 turns x e, which its
// resonances amplify: FP32 incidence cosines, phase rates and phases leave
// coefficient errors of 1e-4 at the 99th percentile, while the FP32 vector
// sweep alone stays near 1e-5. So the accurate mode carries the incidence
// cosine, (n0/n)^2, n/lambda and each layer's phase as hi + lo, and takes the
// sin/cos of the phase on the FMA pipe. The _rn intrinsics are never
// contracted into FMAs, which the error-free transformations below rely on.
// ---------------------------------------------------------------------------
struct F2 {
  float h, l;
};
// p + e = a b exactly
__device__ __forceinline__ F2 two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return F2{p, fmaf(a, b, -p)};
}
// s + e = a + b exactly (Knuth's branch-free sum)
__device__ __forceinline__ F2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return F2{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
// s + e = a + b exactly when |a| >= |b| or a = 0 (Dekker)
__device__ __forceinline__ F2 fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return F2{s, __fsub_rn(b, __fsub_rn(s, a))};
}
// (a.h + a.l)(b.h + b.l) to about 2^-44 relative (lo not renormalized)
__device__ __forceinline__ F2 mul_ff(F2 a, F2 b) {
  const float p = __fmul_rn(a.h, b.h);
  return F2{p, fmaf(a.h, b.l, fmaf(a.l, b.h, fmaf(a.h, b.h, -p)))};
}

// 2 pi log2(e) as hi + lo: an evanescent layer's rate in base-2 exponent units
constexpr float K2PI_LOG2E_H = 9.064720154e+00f;
constexpr float K2PI_LOG2E_L = 1.298458017e-07f;
constexpr float LN2_F = 6.931471825e-01f;

// Accurate material constants: sin2 = sin^2(theta_0), r2 = (n0/n)^2 and
// nl = n / lambda as hi + lo. rad = 1 - r2 sin2 and cos t = sqrt|rad| keep
// ~2^-44 relative error through the cancellation near the critical angle;
// kt + ktl = n cos t / lambda (turns per nm) for a propagating layer, and
// beta log2(e) / (2 pi) x 2 pi = n a / lambda x 2 pi log2(e) (base-2
// exponent per nm) for an evanescent one. The quotients are FP32 as above.
__device__ __forceinline__ MatK mat_const_acc(F2 sin2, float n, float inv_n, F2 r2, F2 nl) {
  MatK k;
  const F2 q = mul_ff(r2, sin2);
  F2 rad = two_sum(1.0f, -q.h);
  rad = fast_two_sum(rad.h, __fsub_rn(rad.l, q.l));
  const bool ev = !(rad.h >= 0.0f);
  const float x = fmaxf(fabsf(rad.h), 1e-30f);
  const float xl = ev ? -rad.l : rad.l;
  float r = rsqrtf(x);
  r = fmaf(0.5f * r, fmaf(-x * r, r, 1.0f), r);
  float c = x * r;
  c = fmaf(0.5f * r, fmaf(-c, c, x), c);
  const float cl = (fmaf(-c, c, x) + xl) * (0.5f * r);  // sqrt(x + xl) = c + cl
  const float nc = n * c;
  float q12 = r * inv_n;
  q12 = fmaf(q12, fmaf(-nc, q12, 1.0f), q12);  // 1 / (n c)
  float q21p = n * r;
  q21p = fmaf(fmaf(-c, q21p, n), r, q21p);     // n / c
  F2 kt = mul_ff(nl, F2{c, cl});
  k.kap = TWO_PI * kt.h;
  if (ev) kt = mul_ff(kt, F2{K2PI_LOG2E_H, K2PI_LOG2E_L});
  k.kt = kt.h;
  k.ktl = kt.l;
  k.q12s = q12;
  k.q21s = ev ? -nc : nc;
  k.q12p = (ev ? -c : c) * inv_n;
  k.q21p = q21p;
  k.evan = ev;
  return k;
}

struct MatTable {
  MatK k[MAX_MAT];
  __device__ __forceinline__ void init(const BlobHeader& h, float cos0, float lam) { init_inv(h, cos0, 1.0f / lam); }
  // the same with 1/lambda given (computed once per cell by the trace kernels)
  __device__ __forceinline__ void init_inv(const BlobHeader& h, float cos0, float inv_lam) {
    const float sin2 = fmaf(-cos0, cos0, 1.0f);
#pragma unroll
    for (int i = 0; i < MAX_MAT; ++i)
      if (i < h.n_mat) k[i] = mat_const(sin2, h.mat_n[i], h.mat_inv_n[i], h.mat_r2[i], inv_lam);
  }
  // accurate mode: cos(theta_0) = c0h + c0l
  __device__ __forceinline__ void init_acc(const BlobHeader& h, float c0h, float c0l, float lam) {
    const F2 p = two_prod(c0h, c0h);
    F2 sin2 = fast_two_sum(1.0f, -p.h);
    sin2.l = fmaf(-2.0f * c0h, c0l, __fsub_rn(sin2.l, p.l));
    const float ilh = __frcp_rn(lam);
    const float ill = fmaf(-ilh, lam, 1.0f) * ilh;  // 1/lam = ilh + ill
#pragma unroll
    for (int i = 0; i < MAX_MAT; ++i)
      if (i < h.n_mat) {
        const float n = h.mat_n[i];
        const F2 nl = two_prod(n, ilh);
        k[i] = mat_const_acc(sin2, n, h.mat_inv_n[i], F2{h.mat_r2[i], h.mat_r2_lo[i]},
                             F2{nl.h, fmaf(n, ill, nl.l)});
      }
  }
  template <bool ACC>
  __device__ __forceinline__ void init_sel(const BlobHeader& h, float c0h, float c0l, float lam) {
    if constexpr (ACC) {
      init_acc(h, c0h, c0l, lam);
    } else {
      init(h, c0h, lam);
    }
  }
  // register select by material id (no local-memory indexing)
  __device__ __forceinline__ MatK get(int m) const {
    MatK r = k[0];
    if (m == 1) r = k[1];
    if (m == 2) r = k[2];
    if (m == 3) r = k[3];
    return r;
  }
};

// sin and cos of 2 pi (p + pl) turns on the FMA pipe (accurate mode), with
// |pl| << 1e-6. p is reduced exactly to r = p - q/4, |r| <= 1/8 turn, with
// q = round(4 p) (from the bits of p 4 + 1.5 2^23); sin(2 pi r) and
// cos(2 pi r) are minimax polynomials in r (max error 5e-9 and 4e-10 on
// |r| <= 1/8, fitted by Lawson's iteratively reweighted least squares with
// the coefficients rounded to FP32 one at a time and the rest refitted);
// pl enters to first order (its square is below 1e-12); the quadrant q mod 4
// then rotates (s, c) by q pi/2.
constexpr float SC_S1 = 6.283185005e+00f, SC_S3 = -4.134150696e+01f, SC_S5 = 8.157170105e+01f,
                SC_S7 = -7.461544800e+01f;
constexpr float SC_C2 = -1.973920822e+01f, SC_C4 = 6.493914032e+01f, SC_C6 = -8.542311859e+01f,
                SC_C8 = 5.856121445e+01f;
__device__ __forceinline__ void sincos_turns_acc(float p, float pl, float& s, float& c) {
  constexpr float MAGIC = 12582912.0f;  // 1.5 x 2^23: the sum's unit is 1
  const float t = fmaf(p, 4.0f, MAGIC);
  const float q = __fsub_rn(t, MAGIC);
  const int qb = __float_as_int(t);
  const float r = fmaf(-0.25f, q, p);  // exact (Sterbenz)
  const float r2 = r * r;
  const float sp = r * fmaf(fmaf(fmaf(SC_S7, r2, SC_S5), r2, SC_S3), r2, SC_S1);
  const float cp = fmaf(fmaf(fmaf(fmaf(SC_C8, r2, SC_C6), r2, SC_C4), r2, SC_C2), r2, 1.0f);
  const float da = TWO_PI * pl;
  const float s1 = fmaf(da, cp, sp), c1 = fmaf(-da, sp, cp);
  const bool sw = qb & 1;
  const float so = sw ? c1 : s1, co = sw ? s1 : c1;
  s = (qb & 2) ? -so : so;          // quadrants 2, 3
  c = ((qb + 1) & 2) ? -co : co;    // quadrants 1, 2
}

// c, s of one layer. Fast mode: the phase reduced exactly to [-1/2, 1/2)
// turn, hardware sin/cos; e^x and e^-x from two independent hardware
// exponentials. Accurate mode: the phase as kt d + (ktl d + the rounding
// error of kt d) turns, sin/cos on the FMA pipe; an evanescent layer's
// exponent in base 2 with the same split, 2^(y + yl) = 2^y (1 + ln2 yl).
// PROP: the caller knows the layer propagates (its evanescent form is
// compiled out; the same values as the general evaluation of such a layer)
template <bool ACC = false, bool PROP = false>
__device__ __forceinline__ void layer_cs(const MatK& k, float d, float& c, float& s) {
  if constexpr (!ACC) {
    const float x = k.kt * d;
    if (PROP || !k.evan) {
      const float f = x - rintf(x);  // exact reduction in turns
      __sincosf(f * TWO_PI, &s, &c);
    } else {
      // e^x and e^-x from two independent hardware exponentials (no
      // dependent reciprocal; both with the same relative accuracy)
      const float e = __expf(x);
      const float ei = __expf(-x);
      c = 0.5f * (e + ei);
      s = 0.5f * (e - ei);
    }
  } else {
    const float p = __fmul_rn(k.kt, d);
    const float pl = fmaf(k.ktl, d, fmaf(k.kt, d, -p));
    if (PROP || !k.evan) {
      sincos_turns_acc(p, pl, s, c);
    } else {
      const float t = LN2_F * pl;
      const float e0 = exp2f(p), ei0 = exp2f(-p);
      const float e = fmaf(e0, t, e0), ei = fmaf(-ei0, t, ei0);
      c = 0.5f * (e + ei);
      s = 0.5f * (e - ei);
    }
  }
}

// ---------------------------------------------------------------------------
// Stack evaluation in vector form. v = [B, C]^T = M_1 ... M_L [1, eta_sub]^T
// is built from the substrate side, v <- M_j v: the substrate-side solution
// grows towards the incident side, so each step keeps its FP32 relative
// error at ~1 ulp (the left-to-right matrix product loses the
// subdominant part behind evanescent barriers). v = (x, y) complex,
// M_j = [[c, i m12], [i m21, c]] real-structured:
//   x' = c x + i m12 y,  y' = i m21 x + c y.
// The vector is carried as (x, z) with z = i y: the step then has real
// coefficients only, x' = c x + m12 z, z' = c z - m21 x, two complex
// multiply-adds per entry that map onto the paired FP32 instructions
// (one issue for the real and imaginary parts; per component the same
// fmaf and product as the scalar form, so the same values).
// ---------------------------------------------------------------------------
struct CV {
  float xr, xi;  // x
  float zr, zi;  // z = i y, i.e. y = (zi, -zr)
};
__device__ __forceinline__ float2 f2b(float a) { return make_float2(a, a); }
__device__ __forceinline__ void cv_step(CV& v, float c, float m12, float m21) {
  const float2 X = make_float2(v.xr, v.xi), Z = make_float2(v.zr, v.zi), cc = f2b(c);
  const float2 X2 = __ffma2_rn(cc, X, __fmul2_rn(f2b(m12), Z));
  const float2 Z2 = __ffma2_rn(cc, Z, __fmul2_rn(f2b(-m21), X));
  v.xr = X2.x;
  v.xi = X2.y;
  v.zr = Z2.x;
  v.zi = Z2.y;
}
__device__ __forceinline__ float cv_maxabs(const CV& v) {
  return fmaxf(fmaxf(fabsf(v.xr), fabsf(v.xi)), fmaxf(fabsf(v.zi), fabsf(v.zr)));
}
// the initial vector (1, eta) of the substrate side: z = i eta
__device__ __forceinline__ CV cv_init(float eta) { return CV{1.0f, 0.0f, 0.0f, eta}; }
constexpr float TWO_P64 = 1.8446744073709552e19f;   // 2^64
constexpr float TWO_M64 = 5.421010862427522e-20f;   // 2^-64
// keep entries below 2^64 by exact power-of-two scaling; e counts the scale
__device__ __forceinline__ void cv_rescale(CV& v, int& e) {
  if (cv_maxabs(v) > TWO_P64) {
    v.xr *= TWO_M64;
    v.xi *= TWO_M64;
    v.zr *= TWO_M64;
    v.zi *= TWO_M64;
    e += 64;
  }
}
// 2^e as a double from its exponent bits (0 below the normal range): exact,
// without the FP64 arithmetic of ldexp (few FP64 units per SM)
__device__ __forceinline__ double pow2d(int e) {
  return e < -1022 ? 0.0 : __longlong_as_double((long long)(1023 + min(e, 1023)) << 52);
}
__device__ __forceinline__ float pow2i(int e) {  // 2^e as float, 0 below the range
  if (e < -149) return 0.0f;
  if (e > 127) return __int_as_float(0x7f800000);
  return ldexpf(1.0f, e);
}
// x * 2^e without forming 2^e when it is out of range (0 * 2^e = 0)
__device__ __forceinline__ float scale2(float x, int e) {
  if (e >= -126 && e <= 127) return x * __int_as_float((e + 127) << 23);
  return ldexpf(x, e);
}

struct Coef {
  float2 rs, rp, ts, tp;
};

// Stack view of one mirror in shared memory: off is the first layer's index
// in the padded layer arrays, shift = off - the first layer's device index
// (the index of the gradient sums).
struct StackView {
  const float* d;
  const uint8_t* m;
  int off, L, shift;
  __device__ __forceinline__ int idx(bool front, int j) const { return front ? off + j : off + L - 1 - j; }
};

// 1 / b for |b| anywhere in the FP32 range: b is scaled by 1/max|b_i| first,
// so |b|^2 cannot overflow (the transfer-matrix vectors reach ~2^70); the
// reciprocals are the fast ones (operands far inside the normal range)
__device__ __forceinline__ float2 crcp_s(float2 b) {
  const float k = __fdividef(1.0f, fmaxf(fabsf(b.x), fabsf(b.y)));
  const float2 s = make_float2(b.x * k, b.y * k);
  const float inv = __fdividef(1.0f, fmaf(s.x, s.x, s.y * s.y)) * k;
  return make_float2(s.x * inv, -s.y * inv);
}

// r = (eta0 B - C)/(eta0 B + C), t = 2 eta0/(eta0 B + C) (Macleod); the
// scale 2^e of v cancels in r and multiplies t by 2^-e.
__device__ __forceinline__ void coef_from_v(const CV& v, float eta0, int e, float2& r, float2& t) {
  // B = x, C = y = (zi, -zr)
  const float2 den = make_float2(fmaf(eta0, v.xr, v.zi), fmaf(eta0, v.xi, -v.zr));
  const float2 num = make_float2(fmaf(eta0, v.xr, -v.zi), fmaf(eta0, v.xi, v.zr));
  const float2 q = crcp_s(den);
  r = cmul(num, q);
  t = cscale(cscale(q, 2.0f * eta0), pow2i(-e));
}

// Segment length of the layer loops: a multiple of the stack's material
// period P, so that every step of a segment uses a fixed material slot held
// in registers (P = 0: any stack; the material is selected per layer).
template <int P>
struct Seg {
  static constexpr int CKP = (P == 3) ? 6 : 8;
  static constexpr int NSLOT = P > 0 ? P : 1;
};

// Material constants of the traversal steps j with j % P == v for a stack
// whose layer i has the material of layer i mod P.
template <int P>
__device__ __forceinline__ void stack_slots(const StackView& st, bool front, const MatTable& mt, MatK* kb) {
#pragma unroll
  for (int v = 0; v < P; ++v) {
    int r = front ? v : (((st.L - 1 - v) % P) + P) % P;
    r = r < st.L ? r : 0;
    kb[v] = mt.get(st.m[st.off + r]);
  }
}

// Traversal step j of a stack (array index i0 + j di), or past the stack's
// end (j >= L, one of the stored pad layers) an identity step: thickness 0
// gives phase 0 and (c, s) = (1, 0) exactly (sin 0 = 0, cos 0 = 1 and
// e^0 = 1 in every evaluation of layer_cs), the identity matrix. Loops over
// whole segments then take no branch and no bounds test on the stack length.
// The material of a periodic stack's step comes from its register slot; a
// general stack reads it.
template <int P, bool ACC, bool PROP = false>
__device__ __forceinline__ void layer_at(const StackView& st, const MatTable& mt, const MatK* kb, int i0, int di,
                                         int j, int u, MatK& k, float& d, float& c, float& s) {
  const int i = i0 + j * di;
  if constexpr (P > 0) {
    k = kb[u % P];
  } else {
    k = mt.get(st.m[i]);
  }
  d = st.d[i];
  layer_cs<ACC, PROP>(k, d, c, s);
}

// The same slots evaluated directly from each slot's material, without a
// table of every material and a select by material id (the values are those
// of MatTable: the same function on the same inputs). inv_lam: 1/lambda of
// the fast evaluation; the accurate one forms 1/lambda as hi + lo from lam.
template <int P, bool ACC>
__device__ __forceinline__ void slot_consts(const BlobHeader& h, const StackView& st, bool front, float c0h,
                                            float c0l, float lam, float inv_lam, MatK* kb) {
  int mv[P];
#pragma unroll
  for (int v = 0; v < P; ++v) {
    int r = front ? v : (((st.L - 1 - v) % P) + P) % P;
    r = r < st.L ? r : 0;
    mv[v] = st.m[st.off + r];
  }
  if constexpr (ACC) {
    const F2 p = two_prod(c0h, c0h);
    F2 sin2 = fast_two_sum(1.0f, -p.h);
    sin2.l = fmaf(-2.0f * c0h, c0l, __fsub_rn(sin2.l, p.l));
    const float ilh = __frcp_rn(lam);
    const float ill = fmaf(-ilh, lam, 1.0f) * ilh;  // 1/lam = ilh + ill
#pragma unroll
    for (int v = 0; v < P; ++v) {
      const int m = mv[v];
      const float n = h.mat_n[m];
      const F2 nl = two_prod(n, ilh);
      kb[v] = mat_const_acc(sin2, n, h.mat_inv_n[m], F2{h.mat_r2[m], h.mat_r2_lo[m]}, F2{nl.h, fmaf(n, ill, nl.l)});
    }
  } else {
    const float sin2 = fmaf(-c0h, c0h, 1.0f);
#pragma unroll
    for (int v = 0; v < P; ++v) {
      const int m = mv[v];
      kb[v] = mat_const(sin2, h.mat_n[m], h.mat_inv_n[m], h.mat_r2[m], inv_lam);
    }
  }
}

// Effective coefficients in the paper's convention (r_p = -r_p(Abeles)).
// kb: the material slots of a periodic stack (P > 0); mt: the material
// table of a general one (P = 0)
template <int P, bool ACC = false>
__device__ __forceinline__ Coef tmm_forward_k(const StackView& st, bool front, const MatTable& mt, const MatK* kb,
                                              float n0, float cos0, int& layer_steps) {
  constexpr int CKP = Seg<P>::CKP;
  const float eta_s = n0 * cos0, eta_p = n0 / cos0;
  CV vs = cv_init(eta_s), vp = cv_init(eta_p);
  int es = 0, ep = 0;
  const int L = st.L;
  const int i0 = front ? st.off : st.off + L - 1, di = front ? 1 : -1;
  const int jtop = L > 0 ? ((L - 1) / CKP) * CKP : -1;
  // P > 0: the thicknesses of the period ahead are loaded one iteration early
  // (the period after the last reads stored pad layers)
  float dn[Seg<P>::NSLOT];
  if constexpr (P > 0) {
#pragma unroll
    for (int v = 0; v < P; ++v) dn[v] = st.d[i0 + (jtop + CKP - P + v) * di];
  }
  for (int j0 = jtop; j0 >= 0; j0 -= CKP) {
    if constexpr (P > 0) {
      // one material period unrolled per iteration (the slots stay static):
      // a shorter loop body for the instruction cache of a kernel whose
      // warps run different phases at once
#pragma unroll 1
      for (int w = CKP / P - 1; w >= 0; --w) {
        float dc[P];
#pragma unroll
        for (int v = 0; v < P; ++v) {
          dc[v] = dn[v];
          dn[v] = st.d[i0 + (j0 + (w - 1) * P + v) * di];
        }
#pragma unroll
        for (int v = P - 1; v >= 0; --v) {
          float c, s;
          const MatK& k = kb[v];
          layer_cs<ACC>(k, dc[v], c, s);
          cv_step(vs, c, s * k.q12s, s * k.q21s);
          cv_step(vp, c, s * k.q12p, s * k.q21p);
        }
      }
    } else {
#pragma unroll
      for (int u = CKP - 1; u >= 0; --u) {
        MatK k;
        float d, c, s;
        layer_at<P, ACC>(st, mt, kb, i0, di, j0 + u, u, k, d, c, s);
        cv_step(vs, c, s * k.q12s, s * k.q21s);
        cv_step(vp, c, s * k.q12p, s * k.q21p);
      }
    }
    cv_rescale(vs, es);
    cv_rescale(vp, ep);
  }
  layer_steps += L;
  Coef out;
  coef_from_v(vs, eta_s, es, out.rs, out.ts);
  float2 rpm;
  coef_from_v(vp, eta_p, ep, rpm, out.tp);
  out.rp = make_float2(-rpm.x, -rpm.y);
  return out;
}
template <int P, bool ACC = false>
__device__ __forceinline__ Coef tmm_forward(const StackView& st, bool front, const MatTable& mt, float n0,
                                            float cos0, int& layer_steps) {
  MatK kb[Seg<P>::NSLOT];
  if constexpr (P > 0) stack_slots<P>(st, front, mt, kb);
  return tmm_forward_k<P, ACC>(st, front, mt, kb, n0, cos0, layer_steps);
}

// ---------------------------------------------------------------------------
// Derivatives with respect to cos(theta_0) of the layer constants and of the
// layer chain (dual numbers), for the mirror-tilt gradient.
// ---------------------------------------------------------------------------
// d/d(cos t0) of a material's constants (value k, the same branch)
struct MatKD {
  float dkt, dq12s, dq21s, dq12p, dq21p;
};
__device__ __forceinline__ MatKD mat_const_d(const MatK& k, float cos0, float n, float inv_n, float r2,
                                             float inv_lam) {
  const float drad = 2.0f * r2 * cos0;  // rad = 1 - r2 (1 - cos0^2)
  MatKD D;
  if (!k.evan) {
    const float eta = k.q21s, ct = fmaxf(eta * inv_n, 1e-20f);
    const float dct = 0.5f * drad / ct, deta = n * dct;
    D.dkt = deta * inv_lam;  // turns per nm
    D.dq12s = -deta * k.q12s * k.q12s;
    D.dq21s = deta;
    D.dq12p = dct * inv_n;
    D.dq21p = -dct * k.q21p / ct;
  } else {
    const float na = -k.q21s, a = fmaxf(na * inv_n, 1e-20f);
    const float da = -0.5f * drad / a, dna = n * da;
    D.dkt = TWO_PI * dna * inv_lam;  // rad per nm, as kt
    D.dq12s = -dna * k.q12s * k.q12s;
    D.dq21s = -dna;
    D.dq12p = -da * inv_n;
    D.dq21p = -da * k.q21p / a;
  }
  return D;
}

struct MatTableD {
  MatKD k[MAX_MAT];
  __device__ __forceinline__ void init(const BlobHeader& h, float cos0, float lam, const MatTable& mt) {
    const float inv_lam = 1.0f / lam;
#pragma unroll
    for (int i = 0; i < MAX_MAT; ++i)
      if (i < h.n_mat) k[i] = mat_const_d(mt.k[i], cos0, h.mat_n[i], h.mat_inv_n[i], h.mat_r2[i], inv_lam);
  }
  __device__ __forceinline__ MatKD get(int m) const {
    MatKD r = k[0];
    if (m == 1) r = k[1];
    if (m == 2) r = k[2];
    if (m == 3) r = k[3];
    return r;
  }
};

// v' = M v and its derivative dv' = dM v + M dv (M = [[c, i m12], [i m21, c]])
__device__ __forceinline__ void cv_step_d(CV& v, CV& dv, float c, float m12, float m21, float dc, float dm12,
                                          float dm21) {
  // in (x, z) form: dx' = dc x + c dx + dm12 z + m12 dz, dz' = dc z + c dz - dm21 x - m21 dx
  const CV o = v;
  cv_step(v, c, m12, m21);
  const float xr = fmaf(dc, o.xr, fmaf(c, dv.xr, fmaf(dm12, o.zr, m12 * dv.zr)));
  const float xi = fmaf(dc, o.xi, fmaf(c, dv.xi, fmaf(dm12, o.zi, m12 * dv.zi)));
  const float zr = fmaf(dc, o.zr, fmaf(c, dv.zr, -fmaf(dm21, o.xr, m21 * dv.xr)));
  const float zi = fmaf(dc, o.zi, fmaf(c, dv.zi, -fmaf(dm21, o.xi, m21 * dv.xi)));
  dv.xr = xr;
  dv.xi = xi;
  dv.zr = zr;
  dv.zi = zi;
}

// r, t and their derivatives from the (scaled) vector and its derivative
__device__ __forceinline__ void coef_from_v_d(const CV& v, const CV& dv, float eta0, float deta0, int e, float2& r,
                                              float2& t, float2& dr, float2& dt) {
  const float2 B = make_float2(v.xr, v.xi), C = make_float2(v.zi, -v.zr);
  const float2 dB = make_float2(dv.xr, dv.xi), dC = make_float2(dv.zi, -dv.zr);
  const float2 den = make_float2(fmaf(eta0, B.x, C.x), fmaf(eta0, B.y, C.y));
  const float2 num = make_float2(fmaf(eta0, B.x, -C.x), fmaf(eta0, B.y, -C.y));
  const float2 dden = make_float2(fmaf(deta0, B.x, fmaf(eta0, dB.x, dC.x)), fmaf(deta0, B.y, fmaf(eta0, dB.y, dC.y)));
  const float2 dnum = make_float2(fmaf(deta0, B.x, fmaf(eta0, dB.x, -dC.x)), fmaf(deta0, B.y, fmaf(eta0, dB.y, -dC.y)));
  const float2 q = crcp_s(den);
  const float sc = pow2i(-e);
  r = cmul(num, q);
  t = cscale(q, 2.0f * eta0 * sc);
  dr = cmul(csub(dnum, cmul(r, dden)), q);
  dt = cmul(csub(make_float2(2.0f * deta0 * sc, 0.0f), cmul(t, dden)), q);
}

// v and its derivative scaled by the same exact power of two
__device__ __forceinline__ void cv_rescale_d(CV& v, CV& dv, int& e) {
  if (fmaxf(cv_maxabs(v), cv_maxabs(dv)) > TWO_P64) {
    v = CV{v.xr * TWO_M64, v.xi * TWO_M64, v.zr * TWO_M64, v.zi * TWO_M64};
    dv = CV{dv.xr * TWO_M64, dv.xi * TWO_M64, dv.zr * TWO_M64, dv.zi * TWO_M64};
    e += 64;
  }
}

// Coefficients in the paper's convention and their derivatives d/d(cos t0):
// the layer loop of tmm_forward (segments of the material period, material
// constants and their derivatives in registers) carrying the dual vector
// (the coating look-up table's entries).
template <int P, bool ACC = false>
__device__ __forceinline__ void tmm_forward_dual(const StackView& st, bool front, const MatTable& mt,
                                                 const MatTableD& mtd, float n0, float cos0, Coef& cf, Coef& dcf) {
  constexpr int CKP = Seg<P>::CKP;
  MatK kb[Seg<P>::NSLOT];
  MatKD kbd[Seg<P>::NSLOT];
  if constexpr (P > 0) {
#pragma unroll
    for (int v = 0; v < P; ++v) {
      int r = front ? v : (((st.L - 1 - v) % P) + P) % P;
      r = r < st.L ? r : 0;
      const int m = st.m[st.off + r];
      kb[v] = mt.get(m);
      kbd[v] = mtd.get(m);
    }
  }
  const float eta_s = n0 * cos0, eta_p = n0 / cos0;
  const float deta_s = n0, deta_p = -eta_p / cos0;
  CV vs = cv_init(eta_s), vp = cv_init(eta_p);
  CV dvs{0.0f, 0.0f, 0.0f, deta_s}, dvp{0.0f, 0.0f, 0.0f, deta_p};
  int es = 0, ep = 0;
  const int L = st.L;
  for (int j0 = L > 0 ? ((L - 1) / CKP) * CKP : -1; j0 >= 0; j0 -= CKP) {
#pragma unroll
    for (int u = CKP - 1; u >= 0; --u) {
      const int j = j0 + u;
      if (j < L) {
        const int i = st.idx(front, j);
        MatK k;
        MatKD kd;
        if constexpr (P > 0) {
          k = kb[u % P];
          kd = kbd[u % P];
        } else {
          const int m = st.m[i];
          k = mt.get(m);
          kd = mtd.get(m);
        }
        const float dthk = st.d[i];
        float c, s, dc, ds;
        layer_cs<ACC>(k, dthk, c, s);
        if (!k.evan) {
          const float dth = TWO_PI * dthk * kd.dkt;  // d(phase)
          dc = -s * dth;
          ds = c * dth;
        } else {
          const float dx = dthk * kd.dkt;
          dc = s * dx;
          ds = c * dx;
        }
        cv_step_d(vs, dvs, c, s * k.q12s, s * k.q21s, dc, fmaf(ds, k.q12s, s * kd.dq12s),
                  fmaf(ds, k.q21s, s * kd.dq21s));
        cv_step_d(vp, dvp, c, s * k.q12p, s * k.q21p, dc, fmaf(ds, k.q12p, s * kd.dq12p),
                  fmaf(ds, k.q21p, s * kd.dq21p));
      }
    }
    cv_rescale_d(vs, dvs, es);
    cv_rescale_d(vp, dvp, ep);
  }
  float2 rpm, drpm;
  coef_from_v_d(vs, dvs, eta_s, deta_s, es, cf.rs, cf.ts, dcf.rs, dcf.ts);
  coef_from_v_d(vp, dvp, eta_p, deta_p, ep, rpm, cf.tp, drpm, dcf.tp);
  cf.rp = make_float2(-rpm.x, -rpm.y);
  dcf.rp = make_float2(-drpm.x, -drpm.y);
}

// ---------------------------------------------------------------------------
// Adjoint of f = 2 Re(A_s c_s + A_p c_p) (c = r or t) with respect to every
// layer thickness. With v_j = M_j ... M_{L-1} u and the row
// a_j = rho M_0 ... M_{j-1}, rho = A (dc/dB, dc/dC):
//   df/dx_j = 2 Re(a_j G_j v_j) = -2 (q12 Im(a_j0 y_j) + q21 Im(a_j1 x_j)),
//   G_j = [[0, i q12], [i q21, 0]] (dM_j/dx = M_j G_j), df/dd_j = kappa_j df/dx_j.
// Sweep 1 runs v from the substrate side and keeps a checkpoint every CK
// layers; sweep 2 runs a from the incident side and takes each segment's v_j
// from a checkpoint: by inverse layer steps from the segment's incident-side
// checkpoint when no layer of the stack is evanescent, else recomputed from
// the checkpoint at its far end.
// sink(layer index, df/dd) receives the gradient (per nm).
// ---------------------------------------------------------------------------
struct Ckpt {
  CV s, p;
  int es, ep;
};

// The row a = (a0, a1) is carried as (a0, b) with b = i a1, i.e. a1 =
// (b.y, -b.x): the step a' = a M, a0' = c a0 + i m21 a1, a1' = i m12 a0 +
// c a1, becomes a0' = c a0 + m21 b, b' = c b - m12 a0 (real coefficients,
// the paired FP32 instructions; per component the scalar form's values).
struct CRow {
  float2 a0, b;
};
__device__ __forceinline__ void row_step(CRow& a, float c, float m12, float m21) {
  const float2 cc = f2b(c);
  const float2 a0 = __ffma2_rn(cc, a.a0, __fmul2_rn(f2b(m21), a.b));
  const float2 b = __ffma2_rn(cc, a.b, __fmul2_rn(f2b(-m12), a.a0));
  a.a0 = a0;
  a.b = b;
}
__device__ __forceinline__ float row_maxabs(const CRow& a) {
  return fmaxf(fmaxf(fabsf(a.a0.x), fabsf(a.a0.y)), fmaxf(fabsf(a.b.y), fabsf(a.b.x)));
}

// rho for one polarization (scaled v, exponent e): returns the row and its exponent
__device__ __forceinline__ CRow coef_row(const CV& v, float eta0, int e, float2 A, int which, int& ea) {
  const float2 B = make_float2(v.xr, v.xi), C = make_float2(v.zi, -v.zr);
  const float2 den = make_float2(fmaf(eta0, B.x, C.x), fmaf(eta0, B.y, C.y));
  CRow a;
  float2 a1;
  if (which == 0) {
    // dr/dB = 2 eta0 C / den^2, dr/dC = -2 eta0 B / den^2
    const float2 dB = cscale(cdiv_s(cdiv_s(C, den), den), 2.0f * eta0);
    const float2 dC = cscale(cdiv_s(cdiv_s(B, den), den), -2.0f * eta0);
    a.a0 = cmul(A, dB);
    a1 = cmul(A, dC);
    ea = -e;
  } else {
    // t = 2 eta0 / den: dt/dB = -eta0 t / den, dt/dC = -t / den
    const float2 t = cdiv_s(make_float2(2.0f * eta0, 0.0f), den);
    const float2 td = cdiv_s(t, den);
    a.a0 = cmul(A, cscale(td, -eta0));
    a1 = cmul(A, cscale(td, -1.0f));
    ea = -2 * e;
  }
  a.b = make_float2(-a1.y, a1.x);  // b = i a1
  return a;
}

// Words per layer of the segment buffer (s and p substrate-side vectors, c, s),
// and the same as pairs of floats
constexpr int kSegWords = 10, kSegPairs = kSegWords / 2;
// a vector from two pairs of a segment-buffer column
__device__ __forceinline__ CV seg_cv(const float2* b) {
  const float2 x = b[0], z = b[32];
  return CV{x.x, x.y, z.x, z.y};
}
// Shared-memory floats of one warp's segment buffers for material period P.
template <int P>
__host__ __device__ constexpr int seg_floats_per_warp() {
  return Seg<P>::CKP * kSegWords * 32;
}

// rho = d ln(cos t)/d(cos t0) of each material for the reverse sweep's
// tilt terms (cos t = sqrt(rad), or a for cos t = -i a; both give
// r2 cos0 / rad). A layer's phase rate and its four quotients all scale
// with it: d(kap)/dcos = rho kap, dq21s = rho q21s, dq12s = -rho q12s,
// dq12p = rho q12p, dq21p = -rho q21p.
struct TiltTable {
  float rho[MAX_MAT];
  __device__ __forceinline__ void init(const BlobHeader& h, float cos0) {
    const float sin2 = fmaf(-cos0, cos0, 1.0f);
#pragma unroll
    for (int i = 0; i < MAX_MAT; ++i) {
      const float rad = fmaf(-h.mat_r2[i], sin2, 1.0f);
      const float q = copysignf(fmaxf(fabsf(rad), 1e-30f), rad);
      rho[i] = i < h.n_mat ? h.mat_r2[i] * cos0 / q : 0.0f;
    }
  }
  __device__ __forceinline__ float get(int m) const {
    float r = rho[0];
    if (m == 1) r = rho[1];
    if (m == 2) r = rho[2];
    if (m == 3) r = rho[3];
    return r;
  }
};

// 2 Re(A dc/d(eta0)) at fixed (B, C) for one polarization: r = (eta0 B - C)/den
// gives 2 B C / den^2, t = 2 eta0 2^-e / den gives 2 C 2^-e / den^2
// (den = eta0 B + C on the scaled vector; A already carries the r_p sign).
__device__ __forceinline__ float coef_deta(const CV& v, float eta0, int e, float2 A, int which) {
  const float2 B = make_float2(v.xr, v.xi), C = make_float2(v.zi, -v.zr);
  const float2 den = make_float2(fmaf(eta0, B.x, C.x), fmaf(eta0, B.y, C.y));
  const float2 cd = cdiv_s(C, den);
  const float2 x = which == 0 ? cmul(cdiv_s(B, den), cd) : cscale(cdiv_s(cd, den), pow2i(-e));
  return 4.0f * fmaf(A.x, x.x, -A.y * x.y);
}


// Exact power-of-two scaling for the adjoint's range management.
// floor(log2 m) of a normal positive float
__device__ __forceinline__ int exp_of(float m) { return ((__float_as_int(m) >> 23) & 0xff) - 127; }
// 2^e for e in [-126, 127]
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((e + 127) << 23); }
// x 2^k for any k in [-252, 254] (two exact factors)
__device__ __forceinline__ float mul_pow2(float x, int k) {
  const int k1 = k / 2;
  return (x * pow2f(k1)) * pow2f(k - k1);
}
// v scaled in one exact step into [1, 2) once its largest entry passes 2^8:
// checkpoints stay small, so that the products of a segment (a vector grown
// by up to 2^31 times a row) leave room below the FP32 range even after the
// tilt terms' factor rho = d ln cos(theta_j)/d cos(theta_0), large near the
// critical angle
constexpr float CK_HI = 256.0f;
__device__ __forceinline__ void cv_fit(CV& v, int& e) {
  const float m = cv_maxabs(v);
  if (m > CK_HI) {
    const int sh = min(exp_of(m), 127);  // m 2^-sh in [1, 2); non-finite stays non-finite
    const float f = pow2f(-sh);
    v.xr *= f;
    v.xi *= f;
    v.zr *= f;
    v.zi *= f;
    e += sh;
  }
}
// the row scaled in one exact step into [2^7, 2^8) when outside [2^-8, 2^8]
constexpr float ROW_HI = 256.0f, ROW_LO = 0.00390625f;
__device__ __forceinline__ void row_fit8(CRow& a, int& e) {
  const float m = row_maxabs(a);
  if ((m > ROW_HI || m < ROW_LO) && m > 0.0f) {
    const int em = m >= 1.17549435e-38f ? exp_of(m) : -126;  // a subnormal row counts as 2^-126
    const int sh = min(em, 127) - 7;
    a.a0 = make_float2(mul_pow2(a.a0.x, -sh), mul_pow2(a.a0.y, -sh));
    a.b = make_float2(mul_pow2(a.b.x, -sh), mul_pow2(a.b.y, -sh));
    e += sh;
  }
}

// Sum over the warp's 32 lanes of R = 8 values per lane, one result per
// value: three transposing exchanges (16, 8, 4 lanes apart) halve the values
// a lane holds while summing pairs, two plain exchanges finish the sums.
// Afterwards lane l holds the sum of value ((l >> 4) & 1) 4 + ((l >> 3) & 1) 2
// + ((l >> 2) & 1), and every lane of a quad holds the same sum.
__device__ __forceinline__ float warp_transpose_sum8(const float (&t)[8], int lane) {
  const bool b16 = lane & 16, b8 = lane & 8, b4 = lane & 4;
  float h[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float send = b16 ? t[k] : t[k + 4];
    h[k] = (b16 ? t[k + 4] : t[k]) + __shfl_xor_sync(0xffffffffu, send, 16);
  }
  float q[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const float send = b8 ? h[k] : h[k + 2];
    q[k] = (b8 ? h[k + 2] : h[k]) + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  float r = (b4 ? q[1] : q[0]) + __shfl_xor_sync(0xffffffffu, b4 ? q[0] : q[1], 4);
  r += __shfl_xor_sync(0xffffffffu, r, 2);
  r += __shfl_xor_sync(0xffffffffu, r, 1);
  return r;
}

// seg: this lane's column of its warp's segment buffer, in pairs of floats
// (pair (u, q) of step u at seg[(u * kSegPairs + q) * 32]; the 32 lanes'
// columns interleave, 8-byte aligned): q = 0, 1: the s vector (x, z); 2, 3:
// the p vector; 4: (c, s) of the layer, whose c word takes the step's term
// once it is used.
// The sink receives each segment's gradient terms at once:
// sink.segment(t, n, i0, di): t[u] = df/dd of layer i0 + u di (per nm), u < n.
// Range management (exact powers of two): the first sweep keeps every
// checkpoint at or below 2^8, the row is brought into [2^-8, 2^8] at each
// segment start; a segment grows either by less than 2^31, so a . v (< 2^78)
// stays far below the FP32 range inside the segment, and each segment's
// terms take one scale factor 2^(e_row + e_v) (computed once; out of the
// normal range a common part is applied to the terms after the segment).
// DUAL: *g_cos also receives df/d(cos t0) of the record through its coating,
// without 2^eA, from the same reverse sweep (reverse-mode, no derivative
// chain): with v_j = M_j v_{j+1} (substrate side) and the row a_j,
//   df/dcos = 2 Re[ A dc/d(eta0) deta0 + sum_j a_j dM_j/dcos v_{j+1} + a_L (0, deta0)^T ],
// where M = c I + s K(q) gives a dM/dcos v_{j+1} = dphi a K v_j (the
// thickness term's product, times dphi/dcos) + s a dK(dq) v_{j+1} (the same
// two products on v_{j+1} with the quotients' derivatives); both scale with
// the material's rho (tt).
template <int P, class Sink, bool DUAL = false, bool ACC = false>
__device__ __forceinline__ void tmm_adjoint(const StackView& st, bool front, const MatTable& mt, float n0,
                                            float cos0, float2 A_s, float2 A_p, int which, Sink& sink,
                                            float2* seg, int eA = 0, const TiltTable* tt = nullptr,
                                            float* g_cos = nullptr, const MatK* slots = nullptr) {
  // (A_s, A_p) * 2^eA are the weights; eA carries the range of dL/dtally;
  // slots (P > 0): the stack slots' material constants when the caller
  // evaluated them directly (else they come from mt)
  constexpr int CKP = Seg<P>::CKP;
  MatK kb[Seg<P>::NSLOT];
  if constexpr (P > 0) {
    if (slots) {
#pragma unroll
      for (int v = 0; v < P; ++v) kb[v] = slots[v];
    } else {
      stack_slots<P>(st, front, mt, kb);
    }
  }
  Ckpt ck[MAX_CK];
  const int L = st.L;
  const int nseg = (L + CKP - 1) / CKP;
  // layer-array index of traversal step j: i0 + j di (the gradient sums take
  // the device index, i0 + j di - st.shift)
  const int i0 = front ? st.off : st.off + L - 1, di = front ? 1 : -1;
  const float eta_s = n0 * cos0, eta_p = n0 / cos0;
  // Stacks without an evanescent layer (P > 0: every slot propagating) take
  // v_{j+1} = M_j^{-1} v_j from the checkpoint at the segment's incident-side
  // end, in registers: M_j = c I + s K with K^2 = -I (q12 q21 = 1) has
  // determinant c^2 + s^2 = 1, and its inverse is the same step with s
  // negated. Its singular values are bounded by the quotients, so the
  // segment's vectors keep about the forward sweep's relative accuracy.
  // Through an evanescent layer (K^2 = I) the inverse would lose the decaying
  // solution, so those stacks recompute each segment from its substrate-side
  // checkpoint instead and keep it in the lane's shared-memory column. The
  // propagating stacks' sweeps also take the layers' propagating form only.
  bool inv = false;
  if constexpr (P > 0) {
    inv = true;
#pragma unroll
    for (int v = 0; v < P; ++v) inv = inv && !kb[v].evan;
  }
  CV vs = cv_init(eta_s), vp = cv_init(eta_p);
  int es = 0, ep = 0;
  ck[nseg] = Ckpt{vs, vp, 0, 0};
  for (int sg = nseg - 1; sg >= 0; --sg) {
    const int j0 = sg * CKP;
    if (inv) {
#pragma unroll
      for (int u = CKP - 1; u >= 0; --u) {
        MatK k;
        float d, c, s;
        layer_at<P, ACC, true>(st, mt, kb, i0, di, j0 + u, u, k, d, c, s);
        cv_step(vs, c, s * k.q12s, s * k.q21s);
        cv_step(vp, c, s * k.q12p, s * k.q21p);
      }
    } else {
#pragma unroll
      for (int u = CKP - 1; u >= 0; --u) {
        MatK k;
        float d, c, s;
        layer_at<P, ACC>(st, mt, kb, i0, di, j0 + u, u, k, d, c, s);
        cv_step(vs, c, s * k.q12s, s * k.q21s);
        cv_step(vp, c, s * k.q12p, s * k.q21p);
      }
    }
    cv_fit(vs, es);
    cv_fit(vp, ep);
    ck[sg] = Ckpt{vs, vp, es, ep};
  }
  // paper convention r_p = -r_p(Abeles): flip A_p for reflection
  const float2 Ap = which == 0 ? make_float2(-A_p.x, -A_p.y) : A_p;
  int eas, eap;
  CRow as = coef_row(vs, eta_s, es, A_s, which, eas);
  CRow ap = coef_row(vp, eta_p, ep, Ap, which, eap);
  const float deta_s = n0, deta_p = -eta_p / cos0;
  float gc = 0.0f, acc_s = 0.0f, acc_p = 0.0f;
  float rb[Seg<P>::NSLOT];
  if constexpr (DUAL) {
    gc = fmaf(deta_s, coef_deta(vs, eta_s, es, A_s, which), deta_p * coef_deta(vp, eta_p, ep, Ap, which));
    if constexpr (P > 0) {
#pragma unroll
      for (int v = 0; v < P; ++v) {
        int r = front ? v : (((st.L - 1 - v) % P) + P) % P;
        r = r < st.L ? r : 0;
        rb[v] = tt->get(st.m[st.off + r]);
      }
    }
  }
  eas += eA;
  eap += eA;
  for (int sg = 0; sg < nseg; ++sg) {
    const int j0 = sg * CKP;
    row_fit8(as, eas);
    row_fit8(ap, eap);
    // the checkpoint the segment's vectors come from; its exponents scale the terms
    const Ckpt cb = ck[inv ? sg : sg + 1];
    // the segment's scale factors of the terms, 2^xs (s) and 2^xp (p), exact
    // powers of two. When either lies outside the normal range the loop
    // applies 2^(xs - xr) and 2^(xp - xr) instead, with xr the larger
    // exponent of the non-zero rows (a row is in [2^7, 2^8) at the segment
    // start unless it is zero, when its exponent means nothing), the other
    // factor clamped to the normal range (a term more than 2^126 below its
    // partner's scale, or a zero row's), and the terms take 2^xr when they
    // are read out: the loop itself never branches on the range
    const int xs = eas + cb.es, xp = eap + cb.ep;
    const bool in_range = xs >= -126 && xs <= 127 && xp >= -126 && xp <= 127;
    int xr = 0;
    if (!in_range) {
      const bool ns = row_maxabs(as) > 0.0f, np = row_maxabs(ap) > 0.0f;
      xr = ns ? (np ? max(xs, xp) : xs) : (np ? xp : 0);
    }
    const float fs = pow2f(min(max(xs - xr, -126), 127)), fp = pow2f(min(max(xp - xr, -126), 127));
    float t[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) t[u] = 0.0f;
    if (inv) {
      CV x = cb.s, y = cb.p;  // v_j of step u
#pragma unroll
      for (int u = 0; u < CKP; ++u) {
        MatK k;
        float d, c, s;
        float rho = 0.0f;
        layer_at<P, ACC, true>(st, mt, kb, i0, di, j0 + u, u, k, d, c, s);
        if constexpr (DUAL) rho = rb[u % P];
        const float m12s = s * k.q12s, m21s = s * k.q21s, m12p = s * k.q12p, m21p = s * k.q21p;
        // v_{j+1} (past the stack's end the identity: v_L)
        CV xn = x, yn = y;
        cv_step(xn, c, -m12s, -m21s);
        cv_step(yn, c, -m12p, -m21p);
        const float gs = fmaf(k.q12s, fmaf(-as.a0.x, x.zr, as.a0.y * x.zi),
                              k.q21s * fmaf(as.b.y, x.xi, -as.b.x * x.xr));
        const float gp = fmaf(k.q12p, fmaf(-ap.a0.x, y.zr, ap.a0.y * y.zi),
                              k.q21p * fmaf(ap.b.y, y.xi, -ap.b.x * y.xr));
        t[u] = -2.0f * k.kap * fmaf(gs, fs, gp * fp);
        if constexpr (DUAL) {
          const float kd = k.kap * d;
          const float qs = fmaf(k.q21s, fmaf(as.b.y, xn.xi, -as.b.x * xn.xr),
                                -k.q12s * fmaf(-as.a0.x, xn.zr, as.a0.y * xn.zi));
          const float qp = fmaf(k.q12p, fmaf(-ap.a0.x, yn.zr, ap.a0.y * yn.zi),
                                -k.q21p * fmaf(ap.b.y, yn.xi, -ap.b.x * yn.xr));
          acc_s = fmaf(rho, fmaf(kd, gs, s * qs), acc_s);
          acc_p = fmaf(rho, fmaf(kd, gp, s * qp), acc_p);
        }
        row_step(as, c, m12s, m21s);
        row_step(ap, c, m12p, m21p);
        x = xn;
        y = yn;
      }
    } else {
      CV ws = cb.s, wp = cb.p;
      // the segment's substrate-side vectors and (c, s), recomputed from the
      // checkpoint at its far end and kept in this lane's shared-memory column
      // (slots past the stack's end hold the checkpoint itself, v_L)
#pragma unroll
      for (int u = CKP - 1; u >= 0; --u) {
        MatK k;
        float d, c, s;
        layer_at<P, ACC>(st, mt, kb, i0, di, j0 + u, u, k, d, c, s);
        cv_step(ws, c, s * k.q12s, s * k.q21s);
        cv_step(wp, c, s * k.q12p, s * k.q21p);
        float2* b = seg + u * kSegPairs * 32;
        b[0 * 32] = make_float2(ws.xr, ws.xi);
        b[1 * 32] = make_float2(ws.zr, ws.zi);
        b[2 * 32] = make_float2(wp.xr, wp.xi);
        b[3 * 32] = make_float2(wp.zr, wp.zi);
        b[4 * 32] = make_float2(c, s);
      }
      // v_j of step u (the row's products with v_{j+1} read the next slot,
      // or the checkpoint for the segment's last step)
      CV x = seg_cv(seg), y = seg_cv(seg + 2 * 32);
#pragma unroll
      for (int u = 0; u < CKP; ++u) {
        const int j = j0 + u;
        CV xn = cb.s, yn = cb.p;
        if (u + 1 < CKP) {
          const float2* bn = seg + (u + 1) * kSegPairs * 32;
          xn = seg_cv(bn);
          yn = seg_cv(bn + 2 * 32);
        }
        {
          // past the stack's end an identity step (the buffer holds c = 1,
          // s = 0 there, the stored thickness is 0): its term is not read,
          // the row and the tilt sums do not change
          MatK k;
          float rho = 0.0f;
          const int i = i0 + j * di;
          if constexpr (P > 0) {
            k = kb[u % P];
            if constexpr (DUAL) rho = rb[u % P];
          } else {
            const int m = st.m[i];
            k = mt.get(m);
            if constexpr (DUAL) rho = tt->get(m);
          }
          const float2 cs = seg[(u * kSegPairs + 4) * 32];
          const float c = cs.x, s = cs.y;
          // Im(a0 y) and Im(a1 x) with y = (zi, -zr), a1 = (b.y, -b.x)
          const float gs = fmaf(k.q12s, fmaf(-as.a0.x, x.zr, as.a0.y * x.zi),
                                k.q21s * fmaf(as.b.y, x.xi, -as.b.x * x.xr));
          const float gp = fmaf(k.q12p, fmaf(-ap.a0.x, y.zr, ap.a0.y * y.zi),
                                k.q21p * fmaf(ap.b.y, y.xi, -ap.b.x * y.xr));
          t[u] = -2.0f * k.kap * fmaf(gs, fs, gp * fp);
          if constexpr (DUAL) {
            // rho (phase term kap d g + quotient term on v_{j+1}), at this
            // segment's exponents
            const float kd = k.kap * st.d[i];
            const float qs = fmaf(k.q21s, fmaf(as.b.y, xn.xi, -as.b.x * xn.xr),
                                  -k.q12s * fmaf(-as.a0.x, xn.zr, as.a0.y * xn.zi));
            const float qp = fmaf(k.q12p, fmaf(-ap.a0.x, yn.zr, ap.a0.y * yn.zi),
                                  -k.q21p * fmaf(ap.b.y, yn.xi, -ap.b.x * yn.xr));
            acc_s = fmaf(rho, fmaf(kd, gs, s * qs), acc_s);
            acc_p = fmaf(rho, fmaf(kd, gp, s * qp), acc_p);
          }
          row_step(as, c, s * k.q12s, s * k.q21s);
          row_step(ap, c, s * k.q12p, s * k.q21p);
        }
        x = xn;
        y = yn;
      }
    }
    if (xr != 0) {
      const int k = min(max(xr, -252), 254);
#pragma unroll
      for (int u = 0; u < 8; ++u) t[u] = mul_pow2(t[u], k);
    }
    sink.segment(t, min(CKP, L - j0), i0 + j0 * di - st.shift, di);
    if constexpr (DUAL) {
      gc = fmaf(-2.0f, scale2(acc_s, eas + cb.es - eA), gc);
      gc = fmaf(-2.0f, scale2(acc_p, eap + cb.ep - eA), gc);
      acc_s = 0.0f;
      acc_p = 0.0f;
    }
  }
  if constexpr (DUAL) {
    // a_L (0, deta0)^T: v_L = (1, eta0) at exponent 0
    gc = fmaf(2.0f * deta_s, scale2(as.b.y, eas - eA), gc);
    gc = fmaf(2.0f * deta_p, scale2(ap.b.y, eap - eA), gc);
    *g_cos = gc;
  }
}

// ---------------------------------------------------------------------------
// Geometry
// ---------------------------------------------------------------------------
struct V3 {
  float x, y, z;
};
__device__ __forceinline__ V3 v3(float x, float y, float z) { return V3{x, y, z}; }
__device__ __forceinline__ float dot3(V3 a, V3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ V3 cross3(V3 a, V3 b) {
  return V3{fmaf(a.y, b.z, -a.z * b.y), fmaf(a.z, b.x, -a.x * b.z), fmaf(a.x, b.y, -a.y * b.x)};
}

// Accurate mode: a direction is carried as d + dl (dl the low parts), a
// mirror normal as N + Nl (FP64 rounded to hi + lo). d . N as hi + lo: the
// three exact products summed with exact sums, then the cross terms.
__device__ __forceinline__ F2 dot3_df(V3 d, V3 dl, V3 N, V3 Nl) {
  const F2 a = two_prod(d.x, N.x), b = two_prod(d.y, N.y), c = two_prod(d.z, N.z);
  const F2 s1 = two_sum(a.h, b.h);
  const F2 s2 = two_sum(s1.h, c.h);
  float lo = __fadd_rn(__fadd_rn(a.l, b.l), __fadd_rn(c.l, __fadd_rn(s1.l, s2.l)));
  lo = fmaf(d.x, Nl.x, fmaf(d.y, Nl.y, fmaf(d.z, Nl.z, lo)));
  lo = fmaf(dl.x, N.x, fmaf(dl.y, N.y, fmaf(dl.z, N.z, lo)));
  return fast_two_sum(s2.h, lo);
}
// one component of d - 2 (d . N) N as hi + lo (m = -2 d . N)
__device__ __forceinline__ F2 reflect1_df(float d, float dl, float n, float nl, F2 m) {
  const F2 p = mul_ff(m, F2{n, nl});
  const F2 s = two_sum(d, p.h);
  return fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(dl, p.l)));
}
__device__ __forceinline__ void reflect_df(V3& d, V3& dl, V3 N, V3 Nl, F2 cd) {
  const F2 m{-2.0f * cd.h, -2.0f * cd.l};
  const F2 x = reflect1_df(d.x, dl.x, N.x, Nl.x, m);
  const F2 y = reflect1_df(d.y, dl.y, N.y, Nl.y, m);
  const F2 z = reflect1_df(d.z, dl.z, N.z, Nl.z, m);
  d = V3{x.h, y.h, z.h};
  dl = V3{x.l, y.l, z.l};
}

// s/p basis of the slab faces for direction d: s = (d_y, -d_x, 0)/|.|, p = s x d
__device__ __forceinline__ void face_basis(V3 d, V3& s, V3& p) {
  const float h2 = fmaf(d.x, d.x, d.y * d.y);
  if (h2 > 1e-30f) {
    const float r = rsqrtf(h2);
    s = V3{d.y * r, -d.x * r, 0.0f};
  } else {
    s = V3{0.0f, 1.0f, 0.0f};
  }
  p = cross3(s, d);
}

// General mirrors, family by family. Within a family the distance
// t_i = (c_i - p.N)/(d.N) is monotone in the index, so the members are
// visited in order of distance from the first one ahead (binary search on c)
// until one acts (the crossing inside its rectangle) or lies beyond the
// nearest surface so far: the same choice as testing every plane, from the
// same t values (one normal per family). Inlined into the kernels
// instantiated for general designs; next_mirror_general is its out-of-line
// form for launches that mix both kinds of design.
__device__ __forceinline__ void next_mirror_families(const Blob& B, V3 p, V3 d, int last, float& best, int& id) {
  const BlobHeader& h = *B.h;
  for (int f = 0; f < h.n_fam; ++f) {
    const FamRec fr = B.fam[f];
    const MirrorRec& m0 = B.mir[fr.k0];
    const float den = fmaf(d.x, m0.nx, fmaf(d.y, m0.ny, d.z * m0.nz));
    if (den == 0.0f) continue;
    const float pn = fmaf(p.x, m0.nx, fmaf(p.y, m0.ny, p.z * m0.nz));
    const bool up = den > 0.0f;  // ahead: c > p.N (den > 0) or c < p.N (den < 0)
    const int step = (up == (fr.dir > 0)) ? 1 : -1;
    // ahead(i) is false then true along the index for step = +1, true then
    // false for step = -1; lo = the index where it switches
    int lo = 0, hi = fr.n;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      const float c = B.mir[fr.k0 + mid].c;
      const bool ahead = up ? (c > pn) : (c < pn);
      if (ahead == (step < 0)) lo = mid + 1;
      else hi = mid;
    }
    for (int i = step > 0 ? lo : lo - 1; i >= 0 && i < fr.n; i += step) {
      const int k = fr.k0 + i;
      const MirrorRec& m = B.mir[k];
      const float t = __fdividef(m.c - pn, den);
      if (!(t < best)) break;
      if (!(t > 0.0f) || S_MIR + k == last) continue;
      const float qx = fmaf(t, d.x, p.x), qy = fmaf(t, d.y, p.y);
      if (!(qx >= m.x0 && qx <= m.x1 && qy >= m.y0 && qy <= m.y1)) continue;
      best = t;
      id = S_MIR + k;
      break;
    }
  }
}
static __device__ __noinline__ void next_mirror_general(const Blob B, V3 p, V3 d, int last, float& best, int& id) {
  next_mirror_families(B, p, d, last, best, id);
}

// Nearest surface along (p, d), excluding `last`. Candidate order and ties
// match the oracle: faces, input mirror, far end, sides, mirrors.
// Nearest surface ahead of the ray (the surface it sits on excluded). With
// reg >= 0 (an ordered design) the ray lies in region reg, between mirror
// plane reg-1 (the input mirror for reg = 0) and mirror plane reg (the end
// face for reg = K); every other plane is behind one of those two inside the
// slab, so only they are tested. reg < 0 tests every plane. Distances use
// the fast quotient (denominators are direction cosines, |x| <= 1).
// GM: 0 PRMA designs only, 1 general designs only (the family search
// inline), 2 either (decided per design; the family search out of line).
template <int GM>
__device__ __forceinline__ int next_surface(const Blob& B, V3 p, V3 d, int last, int reg, float& tmin) {
  const BlobHeader& h = *B.h;
  float best = __int_as_float(0x7f800000);
  int id = -1;
  auto consider = [&](int sid, float t) {
    if (sid != last && t > 0.0f && t < best) {
      best = t;
      id = sid;
    }
  };
  // the face (and side) ahead: the numerator selected, one quotient each
  // (the same values as testing both)
  if (d.z != 0.0f) consider(d.z < 0.0f ? S_BOT : S_TOP, __fdividef(d.z < 0.0f ? -p.z : h.thick - p.z, d.z));
  if (h.dims == 3 && d.y != 0.0f)
    consider(d.y > 0.0f ? S_YPOS : S_YNEG, __fdividef(d.y > 0.0f ? h.half_w - p.y : -h.half_w - p.y, d.y));
  const int K = h.n_mir;
  int k0 = 0, k1 = K;
  bool left = true, right = true;
  if (reg >= 0) {
    k0 = max(reg - 1, 0);
    k1 = min(reg + 1, K);
    left = reg == 0;
    right = reg == K;
  }
  if (left) {
    const float dn = fmaf(d.x, h.ic_nx, d.z * h.ic_nz);
    if (dn > 0.0f) consider(S_LEFT, __fdividef(-fmaf(p.x, h.ic_nx, p.z * h.ic_nz), dn));
  }
  if (right && d.x > 0.0f) consider(S_RIGHT, __fdividef(h.x_end - p.x, d.x));
  auto plane = [&](int k) {
    const float4 m = *reinterpret_cast<const float4*>(&B.mir[k]);  // (nx, ny, nz, c)
    const float den = fmaf(d.x, m.x, fmaf(d.y, m.y, d.z * m.z));
    if (den != 0.0f) consider(S_MIR + k, __fdividef(m.w - fmaf(p.x, m.x, fmaf(p.y, m.y, p.z * m.z)), den));
  };
  auto prma_planes = [&]() {
    if (reg >= 0) {
      // the two planes bounding the region (one at either end), in order
      if (reg > 0) plane(reg - 1);
      if (reg < K) plane(reg);
    } else {
      for (int k = k0; k < k1; ++k) plane(k);
    }
  };
  if constexpr (GM == 0) {
    prma_planes();
  } else if constexpr (GM == 1) {
    next_mirror_families(B, p, d, last, best, id);
  } else {
    if (!h.general) prma_planes();
    else next_mirror_general(B, p, d, last, best, id);
  }
  tmin = best;
  return id;
}

// region after leaving mirror plane k with direction d: the side of the
// plane that d points to (k + 1 = larger x); -1 stays -1 (unordered design)
__device__ __forceinline__ int region_after(const Blob& B, int reg, int k, V3 d) {
  if (reg < 0) return reg;
  const MirrorRec& m = B.mir[k];
  return fmaf(d.x, m.nx, fmaf(d.y, m.ny, d.z * m.nz)) * m.nx > 0.0f ? k + 1 : k;
}

// TIR at a slab face against air: r_s, r_p with u = n cos_i, a = sqrt(n^2 sin^2 - 1)
//   r_s = (u + i a)/(u - i a), r_p = (c + i n a)/(c - i n a)   (cos_t = -i a)
__device__ __forceinline__ void tir_coef(float n, float ci, float sin2, float2& rs, float2& rp) {
  // a from the hardware reciprocal square root (TIR: a^2 > 0; the phase only)
  const float a2 = fmaxf(fmaf(n * n, sin2, -1.0f), 1e-30f);
  const float a = a2 * rsqrtf(a2);
  const float u = n * ci;
  const float iu = __fdividef(1.0f, fmaf(u, u, a * a));
  rs = make_float2(fmaf(u, u, -a * a) * iu, 2.0f * u * a * iu);
  const float na = n * a;
  const float ip = __fdividef(1.0f, fmaf(ci, ci, na * na));
  rp = make_float2(fmaf(ci, ci, -na * na) * ip, 2.0f * ci * na * ip);
}

__device__ __forceinline__ uint32_t fnv(uint32_t h, uint32_t b) { return (h ^ b) * 16777619u; }

// ---------------------------------------------------------------------------
// Forward-mode derivatives for the mirror-tilt gradient. The sampled path is
// held fixed (keys, surfaces, decisions, TIR counts, tally bin), so a tilt
// acts through the incidence angles (the coefficients of every layer stack),
// the local s/p bases, the reflected directions and the angle-dependent TIR
// and exit Fresnel factors; positions do not reach the intensity.
// ---------------------------------------------------------------------------
// d/d(cos i) of the TIR coefficients at a slab face (|r| = 1: r = e^{2i phi},
// dr = 2i r dphi) for cos i = ci
__device__ __forceinline__ void tir_coef_d(float n, float ci, float2 rs, float2 rp, float2& drs, float2& drp) {
  const float a2 = fmaf(n * n, fmaf(-ci, ci, 1.0f), -1.0f);
  const float a = sqrtf(fmaxf(a2, 1e-30f));
  const float da = -n * n * ci / a;
  const float u = n * ci;
  const float dphi = (u * da - a * n) / fmaf(u, u, a * a);
  const float na = n * a;
  const float dpsi = (ci * n * da - na) / fmaf(ci, ci, na * na);
  drs = make_float2(-2.0f * dphi * rs.y, 2.0f * dphi * rs.x);
  drp = make_float2(-2.0f * dpsi * rp.y, 2.0f * dpsi * rp.x);
}

// d/d(cos i) of the exit power transmittances T_s, T_p (glass -> air)
__device__ __forceinline__ void exit_T_d(float n, float ci, float& dTs, float& dTp) {
  const float x = n * n * fmaf(-ci, ci, 1.0f);
  const float ct = sqrtf(fmaxf(1.0f - x, 1e-30f));
  const float dct = n * n * ci / ct;
  const float u = n * ci, du = n;
  const float ts = 2.0f * u / (u + ct), tp = 2.0f * u / fmaf(n, ct, ci);
  const float dts = 2.0f * (du * ct - u * dct) / ((u + ct) * (u + ct));
  const float dtpd = fmaf(n, ct, ci);
  const float dtp = 2.0f * (du * dtpd - u * fmaf(n, dct, 1.0f)) / (dtpd * dtpd);
  const float tf = ct / u, dtf = (dct * u - ct * du) / (u * u);
  dTs = fmaf(dtf, ts * ts, 2.0f * tf * ts * dts);
  dTp = fmaf(dtf, tp * tp, 2.0f * tf * tp * dtp);
}

// tangents of the face basis s = (d_y, -d_x, 0)/h, p = s x d. With
// (d_x, d_y) = h (cos psi, sin psi), s only turns with the azimuth psi:
// ds = (d_x, d_y, 0)/h dpsi, dpsi = (d_x dd_y - d_y dd_x)/h^2. Written this way
// ds stays orthogonal to s for any h (differentiating s/h term by term leaves
// a rounding residue times 1/h along s, which near a vertical direction is
// a spurious scaling of the field), and it is exactly zero in a 2D slab.
__device__ __forceinline__ void face_basis_d(V3 d, V3 dd, V3 s, V3& ds, V3& dp) {
  const float h2 = fmaf(d.x, d.x, d.y * d.y);
  if (h2 > 1e-30f) {
    const float r = rsqrtf(h2);
    const float dpsi = fmaf(d.x, dd.y, -d.y * dd.x) * (r * r);
    ds = V3{d.x * r * dpsi, d.y * r * dpsi, 0.0f};
  } else {
    ds = V3{0.0f, 0.0f, 0.0f};
  }
  const V3 a = cross3(ds, d), b = cross3(s, dd);
  dp = V3{a.x + b.x, a.y + b.y, a.z + b.z};
}

// tangent of w / |w|
__device__ __forceinline__ V3 normalize_d(V3 w, V3 dw) {
  const float r = rsqrtf(dot3(w, w));
  const float k = dot3(w, dw) * r * r;
  return V3{(dw.x - w.x * k) * r, (dw.y - w.y * k) * r, (dw.z - w.z * k) * r};
}

}  // namespace wgk
