// FP64 CPU oracle for the Monte Carlo polarization ray trace through a slab
// waveguide with a partially reflective mirror array (PRMA), its multilayer
// thin-film coatings, and the adjoint of the trace.
//
// TEST INFRASTRUCTURE ONLY. This file is a plain, slow, obviously-correct
// restatement of the method of "End-to-end differentiable design of geometric
// waveguide displays" (Yang et al., arXiv 2601.04370). Only tests/, the smoke
// check in __graft_entry__ and bench.py's CPU-baseline / reference legs may
// load the library built from it. It shares no code, header or constant table
// with the CUDA path.
//
// Sections of the paper followed here:
//   * Methods, "Multilayer thin-film solver": Fresnel coefficients (Eq. 2,
//     fresnel_coefficients), Airy single-layer formulas (Eq. 3, airy_formulas)
//     and the transfer-matrix method (Heavens) for multilayer stacks.
//   * Methods, "Polarization ray tracing": reflected / transmitted complex
//     amplitudes E_r = r_s E_s s + r_p E_p p, E_t = t_s E_s s' + t_p E_p p'
//     (Eq. 4, complex_amplitudes), basis recomputed at every interface.
//   * Methods, "Differentiable Monte Carlo non-sequential ray tracing":
//     reflect with probability w, rescale the amplitude by 1/sqrt(w) or
//     1/sqrt(1-w) (Eq. 5); incoherent intensity I = sum |E|^2.
//   * Results, "System Architecture": slab waveguide, TIR, input mirror,
//     PRMA, eyebox at an eye relief.
//   * Results, Eq. 1 (loss) lives in oracle.py (numpy).
//
// Readings where the paper is silent:
//   - time convention exp(+i w t): the Airy phase factor is exp(-2 i delta) as
//     printed, and an evanescent cos(theta) is -i sqrt(n0^2 sin^2/n^2 - 1);
//   - the p-polarized TMM result is quoted in the paper's Fresnel sign
//     convention (r_p = -r_s at normal incidence): r_p = -r_p(Abeles), and
//     t_p = t_p(Abeles) * cos(theta_0) / cos(theta_sub);
//   - layer 1 faces the mirror's +normal side; a ray arriving from the
//     -normal side sees the stack reversed; pruned layers are skipped;
//   - the mirrors sit inside the glass, so incident = exit medium.
//
// Parity unpinned: nothing. Every public function is pinned by a test in
// tests/test_oracle_*.py (closed forms, textbook identities, brute force,
// finite differences, published Philox known-answer vectors).

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <type_traits>
#include <vector>

namespace ora {

// ---------------------------------------------------------------------------
// Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11,
// "Parallel random numbers: as easy as 1, 2, 3"): ten rounds of two 32x32->64
// multiplies with the key bumped by the Weyl constants between rounds.
// ---------------------------------------------------------------------------
struct U4 {
  uint32_t v[4];
};

static U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += W0;
      k1 += W1;
    }
    uint64_t p0 = (uint64_t)M0 * c.v[0];
    uint64_t p1 = (uint64_t)M1 * c.v[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    U4 n;
    n.v[0] = hi1 ^ c.v[1] ^ k0;
    n.v[1] = lo1;
    n.v[2] = hi0 ^ c.v[3] ^ k1;
    n.v[3] = lo0;
    c = n;
  }
  return c;
}

// Counter layout of the method's random numbers:
//   launch draw : ctr = (ray lo, ray hi, 0, TAG_GEN)
//   mirror hit m: ctr = (ray lo, ray hi, m >> 2, TAG_EVT), word m & 3
static const uint32_t TAG_GEN = 0x47454E30u;  // "GEN0"
static const uint32_t TAG_EVT = 0x45565430u;  // "EVT0"

// uniform in [0,1) with 24 random bits: exactly representable in FP32
static double u24(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0); }

// ---------------------------------------------------------------------------
// Reverse-mode automatic differentiation on a per-thread tape. Used for the
// oracle's adjoint: gradients of the ray intensity with respect to layer
// thicknesses and mirror tilts along each ray's sampled path.
// ---------------------------------------------------------------------------
struct Tape {
  struct Node {
    int a, b;
    double da, db;
  };
  std::vector<Node> nodes;
  int push(int a, double da, int b, double db) {
    nodes.push_back(Node{a, b, da, db});
    return (int)nodes.size() - 1;
  }
};
static thread_local Tape* g_tape = nullptr;

struct Var {
  double v;
  int id;  // < 0: constant
  Var() : v(0.0), id(-1) {}
  Var(double x) : v(x), id(-1) {}
  static Var leaf(double x) {
    Var r;
    r.v = x;
    r.id = g_tape->push(-1, 0.0, -1, 0.0);
    return r;
  }
};

static inline Var mk(double v, int a, double da, int b, double db) {
  if (a < 0 && b < 0) return Var(v);
  Var r;
  r.v = v;
  r.id = g_tape->push(a, da, b, db);
  return r;
}
static inline bool is_const_zero(const Var& x) { return x.id < 0 && x.v == 0.0; }
static inline Var operator+(Var x, Var y) { return mk(x.v + y.v, x.id, 1.0, y.id, 1.0); }
static inline Var operator-(Var x, Var y) { return mk(x.v - y.v, x.id, 1.0, y.id, -1.0); }
static inline Var operator-(Var x) { return mk(-x.v, x.id, -1.0, -1, 0.0); }
static inline Var operator*(Var x, Var y) {
  if (is_const_zero(x) || is_const_zero(y)) return Var(0.0);
  return mk(x.v * y.v, x.id, y.v, y.id, x.v);
}
static inline Var operator/(Var x, Var y) {
  if (is_const_zero(x)) return Var(0.0);
  double q = x.v / y.v;
  return mk(q, x.id, 1.0 / y.v, y.id, -q / y.v);
}
static inline Var sqrt(Var x) {
  double r = std::sqrt(x.v);
  return mk(r, x.id, r > 0 ? 0.5 / r : 0.0, -1, 0.0);
}
static inline Var sin(Var x) { return mk(std::sin(x.v), x.id, std::cos(x.v), -1, 0.0); }
static inline Var cos(Var x) { return mk(std::cos(x.v), x.id, -std::sin(x.v), -1, 0.0); }
static inline Var exp(Var x) {
  double e = std::exp(x.v);
  return mk(e, x.id, e, -1, 0.0);
}

static inline double val(double x) { return x; }
static inline double val(const Var& x) { return x.v; }
using std::cos;
using std::exp;
using std::sin;
using std::sqrt;

// ---------------------------------------------------------------------------
// Complex numbers over a real scalar type T (double or Var).
// ---------------------------------------------------------------------------
template <class T>
struct Cx {
  T re, im;
  Cx() : re(0.0), im(0.0) {}
  Cx(T r) : re(r), im(0.0) {}
  Cx(T r, T i) : re(r), im(i) {}
};
template <class T>
static inline Cx<T> operator+(const Cx<T>& a, const Cx<T>& b) {
  return Cx<T>(a.re + b.re, a.im + b.im);
}
template <class T>
static inline Cx<T> operator-(const Cx<T>& a, const Cx<T>& b) {
  return Cx<T>(a.re - b.re, a.im - b.im);
}
template <class T>
static inline Cx<T> operator-(const Cx<T>& a) {
  return Cx<T>(-a.re, -a.im);
}
template <class T>
static inline Cx<T> operator*(const Cx<T>& a, const Cx<T>& b) {
  return Cx<T>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <class T>
static inline Cx<T> scale(const Cx<T>& a, const T& s) {
  return Cx<T>(a.re * s, a.im * s);
}
template <class T>
static inline Cx<T> operator/(const Cx<T>& a, const Cx<T>& b) {
  T den = b.re * b.re + b.im * b.im;
  return Cx<T>((a.re * b.re + a.im * b.im) / den, (a.im * b.re - a.re * b.im) / den);
}
template <class T>
static inline T abs2(const Cx<T>& a) {
  return a.re * a.re + a.im * a.im;
}
template <class T>
static inline Cx<T> mul_i(const Cx<T>& a) {  // i * a
  return Cx<T>(-a.im, a.re);
}
// cos and sin of a complex argument a + ib:
//   cos(a+ib) = cos a cosh b - i sin a sinh b,  sin(a+ib) = sin a cosh b + i cos a sinh b
template <class T>
static inline void ccos_sin(const Cx<T>& z, Cx<T>& c, Cx<T>& s) {
  T ca = cos(z.re), sa = sin(z.re);
  T ep = exp(z.im), em = exp(-z.im);
  T ch = (ep + em) * T(0.5), sh = (ep - em) * T(0.5);
  c = Cx<T>(ca * ch, -(sa * sh));
  s = Cx<T>(sa * ch, ca * sh);
}

// cos(theta) in a medium of index n for a wave whose transverse invariant is
// n0 sin(theta0), with cos(theta0) real. Propagating: real positive root.
// Evanescent: -i sqrt(n0^2 sin^2 / n^2 - 1) (decays for exp(+i w t)).
template <class T>
static inline Cx<T> snell_cos(double n0, const T& cos0, double n) {
  T sin2 = T(1.0) - cos0 * cos0;
  T rad = T(1.0) - sin2 * T((n0 / n) * (n0 / n));
  if (val(rad) >= 0.0) return Cx<T>(sqrt(rad), T(0.0));
  return Cx<T>(T(0.0), -sqrt(-rad));
}

// ---------------------------------------------------------------------------
// Fresnel coefficients at one interface (Methods, Eq. fresnel_coefficients):
//   r_s = (n_i c_i - n_j c_t)/(n_i c_i + n_j c_t),  t_s = 2 n_i c_i/(n_i c_i + n_j c_t)
//   r_p = (n_j c_i - n_i c_t)/(n_j c_i + n_i c_t),  t_p = 2 n_i c_i/(n_j c_i + n_i c_t)
// with cos(theta_i) possibly complex (inside an evanescent layer).
// ---------------------------------------------------------------------------
template <class T>
struct Fresnel {
  Cx<T> rs, ts, rp, tp;
};
template <class T>
static Fresnel<T> fresnel(double ni, double nj, const Cx<T>& ci, const Cx<T>& ct) {
  Fresnel<T> f;
  Cx<T> ni_ci = scale(ci, T(ni)), nj_ct = scale(ct, T(nj));
  Cx<T> nj_ci = scale(ci, T(nj)), ni_ct = scale(ct, T(ni));
  f.rs = (ni_ci - nj_ct) / (ni_ci + nj_ct);
  f.ts = scale(ni_ci, T(2.0)) / (ni_ci + nj_ct);
  f.rp = (nj_ci - ni_ct) / (nj_ci + ni_ct);
  f.tp = scale(ni_ci, T(2.0)) / (nj_ci + ni_ct);
  return f;
}

// ---------------------------------------------------------------------------
// Multilayer stack by the characteristic-matrix (transfer-matrix) method of
// Heavens / Abeles, per polarization, on an incident medium n0 and exit
// medium nsub, layers listed from the incident side. Per layer
//   delta = 2 pi n d cos(theta) / lambda,
//   M = [[cos delta, i sin delta / eta], [i eta sin delta, cos delta]],
//   eta_s = n cos(theta), eta_p = n / cos(theta).
// [B, C]^T = M_1 ... M_L [1, eta_sub]^T,  r = (eta0 B - C)/(eta0 B + C),
// t = 2 eta0 / (eta0 B + C). Results are returned in the paper's Fresnel
// convention (see file header).
// ---------------------------------------------------------------------------
template <class T>
struct Coef {
  Cx<T> rs, rp, ts, tp;
};
template <class T>
struct M2 {
  Cx<T> a, b, c, d;  // [[a, b], [c, d]]
};
template <class T>
static M2<T> mmul(const M2<T>& x, const M2<T>& y) {
  M2<T> z;
  z.a = x.a * y.a + x.b * y.c;
  z.b = x.a * y.b + x.b * y.d;
  z.c = x.c * y.a + x.d * y.c;
  z.d = x.c * y.b + x.d * y.d;
  return z;
}

// characteristic matrices of the whole stack for s and p
template <class T>
static void stack_matrix(double n0, const T& cos0, int L, const double* n, const T* d,
                         double lambda, M2<T>& Ms, M2<T>& Mp) {
  M2<T> I;
  I.a = Cx<T>(T(1.0));
  I.b = Cx<T>(T(0.0));
  I.c = Cx<T>(T(0.0));
  I.d = Cx<T>(T(1.0));
  Ms = I;
  Mp = I;
  for (int l = 0; l < L; ++l) {
    Cx<T> cl = snell_cos(n0, cos0, n[l]);
    Cx<T> delta = scale(cl, d[l] * T(2.0 * M_PI * n[l] / lambda));
    Cx<T> cd, sd;
    ccos_sin(delta, cd, sd);
    Cx<T> eta_s = scale(cl, T(n[l]));
    Cx<T> eta_p = Cx<T>(T(n[l])) / cl;
    M2<T> ls, lp;
    ls.a = cd;
    ls.b = mul_i(sd / eta_s);
    ls.c = mul_i(eta_s * sd);
    ls.d = cd;
    lp.a = cd;
    lp.b = mul_i(sd / eta_p);
    lp.c = mul_i(eta_p * sd);
    lp.d = cd;
    Ms = mmul(Ms, ls);
    Mp = mmul(Mp, lp);
  }
}

template <class T>
static Coef<T> tmm(double n0, double nsub, const T& cos0, int L, const double* n, const T* d,
                   double lambda) {
  M2<T> Ms, Mp;
  stack_matrix(n0, cos0, L, n, d, lambda, Ms, Mp);
  Cx<T> c0(cos0, T(0.0));
  Cx<T> csub = snell_cos(n0, cos0, nsub);
  Coef<T> out;
  for (int pol = 0; pol < 2; ++pol) {
    const M2<T>& M = pol == 0 ? Ms : Mp;
    Cx<T> eta0 = pol == 0 ? scale(c0, T(n0)) : Cx<T>(T(n0)) / c0;
    Cx<T> etas = pol == 0 ? scale(csub, T(nsub)) : Cx<T>(T(nsub)) / csub;
    Cx<T> B = M.a + M.b * etas;
    Cx<T> C = M.c + M.d * etas;
    Cx<T> den = eta0 * B + C;
    Cx<T> r = (eta0 * B - C) / den;
    Cx<T> t = scale(eta0, T(2.0)) / den;
    if (pol == 0) {
      out.rs = r;
      out.ts = t;
    } else {
      out.rp = -r;
      out.tp = t * (c0 / csub);
    }
  }
  return out;
}

// ---------------------------------------------------------------------------
// 3-vectors
// ---------------------------------------------------------------------------
template <class T>
struct V3 {
  T x, y, z;
  V3() : x(0.0), y(0.0), z(0.0) {}
  V3(T a, T b, T c) : x(a), y(b), z(c) {}
};
template <class T>
static inline V3<T> operator+(const V3<T>& a, const V3<T>& b) {
  return V3<T>(a.x + b.x, a.y + b.y, a.z + b.z);
}
template <class T>
static inline V3<T> operator-(const V3<T>& a, const V3<T>& b) {
  return V3<T>(a.x - b.x, a.y - b.y, a.z - b.z);
}
template <class T>
static inline V3<T> operator*(const V3<T>& a, const T& s) {
  return V3<T>(a.x * s, a.y * s, a.z * s);
}
template <class T>
static inline T dot(const V3<T>& a, const V3<T>& b) {
  return a.x * b.x + a.y * b.y + a.z * b.z;
}
template <class T>
static inline V3<T> cross(const V3<T>& a, const V3<T>& b) {
  return V3<T>(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
template <class T>
static inline V3<T> normalize(const V3<T>& a) {
  T n = sqrt(dot(a, a));
  return V3<T>(a.x / n, a.y / n, a.z / n);
}
// complex field vector
template <class T>
struct E3 {
  Cx<T> x, y, z;
};
template <class T>
static inline Cx<T> edot(const E3<T>& e, const V3<T>& v) {  // E . v (v real)
  return scale(e.x, v.x) + scale(e.y, v.y) + scale(e.z, v.z);
}
template <class T>
static inline E3<T> eaxpy(const Cx<T>& a, const V3<T>& u, const Cx<T>& b, const V3<T>& v) {
  E3<T> r;  // a u + b v
  r.x = scale(a, u.x) + scale(b, v.x);
  r.y = scale(a, u.y) + scale(b, v.y);
  r.z = scale(a, u.z) + scale(b, v.z);
  return r;
}
template <class T>
static inline T enorm2(const E3<T>& e) {
  return abs2(e.x) + abs2(e.y) + abs2(e.z);
}

// s unit vector perpendicular to the plane of incidence spanned by d and the
// surface normal; falls back to any unit vector perpendicular to d at normal
// incidence, where the choice does not change the result.
template <class T>
static V3<T> s_basis(const V3<T>& d, const V3<T>& N) {
  V3<T> s = cross(d, N);
  double m2 = val(dot(s, s));
  if (m2 > 1e-24) return normalize(s);
  V3<T> ax = std::fabs(val(d.x)) < 0.9 ? V3<T>(T(1.0), T(0.0), T(0.0)) : V3<T>(T(0.0), T(1.0), T(0.0));
  return normalize(cross(d, ax));
}

// ---------------------------------------------------------------------------
// Problem description (own POD layout for ctypes; not shared with the GPU).
// ---------------------------------------------------------------------------
extern "C" {
struct OraDesign {
  int32_t dims;            // 2 or 3
  int32_t n_mat;           // materials
  int32_t n_mir;           // PRMA mirrors
  int32_t pad0;
  double n_slab;           // glass index
  double thickness_mm;     // slab thickness, z in [0, t]
  double width_mm;         // 3D lateral width, y in [-w/2, w/2]
  double x_end_mm;         // absorbing right end
  double eye_relief_mm;    // eye plane at z = t + eye_relief
  double ic_tilt_deg;      // input mirror tilt (plane through origin)
  const double* mat_n;     // [n_mat]
  const double* mir_x_mm;  // [n_mir] mirror centre x (at z = t/2)
  const double* mir_tilt_deg;  // [n_mir]
  const float* mir_omega;      // [n_mir] reflection probability (FP32)
  const int32_t* n_layers;     // [n_mir]
  const int32_t* layer_mat;    // [sum n_layers]
  const double* layer_d_nm;    // [sum n_layers]
  const uint8_t* pruned;       // [sum n_layers]
  // NULL: every mirror is a PRMA plane (above). Else row k (14 values) makes
  // mirror k a general plane: normal N0 at the tilt t0, pivot point, tilt
  // axis a (unit, perpendicular to N0), the rectangle [x0, x1] x [y0, y1] of
  // the slab's (x, y) where it acts, and t0 (deg).
  const double* mir_geo;
};
struct OraCfg {
  int32_t n_lam, n_fx, n_fy, pol;  // pol: 0 s+p pair, 1 random linear, 2 s, 3 p
  int64_t n_rays;                  // requested; N_cell = ceil(n_rays / cells)
  uint64_t seed;
  int32_t max_events;
  int32_t eb_nx, eb_ny;
  int32_t lut_bins;  // 0: exact coefficients per hit; N: the coating table (see mirror_coef)
  double pupil_y_mm;
  double eb_cx_mm, eb_cy_mm, eb_w_mm, eb_h_mm;
  const double* lam_nm;   // [n_lam]
  const double* fx_deg;   // [n_fx]
  const double* fy_deg;   // [n_fy]
};
struct OraRayRec {
  uint32_t hash;
  int32_t n_events;
  int32_t n_hits;
  int32_t cat;
  int32_t bin;  // flat tally index or -1
  int32_t pad;
  double I;     // tallied intensity (0 unless cat == EYEBOX)
  double w;     // final |E|^2 (pair-averaged)
};
struct OraStats {
  int64_t n_hits;    // ray-mirror (PRMA) interactions
  int64_t n_events;  // all surface events
  int64_t n_tir;
  int64_t n_rays;
};
}

enum Cat { EYEBOX = 0, MISSED = 1, EXIT_REFL = 2, LEAKED = 3, ABSORBED = 4, TRUNCATED = 5 };
enum Surf { S_BOT = 0, S_TOP = 1, S_LEFT = 2, S_RIGHT = 3, S_YNEG = 4, S_YPOS = 5, S_MIR = 8 };
static const int NLEDGER = 6;

static inline int64_t cells_of(const OraCfg& c) { return (int64_t)c.n_lam * c.n_fx * c.n_fy; }
static inline int64_t n_cell_of(const OraCfg& c) {
  int64_t cells = cells_of(c);
  return (c.n_rays + cells - 1) / cells;
}
static inline int64_t bins_per_cell(const OraCfg& c) { return (int64_t)c.eb_nx * c.eb_ny; }

static inline uint32_t fnv(uint32_t h, uint32_t byte) { return (h ^ byte) * 16777619u; }

// Per-mirror parameters that the adjoint differentiates.
template <class T>
struct Params {
  std::vector<T> d;      // thickness of every layer, all mirrors (nm)
  std::vector<T> tilt;   // tilt of every mirror (rad)
};

template <class T>
struct RayOut {
  T I;
  int bin;
  int cat;
  int n_events, n_hits, n_tir;
  uint32_t hash;
  double w;
};

static const double DEG = M_PI / 180.0;

// ---------------------------------------------------------------------------
// Ray generation (Results, System Architecture: parallel rays per FoV sample
// from the panel, coupled into the slab by the input mirror). The launch
// point is drawn on the input mirror, the field direction is refracted into
// the glass and reflected by the input mirror into the guided direction.
// ---------------------------------------------------------------------------
template <class T>
struct Launch {
  V3<T> p, d;
  int F;          // field vectors carried (2 for the s+p pair)
  E3<T> E[2];
  int lam_i, f;   // wavelength index, field index
  double lambda;
};

template <class T>
static Launch<T> launch(const OraDesign& D, const OraCfg& C, uint64_t ray) {
  Launch<T> L;
  int64_t nf = (int64_t)C.n_fx * C.n_fy;
  int64_t cell = (int64_t)(ray / (uint64_t)n_cell_of(C));
  L.lam_i = (int)(cell / nf);
  L.f = (int)(cell % nf);
  int fy = L.f / C.n_fx, fx = L.f % C.n_fx;
  L.lambda = C.lam_nm[L.lam_i];
  U4 ctr = {{(uint32_t)ray, (uint32_t)(ray >> 32), 0u, TAG_GEN}};
  U4 r0 = philox4x32_10(ctr, (uint32_t)C.seed, (uint32_t)(C.seed >> 32));
  double u0 = u24(r0.v[0]), u1 = u24(r0.v[1]), u2 = u24(r0.v[2]);
  const double half_ulp = 1.0 / 33554432.0;  // 2^-25: keeps the point off the faces
  double a_ic = D.ic_tilt_deg * DEG;
  double z0 = D.thickness_mm * (u0 + half_ulp);
  double x0 = z0 * std::cos(a_ic) / std::sin(a_ic);
  double y0 = D.dims == 3 ? (u1 + half_ulp - 0.5) * C.pupil_y_mm : 0.0;
  L.p = V3<T>(T(x0), T(y0), T(z0));
  double tx = std::tan(C.fx_deg[fx] * DEG);
  double ty = D.dims == 3 ? std::tan(C.fy_deg[fy] * DEG) : 0.0;
  double an = std::sqrt(tx * tx + ty * ty + 1.0);
  double ax = tx / an, ay = ty / an;
  double n = D.n_slab;
  V3<double> dg(ax / n, ay / n, std::sqrt(1.0 - (ax * ax + ay * ay) / (n * n)));
  V3<double> Nic(-std::sin(a_ic), 0.0, std::cos(a_ic));
  V3<double> d = dg - Nic * (2.0 * dot(dg, Nic));
  L.d = V3<T>(T(d.x), T(d.y), T(d.z));
  // transverse basis of the guided ray: e1 along y projected off d, e2 = d x e1
  V3<double> yv(0.0, 1.0, 0.0);
  V3<double> e1 = normalize(yv - d * dot(yv, d));
  V3<double> e2 = cross(d, e1);
  auto setE = [](E3<T>& E, const V3<double>& v, double a) {
    E.x = Cx<T>(T(v.x * a));
    E.y = Cx<T>(T(v.y * a));
    E.z = Cx<T>(T(v.z * a));
  };
  if (C.pol == 0) {
    L.F = 2;
    setE(L.E[0], e1, 1.0);
    setE(L.E[1], e2, 1.0);
  } else {
    L.F = 1;
    V3<double> v = e1;
    if (C.pol == 1) {
      double phi = M_PI * u2;
      v = e1 * std::cos(phi) + e2 * std::sin(phi);
    } else if (C.pol == 3) {
      v = e2;
    }
    setE(L.E[0], v, 1.0);
  }
  return L;
}

// Mirror geometry. PRMA mirror: plane through (x_k, 0, t/2) with normal
// (-sin a, 0, cos a) at tilt a. General mirror (row k of mir_geo): normal
// N(a) = cos(a - a0) N0 + sin(a - a0) (axis x N0), the rotation of N0 about
// the axis by a - a0 (a0 = the row's tilt of N0), normalized, plane through
// the pivot, acting only where the crossing lies in its (x, y) rectangle.
template <class T>
static inline V3<T> mirror_normal(const OraDesign& D, int k, const T& tilt) {
  if (!D.mir_geo) return V3<T>(-sin(tilt), T(0.0), cos(tilt));
  const double* g = D.mir_geo + 14 * k;
  const T del = tilt - T(g[13] * DEG);
  const T c = cos(del), s = sin(del);
  const V3<double> aN = cross(V3<double>(g[6], g[7], g[8]), V3<double>(g[0], g[1], g[2]));
  const V3<T> N(c * T(g[0]) + s * T(aN.x), c * T(g[1]) + s * T(aN.y), c * T(g[2]) + s * T(aN.z));
  // unit to FP64 rounding (the stored values are float32)
  const T inv = T(1.0) / sqrt(N.x * N.x + N.y * N.y + N.z * N.z);
  return V3<T>(N.x * inv, N.y * inv, N.z * inv);
}
static inline V3<double> mirror_pivot(const OraDesign& D, int k) {
  if (!D.mir_geo) return V3<double>(D.mir_x_mm[k], 0.0, 0.5 * D.thickness_mm);
  const double* g = D.mir_geo + 14 * k;
  return V3<double>(g[3], g[4], g[5]);
}

// Nearest surface along the ray; excludes the surface the ray sits on.
template <class T>
static int next_surface(const OraDesign& D, const Params<T>& P, const V3<T>& p, const V3<T>& d,
                        int last, T& tmin) {
  double best = INFINITY;
  int id = -1;
  auto consider = [&](int sid, const T& t) {
    if (sid == last) return;
    double tv = val(t);
    if (tv > 0.0 && tv < best) {
      best = tv;
      id = sid;
      tmin = t;
    }
  };
  double tz = D.thickness_mm;
  if (val(d.z) < 0.0) consider(S_BOT, (T(0.0) - p.z) / d.z);
  if (val(d.z) > 0.0) consider(S_TOP, (T(tz) - p.z) / d.z);
  double a_ic = D.ic_tilt_deg * DEG;
  V3<T> Nic(T(-std::sin(a_ic)), T(0.0), T(std::cos(a_ic)));
  T dn = dot(d, Nic);
  if (val(dn) > 0.0) consider(S_LEFT, -dot(p, Nic) / dn);
  if (val(d.x) > 0.0) consider(S_RIGHT, (T(D.x_end_mm) - p.x) / d.x);
  if (D.dims == 3) {
    double hw = 0.5 * D.width_mm;
    if (val(d.y) > 0.0) consider(S_YPOS, (T(hw) - p.y) / d.y);
    if (val(d.y) < 0.0) consider(S_YNEG, (T(-hw) - p.y) / d.y);
  }
  for (int k = 0; k < D.n_mir; ++k) {
    V3<T> N = mirror_normal(D, k, P.tilt[k]);
    T den = dot(d, N);
    if (val(den) == 0.0) continue;
    const V3<double> pv = mirror_pivot(D, k);
    V3<T> c(T(pv.x), T(pv.y), T(pv.z));
    const T t = dot(c - p, N) / den;
    if (D.mir_geo) {
      // a general mirror acts only inside its rectangle
      const double* g = D.mir_geo + 14 * k;
      const double qx = val(p.x) + val(t) * val(d.x), qy = val(p.y) + val(t) * val(d.y);
      if (!(qx >= g[9] && qx <= g[10] && qy >= g[11] && qy <= g[12])) continue;
    }
    consider(S_MIR + k, t);
  }
  return id;
}

// one surface event of a ray, for geometric checks
extern "C" {
struct OraPathEv {
  int32_t surf;      // surface id (0 bottom, 1 top, 2 input mirror, 3 right end, 4/5 sides, 8+k mirror k)
  int32_t refl;      // 1 if reflected (mirror decision or TIR)
  double p[3];       // event position (mm)
  double d_in[3];    // direction before the event
  double d_out[3];   // direction after the event (air direction for an exit)
};
}

template <class T>
struct TraceCtx {
  const OraDesign* D;
  const OraCfg* C;
  const Params<T>* P;
  std::vector<int> layer_off;  // first layer of each mirror in the flat arrays
  std::vector<OraPathEv>* path = nullptr;
};

template <class T>
static void record(const TraceCtx<T>& X, int sid, bool refl, const V3<T>& p, const V3<T>& din,
                   const V3<double>& dout) {
  if (!X.path) return;
  OraPathEv e;
  e.surf = sid;
  e.refl = refl ? 1 : 0;
  e.p[0] = val(p.x), e.p[1] = val(p.y), e.p[2] = val(p.z);
  e.d_in[0] = val(din.x), e.d_in[1] = val(din.y), e.d_in[2] = val(din.z);
  e.d_out[0] = dout.x, e.d_out[1] = dout.y, e.d_out[2] = dout.z;
  X.path->push_back(e);
}
template <class T>
static V3<double> vval(const V3<T>& v) {
  return V3<double>(val(v.x), val(v.y), val(v.z));
}

// Effective coefficients of mirror k seen from side `front`.
template <class T>
static Coef<T> mirror_coef_at(const TraceCtx<T>& X, int k, bool front, const T& cos_i, double lambda) {
  const OraDesign& D = *X.D;
  int off = X.layer_off[k], L = D.n_layers[k];
  std::vector<double> n;
  std::vector<T> d;
  n.reserve(L);
  d.reserve(L);
  for (int j = 0; j < L; ++j) {
    int l = front ? j : L - 1 - j;
    if (D.pruned[off + l]) continue;
    n.push_back(D.mat_n[D.layer_mat[off + l]]);
    d.push_back(X.P->d[off + l]);
  }
  return tmm(D.n_slab, D.n_slab, cos_i, (int)n.size(), n.data(), d.data(), lambda);
}

// Exact coefficients of mirror k's stack in FP64 at cos(theta_0) = c (the
// thicknesses' values), for the look-up table's grid derivatives.
template <class T>
static Coef<double> mirror_coef_value(const TraceCtx<T>& X, int k, bool front, double c, double lambda) {
  const OraDesign& D = *X.D;
  int off = X.layer_off[k], L = D.n_layers[k];
  std::vector<double> n, d;
  for (int j = 0; j < L; ++j) {
    int l = front ? j : L - 1 - j;
    if (D.pruned[off + l]) continue;
    n.push_back(D.mat_n[D.layer_mat[off + l]]);
    d.push_back(val(X.P->d[off + l]));
  }
  return tmm(D.n_slab, D.n_slab, c, (int)n.size(), n.data(), d.data(), lambda);
}

// d/d(cos t0) of the exact coefficients at c: central differences at h and
// h/2 combined by Richardson extrapolation (error O(h^4) ~ 1e-20 relative
// to the fringe scale, rounding ~1e-11), in FP64.
template <class T>
static Coef<double> mirror_coef_dcos(const TraceCtx<T>& X, int k, bool front, double c, double lambda) {
  auto cd = [&](double h) {
    const Coef<double> p = mirror_coef_value(X, k, front, c + h, lambda);
    const Coef<double> m = mirror_coef_value(X, k, front, c - h, lambda);
    const double s = 1.0 / (2.0 * h);
    Coef<double> r;
    r.rs = scale(p.rs - m.rs, s);
    r.rp = scale(p.rp - m.rp, s);
    r.ts = scale(p.ts - m.ts, s);
    r.tp = scale(p.tp - m.tp, s);
    return r;
  };
  const double h = 1e-5;
  const Coef<double> a = cd(h), b = cd(0.5 * h);
  Coef<double> r;
  r.rs = scale(b.rs, 4.0 / 3.0) - scale(a.rs, 1.0 / 3.0);
  r.rp = scale(b.rp, 4.0 / 3.0) - scale(a.rp, 1.0 / 3.0);
  r.ts = scale(b.ts, 4.0 / 3.0) - scale(a.ts, 1.0 / 3.0);
  r.tp = scale(b.tp, 4.0 / 3.0) - scale(a.tp, 1.0 / 3.0);
  return r;
}

// Coefficients of a hit. With C.lut_bins = N > 0, the coating look-up table
// of the paper's memory-saving variant (Fig. 3c, Results): the stack's
// coefficients and their derivatives with respect to cos(theta_0) are known
// at the N bin centres cos_j = (j + 1/2) / N, and a hit interpolates both
// linearly between the two centres that bracket its cos(theta_0) (weights
// clamped to the end points). The value is that interpolation of the exact
// coefficients (a function of the thicknesses through both entries); its
// derivative with respect to cos(theta_0) (through which the mirror tilts act)
// is the interpolated exact derivative. Written out as that definition.
template <class T>
static Coef<T> mirror_coef(const TraceCtx<T>& X, int k, bool front, const T& cos_i, double lambda) {
  const int N = X.C->lut_bins;
  if (N <= 0) return mirror_coef_at(X, k, front, cos_i, lambda);
  const double ci = val(cos_i);
  const double x = ci * N - 0.5;  // position in bins: cos_j = (j + 1/2) / N
  int j = (int)std::floor(x);
  j = std::min(std::max(j, 0), N - 2);
  const double cj = (j + 0.5) / N, cj1 = (j + 1.5) / N;
  const double f = std::min(std::max((ci - cj) * N, 0.0), 1.0);
  const Coef<T> a = mirror_coef_at(X, k, front, T(cj), lambda);
  const Coef<T> b = mirror_coef_at(X, k, front, T(cj1), lambda);
  Coef<T> c;
  c.rs = a.rs + scale(b.rs - a.rs, T(f));
  c.rp = a.rp + scale(b.rp - a.rp, T(f));
  c.ts = a.ts + scale(b.ts - a.ts, T(f));
  c.tp = a.tp + scale(b.tp - a.tp, T(f));
  if constexpr (!std::is_same<T, double>::value) {
    // the cos(theta_0) dependence: (cos_i - its value) times the interpolated derivative
    const Coef<double> da = mirror_coef_dcos(X, k, front, cj, lambda);
    const Coef<double> db = mirror_coef_dcos(X, k, front, cj1, lambda);
    const T dx = cos_i - T(ci);
    auto term = [&](const Cx<double>& p, const Cx<double>& q) {
      const Cx<double> dd = p + scale(q - p, f);
      return scale(Cx<T>(T(dd.re), T(dd.im)), dx);
    };
    c.rs = c.rs + term(da.rs, db.rs);
    c.rp = c.rp + term(da.rp, db.rp);
    c.ts = c.ts + term(da.ts, db.ts);
    c.tp = c.tp + term(da.tp, db.tp);
  }
  return c;
}

// One Monte Carlo ray (Methods: polarization ray tracing + MC sampling).
template <class T>
static RayOut<T> trace_ray(const TraceCtx<T>& X, uint64_t ray) {
  const OraDesign& D = *X.D;
  const OraCfg& C = *X.C;
  Launch<T> L = launch<T>(D, C, ray);
  RayOut<T> out;
  out.I = T(0.0);
  out.bin = -1;
  out.cat = TRUNCATED;
  out.n_events = out.n_hits = out.n_tir = 0;
  out.hash = 2166136261u;
  out.w = 0.0;
  V3<T> p = L.p, d = L.d;
  E3<T> E[2] = {L.E[0], L.E[1]};
  const int F = L.F;
  const double n = D.n_slab;
  int last = S_LEFT;
  for (int ev = 0; ev < C.max_events; ++ev) {
    T tmin(0.0);
    int sid = next_surface(D, *X.P, p, d, last, tmin);
    out.n_events = ev + 1;
    if (sid < 0) {  // cannot happen inside a closed slab; treat as absorbed
      double w = 0.0;
      for (int f = 0; f < F; ++f) w += val(enorm2(E[f]));
      out.w = w / F;
      out.cat = ABSORBED;
      break;
    }
    p = p + d * tmin;
    last = sid;
    if (sid >= S_MIR) {
      int k = sid - S_MIR;
      V3<T> N = mirror_normal(*X.D, k, X.P->tilt[k]);
      T cd = dot(d, N);
      bool front = val(cd) < 0.0;
      T cos_i = front ? -cd : cd;
      Coef<T> cf = mirror_coef(X, k, front, cos_i, L.lambda);
      V3<T> s = s_basis(d, N);
      V3<T> pv = cross(s, d);
      int m = out.n_hits++;
      U4 ctr = {{(uint32_t)ray, (uint32_t)(ray >> 32), (uint32_t)(m >> 2), TAG_EVT}};
      U4 rr = philox4x32_10(ctr, (uint32_t)C.seed, (uint32_t)(C.seed >> 32));
      double u = u24(rr.v[m & 3]);
      double w = (double)D.mir_omega[k];
      bool refl = u < w;
      out.hash = fnv(out.hash, (uint32_t)sid | (refl ? 0x80u : 0u));
      if (refl) {
        V3<T> d2 = d - N * (cd * T(2.0));
        record(X, sid, true, p, d, vval(d2));
        V3<T> p2 = cross(s, d2);
        T sc = T(1.0 / std::sqrt(w));
        for (int f = 0; f < F; ++f) {
          Cx<T> Es = edot(E[f], s), Ep = edot(E[f], pv);
          E[f] = eaxpy(scale(cf.rs * Es, sc), s, scale(cf.rp * Ep, sc), p2);
        }
        d = d2;
      } else {
        record(X, sid, false, p, d, vval(d));
        T sc = T(1.0 / std::sqrt(1.0 - w));
        for (int f = 0; f < F; ++f) {
          Cx<T> Es = edot(E[f], s), Ep = edot(E[f], pv);
          E[f] = eaxpy(scale(cf.ts * Es, sc), s, scale(cf.tp * Ep, sc), pv);
        }
      }
      continue;
    }
    out.hash = fnv(out.hash, (uint32_t)sid);
    if (sid == S_BOT || sid == S_TOP) {
      V3<T> Nz(T(0.0), T(0.0), T(1.0));
      T cz = d.z;
      T cos_i = val(cz) < 0.0 ? -cz : cz;
      T sin2 = T(1.0) - cz * cz;
      double x = n * n * val(sin2);
      V3<T> s = s_basis(d, Nz);
      V3<T> pv = cross(s, d);
      if (x > 1.0) {  // total internal reflection against air
        out.n_tir++;
        Cx<T> ct(T(0.0), -sqrt(sin2 * T(n * n) - T(1.0)));
        Fresnel<T> fr = fresnel(n, 1.0, Cx<T>(cos_i), ct);
        V3<T> d2(d.x, d.y, -d.z);
        V3<T> p2 = cross(s, d2);
        record(X, sid, true, p, d, vval(d2));
        for (int f = 0; f < F; ++f) {
          Cx<T> Es = edot(E[f], s), Ep = edot(E[f], pv);
          E[f] = eaxpy(fr.rs * Es, s, fr.rp * Ep, p2);
        }
        d = d2;
        continue;
      }
      T w = T(0.0);
      for (int f = 0; f < F; ++f) w = w + enorm2(E[f]);
      w = w * T(1.0 / F);
      out.w = val(w);
      if (sid == S_BOT) {
        record(X, sid, false, p, d, vval(d));
        out.cat = LEAKED;
        break;
      }
      // exit through the eye-side face: Fresnel power transmission glass->air
      T ct = sqrt(T(1.0) - sin2 * T(n * n));
      Fresnel<T> fr = fresnel(n, 1.0, Cx<T>(cos_i), Cx<T>(ct));
      T tf = ct / (cos_i * T(n));
      T Ts = abs2(fr.ts) * tf, Tp = abs2(fr.tp) * tf;
      T I = T(0.0);
      for (int f = 0; f < F; ++f) {
        Cx<T> Es = edot(E[f], s), Ep = edot(E[f], pv);
        I = I + Ts * abs2(Es) + Tp * abs2(Ep);
      }
      I = I * T(1.0 / F);
      // propagate in air to the eye plane
      double ax = n * val(d.x), ay = n * val(d.y), az = val(ct);
      record(X, sid, false, p, d, V3<double>(ax, ay, az));
      double sfac = D.eye_relief_mm / az;
      double qx = val(p.x) + sfac * ax, qy = val(p.y) + sfac * ay;
      int ex = (int)std::floor((qx - (C.eb_cx_mm - 0.5 * C.eb_w_mm)) / C.eb_w_mm * C.eb_nx);
      int ey = 0;
      bool inside = ex >= 0 && ex < C.eb_nx;
      if (D.dims == 3) {
        ey = (int)std::floor((qy - (C.eb_cy_mm - 0.5 * C.eb_h_mm)) / C.eb_h_mm * C.eb_ny);
        inside = inside && ey >= 0 && ey < C.eb_ny;
      }
      out.I = I;
      if (inside) {
        out.cat = EYEBOX;
        int64_t cell = (int64_t)L.lam_i * C.n_fx * C.n_fy + L.f;
        out.bin = (int)(cell * bins_per_cell(C) + (int64_t)ey * C.eb_nx + ex);
      } else {
        out.cat = MISSED;
      }
      break;
    }
    // input-mirror side, right end, lateral sides: absorbed
    record(X, sid, false, p, d, vval(d));
    T w = T(0.0);
    for (int f = 0; f < F; ++f) w = w + enorm2(E[f]);
    out.w = val(w) / F;
    out.cat = ABSORBED;
    break;
  }
  if (out.cat == TRUNCATED) {
    double w = 0.0;
    for (int f = 0; f < F; ++f) w += val(enorm2(E[f]));
    out.w = w / F;
  }
  return out;
}

static void add_ledger(double* led, const RayOut<double>& r) {
  switch (r.cat) {
    case EYEBOX:
      led[EYEBOX] += r.I;
      led[EXIT_REFL] += r.w - r.I;
      break;
    case MISSED:
      led[MISSED] += r.I;
      led[EXIT_REFL] += r.w - r.I;
      break;
    default:
      led[r.cat] += r.w;
  }
}

template <class T>
static TraceCtx<T> make_ctx(const OraDesign& D, const OraCfg& C, const Params<T>& P) {
  TraceCtx<T> X;
  X.D = &D;
  X.C = &C;
  X.P = &P;
  X.layer_off.resize(D.n_mir + 1);
  X.layer_off[0] = 0;
  for (int k = 0; k < D.n_mir; ++k) X.layer_off[k + 1] = X.layer_off[k] + D.n_layers[k];
  return X;
}

static Params<double> params_of(const OraDesign& D) {
  Params<double> P;
  int nl = 0;
  for (int k = 0; k < D.n_mir; ++k) nl += D.n_layers[k];
  P.d.assign(D.layer_d_nm, D.layer_d_nm + nl);
  for (int k = 0; k < D.n_mir; ++k) P.tilt.push_back(D.mir_tilt_deg[k] * DEG);
  return P;
}

static int pick_threads(int nthreads, int64_t work) {
  int hw = (int)std::thread::hardware_concurrency();
  if (hw <= 0) hw = 1;
  int t = nthreads > 0 ? nthreads : hw;
  if ((int64_t)t > work) t = (int)std::max<int64_t>(1, work);
  return t;
}

// Runs fn(thread_index, begin, end) over contiguous ray ranges.
template <class Fn>
static void parallel_rays(int nt, int64_t r0, int64_t r1, Fn fn) {
  std::vector<std::thread> th;
  int64_t n = r1 - r0;
  for (int i = 0; i < nt; ++i) {
    int64_t a = r0 + n * i / nt, b = r0 + n * (i + 1) / nt;
    th.emplace_back([=]() { fn(i, a, b); });
  }
  for (auto& t : th) t.join();
}

// ---------------------------------------------------------------------------
// Brute-force deterministic ray splitting (the exponential-cost reference the
// paper compares the MC estimator with): both branches at every mirror, full
// amplitudes, same launch points and the same event cap.
// ---------------------------------------------------------------------------
struct SplitAcc {
  double* tally;  // local tally for cells [cell0, ...)
  int64_t cell0;
  double* led;
  int64_t branches;
  double prune;
};

static void split_rec(const TraceCtx<double>& X, SplitAcc& A, int cell, double lambda, V3<double> p,
                      V3<double> d, E3<double> E0, E3<double> E1, int F, int last, int ev) {
  const OraDesign& D = *X.D;
  const OraCfg& C = *X.C;
  const double n = D.n_slab;
  E3<double> E[2] = {E0, E1};
  auto wsum = [&]() {
    double w = 0.0;
    for (int f = 0; f < F; ++f) w += enorm2(E[f]);
    return w / F;
  };
  for (; ev < C.max_events; ++ev) {
    double tmin = 0.0;
    int sid = next_surface(D, *X.P, p, d, last, tmin);
    if (sid < 0) {
      A.led[ABSORBED] += wsum();
      return;
    }
    p = p + d * tmin;
    last = sid;
    if (sid >= S_MIR) {
      int k = sid - S_MIR;
      V3<double> N = mirror_normal(*X.D, k, X.P->tilt[k]);
      double cd = dot(d, N);
      bool front = cd < 0.0;
      Coef<double> cf = mirror_coef(X, k, front, front ? -cd : cd, lambda);
      V3<double> s = s_basis(d, N);
      V3<double> pv = cross(s, d);
      V3<double> d2 = d - N * (2.0 * cd);
      V3<double> p2 = cross(s, d2);
      E3<double> Er[2], Et[2];
      for (int f = 0; f < F; ++f) {
        Cx<double> Es = edot(E[f], s), Ep = edot(E[f], pv);
        Er[f] = eaxpy(cf.rs * Es, s, cf.rp * Ep, p2);
        Et[f] = eaxpy(cf.ts * Es, s, cf.tp * Ep, pv);
      }
      A.branches++;
      double wr = 0.0, wt = 0.0;
      for (int f = 0; f < F; ++f) {
        wr += enorm2(Er[f]);
        wt += enorm2(Et[f]);
      }
      wr /= F;
      wt /= F;
      if (wr > A.prune)
        split_rec(X, A, cell, lambda, p, d2, Er[0], Er[1], F, sid, ev + 1);
      else
        A.led[TRUNCATED] += wr;
      if (wt > A.prune)
        split_rec(X, A, cell, lambda, p, d, Et[0], Et[1], F, sid, ev + 1);
      else
        A.led[TRUNCATED] += wt;
      return;
    }
    if (sid == S_BOT || sid == S_TOP) {
      double cz = d.z, cos_i = std::fabs(cz), sin2 = 1.0 - cz * cz;
      V3<double> s = s_basis(d, V3<double>(0.0, 0.0, 1.0));
      V3<double> pv = cross(s, d);
      if (n * n * sin2 > 1.0) {
        Cx<double> ct(0.0, -std::sqrt(n * n * sin2 - 1.0));
        Fresnel<double> fr = fresnel(n, 1.0, Cx<double>(cos_i), ct);
        V3<double> d2(d.x, d.y, -d.z);
        V3<double> p2 = cross(s, d2);
        for (int f = 0; f < F; ++f) {
          Cx<double> Es = edot(E[f], s), Ep = edot(E[f], pv);
          E[f] = eaxpy(fr.rs * Es, s, fr.rp * Ep, p2);
        }
        d = d2;
        continue;
      }
      double w = wsum();
      if (sid == S_BOT) {
        A.led[LEAKED] += w;
        return;
      }
      double ct = std::sqrt(1.0 - n * n * sin2);
      Fresnel<double> fr = fresnel(n, 1.0, Cx<double>(cos_i), Cx<double>(ct));
      double tf = ct / (n * cos_i);
      double Ts = abs2(fr.ts) * tf, Tp = abs2(fr.tp) * tf;
      double I = 0.0;
      for (int f = 0; f < F; ++f) {
        Cx<double> Es = edot(E[f], s), Ep = edot(E[f], pv);
        I += Ts * abs2(Es) + Tp * abs2(Ep);
      }
      I /= F;
      double sfac = D.eye_relief_mm / ct;
      double qx = p.x + sfac * n * d.x, qy = p.y + sfac * n * d.y;
      int ex = (int)std::floor((qx - (C.eb_cx_mm - 0.5 * C.eb_w_mm)) / C.eb_w_mm * C.eb_nx);
      int ey = 0;
      bool inside = ex >= 0 && ex < C.eb_nx;
      if (D.dims == 3) {
        ey = (int)std::floor((qy - (C.eb_cy_mm - 0.5 * C.eb_h_mm)) / C.eb_h_mm * C.eb_ny);
        inside = inside && ey >= 0 && ey < C.eb_ny;
      }
      if (inside) {
        A.tally[(cell - A.cell0) * bins_per_cell(C) + (int64_t)ey * C.eb_nx + ex] += I;
        A.led[EYEBOX] += I;
      } else {
        A.led[MISSED] += I;
      }
      A.led[EXIT_REFL] += w - I;
      return;
    }
    A.led[ABSORBED] += wsum();
    return;
  }
  A.led[TRUNCATED] += wsum();
}

}  // namespace ora

using namespace ora;

extern "C" {

int ora_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
  U4 c = {{ctr[0], ctr[1], ctr[2], ctr[3]}};
  U4 r = philox4x32_10(c, key[0], key[1]);
  for (int i = 0; i < 4; ++i) out[i] = r.v[i];
  return 0;
}

// Fresnel coefficients for real n_i, n_j and real incidence cos_i; cos_t from
// Snell with the evanescent branch. out = rs, ts, rp, tp as (re, im) pairs.
int ora_fresnel(double ni, double nj, double cos_i, double* out) {
  Cx<double> ct = snell_cos(ni, cos_i, nj);
  Fresnel<double> f = fresnel(ni, nj, Cx<double>(cos_i), ct);
  const Cx<double> v[4] = {f.rs, f.ts, f.rp, f.tp};
  for (int i = 0; i < 4; ++i) {
    out[2 * i] = v[i].re;
    out[2 * i + 1] = v[i].im;
  }
  return 0;
}

// Stack coefficients by the characteristic-matrix method.
// out = rs, rp, ts, tp as (re, im) pairs.
int ora_tmm(double n0, double nsub, int L, const double* n, const double* d, double lambda,
            double cos0, double* out) {
  Coef<double> c = tmm(n0, nsub, cos0, L, n, d, lambda);
  const Cx<double> v[4] = {c.rs, c.rp, c.ts, c.tp};
  for (int i = 0; i < 4; ++i) {
    out[2 * i] = v[i].re;
    out[2 * i + 1] = v[i].im;
  }
  return 0;
}

// The two characteristic matrices (s, p): out = [s: a b c d, p: a b c d] as
// (re, im) pairs, 16 values.
int ora_stack_matrix(double n0, int L, const double* n, const double* d, double lambda, double cos0,
                     double* out) {
  M2<double> Ms, Mp;
  stack_matrix(n0, cos0, L, n, d, lambda, Ms, Mp);
  const Cx<double> v[8] = {Ms.a, Ms.b, Ms.c, Ms.d, Mp.a, Mp.b, Mp.c, Mp.d};
  for (int i = 0; i < 8; ++i) {
    out[2 * i] = v[i].re;
    out[2 * i + 1] = v[i].im;
  }
  return 0;
}

// Stack coefficients by repeated application of the paper's Airy formula
// (Eq. airy_formulas): starting at the substrate, each layer with the
// effective interface below it is replaced by one equivalent interface.
// Independent of the matrix route; used to pin ora_tmm.
int ora_airy_stack(double n0, double nsub, int L, const double* n, const double* d, double lambda,
                   double cos0, double* out) {
  // media 0..L+1: incident, layers, substrate
  std::vector<double> nm(L + 2);
  nm[0] = n0;
  for (int l = 0; l < L; ++l) nm[l + 1] = n[l];
  nm[L + 1] = nsub;
  std::vector<Cx<double>> cm(L + 2);
  for (int j = 0; j < L + 2; ++j) cm[j] = snell_cos(n0, cos0, nm[j]);
  for (int pol = 0; pol < 2; ++pol) {
    // effective coefficients of everything below medium j, seen from medium j
    Fresnel<double> fb = fresnel(nm[L], nm[L + 1], cm[L], cm[L + 1]);
    Cx<double> r = pol == 0 ? fb.rs : fb.rp;
    Cx<double> t = pol == 0 ? fb.ts : fb.tp;
    for (int j = L; j >= 1; --j) {
      Fresnel<double> f = fresnel(nm[j - 1], nm[j], cm[j - 1], cm[j]);
      Cx<double> r12 = pol == 0 ? f.rs : f.rp;
      Cx<double> t12 = pol == 0 ? f.ts : f.tp;
      Cx<double> delta = scale(cm[j], 2.0 * M_PI * nm[j] * d[j - 1] / lambda);
      // e^{-i delta} and e^{-2 i delta}
      Cx<double> mid(delta.im, -delta.re);  // -i delta
      double mag = std::exp(mid.re);
      Cx<double> e1(mag * std::cos(mid.im), mag * std::sin(mid.im));
      Cx<double> e2 = e1 * e1;
      Cx<double> den = Cx<double>(1.0) + r12 * r * e2;
      Cx<double> rn = (r12 + r * e2) / den;
      Cx<double> tn = (t12 * t * e1) / den;
      r = rn;
      t = tn;
    }
    if (pol == 0) {
      out[0] = r.re;
      out[1] = r.im;
      out[4] = t.re;
      out[5] = t.im;
    } else {
      out[2] = r.re;
      out[3] = r.im;
      out[6] = t.re;
      out[7] = t.im;
    }
  }
  return 0;
}

// Gradient of f = 2 Re(A_s c_s + A_p c_p) with respect to every layer
// thickness (nm) and to cos(theta_0), where c = r (which == 0) or t (which == 1)
// and A = (A_s, A_p) complex. Reverse-mode AD through ora_tmm's arithmetic.
// out_f receives f.
int ora_tmm_grad(double n0, int L, const double* n, const double* d, double lambda, double cos0,
                 const double* A, int which, double* grad_d, double* grad_cos0, double* out_f) {
  Tape tape;
  Tape* prev = g_tape;
  g_tape = &tape;
  std::vector<Var> dv(L);
  for (int l = 0; l < L; ++l) dv[l] = Var::leaf(d[l]);
  Var c0 = Var::leaf(cos0);
  Coef<Var> c = tmm(n0, n0, c0, L, n, dv.data(), lambda);
  Cx<Var> cs = which == 0 ? c.rs : c.ts;
  Cx<Var> cp = which == 0 ? c.rp : c.tp;
  Cx<Var> As{Var{A[0]}, Var{A[1]}}, Ap{Var{A[2]}, Var{A[3]}};
  Cx<Var> s = As * cs + Ap * cp;
  Var f = s.re * Var(2.0);
  std::vector<double> adj(tape.nodes.size(), 0.0);
  if (f.id >= 0) adj[f.id] = 1.0;
  for (int i = (int)tape.nodes.size() - 1; i >= 0; --i) {
    double g = adj[i];
    if (g == 0.0) continue;
    const Tape::Node& nd = tape.nodes[i];
    if (nd.a >= 0) adj[nd.a] += g * nd.da;
    if (nd.b >= 0) adj[nd.b] += g * nd.db;
  }
  for (int l = 0; l < L; ++l) grad_d[l] = dv[l].id >= 0 ? adj[dv[l].id] : 0.0;
  *grad_cos0 = adj[c0.id];
  *out_f = f.v;
  g_tape = prev;
  return 0;
}

// Monte Carlo forward trace of rays [r0, r1). tally (size cells*bins) and
// ledger[6] are overwritten. recs (nullable) receives one record per ray.
int ora_trace(const OraDesign* D, const OraCfg* C, int64_t r0, int64_t r1, int nthreads,
              double* tally, double* ledger, OraStats* stats, OraRayRec* recs) {
  Params<double> P = params_of(*D);
  TraceCtx<double> X = make_ctx(*D, *C, P);
  int64_t bpc = bins_per_cell(*C), ncell = n_cell_of(*C);
  int64_t total = cells_of(*C) * bpc;
  std::memset(tally, 0, sizeof(double) * total);
  for (int i = 0; i < NLEDGER; ++i) ledger[i] = 0.0;
  int nt = pick_threads(nthreads, r1 - r0);
  struct Part {
    std::vector<double> tally;
    int64_t cell0 = 0;
    double led[NLEDGER] = {0, 0, 0, 0, 0, 0};
    OraStats st = {0, 0, 0, 0};
  };
  std::vector<Part> parts(nt);
  parallel_rays(nt, r0, r1, [&](int ti, int64_t a, int64_t b) {
    Part& pt = parts[ti];
    if (a >= b) return;
    pt.cell0 = a / ncell;
    int64_t cell1 = (b - 1) / ncell;
    pt.tally.assign((cell1 - pt.cell0 + 1) * bpc, 0.0);
    for (int64_t r = a; r < b; ++r) {
      RayOut<double> o = trace_ray(X, (uint64_t)r);
      if (o.cat == EYEBOX) pt.tally[o.bin - pt.cell0 * bpc] += o.I;
      add_ledger(pt.led, o);
      pt.st.n_hits += o.n_hits;
      pt.st.n_events += o.n_events;
      pt.st.n_tir += o.n_tir;
      pt.st.n_rays += 1;
      if (recs) {
        OraRayRec& rc = recs[r - r0];
        rc.hash = o.hash;
        rc.n_events = o.n_events;
        rc.n_hits = o.n_hits;
        rc.cat = o.cat;
        rc.bin = o.cat == EYEBOX ? o.bin : -1;
        rc.pad = 0;
        rc.I = o.cat == EYEBOX ? o.I : 0.0;
        rc.w = o.w;
      }
    }
  });
  OraStats st = {0, 0, 0, 0};
  for (auto& pt : parts) {  // fixed-order reduction
    for (size_t i = 0; i < pt.tally.size(); ++i) tally[pt.cell0 * bpc + (int64_t)i] += pt.tally[i];
    for (int i = 0; i < NLEDGER; ++i) ledger[i] += pt.led[i];
    st.n_hits += pt.st.n_hits;
    st.n_events += pt.st.n_events;
    st.n_tir += pt.st.n_tir;
    st.n_rays += pt.st.n_rays;
  }
  if (stats) *stats = st;
  return 0;
}

// Deterministic splitting expectation for the launch points of rays [r0, r1).
// Branches whose power falls to `prune` or below are booked as truncated
// (prune = 0 keeps every branch).
int ora_split(const OraDesign* D, const OraCfg* C, int64_t r0, int64_t r1, int nthreads, double prune,
              double* tally, double* ledger, int64_t* n_branches) {
  Params<double> P = params_of(*D);
  TraceCtx<double> X = make_ctx(*D, *C, P);
  int64_t bpc = bins_per_cell(*C), ncell = n_cell_of(*C);
  std::memset(tally, 0, sizeof(double) * cells_of(*C) * bpc);
  for (int i = 0; i < NLEDGER; ++i) ledger[i] = 0.0;
  int nt = pick_threads(nthreads, r1 - r0);
  struct Part {
    std::vector<double> tally;
    int64_t cell0 = 0;
    double led[NLEDGER] = {0, 0, 0, 0, 0, 0};
    int64_t br = 0;
  };
  std::vector<Part> parts(nt);
  parallel_rays(nt, r0, r1, [&](int ti, int64_t a, int64_t b) {
    Part& pt = parts[ti];
    if (a >= b) return;
    pt.cell0 = a / ncell;
    int64_t cell1 = (b - 1) / ncell;
    pt.tally.assign((cell1 - pt.cell0 + 1) * bpc, 0.0);
    SplitAcc A;
    A.tally = pt.tally.data();
    A.cell0 = pt.cell0;
    A.led = pt.led;
    A.branches = 0;
    A.prune = prune;
    for (int64_t r = a; r < b; ++r) {
      Launch<double> L = launch<double>(*D, *C, (uint64_t)r);
      int cell = L.lam_i * C->n_fx * C->n_fy + L.f;
      split_rec(X, A, cell, L.lambda, L.p, L.d, L.E[0], L.E[1], L.F, S_LEFT, 0);
    }
    pt.br = A.branches;
  });
  int64_t br = 0;
  for (auto& pt : parts) {
    for (size_t i = 0; i < pt.tally.size(); ++i) tally[pt.cell0 * bpc + (int64_t)i] += pt.tally[i];
    for (int i = 0; i < NLEDGER; ++i) ledger[i] += pt.led[i];
    br += pt.br;
  }
  if (n_branches) *n_branches = br;
  return 0;
}

// Adjoint of the Monte Carlo trace: for the loss gradient G = dL/dtally,
//   grad_d[l]    = sum_rays G[bin(ray)] dI_ray/d d_l      (per nm; 0 for pruned)
//   grad_tilt[k] = sum_rays G[bin(ray)] dI_ray/d tilt_k   (per degree)
// along each ray's sampled path (keys, decisions, surface sequence and bin
// held fixed). mask (nullable, one byte per ray of [r0, r1)) restricts the
// sum to rays with a nonzero mask byte. ray_I (nullable) receives each ray's
// tallied intensity (0 if not tallied).
int ora_trace_grad(const OraDesign* D, const OraCfg* C, int64_t r0, int64_t r1, int nthreads,
                   const double* G, const uint8_t* mask, double* grad_d, double* grad_tilt,
                   double* ray_I) {
  int nl = 0;
  for (int k = 0; k < D->n_mir; ++k) nl += D->n_layers[k];
  int K = D->n_mir;
  for (int i = 0; i < nl; ++i) grad_d[i] = 0.0;
  for (int k = 0; k < K; ++k) grad_tilt[k] = 0.0;
  int nt = pick_threads(nthreads, r1 - r0);
  std::vector<std::vector<double>> gd(nt, std::vector<double>(nl, 0.0));
  std::vector<std::vector<double>> gt(nt, std::vector<double>(K, 0.0));
  parallel_rays(nt, r0, r1, [&](int ti, int64_t a, int64_t b) {
    Tape tape;
    g_tape = &tape;
    std::vector<double> adj;
    for (int64_t r = a; r < b; ++r) {
      tape.nodes.clear();
      Params<Var> P;
      P.d.resize(nl);
      for (int i = 0; i < nl; ++i) P.d[i] = Var::leaf(D->layer_d_nm[i]);
      for (int k = 0; k < K; ++k) P.tilt.push_back(Var::leaf(D->mir_tilt_deg[k] * DEG));
      TraceCtx<Var> X = make_ctx(*D, *C, P);
      RayOut<Var> o = trace_ray(X, (uint64_t)r);
      if (ray_I) ray_I[r - r0] = o.cat == EYEBOX ? o.I.v : 0.0;
      if (o.cat != EYEBOX || o.I.id < 0) continue;
      if (mask && !mask[r - r0]) continue;
      double g = G[o.bin];
      if (g == 0.0) continue;
      adj.assign(tape.nodes.size(), 0.0);
      adj[o.I.id] = g;
      for (int i = (int)tape.nodes.size() - 1; i >= 0; --i) {
        double v = adj[i];
        if (v == 0.0) continue;
        const Tape::Node& nd = tape.nodes[i];
        if (nd.a >= 0) adj[nd.a] += v * nd.da;
        if (nd.b >= 0) adj[nd.b] += v * nd.db;
      }
      for (int i = 0; i < nl; ++i)
        if (!D->pruned[i]) gd[ti][i] += adj[P.d[i].id];
      for (int k = 0; k < K; ++k) gt[ti][k] += adj[P.tilt[k].id] * DEG;
    }
    g_tape = nullptr;
  });
  for (int t = 0; t < nt; ++t) {
    for (int i = 0; i < nl; ++i) grad_d[i] += gd[t][i];
    for (int k = 0; k < K; ++k) grad_tilt[k] += gt[t][k];
  }
  return 0;
}

// Event list of one ray (geometry checks). Returns the number of events
// written (at most cap) and the ray's category in *cat.
int ora_trace_path(const OraDesign* D, const OraCfg* C, int64_t ray, OraPathEv* out, int cap,
                   int* cat, double* intensity) {
  Params<double> P = params_of(*D);
  TraceCtx<double> X = make_ctx(*D, *C, P);
  std::vector<OraPathEv> path;
  X.path = &path;
  RayOut<double> o = trace_ray(X, (uint64_t)ray);
  int n = (int)std::min<size_t>(path.size(), (size_t)cap);
  for (int i = 0; i < n; ++i) out[i] = path[i];
  if (cat) *cat = o.cat;
  if (intensity) *intensity = o.I;
  return n;
}

int ora_hardware_threads(void) {
  int hw = (int)std::thread::hardware_concurrency();
  return hw > 0 ? hw : 1;
}

// ---------------------------------------------------------------------------
// Reflection-probability pre-optimization (Methods, "Learned reflection
// probabilities"): each coating idealized as a scalar reflectance, here equal
// to its mirror's omega, and geometric ray tracing without polarization. At a
// slab face a ray beyond the critical angle reflects completely (TIR);
// otherwise the eye-side face transmits the unpolarized Fresnel power
// (T_s + T_p) / 2 and the ray is tallied at the eye plane, and the back face
// leaks. With the sampling probability equal to the reflectance every path
// has weight one, and the derivative of the expected tally with respect to
// omega_k is the score-function estimator
//   d E[I] / d omega_k = E[ I (n_r,k / omega_k - n_t,k / (1 - omega_k)) ]
// (n_r,k / n_t,k: the path's reflections / transmissions at mirror k).
// ---------------------------------------------------------------------------
// the eye-side exit: unpolarized transmittance and flat tally index (-1 outside the eyebox)
static double geo_exit(const OraDesign& D, const OraCfg& C, const V3<double>& p, const V3<double>& d, int64_t cell,
                       int64_t& flat) {
  const double n = D.n_slab, cos_i = std::fabs(d.z), sin2 = 1.0 - d.z * d.z;
  const double ct = std::sqrt(1.0 - n * n * sin2);
  Fresnel<double> fr = fresnel(n, 1.0, Cx<double>(cos_i), Cx<double>(ct));
  const double tf = ct / (cos_i * n);
  const double T = 0.5 * (abs2(fr.ts) + abs2(fr.tp)) * tf;
  const double ax = n * d.x, ay = n * d.y, az = ct;
  const double sfac = D.eye_relief_mm / az;
  const double qx = p.x + sfac * ax, qy = p.y + sfac * ay;
  int ex = (int)std::floor((qx - (C.eb_cx_mm - 0.5 * C.eb_w_mm)) / C.eb_w_mm * C.eb_nx);
  int ey = 0;
  bool inside = ex >= 0 && ex < C.eb_nx;
  if (D.dims == 3) {
    ey = (int)std::floor((qy - (C.eb_cy_mm - 0.5 * C.eb_h_mm)) / C.eb_h_mm * C.eb_ny);
    inside = inside && ey >= 0 && ey < C.eb_ny;
  }
  flat = inside ? cell * bins_per_cell(C) + (int64_t)ey * C.eb_nx + ex : -1;
  return T;
}

// one Monte Carlo ray of the geometric trace: adds its tallied power to
// tally (local, cells from cell0) and, with G, G[bin] I times its score to grad
static void geo_ray(const TraceCtx<double>& X, uint64_t ray, double* tally, int64_t cell0, const double* G,
                    double* grad) {
  const OraDesign& D = *X.D;
  const OraCfg& C = *X.C;
  Launch<double> L = launch<double>(D, C, ray);
  const int64_t cell = (int64_t)L.lam_i * C.n_fx * C.n_fy + L.f;
  V3<double> p = L.p, d = L.d;
  const double n = D.n_slab;
  std::vector<std::pair<int, bool>> hits;
  int last = S_LEFT, m = 0;
  for (int ev = 0; ev < C.max_events; ++ev) {
    double tmin = 0.0;
    const int sid = next_surface(D, *X.P, p, d, last, tmin);
    if (sid < 0) return;
    p = p + d * tmin;
    last = sid;
    if (sid >= S_MIR) {
      const int k = sid - S_MIR;
      const V3<double> N = mirror_normal(*X.D, k, X.P->tilt[k]);
      const double cd = dot(d, N);
      U4 ctr = {{(uint32_t)ray, (uint32_t)(ray >> 32), (uint32_t)(m >> 2), TAG_EVT}};
      U4 rr = philox4x32_10(ctr, (uint32_t)C.seed, (uint32_t)(C.seed >> 32));
      const bool refl = u24(rr.v[m & 3]) < (double)D.mir_omega[k];
      ++m;
      hits.push_back({k, refl});
      if (refl) d = d - N * (2.0 * cd);
      continue;
    }
    if (sid == S_BOT || sid == S_TOP) {
      if (n * n * (1.0 - d.z * d.z) > 1.0) {
        d = V3<double>(d.x, d.y, -d.z);
        continue;
      }
      if (sid == S_BOT) return;
      int64_t flat;
      const double T = geo_exit(D, C, p, d, cell, flat);
      if (flat < 0) return;
      tally[flat - cell0 * bins_per_cell(C)] += T;
      if (G && grad)
        for (const auto& h : hits) {
          const double w = (double)D.mir_omega[h.first];
          grad[h.first] += G[flat] * T * (h.second ? 1.0 / w : -1.0 / (1.0 - w));
        }
      return;
    }
    return;  // far end, input mirror or a side: absorbed
  }
}

// deterministic splitting of the same model: every branch with its
// probability weight (reflect omega, transmit 1 - omega), pruned below prune
static void geo_split_rec(const TraceCtx<double>& X, double* tally, int64_t cell0, int64_t cell, V3<double> p,
                          V3<double> d, double w, int last, int ev, double prune) {
  const OraDesign& D = *X.D;
  const OraCfg& C = *X.C;
  const double n = D.n_slab;
  for (; ev < C.max_events; ++ev) {
    double tmin = 0.0;
    const int sid = next_surface(D, *X.P, p, d, last, tmin);
    if (sid < 0) return;
    p = p + d * tmin;
    last = sid;
    if (sid >= S_MIR) {
      const int k = sid - S_MIR;
      const V3<double> N = mirror_normal(*X.D, k, X.P->tilt[k]);
      const double om = (double)D.mir_omega[k];
      if (w * om > prune) geo_split_rec(X, tally, cell0, cell, p, d - N * (2.0 * dot(d, N)), w * om, sid, ev + 1, prune);
      if (w * (1.0 - om) > prune) geo_split_rec(X, tally, cell0, cell, p, d, w * (1.0 - om), sid, ev + 1, prune);
      return;
    }
    if (sid == S_BOT || sid == S_TOP) {
      if (n * n * (1.0 - d.z * d.z) > 1.0) {
        d = V3<double>(d.x, d.y, -d.z);
        continue;
      }
      if (sid == S_BOT) return;
      int64_t flat;
      const double T = geo_exit(D, C, p, d, cell, flat);
      if (flat >= 0) tally[flat - cell0 * bins_per_cell(C)] += w * T;
      return;
    }
    return;
  }
}

extern "C" {
// Geometric Monte Carlo trace of rays [r0, r1): tally (full layout, zeroed
// here) and, with G (dL/dtally, full layout), grad_omega[K] = dL/d omega_k.
int ora_geo_trace(const OraDesign* D, const OraCfg* C, int64_t r0, int64_t r1, int nthreads, const double* G,
                  double* tally, double* grad_omega) {
  Params<double> P = params_of(*D);
  TraceCtx<double> X = make_ctx(*D, *C, P);
  const int64_t bpc = bins_per_cell(*C), ncell = n_cell_of(*C);
  std::memset(tally, 0, sizeof(double) * cells_of(*C) * bpc);
  if (grad_omega) std::memset(grad_omega, 0, sizeof(double) * D->n_mir);
  const int nt = pick_threads(nthreads, r1 - r0);
  struct Part {
    std::vector<double> tally, grad;
    int64_t cell0 = 0;
  };
  std::vector<Part> parts(nt);
  parallel_rays(nt, r0, r1, [&](int ti, int64_t a, int64_t b) {
    Part& pt = parts[ti];
    if (a >= b) return;
    pt.cell0 = a / ncell;
    pt.tally.assign(((b - 1) / ncell - pt.cell0 + 1) * bpc, 0.0);
    pt.grad.assign(D->n_mir, 0.0);
    for (int64_t r = a; r < b; ++r) geo_ray(X, (uint64_t)r, pt.tally.data(), pt.cell0, G, pt.grad.data());
  });
  for (auto& pt : parts) {
    for (size_t i = 0; i < pt.tally.size(); ++i) tally[pt.cell0 * bpc + (int64_t)i] += pt.tally[i];
    if (grad_omega)
      for (size_t k = 0; k < pt.grad.size(); ++k) grad_omega[k] += pt.grad[k];
  }
  return 0;
}

// Expected tally of the geometric model for the launches of rays [r0, r1)
// by deterministic splitting (every reflect/transmit branch, weight-pruned).
int ora_geo_split(const OraDesign* D, const OraCfg* C, int64_t r0, int64_t r1, int nthreads, double prune,
                  double* tally) {
  Params<double> P = params_of(*D);
  TraceCtx<double> X = make_ctx(*D, *C, P);
  const int64_t bpc = bins_per_cell(*C), ncell = n_cell_of(*C);
  std::memset(tally, 0, sizeof(double) * cells_of(*C) * bpc);
  const int nt = pick_threads(nthreads, r1 - r0);
  struct Part {
    std::vector<double> tally;
    int64_t cell0 = 0;
  };
  std::vector<Part> parts(nt);
  parallel_rays(nt, r0, r1, [&](int ti, int64_t a, int64_t b) {
    Part& pt = parts[ti];
    if (a >= b) return;
    pt.cell0 = a / ncell;
    pt.tally.assign(((b - 1) / ncell - pt.cell0 + 1) * bpc, 0.0);
    for (int64_t r = a; r < b; ++r) {
      Launch<double> L = launch<double>(*D, *C, (uint64_t)r);
      const int64_t cell = (int64_t)L.lam_i * C->n_fx * C->n_fy + L.f;
      geo_split_rec(X, pt.tally.data(), pt.cell0, cell, L.p, L.d, 1.0, S_LEFT, 0, prune);
    }
  });
  for (auto& pt : parts)
    for (size_t i = 0; i < pt.tally.size(); ++i) tally[pt.cell0 * bpc + (int64_t)i] += pt.tally[i];
  return 0;
}
}  // extern "C"

}  // extern "C"
