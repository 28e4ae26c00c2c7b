// Device building blocks of the shower transport: Philox streams, table lookups, the
// interaction samplers, slab/tube navigation and the analytic helix. Everything is a
// template on the arithmetic type R of the physics: double for the plain FP64 form,
// float for the split form (positions, boundary distances and energies stay double).
#pragma once
#include <cstdint>

#include "layout.h"

namespace adept {

// ---------------------------------------------------------------- constants (PDG/CODATA)
constexpr double kMe = 0.51099895;        // electron mass, MeV
constexpr double kRe = 2.8179403262e-12;  // classical electron radius, mm
constexpr double kAlpha = 1.0 / 137.035999084;
constexpr double kNA = 6.02214076e23;
constexpr double kPi = 3.14159265358979323846;
constexpr double kHelixK = 0.299792458;   // rho[mm] = p[MeV] / (K B[T])
constexpr double kAlphaR = 0.2;           // step function: max(alpha_R R, min(R, rho_f))
constexpr double kRhoF = 1.0;             // mm
constexpr double kBig = 1e300;
// energy grid: ln(1 keV), ln(10)/32 and its inverse, as correctly rounded doubles
constexpr double kLnEmin = -6.907755278982137;
constexpr double kDlog = 0.07195578415606393;
constexpr double kInvDlog = 13.897423420904056;

// numeric helpers per precision
template <class R> struct M;
template <> struct M<double> {
  static __device__ __forceinline__ double log(double x) { return ::log(x); }
  static __device__ __forceinline__ double log1p(double x) { return ::log1p(x); }
  static __device__ __forceinline__ double exp(double x) { return ::exp(x); }
  static __device__ __forceinline__ double sqrt(double x) { return ::sqrt(x); }
  static __device__ __forceinline__ double acos(double x) { return ::acos(x); }
  static __device__ __forceinline__ double atan2(double y, double x) { return ::atan2(y, x); }
  static __device__ __forceinline__ double fmod(double x, double y) { return ::fmod(x, y); }
  static __device__ __forceinline__ void sincos(double x, double* s, double* c) { ::sincos(x, s, c); }
  static __device__ __forceinline__ double cos(double x) { return ::cos(x); }
  static __device__ __forceinline__ double sin(double x) { return ::sin(x); }
  static __device__ __forceinline__ double floor(double x) { return ::floor(x); }
  static __device__ __forceinline__ double fabs(double x) { return ::fabs(x); }
  // "fast" forms: in FP64 the same correctly rounded functions
  static __device__ __forceinline__ double flog(double x) { return ::log(x); }
  static __device__ __forceinline__ double fexp(double x) { return ::exp(x); }
  static __device__ __forceinline__ double fdiv(double a, double b) { return a / b; }
  static __device__ __forceinline__ void fsincos(double x, double* s, double* c) { ::sincos(x, s, c); }
  static __device__ __forceinline__ double fcos(double x) { return ::cos(x); }
  static __host__ __device__ constexpr double big() { return 1e300; }
  static __host__ __device__ constexpr double turn_tol() { return 0.0; }
};
template <> struct M<float> {
  static __device__ __forceinline__ float log(float x) { return ::logf(x); }
  static __device__ __forceinline__ float log1p(float x) { return ::log1pf(x); }
  static __device__ __forceinline__ float exp(float x) { return ::expf(x); }
  static __device__ __forceinline__ float sqrt(float x) { return ::sqrtf(x); }
  static __device__ __forceinline__ float acos(float x) { return ::acosf(x); }
  static __device__ __forceinline__ float atan2(float y, float x) { return ::atan2f(y, x); }
  static __device__ __forceinline__ float fmod(float x, float y) { return ::fmodf(x, y); }
  static __device__ __forceinline__ void sincos(float x, float* s, float* c) { ::sincosf(x, s, c); }
  static __device__ __forceinline__ float cos(float x) { return ::cosf(x); }
  static __device__ __forceinline__ float sin(float x) { return ::sinf(x); }
  static __device__ __forceinline__ float floor(float x) { return ::floorf(x); }
  static __device__ __forceinline__ float fabs(float x) { return ::fabsf(x); }
  // fast forms for the sampling arithmetic (a few ulp; the split form is validated
  // statistically): hardware approximations of log, exp, sin/cos and division. The table
  // grid position, the helix and the boundary geometry keep the accurate functions.
  static __device__ __forceinline__ float flog(float x) { return __logf(x); }
  static __device__ __forceinline__ float fexp(float x) { return __expf(x); }
  static __device__ __forceinline__ float fdiv(float a, float b) { return __fdividef(a, b); }
  static __device__ __forceinline__ void fsincos(float x, float* s, float* c) { __sincosf(x, s, c); }
  static __device__ __forceinline__ float fcos(float x) { return __cosf(x); }
  static __host__ __device__ constexpr float big() { return 1e30f; }
  // a helix root within this many radians below a full turn is the current point seen
  // through FP32 rounding of the phase: treat it as an immediate crossing
  static __host__ __device__ constexpr float turn_tol() { return 2e-5f; }
};

// ---------------------------------------------------------------- FP64 <-> R conversions
// For R = float these work on the bit patterns with integer operations (double -> float
// truncates the significand, float -> double is exact, subnormals flush to zero), which
// keeps the conversions off GB300's narrow FP64 pipe; the values handled (positions,
// energies, path lengths) are far inside the float range.
template <class R> struct Cvt;
template <> struct Cvt<double> {
  static __device__ __forceinline__ double r(double x) { return x; }
  static __device__ __forceinline__ double d(double x) { return x; }
};
template <> struct Cvt<float> {
  static __device__ __forceinline__ float r(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(b >> 32);
    const int e = (int)((hi >> 20) & 0x7FF) - 1023 + 127;
    const unsigned sign = hi & 0x80000000u;
    if (e <= 0) return __uint_as_float(sign);
    if (e >= 255) return __uint_as_float(sign | 0x7F800000u);
    return __uint_as_float(sign | ((unsigned)e << 23) | (unsigned)((b >> 29) & 0x7FFFFFu));
  }
  static __device__ __forceinline__ double d(float f) {
    const unsigned b = __float_as_uint(f);
    const unsigned e = (b >> 23) & 0xFFu;
    const unsigned long long sign = (unsigned long long)(b & 0x80000000u) << 32;
    if (e == 0) return __longlong_as_double((long long)sign);
    const unsigned long long de = e == 255 ? 0x7FFull : (unsigned long long)(e - 127 + 1023);
    return __longlong_as_double((long long)(sign | (de << 52) | ((unsigned long long)(b & 0x7FFFFFu) << 29)));
  }
};
template <class R> __device__ __forceinline__ R to_r(double x) { return Cvt<R>::r(x); }
template <class R> __device__ __forceinline__ double to_d(R x) { return Cvt<R>::d(x); }

// ---------------------------------------------------------------- Philox4x32-10
// Salmon et al., SC'11: ten rounds; each multiplies counter words 0 and 2 by fixed odd
// constants, crosses the high halves with words 1 and 3 and the round key, and bumps
// the key by the Weyl increments 0x9E3779B9 / 0xBB67AE85.
struct U4 { uint32_t a, b, c, d; };

__device__ __forceinline__ U4 philox(U4 x, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * x.a, hi0 = __umulhi(0xD2511F53u, x.a);
    const uint32_t lo1 = 0xCD9E8D57u * x.c, hi1 = __umulhi(0xCD9E8D57u, x.c);
    x = U4{hi1 ^ x.b ^ k0, lo1, hi0 ^ x.d ^ k1, lo0};
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return x;
}

// centred uniforms that can never round to 0 or 1
__device__ __forceinline__ double u01d(uint32_t hi, uint32_t lo) {
  const uint64_t x = ((uint64_t)hi << 20) ^ (uint64_t)(lo >> 12);  // 52 bits
  return ((double)x + 0.5) * (1.0 / 4503599627370496.0);
}
__device__ __forceinline__ float u01f(uint32_t w) {
  return ((float)(w >> 9) + 0.5f) * (1.0f / 8388608.0f);  // 23 bits
}

// Random stream of one (track, step): counter (id lo, id hi, step, block). Block 0 is
// read separately for the interaction length and the process choice; model sampling
// takes blocks 1, 2, ..., two uniforms per block from the word pairs (w0, w1) and
// (w2, w3). The FP32 form takes the top 23 bits of the first word of each pair, so both
// forms walk the same positions of the same stream and a split-precision history stays
// paired with its FP64 counterpart until rounding changes a decision.
template <class R> struct Stream;
template <> struct Stream<double> {
  uint32_t k0, k1, c0, c1, c2, blk;
  U4 w;
  int used;
  __device__ Stream(uint32_t seed, uint32_t ev, uint64_t id, uint32_t step)
      : k0(seed), k1(ev), c0((uint32_t)id), c1((uint32_t)(id >> 32)), c2(step), blk(0), used(4) {}
  __device__ __forceinline__ void block0(double* u0, double* u1) const {
    const U4 r = philox(U4{c0, c1, c2, 0u}, k0, k1);
    *u0 = u01d(r.a, r.b);
    *u1 = u01d(r.c, r.d);
  }
  // the two uniforms of counter block b, outside the sampling sequence
  __device__ __forceinline__ void pair(uint32_t b, double* ua, double* ub) const {
    const U4 r = philox(U4{c0, c1, c2, b}, k0, k1);
    *ua = u01d(r.a, r.b);
    *ub = u01d(r.c, r.d);
  }
  __device__ __forceinline__ double next() {
    if (used >= 4) { w = philox(U4{c0, c1, c2, ++blk}, k0, k1); used = 0; }
    const double u = used == 0 ? u01d(w.a, w.b) : u01d(w.c, w.d);
    used += 2;
    return u;
  }
};
template <> struct Stream<float> {
  uint32_t k0, k1, c0, c1, c2, blk;
  uint32_t w0, w2;
  int used;
  __device__ Stream(uint32_t seed, uint32_t ev, uint64_t id, uint32_t step)
      : k0(seed), k1(ev), c0((uint32_t)id), c1((uint32_t)(id >> 32)), c2(step), blk(0), used(2) {}
  __device__ __forceinline__ void block0(float* u0, float* u1) const {
    const U4 r = philox(U4{c0, c1, c2, 0u}, k0, k1);
    *u0 = u01f(r.a);
    *u1 = u01f(r.c);
  }
  __device__ __forceinline__ void pair(uint32_t b, float* ua, float* ub) const {
    const U4 r = philox(U4{c0, c1, c2, b}, k0, k1);
    *ua = u01f(r.a);
    *ub = u01f(r.c);
  }
  __device__ __forceinline__ float next() {
    if (used >= 2) {
      const U4 r = philox(U4{c0, c1, c2, ++blk}, k0, k1);
      w0 = r.a; w2 = r.c; used = 0;
    }
    return u01f(used++ == 0 ? w0 : w2);
  }
};

// id of the k-th secondary of the interaction at (parent id, parent step)
__device__ __forceinline__ uint64_t child_id(uint32_t seed, uint32_t ev, uint64_t pid,
                                             uint32_t pstep, uint32_t k) {
  const U4 r = philox(U4{(uint32_t)pid, (uint32_t)(pid >> 32), pstep, 0x80000000u | k}, seed, ev);
  return (uint64_t)r.a | ((uint64_t)r.b << 32);
}

// ---------------------------------------------------------------- tables
template <class R> struct Grid {
  static __device__ __forceinline__ R lnEmin() { return (R)kLnEmin; }
  static __device__ __forceinline__ R invd() { return (R)kInvDlog; }
  static __device__ __forceinline__ R dlog() { return (R)kDlog; }
};

// position of E on the grid: bin i in [0, NNODE-2] and fraction t
template <class R>
__device__ __forceinline__ void grid_pos(double E, int* i, R* t);

template <>
__device__ __forceinline__ void grid_pos<double>(double E, int* i, double* t) {
  const double x = (::log(E) - kLnEmin) * kInvDlog;
  int k = (int)::floor(x);
  k = k < 0 ? 0 : (k > kNNode - 2 ? kNNode - 2 : k);
  *i = k;
  *t = x - (double)k;
}

// FP32 form: a float holds the grid coordinate x (up to 288) only to ~2e-5, too coarse for
// a 1e-6 lookup. With E = m 2^k (m in [1/sqrt2, sqrt2), taken from the double's bits),
// x = 96 + k * 32 log10(2) + ln(m) * 32/ln(10); each product is formed exactly with an FMA
// against a two-float constant and the integer parts are set aside, so the fraction t
// carries only the error of logf on m (< 1 ulp) and one rounding of a number below 2.
template <>
__device__ __forceinline__ void grid_pos<float>(double E, int* i, float* t) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(E);
  int k = (int)((b >> 52) & 0x7FF) - 1023;
  float m = __int_as_float(0x3F800000 | (int)((b >> 29) & 0x7FFFFF));       // top 23 mantissa bits
  float mlo = (float)(uint32_t)(b & 0x1FFFFFFFull) * 2.220446049250313e-16f;  // the other 29, * 2^-52
  if (m > 1.41421356f) { m *= 0.5f; mlo *= 0.5f; ++k; }
  const float ln = logf(m) + mlo / m;
  const float kf = (float)k;
  const float c1_hi = 9.632960319519043f, c1_lo = -4.582716428558342e-07f;    // 32 log10(2)
  const float d_hi = 13.89742374420166f, d_lo = -3.232975984701625e-07f;      // 32 / ln(10)
  const float p = kf * c1_hi, pe = fmaf(kf, c1_hi, -p);
  const float q = ln * d_hi, qe = fmaf(ln, d_hi, -q);
  const float ip = floorf(p), iq = floorf(q);
  const float r = ((p - ip) + (q - iq)) + ((pe + kf * c1_lo) + (qe + ln * d_lo));
  const float fr = floorf(r);
  int kk = 96 + (int)ip + (int)iq + (int)fr;
  float tt = r - fr;
  if (kk < 0) { tt += (float)kk; kk = 0; }
  if (kk > kNNode - 2) { tt += (float)(kk - (kNNode - 2)); kk = kNNode - 2; }
  *i = kk;
  *t = tt;
}

template <class R> struct Pair2;
template <> struct Pair2<double> { using T = double2; };
template <> struct Pair2<float> { using T = float2; };

// one interpolated entry of a (value, slope) record
template <class R>
__device__ __forceinline__ R lerp_rec(const typename Pair2<R>::T* rec, int j, R t) {
  const typename Pair2<R>::T v = __ldg(rec + j);
  return v.x + v.y * t;
}

// inverse of the piecewise linear-in-ln(E) range table: 0 below the first node
template <class R>
__device__ __forceinline__ R inverse_range(const R* nodes, R r, int hint_hi) {
  if (!(r >= __ldg(nodes))) return (R)0;
  int lo = 0, hi = hint_hi + 1;
  if (hi > kNNode - 1) hi = kNNode - 1;
  if (r >= __ldg(nodes + hi)) {
    lo = hi;
    hi = kNNode - 1;
    if (r >= __ldg(nodes + hi)) return (R)1e6;
  }
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(nodes + mid) <= r) lo = mid; else hi = mid;
  }
  const R a = __ldg(nodes + lo), b = __ldg(nodes + lo + 1);
  const R t = M<R>::fdiv(r - a, b - a);
  return M<R>::fexp(Grid<R>::lnEmin() + ((R)lo + t) * Grid<R>::dlog());
}

// ---------------------------------------------------------------- direction helpers
// express the local direction (sin t cos f, sin t sin f, cos t) about axis u globally
template <class R>
__device__ __forceinline__ void rotate_to(R ux, R uy, R uz, R cost, R phi, R* ox, R* oy, R* oz) {
  R s2 = (R)1 - cost * cost;
  s2 = s2 < (R)0 ? (R)0 : s2;
  const R sint = M<R>::sqrt(s2);
  R sp, cp;
  M<R>::fsincos(phi, &sp, &cp);
  const R l0 = sint * cp, l1 = sint * sp, l2 = cost;
  const R up2 = ux * ux + uy * uy;
  if (up2 > (R)0) {
    const R up = M<R>::sqrt(up2);
    *ox = M<R>::fdiv(ux * uz * l0 - uy * l1, up) + ux * l2;
    *oy = M<R>::fdiv(uy * uz * l0 + ux * l1, up) + uy * l2;
    *oz = -up * l0 + uz * l2;
  } else if (uz >= (R)0) {
    *ox = l0; *oy = l1; *oz = l2;
  } else {
    *ox = -l0; *oy = l1; *oz = -l2;
  }
}

template <class R>
__device__ __forceinline__ void unit(R* x, R* y, R* z) {
  const R n = M<R>::sqrt(*x * *x + *y * *y + *z * *z);
  *x = M<R>::fdiv(*x, n); *y = M<R>::fdiv(*y, n); *z = M<R>::fdiv(*z, n);
}

// ---------------------------------------------------------------- interactions
// Result of one discrete interaction: the parent's new state and up to two secondaries.
template <class R> struct Ixn {
  bool happened, parent_alive;
  double parent_E;
  R pd[3];
  int n;
  int sp[2];
  double E[2];
  R d[2][3];
};

constexpr int kMaxRej = 1000;

// Compton scattering, Klein-Nishina, sampled by Butcher-Messel composition-rejection
template <class R>
__device__ void compton(Stream<R>& st, double E, const R u[3], Ixn<R>& r) {
  const R Er = to_r<R>(E);
  const R kap = Er / (R)kMe;
  const R e0 = M<R>::fdiv((R)1, (R)1 + (R)2 * kap);
  const R a1 = M<R>::log1p((R)2 * kap);
  const R a2 = (R)0.5 * ((R)1 - e0 * e0);
  R eps = 1, t = 0;
  for (int it = 0; it < kMaxRej; ++it) {
    const R r1 = st.next(), r2 = st.next(), r3 = st.next();
    eps = (r1 * (a1 + a2) < a1) ? M<R>::fexp(-a1 * r2) : M<R>::sqrt(e0 * e0 + ((R)1 - e0 * e0) * r2);
    t = M<R>::fdiv((R)1 - eps, kap * eps);
    const R g = (R)1 - M<R>::fdiv(eps * (t * ((R)2 - t)), (R)1 + eps * eps);
    if (r3 < g) break;
  }
  const R phi = (R)(2.0 * kPi) * st.next();
  const R Epr = eps * Er;
  const double Ep = to_d<R>(Epr);
  rotate_to<R>(u[0], u[1], u[2], (R)1 - t, phi, &r.pd[0], &r.pd[1], &r.pd[2]);
  r.happened = true;
  r.parent_alive = true;
  r.parent_E = Ep;
  r.n = 1;
  r.sp[0] = 1;
  r.E[0] = E - Ep;
  R px = Er * u[0] - Epr * r.pd[0], py = Er * u[1] - Epr * r.pd[1], pz = Er * u[2] - Epr * r.pd[2];
  unit<R>(&px, &py, &pz);
  r.d[0][0] = px; r.d[0][1] = py; r.d[0][2] = pz;
}

// Bethe-Heitler pair: x = E+/E uniform on [m/E, 1 - m/E], accepted with 1 - 4/3 x(1-x)
template <class R>
__device__ void pair(Stream<R>& st, double E, const R u[3], Ixn<R>& r) {
  r.happened = false;
  const R Er = to_r<R>(E);
  if (!(Er > (R)(2.0 * kMe))) return;
  const R a = M<R>::fdiv((R)kMe, Er);
  R x = (R)0.5;
  for (int it = 0; it < kMaxRej; ++it) {
    const R r1 = st.next(), r2 = st.next();
    x = a + ((R)1 - (R)2 * a) * r1;
    if (r2 < (R)1 - (R)(4.0 / 3.0) * x * ((R)1 - x)) break;
  }
  const double Tp = to_d<R>(x * Er) - kMe;
  const double Tm = E - 2.0 * kMe - Tp;
  const R phi = (R)(2.0 * kPi) * st.next();
  r.happened = true;
  r.parent_alive = false;
  r.n = 2;
  r.sp[0] = 2;
  r.E[0] = Tp;
  rotate_to<R>(u[0], u[1], u[2], M<R>::fcos(M<R>::fdiv((R)kMe, to_r<R>(Tp) + (R)kMe)), phi, &r.d[0][0], &r.d[0][1], &r.d[0][2]);
  r.sp[1] = 1;
  r.E[1] = Tm;
  rotate_to<R>(u[0], u[1], u[2], M<R>::fcos(M<R>::fdiv((R)kMe, to_r<R>(Tm) + (R)kMe)), phi + (R)kPi, &r.d[1][0], &r.d[1][1], &r.d[1][2]);
}

template <class R>
__device__ __forceinline__ void photo(double E, const R u[3], Ixn<R>& r) {
  r.happened = true;
  r.parent_alive = false;
  r.n = 1;
  r.sp[0] = 1;
  r.E[0] = E;
  r.d[0][0] = u[0]; r.d[0][1] = u[1]; r.d[0][2] = u[2];
}

// free-electron two-body kinematics of a delta ray of kinetic energy Td
template <class R>
__device__ void delta_ray(Stream<R>& st, double T, double Td, const R u[3], Ixn<R>& r) {
  const R Tr = to_r<R>(T), Tdr = to_r<R>(Td), m2 = (R)(2.0 * kMe);
  R cd = M<R>::sqrt(M<R>::fdiv(Tdr * (Tr + m2), Tr * (Tdr + m2)));
  cd = cd > (R)1 ? (R)1 : cd;
  const R phi = (R)(2.0 * kPi) * st.next();
  R dx, dy, dz;
  rotate_to<R>(u[0], u[1], u[2], cd, phi, &dx, &dy, &dz);
  const R p0 = M<R>::sqrt(Tr * (Tr + m2));
  const R pd = M<R>::sqrt(Tdr * (Tdr + m2));
  R px = p0 * u[0] - pd * dx, py = p0 * u[1] - pd * dy, pz = p0 * u[2] - pd * dz;
  unit<R>(&px, &py, &pz);
  r.happened = true;
  r.parent_alive = true;
  r.parent_E = T - Td;
  r.pd[0] = px; r.pd[1] = py; r.pd[2] = pz;
  r.n = 1;
  r.sp[0] = 1;
  r.E[0] = Td;
  r.d[0][0] = dx; r.d[0][1] = dy; r.d[0][2] = dz;
}

// Moller: eps from 1/eps^2 on [Tc/T, 1/2], accepted with eps^2 f(eps) / (2 + (1-gg)/4)
template <class R>
__device__ void moller(Stream<R>& st, double T, double Tc, const R u[3], Ixn<R>& r) {
  r.happened = false;
  const R Tr = to_r<R>(T);
  if (!(Tr > (R)2 * to_r<R>(Tc))) return;
  const R g = M<R>::fdiv(Tr, (R)kMe) + (R)1;
  const R gg = M<R>::fdiv((R)2 * g - (R)1, g * g);
  const R ec = M<R>::fdiv(to_r<R>(Tc), Tr), em = (R)0.5;
  const R gmax = (R)2 + (R)0.25 * ((R)1 - gg);
  R eps = ec;
  for (int it = 0; it < kMaxRej; ++it) {
    const R r1 = st.next(), r2 = st.next();
    eps = M<R>::fdiv(ec * em, em - (em - ec) * r1);
    const R q = M<R>::fdiv(eps, (R)1 - eps);
    const R f = (R)1 + q * q + ((R)1 - gg) * eps * eps - gg * q;
    if (r2 * gmax < f) break;
  }
  delta_ray<R>(st, T, to_d<R>(eps * Tr), u, r);
}

// Bhabha: eps from 1/eps^2 on [Tc/T, 1], accepted with 1 - b2 eps (B1 - eps (B2 - eps (B3 - eps B4)))
template <class R>
__device__ void bhabha(Stream<R>& st, double T, double Tc, const R u[3], Ixn<R>& r) {
  r.happened = false;
  const R Tr = to_r<R>(T);
  if (!(Tr > to_r<R>(Tc))) return;
  const R tau = M<R>::fdiv(Tr, (R)kMe);
  const R g = tau + (R)1;
  const R b2 = M<R>::fdiv(tau * (tau + (R)2), g * g);
  const R y = M<R>::fdiv((R)1, g + (R)1);
  const R y12 = (R)1 - (R)2 * y;
  const R B1 = (R)2 - y * y, B2 = y12 * ((R)3 + y * y), B4 = y12 * y12 * y12;
  const R B3 = B4 + y12 * y12;
  const R ec = M<R>::fdiv(to_r<R>(Tc), Tr);
  R eps = ec;
  for (int it = 0; it < kMaxRej; ++it) {
    const R r1 = st.next(), r2 = st.next();
    eps = M<R>::fdiv(ec, (R)1 - ((R)1 - ec) * r1);
    const R gf = (R)1 - b2 * eps * (B1 - eps * (B2 - eps * (B3 - eps * B4)));
    if (r2 < gf) break;
  }
  delta_ray<R>(st, T, to_d<R>(eps * Tr), u, r);
}

// Tsai bremsstrahlung: k = kc (T/kc)^r, accepted with 1 - y + 3/4 y^2; photon at angle m/E
template <class R>
__device__ void brem(Stream<R>& st, double T, double kc, const R u[3], Ixn<R>& r) {
  r.happened = false;
  const R Tr = to_r<R>(T), kcR = to_r<R>(kc);
  if (!(Tr > kcR)) return;
  const R Ef = Tr + (R)kMe;
  const R lr = M<R>::flog(M<R>::fdiv(Tr, kcR));
  R k = kcR;
  for (int it = 0; it < kMaxRej; ++it) {
    const R r1 = st.next(), r2 = st.next();
    k = kcR * M<R>::fexp(lr * r1);
    const R y = M<R>::fdiv(k, Ef);
    if (r2 < (R)1 - y + (R)0.75 * y * y) break;
  }
  const double kd = (k >= Tr) ? T : to_d<R>(k);  // FP32 rounding of kc (T/kc)^r can reach T
  const R phi = (R)(2.0 * kPi) * st.next();
  r.happened = true;
  r.parent_alive = true;
  r.parent_E = T - kd;
  r.pd[0] = u[0]; r.pd[1] = u[1]; r.pd[2] = u[2];
  r.n = 1;
  r.sp[0] = 0;
  r.E[0] = kd;
  rotate_to<R>(u[0], u[1], u[2], M<R>::fcos(M<R>::fdiv((R)kMe, Ef)), phi, &r.d[0][0], &r.d[0][1], &r.d[0][2]);
}

// Heitler annihilation in flight: eps = E1/(T+2m) from 1/eps on [eps_min, eps_max],
// accepted with 1 - eps + (2 g eps - 1)/(eps (g+1)^2)
template <class R>
__device__ void annihilate(Stream<R>& st, double T, const R u[3], Ixn<R>& r) {
  const R Tr = to_r<R>(T);
  const R tau = M<R>::fdiv(Tr, (R)kMe);
  const R g = tau + (R)1;
  const R sq = M<R>::sqrt(M<R>::fdiv(tau, tau + (R)2));
  const R emin = (R)0.5 * ((R)1 - sq), emax = (R)0.5 * ((R)1 + sq);
  const R lr = M<R>::flog(M<R>::fdiv(emax, emin));
  const R gp1 = g + (R)1;
  R eps = (R)0.5;
  for (int it = 0; it < kMaxRej; ++it) {
    const R r1 = st.next(), r2 = st.next();
    eps = emin * M<R>::fexp(lr * r1);
    const R gf = (R)1 - eps + M<R>::fdiv((R)2 * g * eps - (R)1, eps * gp1 * gp1);
    if (r2 < gf) break;
  }
  const double Etot = T + 2.0 * kMe;
  const double E1 = to_d<R>(eps * to_r<R>(Etot));
  const double E2 = Etot - E1;
  R c1 = M<R>::fdiv(eps * gp1 - (R)1, eps * M<R>::sqrt(tau * (tau + (R)2)));
  c1 = c1 > (R)1 ? (R)1 : (c1 < (R)-1 ? (R)-1 : c1);
  const R phi = (R)(2.0 * kPi) * st.next();
  r.happened = true;
  r.parent_alive = false;
  r.n = 2;
  r.sp[0] = 0;
  r.E[0] = E1;
  rotate_to<R>(u[0], u[1], u[2], c1, phi, &r.d[0][0], &r.d[0][1], &r.d[0][2]);
  r.sp[1] = 0;
  r.E[1] = E2;
  const R pp = M<R>::sqrt(Tr * (Tr + (R)(2.0 * kMe)));
  const R E1f = (R)E1;
  R x = pp * u[0] - E1f * r.d[0][0], y = pp * u[1] - E1f * r.d[0][1], z = pp * u[2] - E1f * r.d[0][2];
  unit<R>(&x, &y, &z);
  r.d[1][0] = x; r.d[1][1] = y; r.d[1][2] = z;
}

// ---------------------------------------------------------------- optional continuous physics
// Counter blocks of the along-step draws (phase A): they never meet the model-sampling
// blocks 1, 2, ... of phase B, nor the child-id blocks with the top bit set.
constexpr uint32_t kMscBlock = 0x40000000u;
constexpr uint32_t kFluctBlock = 0x40000001u;
constexpr double kTwoPiRe2Me = 2.0 * kPi * kRe * kRe * kMe;  // MeV mm^2

// Highland's width of the projected multiple-scattering angle (PDG, passage of particles
// through matter): 13.6 MeV / (beta c p) sqrt(x/X0) (1 + 0.038 ln(x / (X0 beta^2))) for a
// unit charge at kinetic energy T over path s; the bracket is clamped at 0.
template <class R>
__device__ __forceinline__ R msc_theta0(R T, R inv_x0, R s) {
  const R E = T + (R)kMe, pc2 = T * (T + (R)(2.0 * kMe));
  const R beta2 = M<R>::fdiv(pc2, E * E), bcp = M<R>::fdiv(pc2, E);
  const R x = s * inv_x0;
  if (!(x > (R)0)) return (R)0;
  R br = (R)1 + (R)0.038 * M<R>::flog(M<R>::fdiv(x, beta2));
  br = br < (R)0 ? (R)0 : br;
  return M<R>::fdiv((R)13.6, bcp) * M<R>::sqrt(x) * br;
}

// Bohr's variance of the loss over s to transfers up to min(Tc, largest transfer): T/2 for
// e-, T for e+. xi_coef = 2 pi r_e^2 m c^2 n_el of the material.
template <class R>
__device__ __forceinline__ R fluct_sigma2(R T, R xi_coef, R Tc, R s, bool positron) {
  const R E = T + (R)kMe, beta2 = M<R>::fdiv(T * (T + (R)(2.0 * kMe)), E * E);
  const R tmax = positron ? T : (R)0.5 * T;
  const R tu = Tc < tmax ? Tc : tmax;
  return M<R>::fdiv(xi_coef * s * tu * ((R)1 - (R)0.5 * beta2), beta2);
}

// Multiple scattering at the end of a step: space angle theta0 sqrt(-2 ln ua) (two
// Gaussian projected angles of width theta0), at most pi, azimuth 2 pi ub.
template <class R>
__device__ __forceinline__ void msc_deflect(const Stream<R>& st, R theta0, R u[3]) {
  R ua, ub;
  st.pair(kMscBlock, &ua, &ub);
  R th = theta0 * M<R>::sqrt((R)-2 * M<R>::flog(ua));
  th = th > (R)kPi ? (R)kPi : th;
  R o0, o1, o2;
  rotate_to<R>(u[0], u[1], u[2], M<R>::fcos(th), (R)(2.0 * kPi) * ub, &o0, &o1, &o2);
  unit<R>(&o0, &o1, &o2);
  u[0] = o0; u[1] = o1; u[2] = o2;
}

// Gaussian loss about the mean, redrawn at most 8 times (then the mean) until it lies in
// [0, 2 mean]; one Box-Muller normal per counter block
template <class R>
__device__ __forceinline__ double fluct_loss(const Stream<R>& st, double mean, R sigma) {
  for (uint32_t i = 0; i < 8; ++i) {
    R ua, ub;
    st.pair(kFluctBlock + i, &ua, &ub);
    const R g = M<R>::sqrt((R)-2 * M<R>::flog(ua)) * M<R>::fcos((R)(2.0 * kPi) * ub);
    const double d = mean + to_d<R>(sigma * g);
    if (d >= 0.0 && d <= 2.0 * mean) return d;
  }
  return mean;
}

template <class R>
__device__ void annihilate_at_rest(Stream<R>& st, Ixn<R>& r) {
  const R ct = (R)2 * st.next() - (R)1;
  const R phi = (R)(2.0 * kPi) * st.next();
  R s2 = (R)1 - ct * ct;
  s2 = s2 < (R)0 ? (R)0 : s2;
  const R s = M<R>::sqrt(s2);
  R sp, cp;
  M<R>::fsincos(phi, &sp, &cp);
  r.happened = true;
  r.parent_alive = false;
  r.n = 2;
  r.sp[0] = 0; r.sp[1] = 0;
  r.E[0] = kMe; r.E[1] = kMe;
  r.d[0][0] = s * cp; r.d[0][1] = s * sp; r.d[0][2] = ct;
  r.d[1][0] = -r.d[0][0]; r.d[1][1] = -r.d[0][1]; r.d[1][2] = -r.d[0][2];
}

// ---------------------------------------------------------------- geometry
// Slab: volumes between planes bnd[0..n_vol] along z, |x|,|y| <= half_xy. Tubes: volume
// 0 is r < bnd[0], volume v is bnd[v-1] <= r < bnd[v], |z| <= half_z. next = -1 leaves.
template <class R>
__device__ __forceinline__ R slab_wall(R p, R u, R H) {
  return u > (R)0 ? M<R>::fdiv(H - p, u) : (u < (R)0 ? M<R>::fdiv(-H - p, u) : M<R>::big());
}

// Path lengths are of type R; the FP64 work is the distance to a plane (z_plane - z)
// and the r^2 - R^2 of a cylinder, taken from the FP64 position before rounding.
template <class R>
__device__ R straight_distance(const GeoView& g, double x, double y, double z, const R u[3], int vol,
                               int* next) {
  R s = M<R>::big();
  int nx = vol;
  if (g.kind == 0) {
    if (u[2] > (R)0) {
      s = M<R>::fdiv(to_r<R>(__ldg(g.bnd + vol + 1) - z), u[2]);
      nx = (vol + 1 < g.n_vol) ? vol + 1 : -1;
    } else if (u[2] < (R)0) {
      s = M<R>::fdiv(to_r<R>(__ldg(g.bnd + vol) - z), u[2]);
      nx = vol - 1;
    }
    const R H = (R)g.half_xy;
    const R sx = slab_wall<R>(to_r<R>(x), u[0], H);
    const R sy = slab_wall<R>(to_r<R>(y), u[1], H);
    if (sx < s) { s = sx; nx = -1; }
    if (sy < s) { s = sy; nx = -1; }
  } else {
    const R a = u[0] * u[0] + u[1] * u[1];
    const R b = to_r<R>(x) * u[0] + to_r<R>(y) * u[1];
    const double r2 = x * x + y * y;
    if (a > (R)0) {
      const double Ro = __ldg(g.bnd + vol);
      const R co = to_r<R>(r2 - Ro * Ro);
      R D = b * b - a * co;
      D = D < (R)0 ? (R)0 : D;
      const R sq = M<R>::sqrt(D);
      R so = (b > (R)0) ? -co / (b + sq) : (sq - b) / a;
      so = so < (R)0 ? (R)0 : so;
      s = so;
      nx = (vol + 1 < g.n_vol) ? vol + 1 : -1;
      if (vol > 0 && b < (R)0) {
        const double Ri = __ldg(g.bnd + vol - 1);
        const R ci = to_r<R>(r2 - Ri * Ri);
        const R Di = b * b - a * ci;
        if (Di > (R)0) {
          R si = ci / (M<R>::sqrt(Di) - b);
          si = si < (R)0 ? (R)0 : si;
          if (si < s) { s = si; nx = vol - 1; }
        }
      }
    }
    R sz = M<R>::big();
    if (u[2] > (R)0) sz = to_r<R>(g.half_z - z) / u[2];
    else if (u[2] < (R)0) sz = to_r<R>(-g.half_z - z) / u[2];
    if (sz < s) { s = sz; nx = -1; }
  }
  *next = nx;
  return s < (R)0 ? (R)0 : s;
}

// Helix in B along z: h = -sign(qB) turns the transverse direction, rho = p_T/(K |B|),
// the phase advances by Delta = s u_T / rho over a path s.
template <class R> struct Helix {
  bool straight;
  R uT, rho, h, kpath;
  double cx, cy;
};

template <class R>
__device__ __forceinline__ void helix_setup(double B, double T, int q, const R u[3], double x, double y,
                                            Helix<R>& H) {
  H.straight = true;
  if (B == 0.0 || q == 0) return;
  const R uT = M<R>::sqrt(u[0] * u[0] + u[1] * u[1]);
  if (!(uT > (R)1e-12)) return;
  const R Tr = to_r<R>(T);
  const R pm = M<R>::sqrt(Tr * (Tr + (R)(2.0 * kMe)));
  H.straight = false;
  H.uT = uT;
  H.rho = pm * uT / (R)(kHelixK * fabs(B));
  H.h = ((q > 0) == (B > 0.0)) ? (R)-1 : (R)1;
  H.cx = x - to_d<R>(H.rho * H.h * u[1] / uT);
  H.cy = y + to_d<R>(H.rho * H.h * u[0] / uT);
  H.kpath = uT / H.rho;
}

template <class R>
__device__ __forceinline__ R wrap2pi(R x) {
  const R tp = (R)(2.0 * kPi);
  R r = M<R>::fmod(x, tp);
  if (r < (R)0) r += tp;
  if (r > tp - M<R>::turn_tol()) r = (R)0;
  return r;
}

// First crossing, in the asked direction, of a level set whose crossings sit at phase
// psi_ref -/+ A on the circle; dpsi = psi_ref - psi0. A = acos(C) is taken as
// 2 atan2(sqrt(1 - C), sqrt(1 + C)) from 1 - C and 1 + C computed without cancellation:
// acos itself loses all accuracy in FP32 where A is near 0 or pi (large radii).
template <class R>
__device__ __forceinline__ R helix_hit(const Helix<R>& H, R dpsi, R omc, R opc, bool increasing) {
  if (!(omc >= (R)0 && opc >= (R)0)) return M<R>::big();
  const R A = (R)2 * M<R>::atan2(M<R>::sqrt(omc), M<R>::sqrt(opc));
  const R base = H.h * dpsi;
  const R D = wrap2pi<R>(increasing ? base - A : base + A);
  return D / H.kpath;
}

// 1 - x for a component x of a unit vector whose other component is y
template <class R>
__device__ __forceinline__ R one_minus(R x, R y) { return x > (R)0 ? y * y / ((R)1 + x) : (R)1 - x; }

// phase of direction (ax, ay) minus the particle's phase psi0, in (-pi, pi]
template <class R>
__device__ __forceinline__ R phase_from(R c0, R s0, R ax, R ay) {
  return M<R>::atan2(c0 * ay - s0 * ax, c0 * ax + s0 * ay);
}

template <class R>
__device__ R helix_distance(const GeoView& g, double B, double T, int q, double x, double y,
                                 double z, const R u[3], int vol, int* next) {
  Helix<R> H;
  helix_setup<R>(B, T, q, u, x, y, H);
  if (H.straight) return straight_distance<R>(g, x, y, z, u, vol, next);
  // unit vector from the circle's centre to the particle: (h uy, -h ux) / uT
  const R c0 = H.h * u[1] / H.uT, s0 = -H.h * u[0] / H.uT;
  R s = M<R>::big();
  int nx = vol;
  if (g.kind == 0) {
    if (u[2] > (R)0) {
      s = to_r<R>(__ldg(g.bnd + vol + 1) - z) / u[2];
      nx = (vol + 1 < g.n_vol) ? vol + 1 : -1;
    } else if (u[2] < (R)0) {
      s = to_r<R>(__ldg(g.bnd + vol) - z) / u[2];
      nx = vol - 1;
    }
    const double Hw = g.half_xy;
    if (!(M<R>::fabs(to_r<R>(H.cx)) + H.rho < (R)Hw && M<R>::fabs(to_r<R>(H.cy)) + H.rho < (R)Hw)) {
      // walls x = +Hw, -Hw, y = +Hw, -Hw as n.P = Hw crossed outward; with n.P = n.c +
      // rho cos(psi - psi_n) and n.c = n.p - rho n.e0: C = n.e0 + (Hw - n.p)/rho
      const R nxs[4] = {(R)1, (R)-1, (R)0, (R)0}, nys[4] = {(R)0, (R)0, (R)1, (R)-1};
      const double np[4] = {x, -x, y, -y};
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        const R ne = nxs[w] * c0 + nys[w] * s0;          // n . e0
        const R ne_perp = nxs[w] * s0 - nys[w] * c0;     // the other component of e0
        const R gap = to_r<R>(Hw - np[w]) / H.rho;
        const R omc = one_minus<R>(ne, ne_perp) - gap;
        const R opc = one_minus<R>(-ne, ne_perp) + gap;
        const R sw = helix_hit<R>(H, phase_from<R>(c0, s0, nxs[w], nys[w]), omc, opc, true);
        if (sw < s) { s = sw; nx = -1; }
      }
    }
  } else {
    const double cm2 = H.cx * H.cx + H.cy * H.cy;
    const R cm = M<R>::sqrt(to_r<R>(cm2));
    if (cm > (R)1e-12) {
      const R dpsi = phase_from<R>(c0, s0, to_r<R>(H.cx), to_r<R>(H.cy));
      const R den = (R)2 * H.rho * cm;
      // |P| = R where cos(psi - psi_c) = C = (R^2 - cm^2 - rho^2)/den; 1 - C and 1 + C are
      // formed from FP64 numerators (rho + cm)^2 - R^2 and R^2 - (cm - rho)^2 so that
      // grazing crossings near the circle's far or near point keep their accuracy
      const double rd = to_d<R>(H.rho);
      const double a = cm2 + rd * rd;
      // cm to FP64 accuracy: one Newton step on the float square root
      const double cmf = to_d<R>(cm);
      const double cmd = cmf + (cm2 - cmf * cmf) * to_d<R>((R)0.5 / cm);
      const double b = 2.0 * rd * cmd;
      const double Ro = __ldg(g.bnd + vol);
      {
        const R so = helix_hit<R>(H, dpsi, to_r<R>((a - Ro * Ro) + b) / den, to_r<R>((Ro * Ro - a) + b) / den, true);
        if (so < s) { s = so; nx = (vol + 1 < g.n_vol) ? vol + 1 : -1; }
      }
      if (vol > 0) {
        const double Ri = __ldg(g.bnd + vol - 1);
        const R si = helix_hit<R>(H, dpsi, to_r<R>((a - Ri * Ri) + b) / den, to_r<R>((Ri * Ri - a) + b) / den, false);
        if (si < s) { s = si; nx = vol - 1; }
      }
    }
    R sz = M<R>::big();
    if (u[2] > (R)0) sz = to_r<R>(g.half_z - z) / u[2];
    else if (u[2] < (R)0) sz = to_r<R>(-g.half_z - z) / u[2];
    if (sz < s) { s = sz; nx = -1; }
    if (s >= M<R>::big()) { s = (R)(2.0 * kPi) / H.kpath; nx = vol; }  // closed circle: one turn
  }
  *next = nx;
  return s;
}

// move along the helix (or straight) by s; position stays double, direction in R
template <class R>
__device__ __forceinline__ void helix_move(double B, double T, int q, R s, double* x, double* y,
                                           double* z, R u[3]) {
  Helix<R> H;
  helix_setup<R>(B, T, q, u, *x, *y, H);
  if (H.straight) {
    *x += to_d<R>(s * u[0]); *y += to_d<R>(s * u[1]); *z += to_d<R>(s * u[2]);
    return;
  }
  const R D = s * H.kpath;
  R sd, cd;
  M<R>::sincos(D, &sd, &cd);
  const R sh = M<R>::sin((R)0.5 * D);
  const R cm1 = (R)-2 * sh * sh;
  const R a = u[0] / H.uT, b = u[1] / H.uT;
  *x += to_d<R>(H.rho * (a * sd + H.h * b * cm1));
  *y += to_d<R>(H.rho * (b * sd - H.h * a * cm1));
  *z += to_d<R>(s * u[2]);
  const R u0 = u[0] * cd - H.h * u[1] * sd;
  const R u1 = u[1] * cd + H.h * u[0] * sd;
  u[0] = u0; u[1] = u1;
}

// ---------------------------------------------------------------- chord propagation (optional)
// is (x, y, z) inside (or on the boundary of) volume vol
__device__ __forceinline__ bool inside_volume(const GeoView& g, double x, double y, double z, int vol) {
  if (g.kind == 0)
    return z >= __ldg(g.bnd + vol) && z <= __ldg(g.bnd + vol + 1) && fabs(x) <= g.half_xy && fabs(y) <= g.half_xy;
  const double r2 = x * x + y * y;
  if (fabs(z) > g.half_z) return false;
  const double Ro = __ldg(g.bnd + vol);
  if (r2 > Ro * Ro) return false;
  if (vol == 0) return true;
  const double Ri = __ldg(g.bnd + vol - 1);
  return r2 >= Ri * Ri;
}

// Chord propagation in the field (paper Sec. 2.3): the helix is followed in linear segments
// whose sagitta kappa l^2 / 8 is at most dchord (kappa = |du/ds| = u_T kpath); a segment that
// meets the boundary of the volume (straight distance along it) is refined by bisection
// between an inside and an outside point of the curve until the sagitta is at most dint,
// and the crossing is taken on that last chord. Every segment and every bisection is one
// iteration. Returns 0 (reached s_phys), 1 (crossed into *next) or 2 (more than max_iter
// iterations: the step did not finish; nothing moved). Curve points are evaluated from the
// step's start. Not inlined: it runs only when the chord propagator is chosen, and keeps
// its registers out of the transport kernels.
template <class R>
__device__ __forceinline__ int chord_step(const GeoView& g, double B, double T, int q, R s_phys, int max_iter, R dchord,
                                       R dint, double* x, double* y, double* z, R* u, int vol, int* next, R* s_done) {
  Helix<R> H;
  helix_setup<R>(B, T, q, u, *x, *y, H);
  if (H.straight) {  // no curvature: one straight segment
    int nx;
    const R sg = straight_distance<R>(g, *x, *y, *z, u, vol, &nx);
    const R s = sg <= s_phys ? sg : s_phys;
    *x += to_d<R>(s * u[0]); *y += to_d<R>(s * u[1]); *z += to_d<R>(s * u[2]);
    *next = nx;
    *s_done = s;
    return sg <= s_phys ? 1 : 0;
  }
  const double xs = *x, ys = *y, zs = *z;
  const R us0 = u[0], us1 = u[1], us2 = u[2];
  auto at = [&](R s, double& px, double& py, double& pz, R* pu) {
    px = xs; py = ys; pz = zs;
    pu[0] = us0; pu[1] = us1; pu[2] = us2;
    helix_move<R>(B, T, q, s, &px, &py, &pz, pu);
  };
  const R kappa = H.uT * H.kpath;
  const R lmax = M<R>::sqrt((R)8 * dchord / kappa), lint = M<R>::sqrt((R)8 * dint / kappa);
  R s0 = 0;
  double p0x = xs, p0y = ys, p0z = zs;
  R tmp[3];
  int iters = 0;
  for (;;) {
    if (++iters > max_iter) return 2;
    const R ell = (s_phys - s0 < lmax) ? s_phys - s0 : lmax;
    double p1x, p1y, p1z;
    R u1[3];
    at(s0 + ell, p1x, p1y, p1z, u1);
    const double dx = p1x - p0x, dy = p1y - p0y, dz = p1z - p0z;
    const double L = sqrt(dx * dx + dy * dy + dz * dz);
    int nx = vol;
    R sb = M<R>::big();
    if (L > 0.0) {
      const R d[3] = {to_r<R>(dx / L), to_r<R>(dy / L), to_r<R>(dz / L)};
      sb = straight_distance<R>(g, p0x, p0y, p0z, d, vol, &nx);
    }
    R hi = (R)-1;
    if (sb < to_r<R>(L)) {  // the segment meets the boundary: a curve point outside?
      if (!inside_volume(g, p1x, p1y, p1z, vol)) {
        hi = s0 + ell;
      } else {
        const R sc = s0 + ell * (sb / to_r<R>(L));
        double pcx, pcy, pcz;
        at(sc, pcx, pcy, pcz, tmp);
        if (!inside_volume(g, pcx, pcy, pcz, vol)) hi = sc;
      }
    }
    if (hi < (R)0) {  // no crossing on this segment
      s0 += ell;
      p0x = p1x; p0y = p1y; p0z = p1z;
      if (s0 >= s_phys) {
        *x = p1x; *y = p1y; *z = p1z;
        u[0] = u1[0]; u[1] = u1[1]; u[2] = u1[2];
        *s_done = s_phys;
        return 0;
      }
      continue;
    }
    R lo = s0;
    double plx = p0x, ply = p0y, plz = p0z, phx, phy, phz;
    at(hi, phx, phy, phz, tmp);
    while (hi - lo > lint) {
      if (++iters > max_iter) return 2;
      const R mid = (R)0.5 * (lo + hi);
      double pmx, pmy, pmz;
      at(mid, pmx, pmy, pmz, tmp);
      if (inside_volume(g, pmx, pmy, pmz, vol)) { lo = mid; plx = pmx; ply = pmy; plz = pmz; }
      else { hi = mid; phx = pmx; phy = pmy; phz = pmz; }
    }
    const double ex = phx - plx, ey = phy - ply, ez = phz - plz;
    const double Le = sqrt(ex * ex + ey * ey + ez * ez);
    R sx = hi;
    if (Le > 0.0) {
      const R e[3] = {to_r<R>(ex / Le), to_r<R>(ey / Le), to_r<R>(ez / Le)};
      R sbe = straight_distance<R>(g, plx, ply, plz, e, vol, &nx);
      if (sbe > to_r<R>(Le)) sbe = to_r<R>(Le);
      sx = lo + (sbe / to_r<R>(Le)) * (hi - lo);
      *x = plx + to_d<R>(sbe) * (ex / Le); *y = ply + to_d<R>(sbe) * (ey / Le); *z = plz + to_d<R>(sbe) * (ez / Le);
    } else {
      *x = phx; *y = phy; *z = phz;
    }
    double qx, qy, qz;
    at(sx, qx, qy, qz, u);
    *next = nx;
    *s_done = sx;
    return 1;
  }
}

// locate a point: on a surface, the volume the direction points into
__device__ __forceinline__ int locate(const GeoView& g, double x, double y, double z, double ux, double uy,
                                      double uz) {
  if (g.kind == 0) {
    if (fabs(x) > g.half_xy || fabs(y) > g.half_xy) return -1;
    if (z < g.bnd[0] || z > g.bnd[g.n_vol]) return -1;
    int lo = 0, hi = g.n_vol;  // find k with bnd[k] <= z < bnd[k+1]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (g.bnd[mid] <= z) lo = mid; else hi = mid;
    }
    if (z == g.bnd[g.n_vol]) lo = g.n_vol;
    if (z == g.bnd[lo]) {
      const int v = uz >= 0.0 ? lo : lo - 1;
      return (v < 0 || v >= g.n_vol) ? -1 : v;
    }
    return lo;
  }
  if (fabs(z) > g.half_z) return -1;
  const double r = sqrt(x * x + y * y);
  const double radial = x * ux + y * uy;
  int v = 0;
  for (int k = 0; k < g.n_vol; ++k) {
    const double b = g.bnd[k];
    if (fabs(r - b) <= 1e-9 * b) {
      v = radial > 0.0 ? k + 1 : k;
      return v >= g.n_vol ? -1 : v;
    }
    if (b < r) v = k + 1;
  }
  return v >= g.n_vol ? -1 : v;
}

}  // namespace adept
