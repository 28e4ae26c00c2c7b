/*
 * FP64 CPU oracle for electromagnetic shower transport (AdePT, arXiv 2209.15445).
 * TEST INFRASTRUCTURE ONLY: see oracle.h for who may call it.
 *
 * Plain, slow and direct: one event at a time, a LIFO stack of tracks, one step
 * of one track at a time (paper Sec. 3 describes the GPU departing from exactly
 * this CPU model). All arithmetic is double precision with no FMA contraction
 * (built with -ffp-contract=off) so that x86 and Arm hosts agree bit for bit.
 *
 * Units: MeV, mm, tesla. Constants: CODATA/PDG.
 */
#include "oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ constants */
static const double kMe = 0.51099895;          /* electron mass [MeV] */
static const double kRe = 2.8179403262e-12;    /* classical electron radius [mm] */
static const double kAlpha = 1.0 / 137.035999084;
static const double kNA = 6.02214076e23;       /* 1/mol */
static const double kPi = 3.14159265358979323846;
static const double kHelixK = 0.299792458;     /* rho[mm] = p[MeV] / (K * B[T]) */
static const double kEmin = 1e-3, kEmax = 1e6; /* table grid, MeV */
static const double kAlphaR = 0.2, kRhoF = 1.0;/* step function: max(alpha_R R, min(R, rho_f)) */

static double lnEmin(void) { return log(1e-3); }
static double dlog(void) { return log(10.0) / 32.0; }
static double inv_dlog(void) { return 32.0 / log(10.0); }

/* ------------------------------------------------------------------ Philox4x32-10
 * Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11:
 * a 10-round Feistel-like bijection of a 128-bit counter under a 64-bit key. Each
 * round multiplies two counter words by fixed odd constants, mixes the high halves
 * with the other words and the round key, and the key is bumped by the Weyl
 * constants between rounds. */
static void philox_round(uint32_t c[4], const uint32_t k[2]) {
  const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
  const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
  const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
  const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
  uint32_t n0 = hi1 ^ c[1] ^ k[0];
  uint32_t n1 = lo1;
  uint32_t n2 = hi0 ^ c[3] ^ k[1];
  uint32_t n3 = lo0;
  c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
}

void or_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
  uint32_t k[2] = {key[0], key[1]};
  for (int r = 0; r < 10; ++r) {
    philox_round(c, k);
    k[0] += 0x9E3779B9u;
    k[1] += 0xBB67AE85u;
  }
  out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* 52 random bits from two words, centred in (0,1): (x + 0.5) 2^-52, which is exact in
 * double precision (x + 0.5 needs 53 significant bits), so u lies in [2^-53, 1 - 2^-53] */
double or_u01_f64(uint32_t w0, uint32_t w1) {
  const uint64_t x = ((uint64_t)w0 << 20) ^ (uint64_t)(w1 >> 12);
  return ((double)x + 0.5) * (1.0 / 4503599627370496.0);
}
/* 23 random bits from one word: (x + 0.5) 2^-23, exact in single precision */
float or_u01_f32(uint32_t w) { return ((float)(w >> 9) + 0.5f) * (1.0f / 8388608.0f); }

uint64_t or_child_id(uint32_t seed, uint32_t event, uint64_t parent_id, uint32_t parent_step,
                     uint32_t k) {
  const uint32_t key[2] = {seed, event};
  const uint32_t ctr[4] = {(uint32_t)parent_id, (uint32_t)(parent_id >> 32), parent_step,
                           0x80000000u | k};
  uint32_t w[4];
  or_philox(ctr, key, w);
  return (uint64_t)w[0] | ((uint64_t)w[1] << 32);
}

/* The uniform stream of one (track, step): block 0 gives u0 (interaction length) and u1
 * (process choice); model sampling draws from blocks 1, 2, ... two doubles per block. */
typedef struct {
  uint32_t key[2];
  uint32_t ctr[4];
  uint32_t w[4];
  int next;
} stream_t;

static void stream_init(stream_t* s, uint32_t seed, uint32_t event, uint64_t id, uint32_t step) {
  s->key[0] = seed; s->key[1] = event;
  s->ctr[0] = (uint32_t)id; s->ctr[1] = (uint32_t)(id >> 32); s->ctr[2] = step; s->ctr[3] = 0;
  s->next = 4;
}
static void stream_block0(stream_t* s, double* u0, double* u1) {
  uint32_t c[4] = {s->ctr[0], s->ctr[1], s->ctr[2], 0};
  uint32_t w[4];
  or_philox(c, s->key, w);
  *u0 = or_u01_f64(w[0], w[1]);
  *u1 = or_u01_f64(w[2], w[3]);
}
static double stream_u(stream_t* s) {
  if (s->next >= 4) {
    s->ctr[3] += 1;
    or_philox(s->ctr, s->key, s->w);
    s->next = 0;
  }
  const double u = or_u01_f64(s->w[s->next], s->w[s->next + 1]);
  s->next += 2;
  return u;
}

/* ------------------------------------------------------------------ context */
typedef struct {
  int Z;               /* > 0 for matter (a compound's mean Z); 0 vacuum */
  double A, rho, I;
  int n_elem;          /* elements: Z, A, atoms per mm^3 */
  int eZ[OR_MAX_ELEM];
  double eA[OR_MAX_ELEM], en_at[OR_MAX_ELEM];
  double ZoA;          /* <Z/A> by mass */
  double n_at, n_el;   /* 1/mm^3 */
  double invX0;        /* 1/mm */
  double Cbar, x0, x1, a_d; /* Sternheimer-Peierls density effect */
} mat_t;

struct or_ctx {
  int n_mat;
  mat_t mat[OR_MAX_MAT];
  int kind;
  int n_vol;              /* volumes 0..n_vol-1 */
  double bnd[OR_MAX_VOL + 1];
  int vol_mat[OR_MAX_VOL];
  int vol_bin[OR_MAX_VOL];
  int n_bins;
  double half_xy, half_z;
  double field_T, tcut;
  double Tc[OR_MAX_MAT], kc[OR_MAX_MAT];
  double gam[OR_MAX_MAT][3][OR_NNODE];
  double ele[OR_MAX_MAT][4][OR_NNODE];
  double pos[OR_MAX_MAT][5][OR_NNODE];
  double rfull[OR_MAX_MAT][OR_NNODE];
};

double or_node_energy(int i) { return exp(lnEmin() + i * dlog()); }

/* ------------------------------------------------------------------ cross sections */
/* Klein-Nishina total cross section per electron [mm^2] (Klein & Nishina 1929; any
 * textbook, e.g. Heitler, "The Quantum Theory of Radiation"):
 *   sigma = 2 pi re^2 b(k),
 *   b = (1+k)/k^2 [2(1+k)/(1+2k) - ln(1+2k)/k] + ln(1+2k)/(2k) - (1+3k)/(1+2k)^2.
 * The closed form cancels terms of size 1/k^2 down to O(1): in FP64 it keeps about
 * 1e-16/k^2 relative accuracy (7e-13 at k = 0.02, 4e-14 at k = 0.1, 1e-14 at 0.2).
 * Below k = 0.2 b is summed as its Taylor series instead. With x = 2k, expanding
 * ln(1+x), 1/(1+x) and 1/(1+x)^2 term by term (the bracket's first two orders cancel
 * exactly) gives
 *   b = sum_n (-x)^n d_n,  d_n = 4(n+1)/(n+3) + 1/(n+1) - 2n/(n+2) + n/2 - 1,
 * with d_0 = 4/3 (the Thomson limit). It converges for x < 1; at x = 0.4, 60 terms leave
 * below 1e-22. */
double or_sigma_kn_direct(double k) {
  const double l = log1p(2.0 * k);
  const double b = (1.0 + k) / (k * k) * (2.0 * (1.0 + k) / (1.0 + 2.0 * k) - l / k) +
                   l / (2.0 * k) - (1.0 + 3.0 * k) / ((1.0 + 2.0 * k) * (1.0 + 2.0 * k));
  return 2.0 * kPi * kRe * kRe * b;
}
static double kn_series_coef(int n) {
  return 4.0 * (n + 1) / (n + 3) + 1.0 / (n + 1) - 2.0 * n / (n + 2) + 0.5 * n - 1.0;
}
double or_sigma_kn(double k) {
  if (k >= 0.2) return or_sigma_kn_direct(k);
  const double x = 2.0 * k;
  double s = kn_series_coef(59);
  for (int n = 58; n >= 0; --n) s = s * (-x) + kn_series_coef(n); /* Horner */
  return 2.0 * kPi * kRe * kRe * s;
}

double or_mu_compton(const or_ctx* c, int m, double E) {
  return c->mat[m].n_el * or_sigma_kn(E / kMe);
}

/* Radiation length, Tsai (Rev. Mod. Phys. 46 (1974) 815) as quoted by the PDG:
 * 1/X0 = 4 alpha re^2 (NA rho / A) [Z^2 (Lrad - f(Z)) + Z L'rad],
 * Lrad = ln(184.15 Z^-1/3), L'rad = ln(1194 Z^-2/3), f = Davies-Bethe-Maximon Coulomb
 * correction a^2[(1+a^2)^-1 + 0.20206 - 0.0369 a^2 + 0.0083 a^4 - 0.002 a^6], a = alpha Z. */
static double inv_x0_per_atom(double Z) {
  const double lz = log(Z);
  const double Lrad = log(184.15) - lz / 3.0;
  const double Lp = log(1194.0) - 2.0 * lz / 3.0;
  const double a2 = (kAlpha * Z) * (kAlpha * Z);
  const double f = a2 * (1.0 / (1.0 + a2) + 0.20206 - 0.0369 * a2 + 0.0083 * a2 * a2 -
                         0.002 * a2 * a2 * a2);
  return 4.0 * kAlpha * kRe * kRe * (Z * Z * (Lrad - f) + Z * Lp);
}
/* a compound adds its elements' terms by atom density: 1/X0 = sum_i w_i / X0_i (Bragg
 * additivity, as the PDG gives it for mixtures) */
static double inv_x0(const mat_t* t) {
  double s = 0.0;
  for (int i = 0; i < t->n_elem; ++i) s += t->en_at[i] * inv_x0_per_atom(t->eZ[i]);
  return s;
}
double or_inv_X0(const or_ctx* c, int m) { return c->mat[m].invX0; }

/* Bethe-Heitler pair production in complete screening (PDG "Passage of particles",
 * photon pair production): dsigma/dx = (A / (X0 NA rho)) [1 - 4/3 x(1-x)], x the
 * positron's total-energy fraction, here restricted to the kinematic range
 * [m/E, 1 - m/E]. Integrating with w = 1 - 2m/E and a = m/E gives
 * mu = (w / X0) (7 - 4 a (1 - a)) / 9, which tends to 7/(9 X0). */
double or_mu_pair(const or_ctx* c, int m, double E) {
  if (!(E > 2.0 * kMe)) return 0.0;
  const double a = kMe / E;
  const double w = (E - 2.0 * kMe) / E;
  return c->mat[m].invX0 * w * (7.0 - 4.0 * a * (1.0 - a)) / 9.0;
}

/* Photoabsorption, Born approximation for the two K electrons (Heitler):
 * sigma = 4 sqrt(2) alpha^4 Z^5 sigma_Th (m/E)^(7/2), no edges. */
double or_mu_photo(const or_ctx* c, int m, double E) {
  const double q = kMe / E;
  const double sth = 8.0 * kPi / 3.0 * kRe * kRe;
  const double a4 = kAlpha * kAlpha * kAlpha * kAlpha;
  const mat_t* t = &c->mat[m];
  double s = 0.0; /* a compound: the sum over its atoms */
  for (int i = 0; i < t->n_elem; ++i) {
    const double Z = t->eZ[i];
    s += t->en_at[i] * 4.0 * sqrt(2.0) * a4 * (Z * Z * Z * Z * Z) * sth * (q * q * q * sqrt(q));
  }
  return s;
}

/* Sternheimer & Peierls (Phys. Rev. B 3 (1971) 3681) general density-effect
 * parameterisation for condensed media from I, rho and Z/A. */
static void density_params(mat_t* t) {
  const double hwp = 28.816 * sqrt(t->rho * t->ZoA); /* eV */
  t->Cbar = 2.0 * log(t->I / hwp) + 1.0;
  if (t->I < 100.0) {
    t->x1 = 2.0;
    t->x0 = (t->Cbar < 3.681) ? 0.2 : 0.326 * t->Cbar - 1.0;
  } else {
    t->x1 = 3.0;
    t->x0 = (t->Cbar < 5.215) ? 0.2 : 0.326 * t->Cbar - 1.5;
  }
  const double d = t->x1 - t->x0;
  t->a_d = (t->Cbar - 2.0 * log(10.0) * t->x0) / (d * d * d);
}

static double delta_of(const mat_t* t, double T) {
  const double tau = T / kMe;
  const double x = 0.5 * log(tau * (tau + 2.0)) / log(10.0); /* log10(beta gamma) */
  if (x < t->x0) return 0.0;
  const double lin = 2.0 * log(10.0) * x - t->Cbar;
  if (x >= t->x1) return lin;
  const double r = t->x1 - x;
  return lin + t->a_d * r * r * r;
}
double or_density_delta(const or_ctx* c, int m, double T) { return delta_of(&c->mat[m], T); }

/* Restricted collision stopping power, Berger-Seltzer (ICRU Report 37) form:
 * dE/dx = 2 pi re^2 m n_el / beta^2 [ ln(2(tau+2)/(I/m)^2) + F(tau, D) - delta ],
 * D = min(cut, T/2) / m for electrons (Moller), min(cut, T) / m for positrons (Bhabha).
 * F- = -1 - b2 + ln((tau-D)D) + tau/(tau-D) + [D^2/2 + (2tau+1) ln(1 - D/tau)] / g^2
 * F+ = ln(tau D) - (b2/tau)[tau + 2D - 3D^2 y/2 - (D - D^3/3) y^2
 *                          - (D^2/2 - tau D^3/3 + D^4/4) y^3],  y = 1/(g+1). */
static double dedx_col(const mat_t* t, double T, double cut, int positron) {
  const double tau = T / kMe;
  const double g = tau + 1.0;
  const double b2 = tau * (tau + 2.0) / (g * g);
  const double Im = t->I * 1e-6 / kMe;
  double D = positron ? T : 0.5 * T;
  if (cut < D) D = cut;
  D /= kMe;
  double F;
  if (!positron) {
    F = -1.0 - b2 + log((tau - D) * D) + tau / (tau - D) +
        (0.5 * D * D + (2.0 * tau + 1.0) * log1p(-D / tau)) / (g * g);
  } else {
    const double y = 1.0 / (g + 1.0);
    const double D2 = D * D, D3 = D2 * D, D4 = D3 * D;
    F = log(tau * D) - (b2 / tau) * (tau + 2.0 * D - 1.5 * D2 * y - (D - D3 / 3.0) * y * y -
                                     (0.5 * D2 - tau * D3 / 3.0 + 0.25 * D4) * y * y * y);
  }
  double br = log(2.0 * (tau + 2.0) / (Im * Im)) + F - delta_of(t, T);
  if (br < 0.0) br = 0.0;
  return 2.0 * kPi * kRe * kRe * kMe * t->n_el / b2 * br;
}
double or_dedx_col(const or_ctx* c, int m, double T, double cut, int positron) {
  return dedx_col(&c->mat[m], T, cut, positron);
}

/* Radiative loss to photons below k (Tsai complete screening, see or_lambda_brem):
 * (1/X0) [4/3 k - 2/3 k^2/E + k^3/(3E^2)], k = min(kcut, T). */
static double dedx_rad(const mat_t* t, double T, double kcut) {
  const double k = kcut < T ? kcut : T;
  const double E = T + kMe;
  return t->invX0 * (4.0 / 3.0 * k - 2.0 / 3.0 * k * k / E + k * k * k / (3.0 * E * E));
}
double or_dedx_rad(const or_ctx* c, int m, double T, double kcut) {
  return dedx_rad(&c->mat[m], T, kcut);
}

/* Moller (e-e-) and Bhabha (e+e-) cross sections for delta rays above the cut, integrated
 * in closed form over eps = T_delta / T:
 * Moller: dsig/deps = 2 pi re^2 m/(b2 T) [(1-gg) + 1/eps^2 + 1/(1-eps)^2 - gg/(eps(1-eps))],
 *   gg = (2g-1)/g^2, eps in [cut/T, 1/2];
 * Bhabha: dsig/deps = 2 pi re^2 m/T [1/(b2 eps^2) - B1/eps + B2 - B3 eps + B4 eps^2],
 *   y = 1/(g+1), B1 = 2-y^2, B2 = (1-2y)(3+y^2), B4 = (1-2y)^3, B3 = B4 + (1-2y)^2,
 *   eps in [cut/T, 1]. The integrals are written in w = 1 - 2 eps_c (Moller) and
 *   v = 1 - eps_c (Bhabha) so that they vanish smoothly at threshold. */
static double lambda_ioni(const mat_t* t, double T, double cut, int positron) {
  const double g = T / kMe + 1.0;
  const double tau = T / kMe;
  const double b2 = tau * (tau + 2.0) / (g * g);
  const double ec = cut / T;
  double br;
  if (!positron) {
    if (!(T > 2.0 * cut)) return 0.0;
    const double w = (T - 2.0 * cut) / T;
    const double gg = (2.0 * g - 1.0) / (g * g);
    br = (1.0 - gg) * 0.5 * w + w / (ec * (1.0 - ec)) - gg * log1p(w / ec);
    return t->n_el * 2.0 * kPi * kRe * kRe * kMe / (b2 * T) * br;
  }
  if (!(T > cut)) return 0.0;
  const double v = (T - cut) / T;
  const double y = 1.0 / (g + 1.0);
  const double y12 = 1.0 - 2.0 * y;
  const double B1 = 2.0 - y * y, B2 = y12 * (3.0 + y * y), B4 = y12 * y12 * y12;
  const double B3 = B4 + y12 * y12;
  br = v / (b2 * ec) - B1 * log1p(v / ec) + B2 * v - 0.5 * B3 * v * (1.0 + ec) +
       B4 / 3.0 * v * (1.0 + ec + ec * ec);
  return t->n_el * 2.0 * kPi * kRe * kRe * kMe / T * br;
}
double or_lambda_ioni(const or_ctx* c, int m, double T, double cut, int positron) {
  return lambda_ioni(&c->mat[m], T, cut, positron);
}

/* Tsai complete-screening bremsstrahlung (PDG): dsig/dk = (A/(X0 NA rho k))[4/3 - 4/3 y + y^2],
 * y = k/E with E the total energy. Integrated over k in [kcut, T]. */
static double lambda_brem(const mat_t* t, double T, double kcut) {
  if (!(T > kcut)) return 0.0;
  const double E = T + kMe;
  const double d = T - kcut;
  return t->invX0 *
         (4.0 / 3.0 * log1p(d / kcut) - 4.0 / 3.0 * d / E + d * (T + kcut) / (2.0 * E * E));
}
double or_lambda_brem(const or_ctx* c, int m, double T, double kcut) {
  return lambda_brem(&c->mat[m], T, kcut);
}

/* Heitler two-photon annihilation in flight, per electron:
 * sigma = pi re^2/(g+1) [ (g^2+4g+1)/(g^2-1) ln(g + sqrt(g^2-1)) - (g+3)/sqrt(g^2-1) ]. */
static double lambda_annih(const mat_t* t, double T) {
  const double tau = T / kMe;
  const double g = tau + 1.0;
  const double s2 = tau * (tau + 2.0);
  const double s = sqrt(s2);
  const double sig = kPi * kRe * kRe / (g + 1.0) *
                     ((g * g + 4.0 * g + 1.0) / s2 * log1p(tau + s) - (g + 3.0) / s);
  return t->n_el * sig;
}
double or_lambda_annih(const or_ctx* c, int m, double T) { return lambda_annih(&c->mat[m], T); }

/* ------------------------------------------------------------------ tables */
static double interp_nodes(const double* v, double E) {
  const double x = (log(E) - lnEmin()) * inv_dlog();
  int i = (int)floor(x);
  if (i < 0) i = 0;
  if (i > OR_NNODE - 2) i = OR_NNODE - 2;
  const double t = x - (double)i;
  return v[i] + (v[i + 1] - v[i]) * t;
}

/* inverse of the piecewise linear-in-ln(E) range table; 0 below the first node */
static double inverse_range_nodes(const double* R, double r) {
  if (!(r >= R[0])) return 0.0;
  int lo = 0, hi = OR_NNODE - 1;
  if (r >= R[hi]) return kEmax;
  while (hi - lo > 1) {
    const int mid = (lo + hi) / 2;
    if (R[mid] <= r) lo = mid; else hi = mid;
  }
  const double t = (r - R[lo]) / (R[lo + 1] - R[lo]);
  return exp(lnEmin() + ((double)lo + t) * dlog());
}

typedef double (*stop_fn)(const mat_t*, double, double, double, int);
static double s_unrestricted(const mat_t* t, double T, double Tc, double kc, int pos) {
  (void)Tc; (void)kc;
  return dedx_col(t, T, T, pos) + dedx_rad(t, T, T);
}
static double s_restricted(const mat_t* t, double T, double Tc, double kc, int pos) {
  return dedx_col(t, T, Tc, pos) + dedx_rad(t, T, kc);
}

/* Range by quadrature of dT/S(T) in ln T: composite Simpson with 8 panels per bin;
 * below the first node S is taken proportional to 1/T, which gives R(E0) = E0/(2 S(E0)). */
static void build_range(const mat_t* t, stop_fn S, double Tc, double kc, int pos, double* R) {
  const double E0 = or_node_energy(0);
  R[0] = E0 / (2.0 * S(t, E0, Tc, kc, pos));
  const double h = dlog() / 8.0;
  for (int i = 0; i < OR_NNODE - 1; ++i) {
    double acc = 0.0;
    for (int j = 0; j <= 8; ++j) {
      const double lt = lnEmin() + (double)i * dlog() + (double)j * h;
      const double T = exp(lt);
      const double f = T / S(t, T, Tc, kc, pos);
      const double w = (j == 0 || j == 8) ? 1.0 : ((j & 1) ? 4.0 : 2.0);
      acc += w * f;
    }
    R[i + 1] = R[i] + acc * h / 3.0;
  }
}

static double clamp_cut(double x) {
  if (x < 0.99e-3) return 0.99e-3;
  if (x > 1e4) return 1e4;
  return x;
}

/* Production thresholds from a range cut (Geant4-style "cut in range"):
 * e+-: the energy whose unrestricted CSDA range equals the cut (exact inversion of the
 *      interpolated range table); gamma: the energy where 5 absorption lengths equal the
 *      cut, on the decreasing low-energy branch of mu_total (exact inversion of the
 *      interpolated table). Both clamped to [0.99 keV, 10 GeV]; positrons use the
 *      electron threshold. */
static void compute_cuts(or_ctx* c, int m, double range_cut) {
  double* Rf = c->rfull[m];
  double Tc;
  if (range_cut <= Rf[0]) {
    Tc = or_node_energy(0);
  } else {
    Tc = kEmax;
    for (int i = 0; i < OR_NNODE - 1; ++i) {
      if (Rf[i + 1] >= range_cut) {
        const double t = (range_cut - Rf[i]) / (Rf[i + 1] - Rf[i]);
        Tc = exp(lnEmin() + ((double)i + t) * dlog());
        break;
      }
    }
  }
  const double target = 5.0 / range_cut;
  double mu[OR_NNODE];
  for (int i = 0; i < OR_NNODE; ++i) mu[i] = c->gam[m][0][i] + c->gam[m][1][i] + c->gam[m][2][i];
  double kc;
  if (mu[0] <= target) {
    kc = or_node_energy(0);
  } else {
    kc = kEmax;
    for (int i = 0; i < OR_NNODE - 1; ++i) {
      if (mu[i + 1] <= target) {
        const double t = (mu[i] - target) / (mu[i] - mu[i + 1]);
        kc = exp(lnEmin() + ((double)i + t) * dlog());
        break;
      }
    }
  }
  c->Tc[m] = clamp_cut(Tc);
  c->kc[m] = clamp_cut(kc);
}

static void build_tables(or_ctx* c, double range_cut) {
  for (int m = 0; m < c->n_mat; ++m) {
    const mat_t* t = &c->mat[m];
    if (t->Z <= 0) continue;
    for (int i = 0; i < OR_NNODE; ++i) {
      const double E = or_node_energy(i);
      c->gam[m][0][i] = or_mu_compton(c, m, E);
      c->gam[m][1][i] = or_mu_pair(c, m, E);
      c->gam[m][2][i] = or_mu_photo(c, m, E);
    }
    build_range(t, s_unrestricted, 0.0, 0.0, 0, c->rfull[m]);
    compute_cuts(c, m, range_cut);
    const double Tc = c->Tc[m], kc = c->kc[m];
    for (int i = 0; i < OR_NNODE; ++i) {
      const double T = or_node_energy(i);
      c->ele[m][0][i] = s_restricted(t, T, Tc, kc, 0);
      c->ele[m][2][i] = lambda_ioni(t, T, Tc, 0);
      c->ele[m][3][i] = lambda_brem(t, T, kc);
      c->pos[m][0][i] = s_restricted(t, T, Tc, kc, 1);
      c->pos[m][2][i] = lambda_ioni(t, T, Tc, 1);
      c->pos[m][3][i] = lambda_brem(t, T, kc);
      c->pos[m][4][i] = lambda_annih(t, T);
    }
    build_range(t, s_restricted, Tc, kc, 0, c->ele[m][1]);
    build_range(t, s_restricted, Tc, kc, 1, c->pos[m][1]);
  }
}

void or_cuts(const or_ctx* c, int m, double* Tc, double* kc) {
  *Tc = c->Tc[m];
  *kc = c->kc[m];
}

static const double* table_ptr(const or_ctx* c, int species, int table, int m) {
  if (m < 0 || m >= c->n_mat || c->mat[m].Z <= 0) return NULL;
  if (species == 0 && table >= 0 && table < 3) return c->gam[m][table];
  if (species == 1 && table >= 0 && table < 4) return c->ele[m][table];
  if (species == 2 && table >= 0 && table < 5) return c->pos[m][table];
  if (species == 3 && table == 0) return c->rfull[m];
  return NULL;
}

int or_table(const or_ctx* c, int species, int table, int m, double* out) {
  const double* p = table_ptr(c, species, table, m);
  if (!p) return -1;
  memcpy(out, p, sizeof(double) * OR_NNODE);
  return 0;
}
double or_interp(const or_ctx* c, int species, int table, int m, double E) {
  const double* p = table_ptr(c, species, table, m);
  return p ? interp_nodes(p, E) : NAN;
}
double or_inverse_range(const or_ctx* c, int species, int m, double R) {
  const double* p = table_ptr(c, species, 1, m);
  return p ? inverse_range_nodes(p, R) : NAN;
}

/* ------------------------------------------------------------------ geometry */
int or_n_volumes(const or_ctx* c) { return c->n_vol; }
int or_n_bins(const or_ctx* c) { return c->n_bins; }

/* Slab: volumes between the planes bnd[0..n_vol]; tubes: volume 0 is r < bnd[0] and
 * volume v > 0 is bnd[v-1] <= r < bnd[v]; the world ends at bnd[n_vol-1].
 * A point on a surface belongs to the volume its direction points into. */
int or_locate(const or_ctx* c, const double p[3], const double u[3]) {
  if (c->kind == 0) {
    if (fabs(p[0]) > c->half_xy || fabs(p[1]) > c->half_xy) return -1;
    const double z = p[2];
    if (z < c->bnd[0] || z > c->bnd[c->n_vol]) return -1;
    for (int k = 0; k <= c->n_vol; ++k) {
      if (z == c->bnd[k]) {
        const int v = (u[2] >= 0.0) ? k : k - 1;
        return (v < 0 || v >= c->n_vol) ? -1 : v;
      }
    }
    int v = 0;
    while (v < c->n_vol && c->bnd[v + 1] <= z) ++v;
    return v;
  }
  if (fabs(p[2]) > c->half_z) return -1;
  const double r = sqrt(p[0] * p[0] + p[1] * p[1]);
  const double radial = p[0] * u[0] + p[1] * u[1];
  int v = 0;
  for (int k = 0; k < c->n_vol; ++k) {
    const double b = c->bnd[k];
    if (fabs(r - b) <= 1e-9 * b) {
      v = (radial > 0.0) ? k + 1 : k;
      return v >= c->n_vol ? -1 : v;
    }
    if (b < r) v = k + 1;
  }
  return v >= c->n_vol ? -1 : v;
}

static const double kInf = 1e300;

double or_distance(const or_ctx* c, const double p[3], const double u[3], int vol, int* next) {
  double s = kInf;
  int nx = vol;
  if (c->kind == 0) {
    if (u[2] > 0.0) {
      s = (c->bnd[vol + 1] - p[2]) / u[2];
      nx = (vol + 1 < c->n_vol) ? vol + 1 : -1;
    } else if (u[2] < 0.0) {
      s = (c->bnd[vol] - p[2]) / u[2];
      nx = vol - 1;
    }
    const double H = c->half_xy;
    for (int a = 0; a < 2; ++a) {
      double sw = kInf;
      if (u[a] > 0.0) sw = (H - p[a]) / u[a];
      else if (u[a] < 0.0) sw = (-H - p[a]) / u[a];
      if (sw < s) { s = sw; nx = -1; }
    }
  } else {
    const double a = u[0] * u[0] + u[1] * u[1];
    const double b = p[0] * u[0] + p[1] * u[1];
    const double r2 = p[0] * p[0] + p[1] * p[1];
    if (a > 0.0) {
      const double Ro = c->bnd[vol];
      const double co = r2 - Ro * Ro;
      double D = b * b - a * co;
      if (D < 0.0) D = 0.0;
      const double sq = sqrt(D);
      double so = (b > 0.0) ? -co / (b + sq) : (sq - b) / a;
      if (so < 0.0) so = 0.0;
      s = so;
      nx = (vol + 1 < c->n_vol) ? vol + 1 : -1;
      if (vol > 0 && b < 0.0) {
        const double Ri = c->bnd[vol - 1];
        const double ci = r2 - Ri * Ri;
        const double Di = b * b - a * ci;
        if (Di > 0.0) {
          double si = ci / (sqrt(Di) - b);
          if (si < 0.0) si = 0.0;
          if (si < s) { s = si; nx = vol - 1; }
        }
      }
    }
    double sz = kInf;
    if (u[2] > 0.0) sz = (c->half_z - p[2]) / u[2];
    else if (u[2] < 0.0) sz = (-c->half_z - p[2]) / u[2];
    if (sz < s) { s = sz; nx = -1; }
  }
  if (s < 0.0) s = 0.0;
  *next = nx;
  return s;
}

/* Helix in the uniform field B along z (paper Sec. 2.3 propagates in a constant field; the
 * closed form replaces its chord segments). h = -sign(qB) is the sense of rotation of the
 * transverse direction, rho = p_T / (0.299792458 |B|) the radius in mm, and the transverse
 * direction turns by Delta = s u_T / rho over a path s. */
typedef struct {
  int straight;
  double uT, rho, h, psi0, cx, cy, kpath;
} helix_t;

static void helix_setup(double B, double T, int q, const double u[3], const double p[3],
                        helix_t* H) {
  H->straight = 1;
  if (B == 0.0 || q == 0) return;
  const double uT = sqrt(u[0] * u[0] + u[1] * u[1]);
  if (!(uT > 1e-12)) return;
  const double pm = sqrt(T * (T + 2.0 * kMe));
  H->straight = 0;
  H->uT = uT;
  H->rho = pm * uT / (kHelixK * fabs(B));
  H->h = ((q > 0) == (B > 0.0)) ? -1.0 : 1.0;
  H->psi0 = atan2(-H->h * u[0], H->h * u[1]);
  H->cx = p[0] - H->rho * H->h * u[1] / uT;
  H->cy = p[1] + H->rho * H->h * u[0] / uT;
  H->kpath = uT / H->rho;
}

void or_helix_move(double B, double T, int q, double s, double p[3], double u[3]) {
  helix_t H;
  helix_setup(B, T, q, u, p, &H);
  if (H.straight) {
    p[0] += s * u[0]; p[1] += s * u[1]; p[2] += s * u[2];
    return;
  }
  const double D = s * H.kpath;
  const double sd = sin(D), cd = cos(D);
  const double sh = sin(0.5 * D);
  const double cm1 = -2.0 * sh * sh; /* cos D - 1 */
  const double a = u[0] / H.uT, b = u[1] / H.uT;
  p[0] += H.rho * (a * sd + H.h * b * cm1);
  p[1] += H.rho * (b * sd - H.h * a * cm1);
  p[2] += s * u[2];
  const double u0 = u[0] * cd - H.h * u[1] * sd;
  const double u1 = u[1] * cd + H.h * u[0] * sd;
  u[0] = u0; u[1] = u1;
}

static double mod2pi(double x) {
  const double tp = 2.0 * kPi;
  double r = fmod(x, tp);
  if (r < 0.0) r += tp;
  return r;
}

/* first crossing of the helix with a level set n.P = d (straight wall) or |P| = R
 * (cylinder) in the crossing direction asked for; the crossing's phase on the circle is
 * psi_ref -/+ acos(C): the first for an increasing, the second for a decreasing level */
static double helix_phase_hit(const helix_t* H, double psi_ref, double C, int increasing) {
  if (!(C >= -1.0 && C <= 1.0)) return kInf;
  const double A = acos(C);
  const double D = increasing ? mod2pi(H->h * (psi_ref - H->psi0) - A)
                              : mod2pi(H->h * (psi_ref - H->psi0) + A);
  return D / H->kpath;
}

double or_helix_distance(const or_ctx* c, double T, int q, const double p[3], const double u[3],
                         int vol, int* next) {
  helix_t H;
  helix_setup(c->field_T, T, q, u, p, &H);
  if (H.straight) return or_distance(c, p, u, vol, next);
  double s = kInf;
  int nx = vol;
  if (c->kind == 0) {
    if (u[2] > 0.0) {
      s = (c->bnd[vol + 1] - p[2]) / u[2];
      nx = (vol + 1 < c->n_vol) ? vol + 1 : -1;
    } else if (u[2] < 0.0) {
      s = (c->bnd[vol] - p[2]) / u[2];
      nx = vol - 1;
    }
    const double Hw = c->half_xy;
    if (!(fabs(H.cx) + H.rho < Hw && fabs(H.cy) + H.rho < Hw)) {
      /* walls x = +H, x = -H, y = +H, y = -H as n.P = H with n = +x, -x, +y, -y */
      const double nxs[4] = {1.0, -1.0, 0.0, 0.0}, nys[4] = {0.0, 0.0, 1.0, -1.0};
      const double psin[4] = {0.0, kPi, 0.5 * kPi, -0.5 * kPi};
      for (int w = 0; w < 4; ++w) {
        const double nc = nxs[w] * H.cx + nys[w] * H.cy;
        const double sw = helix_phase_hit(&H, psin[w], (Hw - nc) / H.rho, 1);
        if (sw < s) { s = sw; nx = -1; }
      }
    }
  } else {
    const double cm = sqrt(H.cx * H.cx + H.cy * H.cy);
    if (cm > 1e-12) {
      const double psic = atan2(H.cy, H.cx);
      const double Ro = c->bnd[vol];
      const double so = helix_phase_hit(&H, psic, (Ro * Ro - cm * cm - H.rho * H.rho) / (2.0 * H.rho * cm), 1);
      if (so < s) { s = so; nx = (vol + 1 < c->n_vol) ? vol + 1 : -1; }
      if (vol > 0) {
        const double Ri = c->bnd[vol - 1];
        const double si = helix_phase_hit(&H, psic, (Ri * Ri - cm * cm - H.rho * H.rho) / (2.0 * H.rho * cm), 0);
        if (si < s) { s = si; nx = vol - 1; }
      }
    }
    double sz = kInf;
    if (u[2] > 0.0) sz = (c->half_z - p[2]) / u[2];
    else if (u[2] < 0.0) sz = (-c->half_z - p[2]) / u[2];
    if (sz < s) { s = sz; nx = -1; }
    if (s >= kInf) { s = 2.0 * kPi / H.kpath; nx = vol; } /* a closed circle: one turn */
  }
  *next = nx;
  return s;
}

/* ------------------------------------------------------------------ ray tracing */
static void normalize3(double v[3]);
/* entry of the ray p + t u (t >= 0) into the world, snapped onto the entry face; returns
 * 0 if the ray misses it */
static int world_entry(const or_ctx* c, const double p[3], const double u[3], double q[3]) {
  double t0 = 0.0, t1 = kInf;
  int face = -1; /* 0/1/2: axis of the entry plane (box) or z cap; 3: the cylinder */
  double fval = 0.0;
  if (c->kind == 0) {
    const double lo[3] = {-c->half_xy, -c->half_xy, c->bnd[0]};
    const double hi[3] = {c->half_xy, c->half_xy, c->bnd[c->n_vol]};
    for (int a = 0; a < 3; ++a) {
      if (u[a] == 0.0) {
        if (p[a] < lo[a] || p[a] > hi[a]) return 0;
        continue;
      }
      double ta = (lo[a] - p[a]) / u[a], tb = (hi[a] - p[a]) / u[a];
      double va = lo[a], vb = hi[a];
      if (ta > tb) { double x = ta; ta = tb; tb = x; x = va; va = vb; vb = x; }
      if (ta > t0) { t0 = ta; face = a; fval = va; }
      if (tb < t1) t1 = tb;
    }
  } else {
    const double R = c->bnd[c->n_vol - 1];
    const double a = u[0] * u[0] + u[1] * u[1], b = p[0] * u[0] + p[1] * u[1];
    const double cc = p[0] * p[0] + p[1] * p[1] - R * R;
    if (a > 0.0) {
      const double D = b * b - a * cc;
      if (D < 0.0) return 0;
      const double sq = sqrt(D);
      const double ta = (-b - sq) / a, tb = (-b + sq) / a;
      if (ta > t0) { t0 = ta; face = 3; }
      if (tb < t1) t1 = tb;
    } else if (cc > 0.0) {
      return 0;
    }
    if (u[2] != 0.0) {
      double ta = (-c->half_z - p[2]) / u[2], tb = (c->half_z - p[2]) / u[2];
      double va = -c->half_z, vb = c->half_z;
      if (ta > tb) { double x = ta; ta = tb; tb = x; x = va; va = vb; vb = x; }
      if (ta > t0) { t0 = ta; face = 2; fval = va; }
      if (tb < t1) t1 = tb;
    } else if (fabs(p[2]) > c->half_z) {
      return 0;
    }
  }
  if (!(t0 <= t1)) return 0;
  for (int a = 0; a < 3; ++a) q[a] = p[a] + t0 * u[a];
  if (face >= 0 && face < 3) q[face] = fval;
  if (face == 3) {
    const double R = c->bnd[c->n_vol - 1], r = sqrt(q[0] * q[0] + q[1] * q[1]);
    if (r > 0.0) { q[0] *= R / r; q[1] *= R / r; }
  }
  return 1;
}

void or_raytrace(const or_ctx* c, const double cam[11], int nx, int ny, double* out) {
  double d[3] = {cam[3], cam[4], cam[5]}, up[3] = {cam[6], cam[7], cam[8]};
  normalize3(d);
  double rt[3] = {d[1] * up[2] - d[2] * up[1], d[2] * up[0] - d[0] * up[2], d[0] * up[1] - d[1] * up[0]};
  normalize3(rt);
  const double u2[3] = {rt[1] * d[2] - rt[2] * d[1], rt[2] * d[0] - rt[0] * d[2], rt[0] * d[1] - rt[1] * d[0]};
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      const double a = ((i + 0.5) / nx - 0.5) * cam[9], b = ((j + 0.5) / ny - 0.5) * cam[10];
      const double p[3] = {cam[0] + a * rt[0] + b * u2[0], cam[1] + a * rt[1] + b * u2[1],
                           cam[2] + a * rt[2] + b * u2[2]};
      double q[3], mass = 0.0, n = 0.0;
      if (world_entry(c, p, d, q)) {
        int vol = or_locate(c, q, d);
        for (int k = 0; vol >= 0 && k < 100000; ++k) {
          n += 1.0;
          int next;
          const double s = or_distance(c, q, d, vol, &next);
          const int m = c->vol_mat[vol];
          if (m >= 0) mass += c->mat[m].rho * s * 0.1;
          for (int e = 0; e < 3; ++e) q[e] += s * d[e];
          if (c->kind == 0 && next >= 0) q[2] = c->bnd[d[2] > 0.0 ? vol + 1 : vol];
          vol = next;
        }
      }
      out[2 * ((size_t)j * nx + i)] = mass;
      out[2 * ((size_t)j * nx + i) + 1] = n;
    }
}

/* ------------------------------------------------------------------ chord propagation */
/* is p inside (or on the boundary of) volume vol */
static int inside_volume(const or_ctx* c, const double p[3], int vol) {
  if (c->kind == 0) {
    return p[2] >= c->bnd[vol] && p[2] <= c->bnd[vol + 1] && fabs(p[0]) <= c->half_xy &&
           fabs(p[1]) <= c->half_xy;
  }
  const double r2 = p[0] * p[0] + p[1] * p[1];
  if (fabs(p[2]) > c->half_z) return 0;
  if (r2 > c->bnd[vol] * c->bnd[vol]) return 0;
  return vol == 0 || r2 >= c->bnd[vol - 1] * c->bnd[vol - 1];
}

/* the point and direction at path s along the helix from (p0, u0) */
static void helix_at(double B, double T, int q, const double p0[3], const double u0[3], double s, double p[3],
                     double u[3]) {
  memcpy(p, p0, 3 * sizeof(double));
  memcpy(u, u0, 3 * sizeof(double));
  or_helix_move(B, T, q, s, p, u);
}

int or_chord_step(const or_ctx* c, double T, int q, double s_phys, int max_iter, double delta_chord,
                  double delta_int, double p[3], double u[3], int vol, int* next, double* s_done,
                  int* iters) {
  const double B = c->field_T;
  helix_t H;
  helix_setup(B, T, q, u, p, &H);
  *iters = 0;
  if (H.straight) { /* no curvature: one straight segment */
    *iters = 1;
    const double sg = or_distance(c, p, u, vol, next);
    const double s = sg <= s_phys ? sg : s_phys;
    p[0] += s * u[0]; p[1] += s * u[1]; p[2] += s * u[2];
    *s_done = s;
    return sg <= s_phys ? 1 : 0;
  }
  double ps[3], us[3], tmp[3];                           /* the state at the step's start */
  memcpy(ps, p, sizeof(ps));
  memcpy(us, u, sizeof(us));
  const double kappa = H.uT * H.kpath;                   /* |du/ds| of the helix */
  const double lmax = sqrt(8.0 * delta_chord / kappa);   /* sagitta kappa l^2 / 8 <= delta_chord */
  const double lint = sqrt(8.0 * delta_int / kappa);
  double s0 = 0.0, P0[3];
  memcpy(P0, ps, sizeof(P0));
  for (;;) {
    if (++*iters > max_iter) return 2;
    const double ell = (s_phys - s0 < lmax) ? s_phys - s0 : lmax;
    double P1[3], U1[3];
    helix_at(B, T, q, ps, us, s0 + ell, P1, U1);
    double d[3] = {P1[0] - P0[0], P1[1] - P0[1], P1[2] - P0[2]};
    const double L = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    int nx = vol;
    double sb = kInf;
    if (L > 0.0) {
      d[0] /= L; d[1] /= L; d[2] /= L;
      sb = or_distance(c, P0, d, vol, &nx);
    }
    /* a segment that meets the boundary: look for a curve point outside the volume, at the
     * segment's end or where the segment meets the boundary */
    double hi = -1.0;
    if (sb < L) {
      if (!inside_volume(c, P1, vol)) {
        hi = s0 + ell;
      } else {
        const double sc = s0 + ell * (sb / L);
        double Pc[3];
        helix_at(B, T, q, ps, us, sc, Pc, tmp);
        if (!inside_volume(c, Pc, vol)) hi = sc;
      }
    }
    if (hi < 0.0) { /* no crossing on this segment */
      s0 += ell;
      memcpy(P0, P1, sizeof(P0));
      if (s0 >= s_phys) {
        memcpy(p, P1, sizeof(P1));
        memcpy(u, U1, sizeof(U1));
        *s_done = s_phys;
        return 0;
      }
      continue;
    }
    /* refine: bisection between an inside (lo) and an outside (hi) point of the curve until
     * the chord between them has a sagitta of at most delta_int */
    double lo = s0, Plo[3], Phi[3];
    memcpy(Plo, P0, sizeof(Plo));
    helix_at(B, T, q, ps, us, hi, Phi, tmp);
    while (hi - lo > lint) {
      if (++*iters > max_iter) return 2;
      const double mid = 0.5 * (lo + hi);
      double Pm[3];
      helix_at(B, T, q, ps, us, mid, Pm, tmp);
      if (inside_volume(c, Pm, vol)) { lo = mid; memcpy(Plo, Pm, sizeof(Plo)); }
      else { hi = mid; memcpy(Phi, Pm, sizeof(Phi)); }
    }
    /* the crossing lies on that chord; the direction is the curve's at the matching path */
    double e[3] = {Phi[0] - Plo[0], Phi[1] - Plo[1], Phi[2] - Plo[2]};
    const double Le = sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
    double sx = hi;
    if (Le > 0.0) {
      e[0] /= Le; e[1] /= Le; e[2] /= Le;
      double sbe = or_distance(c, Plo, e, vol, &nx);
      if (sbe > Le) sbe = Le;
      sx = lo + (sbe / Le) * (hi - lo);
      p[0] = Plo[0] + sbe * e[0]; p[1] = Plo[1] + sbe * e[1]; p[2] = Plo[2] + sbe * e[2];
    } else {
      memcpy(p, Phi, sizeof(Phi));
    }
    double Px[3];
    helix_at(B, T, q, ps, us, sx, Px, u);
    *next = nx;
    *s_done = sx;
    return 1;
  }
}

/* ------------------------------------------------------------------ kinematics helpers */
/* rotate the local direction (sin t cos f, sin t sin f, cos t) from the frame whose z axis
 * is u into the global frame */
static void rotate_to(const double u[3], double cost, double phi, double out[3]) {
  double s2 = 1.0 - cost * cost;
  if (s2 < 0.0) s2 = 0.0;
  const double sint = sqrt(s2);
  const double l0 = sint * cos(phi), l1 = sint * sin(phi), l2 = cost;
  const double up2 = u[0] * u[0] + u[1] * u[1];
  if (up2 > 0.0) {
    const double up = sqrt(up2);
    out[0] = (u[0] * u[2] * l0 - u[1] * l1) / up + u[0] * l2;
    out[1] = (u[1] * u[2] * l0 + u[0] * l1) / up + u[1] * l2;
    out[2] = -up * l0 + u[2] * l2;
  } else if (u[2] >= 0.0) {
    out[0] = l0; out[1] = l1; out[2] = l2;
  } else {
    out[0] = -l0; out[1] = l1; out[2] = -l2;
  }
}

static void normalize3(double v[3]) {
  const double n = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  v[0] /= n; v[1] /= n; v[2] /= n;
}

typedef struct {
  int happened;
  int n;
  int species[2];
  double T[2];
  double dir[2][3];
  int parent_alive;
  double parent_T;
  double parent_dir[3];
} ixn_t;

static const int kMaxRejections = 1000;

/* ------------------------------------------------------------------ continuous physics */
/* the uniform pair of counter block blk of a (track, step) stream */
static void stream_block(const stream_t* s, uint32_t blk, double* ua, double* ub) {
  const uint32_t c[4] = {s->ctr[0], s->ctr[1], s->ctr[2], blk};
  uint32_t w[4];
  or_philox(c, s->key, w);
  *ua = or_u01_f64(w[0], w[1]);
  *ub = or_u01_f64(w[2], w[3]);
}

/* Highland's width of the projected scattering angle (PDG Review of Particle Physics,
 * "Passage of particles through matter", multiple scattering through small angles):
 * theta0 = 13.6 MeV / (beta c p) * z * sqrt(x/X0) * (1 + 0.038 ln(x z^2 / (X0 beta^2))),
 * z = 1, at the pre-step energy. The bracket, negative only below x/X0 ~ 1e-11, is
 * clamped at 0. */
double or_msc_theta0(const or_ctx* c, int m, double T, double s) {
  const double E = T + kMe, pc2 = T * (T + 2.0 * kMe);
  const double beta2 = pc2 / (E * E), bcp = pc2 / E;
  const double x = s * c->mat[m].invX0;
  if (!(x > 0.0)) return 0.0;
  double br = 1.0 + 0.038 * log(x / beta2);
  if (br < 0.0) br = 0.0;
  return 13.6 / bcp * sqrt(x) * br;
}

/* Bohr's variance of the energy lost over s to transfers up to Tu (the part of the loss
 * that is continuous: Tu = min(production cut, largest transfer), T/2 for e-, T for e+):
 * sigma^2 = 2 pi r_e^2 m c^2 n_el s Tu (1 - beta^2/2) / beta^2. */
double or_fluct_sigma2(const or_ctx* c, int m, double T, double s, int positron) {
  const mat_t* t = &c->mat[m];
  const double E = T + kMe, beta2 = T * (T + 2.0 * kMe) / (E * E);
  const double tmax = positron ? T : 0.5 * T;
  const double tu = c->Tc[m] < tmax ? c->Tc[m] : tmax;
  return 2.0 * kPi * kRe * kRe * kMe * t->n_el * s * tu * (1.0 - 0.5 * beta2) / beta2;
}

/* deflection by theta = theta0 sqrt(-2 ln ua) (the space angle of two independent Gaussian
 * projected angles of width theta0), at most pi, azimuth 2 pi ub */
static void msc_deflect(const stream_t* rs, double theta0, double u[3]) {
  double ua, ub;
  stream_block(rs, OR_MSC_BLOCK, &ua, &ub);
  double th = theta0 * sqrt(-2.0 * log(ua));
  if (th > kPi) th = kPi;
  double out[3];
  rotate_to(u, cos(th), 2.0 * kPi * ub, out);
  normalize3(out);
  memcpy(u, out, sizeof(out));
}

/* Gaussian loss about the mean, redrawn (at most 8 times, then the mean) until it lies in
 * [0, 2 mean]; one Box-Muller normal per counter block */
static double fluct_loss(const stream_t* rs, double mean, double sigma) {
  for (uint32_t i = 0; i < 8; ++i) {
    double ua, ub;
    stream_block(rs, OR_FLUCT_BLOCK + i, &ua, &ub);
    const double g = sqrt(-2.0 * log(ua)) * cos(2.0 * kPi * ub);
    const double d = mean + sigma * g;
    if (d >= 0.0 && d <= 2.0 * mean) return d;
  }
  return mean;
}

/* Compton, Klein-Nishina via Butcher & Messel composition-rejection (Nucl. Phys. 20 (1960)
 * 15; EGS4 SLAC-265 Sec. 2.9): eps = E'/E in [eps0, 1], eps0 = 1/(1+2 kappa), is drawn from
 * 1/eps (weight ln(1/eps0)) or from eps (weight (1-eps0^2)/2), then accepted with
 * 1 - eps sin^2(theta) / (1 + eps^2). */
static void sample_compton(stream_t* st, double E, const double u[3], ixn_t* r) {
  const double kap = E / kMe;
  const double e0 = 1.0 / (1.0 + 2.0 * kap);
  const double a1 = log1p(2.0 * kap);
  const double a2 = 0.5 * (1.0 - e0 * e0);
  double eps = 1.0, t = 0.0;
  for (int it = 0; it < kMaxRejections; ++it) {
    const double r1 = stream_u(st), r2 = stream_u(st), r3 = stream_u(st);
    if (r1 * (a1 + a2) < a1) {
      eps = exp(-a1 * r2);
    } else {
      eps = sqrt(e0 * e0 + (1.0 - e0 * e0) * r2);
    }
    t = (1.0 - eps) / (kap * eps);
    const double sin2 = t * (2.0 - t);
    const double g = 1.0 - eps * sin2 / (1.0 + eps * eps);
    if (r3 < g) break;
  }
  const double phi = 2.0 * kPi * stream_u(st);
  const double Ep = eps * E;
  double ud[3];
  rotate_to(u, 1.0 - t, phi, ud);
  r->happened = 1;
  r->parent_alive = 1;
  r->parent_T = Ep;
  r->parent_dir[0] = ud[0]; r->parent_dir[1] = ud[1]; r->parent_dir[2] = ud[2];
  const double Te = E - Ep;
  double pe[3] = {E * u[0] - Ep * ud[0], E * u[1] - Ep * ud[1], E * u[2] - Ep * ud[2]};
  normalize3(pe);
  r->n = 1;
  r->species[0] = 1;
  r->T[0] = Te;
  memcpy(r->dir[0], pe, sizeof(pe));
}

/* Bethe-Heitler pair: x = E+/E drawn uniformly on [m/E, 1-m/E] and accepted with
 * 1 - 4/3 x(1-x) (efficiency >= 2/3); leptons at the characteristic angle m/E+-. */
static void sample_pair(stream_t* st, double E, const double u[3], ixn_t* r) {
  r->happened = 0;
  if (!(E > 2.0 * kMe)) return;
  const double a = kMe / E;
  double x = 0.5;
  for (int it = 0; it < kMaxRejections; ++it) {
    const double r1 = stream_u(st), r2 = stream_u(st);
    x = a + (1.0 - 2.0 * a) * r1;
    if (r2 < 1.0 - 4.0 / 3.0 * x * (1.0 - x)) break;
  }
  const double Tp = x * E - kMe;
  const double Tm = E - 2.0 * kMe - Tp;
  const double phi = 2.0 * kPi * stream_u(st);
  r->happened = 1;
  r->parent_alive = 0;
  r->n = 2;
  r->species[0] = 2;
  r->T[0] = Tp;
  rotate_to(u, cos(kMe / (Tp + kMe)), phi, r->dir[0]);
  r->species[1] = 1;
  r->T[1] = Tm;
  rotate_to(u, cos(kMe / (Tm + kMe)), phi + kPi, r->dir[1]);
}

static void sample_photo(double E, const double u[3], ixn_t* r) {
  r->happened = 1;
  r->parent_alive = 0;
  r->n = 1;
  r->species[0] = 1;
  r->T[0] = E;
  memcpy(r->dir[0], u, 3 * sizeof(double));
}

/* delta-ray kinematics shared by Moller and Bhabha: free-electron two-body scattering */
static void delta_kinematics(stream_t* st, double T, double Td, const double u[3], ixn_t* r) {
  const double cd = sqrt(Td * (T + 2.0 * kMe) / (T * (Td + 2.0 * kMe)));
  const double phi = 2.0 * kPi * stream_u(st);
  double dd[3];
  rotate_to(u, cd > 1.0 ? 1.0 : cd, phi, dd);
  const double p0 = sqrt(T * (T + 2.0 * kMe));
  const double pd = sqrt(Td * (Td + 2.0 * kMe));
  double pp[3] = {p0 * u[0] - pd * dd[0], p0 * u[1] - pd * dd[1], p0 * u[2] - pd * dd[2]};
  normalize3(pp);
  r->happened = 1;
  r->parent_alive = 1;
  r->parent_T = T - Td;
  memcpy(r->parent_dir, pp, sizeof(pp));
  r->n = 1;
  r->species[0] = 1;
  r->T[0] = Td;
  memcpy(r->dir[0], dd, sizeof(dd));
}

/* Moller: eps from 1/eps^2 on [Tc/T, 1/2] by inversion, accepted with
 * eps^2 f(eps) / (2 + (1-gg)/4), the bound taking each positive term at eps = 1/2 */
static void sample_moller(stream_t* st, double T, double Tc, const double u[3], ixn_t* r) {
  r->happened = 0;
  if (!(T > 2.0 * Tc)) return;
  const double g = T / kMe + 1.0;
  const double gg = (2.0 * g - 1.0) / (g * g);
  const double ec = Tc / T, em = 0.5;
  const double gmax = 2.0 + 0.25 * (1.0 - gg);
  double eps = ec;
  for (int it = 0; it < kMaxRejections; ++it) {
    const double r1 = stream_u(st), r2 = stream_u(st);
    eps = ec * em / (em - (em - ec) * r1);
    const double q = eps / (1.0 - eps);
    const double f = 1.0 + q * q + (1.0 - gg) * eps * eps - gg * q;
    if (r2 * gmax < f) break;
  }
  delta_kinematics(st, T, eps * T, u, r);
}

/* Bhabha: eps from 1/eps^2 on [Tc/T, 1] by inversion, accepted with
 * b2 eps^2 f(eps) = 1 - b2 eps (B1 - eps (B2 - eps (B3 - eps B4))) <= 1 */
static void sample_bhabha(stream_t* st, double T, double Tc, const double u[3], ixn_t* r) {
  r->happened = 0;
  if (!(T > Tc)) return;
  const double tau = T / kMe;
  const double g = tau + 1.0;
  const double b2 = tau * (tau + 2.0) / (g * g);
  const double y = 1.0 / (g + 1.0);
  const double y12 = 1.0 - 2.0 * y;
  const double B1 = 2.0 - y * y, B2 = y12 * (3.0 + y * y), B4 = y12 * y12 * y12;
  const double B3 = B4 + y12 * y12;
  const double ec = Tc / T;
  double eps = ec;
  for (int it = 0; it < kMaxRejections; ++it) {
    const double r1 = stream_u(st), r2 = stream_u(st);
    eps = ec / (1.0 - (1.0 - ec) * r1);
    const double gfun = 1.0 - b2 * eps * (B1 - eps * (B2 - eps * (B3 - eps * B4)));
    if (r2 < gfun) break;
  }
  delta_kinematics(st, T, eps * T, u, r);
}

/* Tsai bremsstrahlung: k = kc (T/kc)^r (a 1/k draw), accepted with 1 - y + 3/4 y^2, y = k/E;
 * the photon leaves at the characteristic angle m/E, the lepton keeps its direction */
static void sample_brem(stream_t* st, double T, double kc, const double u[3], ixn_t* r) {
  r->happened = 0;
  if (!(T > kc)) return;
  const double E = T + kMe;
  const double lr = log(T / kc);
  double k = kc;
  for (int it = 0; it < kMaxRejections; ++it) {
    const double r1 = stream_u(st), r2 = stream_u(st);
    k = kc * exp(lr * r1);
    const double y = k / E;
    if (r2 < 1.0 - y + 0.75 * y * y) break;
  }
  const double phi = 2.0 * kPi * stream_u(st);
  r->happened = 1;
  r->parent_alive = 1;
  r->parent_T = T - k;
  memcpy(r->parent_dir, u, 3 * sizeof(double));
  r->n = 1;
  r->species[0] = 0;
  r->T[0] = k;
  rotate_to(u, cos(kMe / E), phi, r->dir[0]);
}

/* Heitler two-photon annihilation in flight: eps = E1/(T + 2m) drawn from 1/eps on
 * [eps_min, eps_max] = (1 -+ sqrt((g-1)/(g+1)))/2 and accepted with
 * 1 - eps + (2 g eps - 1)/(eps (g+1)^2) (maximum (g^2+1)/(g+1)^2 <= 1);
 * photon 1 from two-body kinematics, photon 2 from momentum conservation. */
static void sample_annih(stream_t* st, double T, const double u[3], ixn_t* r) {
  const double tau = T / kMe;
  const double g = tau + 1.0;
  const double sq = sqrt(tau / (tau + 2.0));
  const double emin = 0.5 * (1.0 - sq), emax = 0.5 * (1.0 + sq);
  const double lr = log(emax / emin);
  const double gp1 = g + 1.0;
  double eps = 0.5;
  for (int it = 0; it < kMaxRejections; ++it) {
    const double r1 = stream_u(st), r2 = stream_u(st);
    eps = emin * exp(lr * r1);
    const double gfun = 1.0 - eps + (2.0 * g * eps - 1.0) / (eps * gp1 * gp1);
    if (r2 < gfun) break;
  }
  const double Etot = T + 2.0 * kMe;
  const double E1 = eps * Etot;
  const double E2 = Etot - E1;
  const double pp = sqrt(T * (T + 2.0 * kMe));
  double c1 = (eps * gp1 - 1.0) / (eps * sqrt(tau * (tau + 2.0)));
  if (c1 > 1.0) c1 = 1.0;
  if (c1 < -1.0) c1 = -1.0;
  const double phi = 2.0 * kPi * stream_u(st);
  r->happened = 1;
  r->parent_alive = 0;
  r->n = 2;
  r->species[0] = 0;
  r->T[0] = E1;
  rotate_to(u, c1, phi, r->dir[0]);
  r->species[1] = 0;
  r->T[1] = E2;
  double p2[3] = {pp * u[0] - E1 * r->dir[0][0], pp * u[1] - E1 * r->dir[0][1],
                  pp * u[2] - E1 * r->dir[0][2]};
  normalize3(p2);
  memcpy(r->dir[1], p2, sizeof(p2));
}

/* at rest: two photons of m each, back to back, isotropic */
static void sample_annih_rest(stream_t* st, ixn_t* r) {
  const double ct = 2.0 * stream_u(st) - 1.0;
  const double phi = 2.0 * kPi * stream_u(st);
  double s2 = 1.0 - ct * ct;
  if (s2 < 0.0) s2 = 0.0;
  const double st_ = sqrt(s2);
  r->happened = 1;
  r->parent_alive = 0;
  r->n = 2;
  r->species[0] = 0; r->species[1] = 0;
  r->T[0] = kMe; r->T[1] = kMe;
  r->dir[0][0] = st_ * cos(phi); r->dir[0][1] = st_ * sin(phi); r->dir[0][2] = ct;
  r->dir[1][0] = -r->dir[0][0]; r->dir[1][1] = -r->dir[0][1]; r->dir[1][2] = -r->dir[0][2];
}

void or_sample_continuous(const or_ctx* c, int which, int species, int m, double T, double s,
                          uint32_t seed, uint32_t event, int n, double* out) {
  for (int i = 0; i < n; ++i) {
    stream_t st;
    stream_init(&st, seed, event, (uint64_t)(i + 1), 0);
    if (which == 0) {
      double u[3] = {0.0, 0.0, 1.0};
      msc_deflect(&st, or_msc_theta0(c, m, T, s), u);
      memcpy(out + 3 * i, u, sizeof(u));
    } else {
      const double* Rt = species == 2 ? c->pos[m][1] : c->ele[m][1];
      const double R = interp_nodes(Rt, T);
      double Ep = s < R ? inverse_range_nodes(Rt, R - s) : 0.0;
      if (Ep > T) Ep = T;
      const double mean = T - Ep;
      out[2 * i] = fluct_loss(&st, mean, sqrt(or_fluct_sigma2(c, m, T, s, species == 2)));
      out[2 * i + 1] = mean;
    }
  }
}

void or_sample(const or_ctx* c, int which, int m, double E, uint32_t seed, uint32_t event, int n,
               double* out) {
  const double u[3] = {0.0, 0.0, 1.0};
  for (int i = 0; i < n; ++i) {
    stream_t st;
    stream_init(&st, seed, event, (uint64_t)(i + 1), 0);
    ixn_t r;
    memset(&r, 0, sizeof(r));
    switch (which) {
      case 0: sample_compton(&st, E, u, &r); break;
      case 1: sample_pair(&st, E, u, &r); break;
      case 2: sample_moller(&st, E, c->Tc[m], u, &r); break;
      case 3: sample_bhabha(&st, E, c->Tc[m], u, &r); break;
      case 4: sample_brem(&st, E, c->kc[m], u, &r); break;
      case 5: sample_annih(&st, E, u, &r); break;
      default: sample_annih_rest(&st, &r); break;
    }
    double* o = out + 12 * i;
    o[0] = r.happened;
    o[1] = r.parent_alive ? r.parent_T : -1.0;
    o[2] = r.parent_dir[0]; o[3] = r.parent_dir[1]; o[4] = r.parent_dir[2];
    o[5] = r.n > 0 ? r.T[0] : -1.0;
    o[6] = r.dir[0][0]; o[7] = r.dir[0][1]; o[8] = r.dir[0][2];
    o[9] = r.n > 1 ? r.T[1] : -1.0;
    o[10] = r.n > 1 ? r.dir[1][2] : 0.0;
    o[11] = r.n > 1 ? r.dir[1][0] * r.dir[0][0] + r.dir[1][1] * r.dir[0][1] + r.dir[1][2] * r.dir[0][2] : 0.0;
  }
}

/* ------------------------------------------------------------------ setup */
or_ctx* or_create(int n_mat, const int* mat_Z, const double* mat_A, const double* mat_rho,
                  const double* mat_I_eV, const int* mat_n_elem, const int* elem_Z, const double* elem_A,
                  const double* elem_atoms, int kind, int n_layers, int n_sub, const int* sub_mat,
                  const double* sub_thick, double half_xy, double half_z, const double* layer_r,
                  double range_cut_mm, double field_T, double tracking_cut_MeV) {
  if (n_mat <= 0 || n_mat > OR_MAX_MAT || n_layers <= 0 || n_sub <= 0) return NULL;
  or_ctx* c = (or_ctx*)calloc(1, sizeof(or_ctx));
  if (!c) return NULL;
  c->n_mat = n_mat;
  int e0 = 0; /* first element of material m */
  for (int m = 0; m < n_mat; ++m) {
    mat_t* t = &c->mat[m];
    t->Z = mat_Z[m];
    t->A = mat_A[m];
    t->rho = mat_rho[m];
    t->I = mat_I_eV[m];
    const int ne = mat_n_elem ? mat_n_elem[m] : 0;
    if (ne < 0 || ne > OR_MAX_ELEM) { free(c); return NULL; }
    if (ne > 0) {
      /* a compound: atoms per mm^3 of each element from the formula's mass fractions */
      double M = 0.0, natoms = 0.0, zsum = 0.0;
      for (int i = 0; i < ne; ++i) {
        M += elem_atoms[e0 + i] * elem_A[e0 + i];
        natoms += elem_atoms[e0 + i];
        zsum += elem_atoms[e0 + i] * elem_Z[e0 + i];
      }
      t->n_elem = ne;
      t->ZoA = 0.0;
      t->n_at = 0.0;
      t->n_el = 0.0;
      for (int i = 0; i < ne; ++i) {
        const double w = elem_atoms[e0 + i] * elem_A[e0 + i] / M;
        t->eZ[i] = elem_Z[e0 + i];
        t->eA[i] = elem_A[e0 + i];
        t->en_at[i] = kNA * t->rho * w / elem_A[e0 + i] * 1e-3;
        t->ZoA += w * elem_Z[e0 + i] / elem_A[e0 + i];
        t->n_at += t->en_at[i];
        t->n_el += elem_Z[e0 + i] * t->en_at[i];
      }
      t->A = M / natoms;
      t->Z = (int)(zsum / natoms + 0.5);
      if (t->Z < 1) t->Z = 1;
      e0 += ne;
    } else if (t->Z > 0) {
      t->n_at = kNA * t->rho / t->A * 1e-3;
      t->n_el = t->Z * t->n_at;
      t->n_elem = 1;
      t->eZ[0] = t->Z;
      t->eA[0] = t->A;
      t->en_at[0] = t->n_at;
      t->ZoA = t->Z / t->A;
    }
    if (t->Z > 0) {
      t->invX0 = inv_x0(t);
      density_params(t);
    }
  }
  c->kind = kind;
  c->half_xy = half_xy;
  c->half_z = half_z;
  c->field_T = field_T;
  c->tcut = tracking_cut_MeV;
  if (kind == 0) {
    int v = 0;
    c->bnd[0] = 0.0;
    double z = 0.0;
    for (int l = 0; l < n_layers; ++l)
      for (int s = 0; s < n_sub; ++s) {
        if (v >= OR_MAX_VOL) { free(c); return NULL; }
        z += sub_thick[s];
        c->vol_mat[v] = sub_mat[s];
        c->vol_bin[v] = l * n_sub + s;
        c->bnd[++v] = z;
      }
    c->n_vol = v;
  } else {
    /* volume 0 is the vacuum inside the first layer; each layer adds its sublayers and,
     * except after the last one, the vacuum gap up to the next layer */
    int v = 0;
    c->vol_mat[0] = -1;
    c->vol_bin[0] = -1;
    c->bnd[0] = layer_r[0];
    v = 1;
    for (int l = 0; l < n_layers; ++l) {
      double r = layer_r[l];
      for (int s = 0; s < n_sub; ++s) {
        if (v + 1 >= OR_MAX_VOL) { free(c); return NULL; }
        r += sub_thick[s];
        c->vol_mat[v] = sub_mat[s];
        c->vol_bin[v] = l * n_sub + s;
        c->bnd[v] = r;
        ++v;
      }
      if (l + 1 < n_layers) {
        c->vol_mat[v] = -1;
        c->vol_bin[v] = -1;
        c->bnd[v] = layer_r[l + 1];
        ++v;
      }
    }
    c->n_vol = v;
  }
  for (int v = 0; v < c->n_vol; ++v)
    if (c->vol_mat[v] >= 0 && c->mat[c->vol_mat[v]].Z <= 0) { c->vol_mat[v] = -1; c->vol_bin[v] = -1; }
  c->n_bins = n_layers * n_sub;
  build_tables(c, range_cut_mm);
  return c;
}

void or_destroy(or_ctx* c) { free(c); }

/* ------------------------------------------------------------------ transport */
typedef struct {
  double x[3], u[3];
  double T;
  uint64_t id;
  uint32_t step;
  int vol, species, vac, gen;
} trk_t;

typedef struct {
  trk_t* v;
  size_t n, cap;
} stack_t_;

static void push(stack_t_* s, const trk_t* t) {
  if (s->n == s->cap) {
    s->cap = s->cap ? 2 * s->cap : 1024;
    s->v = (trk_t*)realloc(s->v, s->cap * sizeof(trk_t));
  }
  s->v[s->n++] = *t;
}

typedef struct {
  const or_ctx* c;
  const or_run_opts* o;
  uint32_t event;
  double* edep;  /* this event's bins */
  double leaked, killed;
  uint64_t steps[3], created[3], boundary[3];
  uint64_t* gen_hist; /* shared, atomically updated */
  uint64_t* steplen;  /* shared */
  or_result* res;     /* outgoing-particle list (shared, atomically indexed) */
  int slot;
} ev_t;

/* an outgoing particle: the track as it leaves the calorimeter */
static void record_leak(ev_t* e, const trk_t* t) {
  or_result* r = e->res;
  if (!r->leak_out) return;
  const uint64_t i = __atomic_fetch_add(&r->leak_n, 1, __ATOMIC_RELAXED);
  if (i >= r->leak_cap) return;
  double* o = r->leak_out + 9 * i;
  o[0] = e->slot;
  o[1] = t->species == 0 ? 22 : (t->species == 1 ? 11 : -11);
  o[2] = t->T;
  for (int a = 0; a < 3; ++a) { o[3 + a] = t->x[a]; o[6 + a] = t->u[a]; }
}

static int enabled(const or_run_opts* o, uint32_t bit) {
  return o->process_mask == 0 || (o->process_mask & bit);
}

static void deposit(ev_t* e, int vol, double dE) {
  if (dE == 0.0) return;
  const int b = e->c->vol_bin[vol];
  if (b >= 0) e->edep[b] += dE;
  else e->killed += dE; /* cannot happen: no energy loss in vacuum */
}

static void emit(ev_t* e, stack_t_* st, const trk_t* parent, const ixn_t* r, uint32_t step) {
  for (int k = 0; k < r->n; ++k) {
    const int sp = r->species[k];
    const double T = r->T[k];
    if (sp != 2 && T < e->c->tcut) { deposit(e, parent->vol, T); continue; }
    trk_t t;
    memcpy(t.x, parent->x, sizeof(t.x));
    memcpy(t.u, r->dir[k], sizeof(t.u));
    t.T = T;
    t.id = or_child_id(e->o->seed, e->event, parent->id, step, (uint32_t)k);
    t.step = 0;
    t.vol = parent->vol;
    t.species = sp;
    t.vac = 0;
    t.gen = parent->gen + 1;
    push(st, &t);
    e->created[sp]++;
  }
}

static void record(ev_t* e, const trk_t* t, double s) {
  e->steps[t->species]++;
  if (e->gen_hist && t->gen < e->o->max_gen)
    __atomic_fetch_add(&e->gen_hist[3 * t->gen + t->species], 1, __ATOMIC_RELAXED);
  if (e->steplen && s > 0.0 && s < 1e299) {
    int ex;
    frexp(s, &ex);
    int b = ex - 1 + 40;
    if (b < 0) b = 0;
    if (b > 63) b = 63;
    __atomic_fetch_add(&e->steplen[64 * t->species + b], 1, __ATOMIC_RELAXED);
  }
}

/* One step of one track (paper Sec. 3). Returns 1 while the track is alive. */
static int step_track(ev_t* e, trk_t* t, stack_t_* st) {
  const or_ctx* c = e->c;
  const or_run_opts* o = e->o;
  const int sp = t->species;
  const int q = sp == 1 ? -1 : (sp == 2 ? 1 : 0);
  const double rest = (sp == 2) ? 2.0 * kMe : 0.0;
  const int m = c->vol_mat[t->vol];
  const uint32_t step = t->step;

  /* looper caps: the paper kills and accounts tracks whose field integration does not
   * finish (Sec. 2.3); here a per-track step cap and a consecutive-vacuum-step cap */
  if (step >= o->max_steps) { record(e, t, 0.0); e->killed += t->T + rest; return 0; }
  if (m < 0) {
    if ((uint32_t)t->vac >= o->max_vacuum_steps) { record(e, t, 0.0); e->killed += t->T + rest; return 0; }
    t->vac++;
  } else {
    t->vac = 0;
  }

  stream_t rs;
  stream_init(&rs, o->seed, e->event, t->id, step);

  /* below the tracking cut: deposit; a positron annihilates at rest */
  if (t->T < c->tcut) {
    record(e, t, 0.0);
    deposit(e, t->vol, t->T);
    if (sp == 2) {
      ixn_t r; memset(&r, 0, sizeof(r));
      sample_annih_rest(&rs, &r);
      emit(e, st, t, &r, step);
    }
    return 0;
  }

  double u0, u1;
  stream_block0(&rs, &u0, &u1);

  /* cross sections at the pre-step energy (constant along the step) */
  double sig[3] = {0.0, 0.0, 0.0};
  double R = 0.0;
  int nproc = 0;
  if (m >= 0) {
    if (sp == 0) {
      nproc = 3;
      if (enabled(o, OR_P_COMPT)) sig[0] = interp_nodes(c->gam[m][0], t->T);
      if (enabled(o, OR_P_CONV)) sig[1] = interp_nodes(c->gam[m][1], t->T);
      if (enabled(o, OR_P_PHOTO)) sig[2] = interp_nodes(c->gam[m][2], t->T);
    } else if (sp == 1) {
      nproc = 2;
      R = interp_nodes(c->ele[m][1], t->T);
      if (enabled(o, OR_P_EIONI)) sig[0] = interp_nodes(c->ele[m][2], t->T);
      if (enabled(o, OR_P_EBREM)) sig[1] = interp_nodes(c->ele[m][3], t->T);
    } else {
      nproc = 3;
      R = interp_nodes(c->pos[m][1], t->T);
      if (enabled(o, OR_P_PIONI)) sig[0] = interp_nodes(c->pos[m][2], t->T);
      if (enabled(o, OR_P_PBREM)) sig[1] = interp_nodes(c->pos[m][3], t->T);
      if (enabled(o, OR_P_ANNIH)) sig[2] = interp_nodes(c->pos[m][4], t->T);
    }
  }
  for (int i = 0; i < 3; ++i) if (sig[i] < 0.0) sig[i] = 0.0;
  const double stot = sig[0] + sig[1] + sig[2];
  const double s_int = stot > 0.0 ? -log(u0) / stot : kInf;
  double s_phys = s_int;
  int limited = 0; /* the step limit, not the sampled interaction length, ends the step */
  const int msc = (o->physics & OR_PHYS_MSC) != 0, fluct = (o->physics & OR_PHYS_FLUCT) != 0;
  if (q != 0 && m >= 0) {
    double smax = (R <= kRhoF) ? R : ((kAlphaR * R > kRhoF) ? kAlphaR * R : kRhoF);
    if (msc) {  /* multiple-scattering step limit */
      const double f = o->msc_range_factor > 0.0 ? o->msc_range_factor : 0.04;
      const double sm = (f * R > 0.01) ? f * R : 0.01;
      if (sm < smax) smax = sm;
    }
    if (smax < s_phys) { s_phys = smax; limited = 1; }
  }

  int next;
  const int field = (q != 0 && c->field_T != 0.0);
  int boundary;
  double s;
  if (field && o->field_max_iter > 0) {
    /* chord propagation (paper Sec. 2.3): a step whose integration does not finish within
     * the iteration cap is killed and its energy accounted */
    double sd;
    int iters;
    const int rc = or_chord_step(c, t->T, q, s_phys, o->field_max_iter,
                                 o->delta_chord > 0.0 ? o->delta_chord : 0.25,
                                 o->delta_int > 0.0 ? o->delta_int : 0.001, t->x, t->u, t->vol, &next, &sd,
                                 &iters);
    if (rc == 2) { record(e, t, 0.0); e->killed += t->T + rest; return 0; }
    boundary = (rc == 1);
    s = sd;
    record(e, t, s);
  } else {
    const double s_geom = field ? or_helix_distance(c, t->T, q, t->x, t->u, t->vol, &next)
                                : or_distance(c, t->x, t->u, t->vol, &next);
    boundary = (s_geom <= s_phys);
    s = boundary ? s_geom : s_phys;
    record(e, t, s);
    /* move */
    if (field) {
      or_helix_move(c->field_T, t->T, q, s, t->x, t->u);
    } else {
      t->x[0] += s * t->u[0]; t->x[1] += s * t->u[1]; t->x[2] += s * t->u[2];
    }
  }
  if (boundary && c->kind == 0 && next >= 0) {
    /* a crossing into another slab is through a z plane: land exactly on it */
    t->x[2] = c->bnd[t->u[2] > 0.0 ? t->vol + 1 : t->vol];
  }
  t->step = step + 1;

  /* continuous energy loss through the range table; with fluctuations, a Gaussian loss
   * about that mean for a track that survives the mean loss */
  const double Tpre = t->T;
  if (q != 0 && m >= 0) {
    const double* Rt = (sp == 1) ? c->ele[m][1] : c->pos[m][1];
    double Epost = 0.0;
    if (s < R) Epost = inverse_range_nodes(Rt, R - s);
    if (Epost > t->T) Epost = t->T;
    if (fluct && s < R && Epost >= c->tcut)
      Epost = t->T - fluct_loss(&rs, t->T - Epost, sqrt(or_fluct_sigma2(c, m, t->T, s, sp == 2)));
    deposit(e, t->vol, t->T - Epost);
    t->T = Epost;
    if (t->T < c->tcut) {
      deposit(e, t->vol, t->T);
      t->T = 0.0;
      if (sp == 2) {
        ixn_t r; memset(&r, 0, sizeof(r));
        sample_annih_rest(&rs, &r);
        emit(e, st, t, &r, step);
      }
      return 0;
    }
    /* multiple scattering: the direction at the end of the step */
    if (msc && s > 0.0) msc_deflect(&rs, or_msc_theta0(c, m, Tpre, s), t->u);
  }

  if (boundary) {
    if (next < 0) { e->leaked += t->T + rest; record_leak(e, t); return 0; }
    t->vol = next;
    e->boundary[sp]++;
    return 1;
  }
  /* a step cut short by the step limit ends with its continuous loss only */
  if (limited) return 1;

  /* discrete interaction: process chosen by u1 over the fixed order */
  const double x = u1 * stot;
  int proc = nproc - 1;
  double acc = 0.0;
  for (int i = 0; i < nproc; ++i) {
    acc += sig[i];
    if (x < acc) { proc = i; break; }
  }
  ixn_t r;
  memset(&r, 0, sizeof(r));
  if (sp == 0) {
    if (proc == 0) sample_compton(&rs, t->T, t->u, &r);
    else if (proc == 1) sample_pair(&rs, t->T, t->u, &r);
    else sample_photo(t->T, t->u, &r);
  } else if (sp == 1) {
    if (proc == 0) sample_moller(&rs, t->T, c->Tc[m], t->u, &r);
    else sample_brem(&rs, t->T, c->kc[m], t->u, &r);
  } else {
    if (proc == 0) sample_bhabha(&rs, t->T, c->Tc[m], t->u, &r);
    else if (proc == 1) sample_brem(&rs, t->T, c->kc[m], t->u, &r);
    else sample_annih(&rs, t->T, t->u, &r);
  }
  if (!r.happened) return 1;
  emit(e, st, t, &r, step);
  if (!r.parent_alive) return 0;
  t->T = r.parent_T;
  memcpy(t->u, r.parent_dir, sizeof(t->u));
  if (sp == 0 && t->T < c->tcut) { deposit(e, t->vol, t->T); return 0; }
  return 1;
}

typedef struct {
  const or_ctx* c;
  const or_run_opts* o;
  int n, n_events;
  const int* pdg;
  const double *E, *pos, *dir;
  const uint32_t* key;
  const int* slot;
  int* order;      /* track indices grouped by event */
  int* ev_begin;   /* [n_events + 1] */
  or_result* r;
  int next_event;
  pthread_mutex_t mu;
} job_t;

static void run_event(job_t* j, int ev, stack_t_* st) {
  const or_ctx* c = j->c;
  ev_t e;
  memset(&e, 0, sizeof(e));
  e.c = c;
  e.o = j->o;
  e.edep = j->r->edep + (size_t)ev * c->n_bins;
  e.gen_hist = j->r->gen_hist;
  e.steplen = j->r->steplen_hist;
  e.res = j->r;
  e.slot = ev; /* tracks are grouped by event slot */
  st->n = 0;
  for (int k = j->ev_begin[ev + 1] - 1; k >= j->ev_begin[ev]; --k) {
    const int i = j->order[k];
    trk_t t;
    memset(&t, 0, sizeof(t));
    for (int a = 0; a < 3; ++a) { t.x[a] = j->pos[3 * i + a]; t.u[a] = j->dir[3 * i + a]; }
    t.T = j->E[i];
    t.species = j->pdg[i] == 22 ? 0 : (j->pdg[i] == 11 ? 1 : 2);
    t.id = (uint64_t)(k - j->ev_begin[ev] + 1);
    e.event = j->key[i];
    t.vol = or_locate(c, t.x, t.u);
    if (t.vol < 0) { e.leaked += t.T + (t.species == 2 ? 2.0 * kMe : 0.0); record_leak(&e, &t); continue; }
    push(st, &t);
  }
  while (st->n > 0) {
    trk_t t = st->v[--st->n];
    while (step_track(&e, &t, st)) t.gen++;
  }
  j->r->leaked[ev] = e.leaked;
  j->r->killed[ev] = e.killed;
  pthread_mutex_lock(&j->mu);
  for (int s = 0; s < 3; ++s) {
    j->r->steps[s] += e.steps[s];
    j->r->created[s] += e.created[s];
    j->r->boundary_steps[s] += e.boundary[s];
  }
  pthread_mutex_unlock(&j->mu);
}

static void* worker(void* arg) {
  job_t* j = (job_t*)arg;
  stack_t_ st = {NULL, 0, 0};
  for (;;) {
    const int ev = __atomic_fetch_add(&j->next_event, 1, __ATOMIC_RELAXED);
    if (ev >= j->n_events) break;
    run_event(j, ev, &st);
  }
  free(st.v);
  return NULL;
}

int or_transport(const or_ctx* c, int n, const int* pdg, const double* E, const double* pos,
                 const double* dir, const uint32_t* event_key, const int* event_slot, int n_events,
                 const or_run_opts* o, or_result* r) {
  if (n < 0 || n_events < 0) return -1;
  for (int i = 0; i < n; ++i)
    if (event_slot[i] < 0 || event_slot[i] >= n_events) return -1;
  job_t j;
  memset(&j, 0, sizeof(j));
  j.c = c; j.o = o; j.n = n; j.n_events = n_events;
  j.pdg = pdg; j.E = E; j.pos = pos; j.dir = dir; j.key = event_key; j.slot = event_slot;
  j.r = r;
  j.order = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  j.ev_begin = (int*)calloc((size_t)n_events + 1, sizeof(int));
  for (int i = 0; i < n; ++i) j.ev_begin[event_slot[i] + 1]++;
  for (int ev = 0; ev < n_events; ++ev) j.ev_begin[ev + 1] += j.ev_begin[ev];
  int* fill = (int*)calloc((size_t)n_events + 1, sizeof(int));
  for (int i = 0; i < n; ++i) {
    const int ev = event_slot[i];
    j.order[j.ev_begin[ev] + fill[ev]++] = i;
  }
  free(fill);
  memset(r->edep, 0, sizeof(double) * (size_t)n_events * c->n_bins);
  for (int s = 0; s < 3; ++s) { r->steps[s] = 0; r->created[s] = 0; r->boundary_steps[s] = 0; }
  pthread_mutex_init(&j.mu, NULL);
  int nt = o->n_threads > 0 ? o->n_threads : 1;
  if (nt > 256) nt = 256;
  pthread_t th[256];
  for (int k = 0; k < nt; ++k) pthread_create(&th[k], NULL, worker, &j);
  for (int k = 0; k < nt; ++k) pthread_join(th[k], NULL);
  pthread_mutex_destroy(&j.mu);
  free(j.order);
  free(j.ev_begin);
  return 0;
}
