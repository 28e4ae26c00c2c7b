// Double-precision closed forms used to build the physics tables on the device at
// initialisation (the paper keeps G4HepEm's initialisation separate from its run-time
// functions and uploads the tables to the GPU, Sec. 2.2; here the tables are built
// directly on the GPU). The models are the textbook forms named with each function.
#pragma once
#include "device.cuh"

namespace adept {
namespace init {

// Klein-Nishina total cross section per electron [mm^2], 2 pi re^2 b(k). The closed form
// of b cancels terms of size 1/k^2 down to O(1) (relative error about 1e-16/k^2 in FP64),
// so below k = 0.2 b is taken from its Taylor series in x = 2k instead: term by term from
// the expansions of ln(1+x), 1/(1+x) and 1/(1+x)^2, b = sum_n (-x)^n d_n with
// d_n = 4(n+1)/(n+3) + 1/(n+1) - 2n/(n+2) + n/2 - 1 (d_0 = 4/3, Thomson), 60 terms.
__device__ inline double kn_series_term(int n) {
  const double dn = (double)n;
  return 4.0 * (dn + 1.0) / (dn + 3.0) + 1.0 / (dn + 1.0) - 2.0 * dn / (dn + 2.0) + 0.5 * dn - 1.0;
}
__device__ inline double sigma_kn(double k) {
  double b;
  if (k >= 0.2) {
    const double l = log1p(2.0 * k);
    const double a = 1.0 + 2.0 * k;
    b = (1.0 + k) / (k * k) * (2.0 * (1.0 + k) / a - l / k) + l / (2.0 * k) - (1.0 + 3.0 * k) / (a * a);
  } else {
    const double mx = -2.0 * k;
    b = kn_series_term(59);
    for (int n = 58; n >= 0; --n) b = fma(b, mx, kn_series_term(n));
  }
  return 2.0 * kPi * kRe * kRe * b;
}

// Tsai radiation length per atom (PDG): Lrad = ln(184.15 Z^-1/3), L'rad = ln(1194 Z^-2/3),
// Coulomb correction f(Z) of Davies, Bethe and Maximon; 1/X0 = n_at x this
__device__ inline double inv_x0_per_atom(double Z) {
  const double lz = log(Z);
  const double a2 = (kAlpha * Z) * (kAlpha * Z);
  const double f = a2 * (1.0 / (1.0 + a2) + 0.20206 - 0.0369 * a2 + 0.0083 * a2 * a2 - 0.002 * a2 * a2 * a2);
  return 4.0 * kAlpha * kRe * kRe * (Z * Z * ((log(184.15) - lz / 3.0) - f) + Z * (log(1194.0) - 2.0 * lz / 3.0));
}

// in: a kMatRec material record. An element (n_elem = 0) is one atom kind; a compound
// lists its elements with their atoms per formula unit, and its atom densities follow from
// the formula's mass fractions.
__device__ inline void setup_material(const double* in, MatDev* m) {
  m->Z = in[0]; m->A = in[1]; m->rho = in[2]; m->I = in[3];
  const int ne = (int)in[4];
  m->vacuum = !(m->Z > 0.0) && ne == 0;
  m->n_elem = 0;
  if (m->vacuum) return;
  if (ne > 0) {
    double M = 0.0, natoms = 0.0, zsum = 0.0;
    for (int i = 0; i < ne; ++i) {
      M += in[5 + 3 * i + 2] * in[5 + 3 * i + 1];
      natoms += in[5 + 3 * i + 2];
      zsum += in[5 + 3 * i + 2] * in[5 + 3 * i];
    }
    m->n_elem = ne;
    m->ZoA = 0.0; m->n_at = 0.0; m->n_el = 0.0;
    for (int i = 0; i < ne; ++i) {
      const double Zi = in[5 + 3 * i], Ai = in[5 + 3 * i + 1];
      const double w = in[5 + 3 * i + 2] * Ai / M;
      m->eZ[i] = Zi;
      m->en_at[i] = kNA * m->rho * w / Ai * 1e-3;
      m->ZoA += w * Zi / Ai;
      m->n_at += m->en_at[i];
      m->n_el += Zi * m->en_at[i];
    }
    m->A = M / natoms;
    m->Z = zsum / natoms;
  } else {
    m->n_at = kNA * m->rho / m->A * 1e-3;
    m->n_el = m->Z * m->n_at;
    m->n_elem = 1;
    m->eZ[0] = m->Z;
    m->en_at[0] = m->n_at;
    m->ZoA = m->Z / m->A;
  }
  // a compound adds its elements' terms by atom density (Bragg additivity of 1/X0)
  m->inv_x0 = 0.0;
  for (int i = 0; i < m->n_elem; ++i) m->inv_x0 += m->en_at[i] * inv_x0_per_atom(m->eZ[i]);
  // Sternheimer-Peierls general density-effect parameters for condensed media
  const double hwp = 28.816 * sqrt(m->rho * m->ZoA);
  m->cbar = 2.0 * log(m->I / hwp) + 1.0;
  if (m->I < 100.0) {
    m->x1 = 2.0;
    m->x0 = m->cbar < 3.681 ? 0.2 : 0.326 * m->cbar - 1.0;
  } else {
    m->x1 = 3.0;
    m->x0 = m->cbar < 5.215 ? 0.2 : 0.326 * m->cbar - 1.5;
  }
  const double d = m->x1 - m->x0;
  m->a_d = (m->cbar - 2.0 * log(10.0) * m->x0) / (d * d * d);
}

__device__ inline double mu_compton(const MatDev& m, double E) { return m.n_el * sigma_kn(E / kMe); }

// Bethe-Heitler in complete screening over the kinematic range of the positron fraction:
// (w/X0)(7 - 4a(1-a))/9 with a = m/E, w = 1 - 2a
__device__ inline double mu_pair(const MatDev& m, double E) {
  if (!(E > 2.0 * kMe)) return 0.0;
  const double a = kMe / E;
  return m.inv_x0 * ((E - 2.0 * kMe) / E) * (7.0 - 4.0 * a * (1.0 - a)) / 9.0;
}

// Born-approximation K-shell photoabsorption: 4 sqrt(2) alpha^4 Z^5 sigma_Th (m/E)^3.5
// (a compound: the sum over its atoms)
__device__ inline double mu_photo(const MatDev& m, double E) {
  const double q = kMe / E;
  const double a2 = kAlpha * kAlpha;
  double s = 0.0;
  for (int i = 0; i < m.n_elem; ++i) {
    const double Z = m.eZ[i], z2 = Z * Z;
    s += m.en_at[i] * 4.0 * sqrt(2.0) * (a2 * a2) * (z2 * z2 * Z) * (8.0 * kPi / 3.0 * kRe * kRe) *
         (q * q * q * sqrt(q));
  }
  return s;
}

__device__ inline double density_delta(const MatDev& m, double T) {
  const double tau = T / kMe;
  const double x = 0.5 * log(tau * (tau + 2.0)) / log(10.0);
  if (x < m.x0) return 0.0;
  const double lin = 2.0 * log(10.0) * x - m.cbar;
  if (x >= m.x1) return lin;
  const double r = m.x1 - x;
  return lin + m.a_d * r * r * r;
}

// Berger-Seltzer restricted collision stopping power (ICRU 37), electrons (Moller,
// D = min(cut, T/2)) or positrons (Bhabha, D = min(cut, T)), with the density effect
__device__ inline double dedx_col(const MatDev& m, double T, double cut, bool positron) {
  const double tau = T / kMe, g = tau + 1.0;
  const double b2 = tau * (tau + 2.0) / (g * g);
  const double Im = m.I * 1e-6 / kMe;
  double D = positron ? T : 0.5 * T;
  D = (cut < D ? cut : D) / kMe;
  double F;
  if (!positron) {
    F = -1.0 - b2 + log((tau - D) * D) + tau / (tau - D) +
        (0.5 * D * D + (2.0 * tau + 1.0) * log1p(-D / tau)) / (g * g);
  } else {
    const double y = 1.0 / (g + 1.0);
    const double D2 = D * D, D3 = D2 * D;
    F = log(tau * D) - (b2 / tau) * (tau + 2.0 * D - 1.5 * D2 * y - (D - D3 / 3.0) * y * y -
                                     (0.5 * D2 - tau * D3 / 3.0 + 0.25 * D3 * D) * y * y * y);
  }
  double br = log(2.0 * (tau + 2.0) / (Im * Im)) + F - density_delta(m, T);
  br = br < 0.0 ? 0.0 : br;
  return 2.0 * kPi * kRe * kRe * kMe * m.n_el / b2 * br;
}

// Tsai radiative loss to photons below min(kc, T)
__device__ inline double dedx_rad(const MatDev& m, double T, double kc) {
  const double k = kc < T ? kc : T;
  const double E = T + kMe;
  return m.inv_x0 * (4.0 / 3.0 * k - 2.0 / 3.0 * k * k / E + k * k * k / (3.0 * E * E));
}

// Moller / Bhabha delta-ray cross sections above the cut, integrated in closed form
__device__ inline double lambda_ioni(const MatDev& m, double T, double cut, bool positron) {
  const double tau = T / kMe, g = tau + 1.0;
  const double b2 = tau * (tau + 2.0) / (g * g);
  const double ec = cut / T;
  const double pref = m.n_el * 2.0 * kPi * kRe * kRe * kMe / T;
  if (!positron) {
    if (!(T > 2.0 * cut)) return 0.0;
    const double w = (T - 2.0 * cut) / T;
    const double gg = (2.0 * g - 1.0) / (g * g);
    return pref / b2 * ((1.0 - gg) * 0.5 * w + w / (ec * (1.0 - ec)) - gg * log1p(w / ec));
  }
  if (!(T > cut)) return 0.0;
  const double v = (T - cut) / T;
  const double y = 1.0 / (g + 1.0), y12 = 1.0 - 2.0 * y;
  const double B1 = 2.0 - y * y, B2 = y12 * (3.0 + y * y), B4 = y12 * y12 * y12, B3 = B4 + y12 * y12;
  return pref * (v / (b2 * ec) - B1 * log1p(v / ec) + B2 * v - 0.5 * B3 * v * (1.0 + ec) +
                 B4 / 3.0 * v * (1.0 + ec + ec * ec));
}

// Tsai bremsstrahlung above kc
__device__ inline double lambda_brem(const MatDev& m, double T, double kc) {
  if (!(T > kc)) return 0.0;
  const double E = T + kMe, d = T - kc;
  return m.inv_x0 * (4.0 / 3.0 * log1p(d / kc) - 4.0 / 3.0 * d / E + d * (T + kc) / (2.0 * E * E));
}

// Heitler two-photon annihilation in flight, per electron times n_el
__device__ inline double lambda_annih(const MatDev& m, double T) {
  const double tau = T / kMe, g = tau + 1.0;
  const double s2 = tau * (tau + 2.0), s = sqrt(s2);
  return m.n_el * kPi * kRe * kRe / (g + 1.0) *
         ((g * g + 4.0 * g + 1.0) / s2 * log1p(tau + s) - (g + 3.0) / s);
}

// ---------------------------------------------------------------- range and thresholds
// Shared by the arena build (kernels.cu) and the allocation-free build (noalloc.cu), so
// that both builds follow one set of rules.

// energy of grid node i
__device__ inline double node_E(int i) { return exp(kLnEmin + (double)i * kDlog); }

// Simpson rule with 8 panels of T/S(T) over bin i in ln T: the range gained across bin i
template <class F>
__device__ inline double bin_integral(int i, F S) {
  const double h = kDlog / 8.0;
  double acc = 0.0;
  for (int j = 0; j <= 8; ++j) {
    const double T = exp(kLnEmin + (double)i * kDlog + (double)j * h);
    const double w = (j == 0 || j == 8) ? 1.0 : ((j & 1) ? 4.0 : 2.0);
    acc += w * (T / S(T));
  }
  return acc * h / 3.0;
}

// range of a stopping-power row: R(E0) = E0/(2 S(E0)) (S taken as 1/T below the grid),
// then the running sum of the bin integrals
__device__ inline void prefix_range(const double* S, const double* bins, double* R) {
  double r = node_E(0) / (2.0 * S[0]);
  R[0] = r;
  for (int i = 0; i < kNNode - 1; ++i) {
    r += bins[i];
    R[i + 1] = r;
  }
}

// production thresholds are clamped to [0.99 keV, 10 GeV]
__device__ inline double clamp_cut(double x) { return x < 0.99e-3 ? 0.99e-3 : (x > 1e4 ? 1e4 : x); }

// e+- threshold: the energy whose unrestricted range R (node values, rising) equals the
// range cut, by exact inversion of the range interpolated linearly in ln E
__device__ inline double range_threshold(const double* R, double range_cut) {
  if (range_cut <= R[0]) return node_E(0);
  for (int i = 0; i < kNNode - 1; ++i)
    if (R[i + 1] >= range_cut) {
      const double t = (range_cut - R[i]) / (R[i + 1] - R[i]);
      return exp(kLnEmin + ((double)i + t) * kDlog);
    }
  return 1e6;
}

// gamma threshold: five mean free paths equal the range cut, on the falling low-energy
// branch of the total attenuation mu(i) (node values)
template <class F>
__device__ inline double gamma_threshold(F mu, double range_cut) {
  const double target = 5.0 / range_cut;
  if (mu(0) <= target) return node_E(0);
  for (int i = 0; i < kNNode - 1; ++i)
    if (mu(i + 1) <= target) {
      const double a = mu(i), b = mu(i + 1);
      return exp(kLnEmin + ((double)i + (a - target) / (a - b)) * kDlog);
    }
  return 1e6;
}

}  // namespace init
}  // namespace adept
