/*
 * FP64 CPU oracle for electromagnetic shower transport (AdePT, arXiv 2209.15445).
 *
 * TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library. The product
 * path (the CUDA library and its Python binding) never links, imports or calls it,
 * and the two share no source, header, table or constant generator.
 *
 * What it computes: the per-step transport of e-, e+ and gamma tracks through a
 * layered calorimeter (paper Sec. 3, "Stepping workflow"), one event at a time,
 * with a LIFO stack of tracks, in plain double precision. The physics models are
 * the textbook forms that the paper leaves unstated (it only names G4HepEm, Sec. 2.2):
 *   Klein-Nishina Compton, Bethe-Heitler pair (complete screening), Born K-shell
 *   photoabsorption, Moller/Bhabha ionisation above a production cut, Tsai
 *   complete-screening bremsstrahlung, Heitler two-photon annihilation,
 *   Berger-Seltzer restricted collision stopping power with the Sternheimer-Peierls
 *   density effect, and a piecewise linear-in-ln(E) range table.
 * The random numbers come from Philox4x32-10 (Salmon et al., SC'11), keyed by
 * (seed, event) with counter (track id lo, track id hi, step, block); the paper
 * uses RANLUX++ (Sec. 2.2) and this build fixes a counter-based generator instead.
 *
 * Every function below is pinned by a CPU test in tests/test_oracle_*.py, with one
 * exception: the overall constant of the photoabsorption cross section (or_mu_photo) is
 * parity unpinned -- its Z^5 and E^-3.5 dependence and its order of magnitude are pinned,
 * but no published value of this Born K-shell form is available to fix the prefactor.
 */
#ifndef ORACLE_H
#define ORACLE_H
#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OR_NNODE 289          /* 1 keV .. 1 TeV, 32 bins per decade */
#define OR_MAX_MAT 8
#define OR_MAX_ELEM 8         /* elements of a compound */
#define OR_MAX_VOL 512

/* process bits for the single-interaction tests (0 = all enabled) */
#define OR_P_COMPT   (1u << 0)
#define OR_P_CONV    (1u << 1)
#define OR_P_PHOTO   (1u << 2)
#define OR_P_EIONI   (1u << 3)
#define OR_P_EBREM   (1u << 4)
#define OR_P_PIONI   (1u << 5)
#define OR_P_PBREM   (1u << 6)
#define OR_P_ANNIH   (1u << 7)

typedef struct or_ctx or_ctx;

/* ---- Philox4x32-10 and the uniform maps ---- */
void or_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double or_u01_f64(uint32_t w0, uint32_t w1);
float or_u01_f32(uint32_t w);
uint64_t or_child_id(uint32_t seed, uint32_t event, uint64_t parent_id, uint32_t parent_step, uint32_t k);

/* ---- setup: materials, geometry, cuts, tables ---- */
/* mat_* arrays have n_mat entries; Z = 0 (and no elements) marks vacuum. A compound is given
 * by mat_n_elem[m] > 0 elements, taken in order from elem_Z / elem_A / elem_atoms (atoms per
 * formula unit); its own mat_Z and mat_A are then ignored. mat_n_elem = NULL: all elements. 
 * geometry: kind 0 = slab stack along z starting at z = 0, |x|,|y| <= half_xy;
 *           kind 1 = concentric tubes around z, |z| <= half_z, layer_r[n_layers] inner radii.
 * sub_mat/sub_thick: the sublayers of one layer (same for every layer). */
or_ctx* or_create(int n_mat, const int* mat_Z, const double* mat_A, const double* mat_rho,
                  const double* mat_I_eV, const int* mat_n_elem, const int* elem_Z, const double* elem_A,
                  const double* elem_atoms, int kind, int n_layers, int n_sub, const int* sub_mat,
                  const double* sub_thick, double half_xy, double half_z, const double* layer_r,
                  double range_cut_mm, double field_T, double tracking_cut_MeV);
void or_destroy(or_ctx* c);

/* closed forms (per material index) */
double or_mu_compton(const or_ctx* c, int m, double E);
double or_mu_pair(const or_ctx* c, int m, double E);
double or_mu_photo(const or_ctx* c, int m, double E);
double or_inv_X0(const or_ctx* c, int m);
double or_dedx_col(const or_ctx* c, int m, double T, double cut, int positron);
double or_dedx_rad(const or_ctx* c, int m, double T, double kcut);
double or_density_delta(const or_ctx* c, int m, double T);
double or_lambda_ioni(const or_ctx* c, int m, double T, double cut, int positron);
double or_lambda_brem(const or_ctx* c, int m, double T, double kcut);
double or_lambda_annih(const or_ctx* c, int m, double T);
double or_sigma_kn(double kappa);       /* per electron, mm^2 */
double or_sigma_kn_direct(double kappa);/* the unexpanded closed form, for the series pin */

/* cuts and tables */
void or_cuts(const or_ctx* c, int m, double* Tc, double* kc);
/* species 0 gamma (tables: compton, pair, photo), 1 e- (dedx, range, ioni, brem),
 * 2 e+ (dedx, range, ioni, brem, annih), 3 = unrestricted e- range (1 table) */
int or_table(const or_ctx* c, int species, int table, int m, double* out /* OR_NNODE */);
double or_interp(const or_ctx* c, int species, int table, int m, double E);
double or_inverse_range(const or_ctx* c, int species, int m, double R);
double or_node_energy(int i);

/* ---- samplers (for the KS pins): n draws, stream i keyed (seed, event) counter (i+1, 0, step, .) ----
 * out layout per draw, see oracle.c */
void or_sample(const or_ctx* c, int which, int m, double E, uint32_t seed, uint32_t event, int n,
               double* out);

/* ---- optional continuous physics (off unless or_run_opts.physics sets it) ----
 * OR_PHYS_MSC: multiple Coulomb scattering of e+-, a Gaussian (Highland) deflection at the
 *   end of every charged step, with the step limit s <= max(f R, 0.01 mm);
 * OR_PHYS_FLUCT: Gaussian (Bohr) fluctuations of the restricted continuous loss. */
#define OR_PHYS_MSC   (1u << 0)
#define OR_PHYS_FLUCT (1u << 1)
#define OR_MSC_BLOCK   0x40000000u /* Philox counter block of the deflection */
#define OR_FLUCT_BLOCK 0x40000001u /* first block of the fluctuation draws */
/* Highland's theta0 [rad] of an e+- of kinetic energy T over path s in material m */
double or_msc_theta0(const or_ctx* c, int m, double T, double s);
/* Bohr variance [MeV^2] of the restricted loss of an e- (positron = 0) or e+ over s */
double or_fluct_sigma2(const or_ctx* c, int m, double T, double s, int positron);
/* n draws, draw i from the stream keyed (seed, event), counter (i+1, 0, 0, .):
 * which 0: deflected direction of (0,0,1) after a step s at energy T (out: 3 per draw);
 * which 1: sampled loss of a step s at energy T, species 1 (e-) or 2 (e+) (out: 2 per draw:
 *          the loss, and the mean loss it fluctuates about) */
void or_sample_continuous(const or_ctx* c, int which, int species, int m, double T, double s,
                          uint32_t seed, uint32_t event, int n, double* out);

/* ---- geometry ---- */
int or_n_volumes(const or_ctx* c);
int or_locate(const or_ctx* c, const double pos[3], const double dir[3]);
/* distance to the next boundary along a straight line; next volume in *next (-1 = leaves world) */
double or_distance(const or_ctx* c, const double pos[3], const double dir[3], int vol, int* next);
/* helix: charged track of kinetic energy T and charge q in the uniform field along z.
 * propagate by path length s: pos/dir updated in place. */
void or_helix_move(double field_T, double T, int charge, double s, double pos[3], double dir[3]);
double or_helix_distance(const or_ctx* c, double T, int charge, const double pos[3],
                         const double dir[3], int vol, int* next);

/* chord propagation in the field (paper Sec. 2.3): the path of a charged track is
 * followed in linear segments whose sagitta is at most delta_chord; a segment that meets
 * the boundary of the volume is refined until the crossing is within delta_int of the
 * curve. Each segment and each refinement is one iteration; a step needing more than
 * max_iter does not finish. Starting at p/u in volume vol with a physics step s_phys:
 * returns 0 (reached s_phys), 1 (crossed into *next, -1 = left the world) or 2 (cap hit,
 * p/u unchanged); *s_done = path length, *iters = iterations used. */
int or_chord_step(const or_ctx* c, double T, int q, double s_phys, int max_iter, double delta_chord,
                  double delta_int, double p[3], double u[3], int vol, int* next, double* s_done,
                  int* iters);

/* ---- ray tracing of the geometry (paper Sec. 2.1: navigation validated on ray-traced
 * images, GPU against CPU and single against double precision) ----
 * Orthographic camera cam = {origin[3], view direction[3], up[3], width, height} (mm): the
 * ray of pixel (i, j) starts at origin + ((i+0.5)/nx - 0.5) width right + ((j+0.5)/ny - 0.5)
 * height up', right = dir x up / |.|, up' = right x dir, and runs along dir. It enters the
 * world (box or cylinder) analytically, snapped onto the face it enters, and then crosses
 * volume after volume with or_distance. out[2 (j nx + i) + {0, 1}] = the mass thickness it
 * traverses (g/cm^2) and the number of volumes it enters (0: it misses the world). */
void or_raytrace(const or_ctx* c, const double cam[11], int nx, int ny, double* out);

/* ---- transport ---- */
typedef struct {
  uint32_t seed;
  uint32_t process_mask;     /* 0 = all processes */
  uint32_t max_steps;        /* per track */
  uint32_t max_vacuum_steps; /* consecutive steps in vacuum */
  int n_threads;
  int max_gen;               /* size of the gen_hist rows (0 = none) */
  uint32_t physics;          /* OR_PHYS_* bits (0 = the paper's list only) */
  double msc_range_factor;   /* f of the MSC step limit (0 = 0.04) */
  int field_max_iter;        /* 0: analytic helix; N > 0: chord propagation, at most N iterations */
  double delta_chord;        /* chord sagitta limit [mm] (0 = 0.25) */
  double delta_int;          /* intersection accuracy [mm] (0 = 0.001) */
} or_run_opts;

typedef struct {
  double* edep;        /* [n_events][n_bins] */
  double* leaked;      /* [n_events] */
  double* killed;      /* [n_events] */
  uint64_t steps[3];   /* gamma, e-, e+ */
  uint64_t created[3]; /* secondaries pushed per species */
  uint64_t* gen_hist;  /* [max_gen][3] steps per generation and species, or NULL */
  uint64_t* steplen_hist; /* [3][64] log2 bins of step length in um, or NULL */
  /* outgoing particles (tracks that leave the calorimeter, primaries submitted outside it):
   * 9 doubles each (event slot, pdg, kinetic energy, position[3], direction[3]) at the point
   * where they leave; up to leak_cap records, leak_n counts all (NULL: not recorded) */
  double* leak_out;
  uint64_t leak_cap;
  uint64_t leak_n;
  uint64_t boundary_steps[3]; /* steps that ended on a boundary inside the world */
} or_result;

/* tracks: pdg (22, 11, -11), kinetic energy, position, direction, RNG event key, event slot */
int or_transport(const or_ctx* c, int n, const int* pdg, const double* E, const double* pos,
                 const double* dir, const uint32_t* event_key, const int* event_slot, int n_events,
                 const or_run_opts* o, or_result* r);
int or_n_bins(const or_ctx* c);

#ifdef __cplusplus
}
#endif
#endif
