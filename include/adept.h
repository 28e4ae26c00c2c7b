/*
 * adept.h -- C ABI of the GB300 electromagnetic shower transport library (libadept.so).
 *
 * The library transports electrons, positrons and photons through a layered
 * calorimeter on one GPU and returns the energy they deposit per layer and material.
 * It follows the problem statement of AdePT (arXiv 2209.15445): particles are taken in,
 * buffered until a flush, transported on the GPU, and energy deposits come back to the
 * host per event (Sec. 4, "Geant4 integration"); transport advances the whole track
 * population one step at a time from per-species queues (Sec. 3, "Stepping workflow").
 *
 * Conventions for every entry point:
 *  - Return value: ADEPT_OK (0) or a negative ADEPT_E* code. No C++ exception crosses
 *    the ABI. adept_last_error() gives a per-context message for the last failure.
 *  - Units: MeV, mm, tesla.
 *  - Pointers named host_* or documented as host memory are ordinary CPU memory owned
 *    by the caller and only read (or written) during the call. dev_arena is device
 *    memory owned by the caller (e.g. a torch CUDA tensor); its contents belong to the
 *    library from adept_init until adept_destroy.
 *  - stream is a cudaStream_t passed as void* (e.g. torch.cuda.Stream.cuda_stream);
 *    all device work of the context is ordered on it.
 *  - Threading: adept_submit, adept_submit_device, adept_poll, adept_wait,
 *    adept_get_leaked and adept_get_scoring are thread-safe; adept_transport must be
 *    called from one thread at a time per context.
 */
#ifndef ADEPT_H
#define ADEPT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define ADEPT_OK 0
#define ADEPT_EINVAL (-1)   /* invalid argument (null pointer, bad size, bad geometry) */
#define ADEPT_ENOMEM (-2)   /* arena too small, or the track queues or the outgoing-particle
                                ring overflowed during transport */
#define ADEPT_ESTATE (-3)   /* call out of order (e.g. transport before adept_build_tables) */
#define ADEPT_ECUDA (-4)    /* a CUDA runtime call failed; see adept_last_error */
#define ADEPT_ETIMEOUT (-5) /* adept_transport hit its time budget with work left */
#define ADEPT_EBUSY (-6)    /* the request exists but has not finished */
#define ADEPT_ENOTFOUND (-7)/* unknown request id (or its results were already taken) */

/* ---- particle codes (PDG) ---- */
#define ADEPT_GAMMA 22
#define ADEPT_ELECTRON 11
#define ADEPT_POSITRON (-11)

/* ---- process bits for adept_options.process_mask (0 = all processes on) ---- */
#define ADEPT_P_COMPTON (1u << 0)
#define ADEPT_P_CONVERSION (1u << 1)
#define ADEPT_P_PHOTOELECTRIC (1u << 2)
#define ADEPT_P_E_IONI (1u << 3)
#define ADEPT_P_E_BREM (1u << 4)
#define ADEPT_P_POS_IONI (1u << 5)
#define ADEPT_P_POS_BREM (1u << 6)
#define ADEPT_P_ANNIHILATION (1u << 7)

/* Optional continuous physics (adept_options.physics). The paper's process list has
 * neither; both are off by default.
 *  ADEPT_PHYS_MSC: multiple Coulomb scattering of e+-: at the end of every charged step in
 *    matter the direction turns by a space angle theta0 sqrt(-2 ln u) (two Gaussian
 *    projected angles of Highland's width theta0 at the pre-step energy, PDG), at most pi,
 *    with uniform azimuth; charged steps are limited to max(f R, 0.01 mm), f =
 *    msc_range_factor.
 *  ADEPT_PHYS_FLUCT: Gaussian fluctuations of the continuous (restricted) loss: Bohr's
 *    variance for transfers up to min(production cut, largest transfer), the loss redrawn
 *    into [0, 2 x mean] (at most 8 draws, then the mean), for tracks that survive the mean
 *    loss of a step shorter than their range.
 * Their random numbers come from counter blocks 0x40000000 (deflection) and 0x40000001.. of
 * the step's stream, apart from the interaction sampling. */
#define ADEPT_PHYS_MSC (1u << 0)
#define ADEPT_PHYS_FLUCT (1u << 1)

typedef struct adept_ctx adept_ctx; /* opaque, library-owned */

/* Calorimeter geometry. kind 0: a stack of n_layers identical layers along +z starting
 * at z = 0, |x|,|y| <= transverse_half_mm. kind 1: n_layers concentric tube layers
 * around the z axis, |z| <= half_length_mm, layer l starting at radius
 * layer_inner_r_mm[l] (increasing), vacuum inside the first layer and between layers.
 * Each layer consists of n_mat_per_layer sublayers (inner to outer / front to back)
 * of material layer_materials[s] and thickness thickness_mm[s]. Leaving the calorimeter
 * ends a track ("leaked"). A material with Z = 0 is vacuum. Host memory, read at init. */
typedef struct {
  int32_t kind;
  int32_t n_layers;
  int32_t n_mat_per_layer;
  const int32_t* layer_materials; /* [n_mat_per_layer] index into the material array */
  const double* thickness_mm;     /* [n_mat_per_layer] */
  double transverse_half_mm;      /* kind 0 */
  double half_length_mm;          /* kind 1 */
  const double* layer_inner_r_mm; /* kind 1: [n_layers] */
} adept_geometry;

/* An elemental material (Z, molar mass, density, mean excitation energy). */
typedef struct {
  int32_t Z;
  double A_g_mol;
  double density_g_cm3;
  double I_eV;
  /* A compound (n_elements 1..8): its elements' Z, molar mass (g/mol) and atoms per formula
   * unit, caller-owned and read only by adept_init; Z and A_g_mol are then ignored. The
   * per-electron processes use the compound's electron density, photoabsorption sums over
   * its atoms, 1/X0 adds its elements' terms by atom density (Bragg additivity), and the
   * density effect takes its I and rho <Z/A>. n_elements = 0: a single element Z (Z = 0:
   * vacuum). */
  int32_t n_elements;
  const int32_t* element_Z;
  const double* element_A;
  const double* element_atoms;
} adept_material;

/* Production cut as a range (converted to energy thresholds per material), uniform
 * field along +z, and the tracking cut below which a particle deposits its energy. */
typedef struct {
  double range_cut_mm;
  double field_T;
  double tracking_cut_MeV; /* must equal 1e-3: the tables start at 1 keV */
} adept_cuts;

/* Run options. Zero-initialised fields take the default in brackets. */
typedef struct {
  int32_t precision;          /* 0: plain FP64 everywhere; 1: split, FP32 physics and helix
                                 with FP64 positions, boundary distances and energy [0] */
  int32_t block_size;         /* threads per block of the step kernel [256] */
  int32_t blocks_per_sm;      /* transport-kernel variant compiled for 1..4 resident
                                 256-thread blocks per SM (register cap 255/128/85/64); the
                                 persistent grid is SMs x its occupancy [3 split, 2 FP64] */
  int32_t graph_generations;  /* generations per captured CUDA graph [32]; -1 = no graphs:
                                 launch each generation and read the queue sizes after it */
  uint32_t seed;              /* Philox key word 0 [1] */
  uint32_t process_mask;      /* ADEPT_P_* bits, 0 = all [0]; a process switched off has zero
                                 cross-section tables in the context (adept_get_table) */
  uint32_t max_steps;         /* per-track step cap; the rest of the energy is "killed" [100000] */
  uint32_t max_vacuum_steps;  /* consecutive vacuum-step cap [1000] */
  uint32_t max_events;        /* event slots (events in flight) [65536] */
  uint32_t max_generation_log;/* per-generation queue-size log length [4096] */
  uint64_t track_capacity;    /* tracks per species per buffer [derived from arena] */
  double tracks_per_MeV;      /* admission estimate of peak live tracks per MeV [0.25] */
  int32_t flags;              /* ADEPT_FLAG_* bits [0] */
  int32_t blocks_per_sm_species[3]; /* per-species override of blocks_per_sm (gamma, e-, e+) [0] */
  int32_t fused;              /* 0: per generation, three species kernels run concurrently;
                                 1: one kernel per generation for all three species;
                                 blocks_per_sm picks its variant (2 or 3 split, 1 or 2 FP64) [0] */
  uint32_t physics;           /* ADEPT_PHYS_* bits [0] */
  double msc_range_factor;    /* f of the multiple-scattering step limit [0.04] */
  int32_t field_max_iterations; /* charged tracks in the field: 0 = the analytic helix [0];
                                 N > 0 = the paper's chord propagation (Sec. 2.3): linear
                                 segments of sagitta <= delta_chord_mm, a crossing refined to
                                 delta_intersection_mm, at most N segments and refinements per
                                 step; a track whose step needs more is killed, its energy
                                 counted in killed_MeV */
  double delta_chord_mm;      /* [0.25] */
  double delta_intersection_mm; /* [0.001] */
  uint32_t max_outgoing;      /* outgoing particles kept between two status reads (a ring in the
                                 arena, 64 bytes each); more make adept_transport return
                                 ADEPT_ENOMEM [arena_bytes / 1024, within 2^16 .. 2^26] */
  int32_t tail_tracks;        /* when fewer tracks than this, and than an eighth of the peak
                                 since the queues were last empty, are live (at the last status,
                                 plus an estimate for requests admitted since), the next chunk
                                 runs as a tail chunk: one generation per iteration of a
                                 conditional graph loop that stops as soon as the queues are
                                 empty (no empty generations at the end of a transport), once
                                 4 x tail_tracks are live, or after graph_generations
                                 generations; < 0: never [16384] */
} adept_options;

/* adept_options.flags: time every generation (its three transport kernels, from the fork to
 * the join) with CUDA events recorded inside the captured graphs; totals in adept_stats */
#define ADEPT_FLAG_TIME_STEPS 1
/* also time each species kernel separately (two more events per generation) */
#define ADEPT_FLAG_TIME_SPECIES 4
/* histogram the length of every step (validation; costs one atomic per step; runs kernels
 * compiled with the histogram, so not with fused = 1 or field_max_iterations > 0, which
 * adept_init refuses with ADEPT_EINVAL) */
#define ADEPT_FLAG_STEP_HISTOGRAM 8

/* One particle handed to the library. event is the caller's event number; it keys the
 * random streams together with the seed, so equal (seed, event, track order) inputs
 * give equal results whatever else is in flight. Tracks of one event within one
 * adept_submit are numbered 1, 2, ... in submission order (their track ids). */
typedef struct {
  int32_t pdg;
  double E_kin_MeV;
  double pos_mm[3];
  double dir[3]; /* unit vector */
  uint32_t event;
} adept_track;

/* Per-request summary written by adept_get_scoring. */
typedef struct {
  uint32_t request;
  uint32_t n_events;   /* events of the request, in first-appearance order */
  uint32_t n_bins;     /* n_layers * n_mat_per_layer */
  double deposited_MeV;
  double leaked_MeV;   /* energy carried out of the calorimeter (a positron adds 2 m c^2) */
  double killed_MeV;   /* energy of tracks stopped by the step caps or by overflow */
  double latency_us;   /* from adept_submit to completion being seen by the host */
} adept_result;

/* Outgoing particles of a finished request (paper Sec. 4: the particles that leave the GPU
 * region go back to the host): every track that left the calorimeter, at the point where it
 * left, and every primary submitted outside it, with the caller's event number. Writes
 * min(n_max, count) of them to out (unordered) and the count to *n_out. Call it before
 * adept_get_scoring, which releases the request. ADEPT_EBUSY before the request is done. */
int adept_get_leaked(adept_ctx* ctx, uint32_t request, adept_track* out, size_t n_max, size_t* n_out);

/* Global counters since adept_init. */
typedef struct {
  uint64_t steps[3];      /* tracked steps: gamma, e-, e+ */
  uint64_t secondaries[3];/* secondaries pushed onto the queues */
  uint64_t generations;   /* step-kernel generations run */
  uint64_t overflow;      /* tracks dropped for lack of capacity (transport then failed) */
  uint64_t requests_done;
  uint64_t launches;      /* kernels launched by the library */
  uint64_t step_launches; /* generations timed (ADEPT_FLAG_TIME_STEPS or _SPECIES) */
  double step_kernel_ms;  /* summed CUDA-event durations of their generations (fork to the
                             end of the last of the three concurrent species kernels, or the
                             fused kernel) */
  double species_ms[3];   /* per species kernel (gamma, e-, e+): fork to its end, summed
                             (ADEPT_FLAG_TIME_SPECIES only) */
} adept_stats;

/* Create a context: validates geometry and materials, lays out dev_arena (device memory
 * of arena_bytes owned by the caller, 256-byte aligned) for tables, track queues, event
 * slots and scoring. Returns ADEPT_ENOMEM if the arena cannot hold the minimum layout,
 * ADEPT_EINVAL (with adept_last_error) for invalid input, and writes *out only on
 * success; the caller keeps ownership of every input array and of the arena, which must
 * outlive the context. No device work yet beyond memory layout. Paper: the
 * initialisation phase that sets up the geometry and materials once, kept apart from the
 * run-time transport (Sec. 2.2), and the detector region handed to the GPU (Sec. 4). */
int adept_init(adept_ctx** out, const adept_geometry* geometry, const adept_material* materials,
               int32_t n_materials, const adept_cuts* cuts, const adept_options* options,
               void* dev_arena, size_t arena_bytes, void* stream);

/* Build the physics tables on the device in FP64 (cross sections, stopping powers and
 * ranges on a 1 keV - 1 TeV log grid, 32 bins per decade; production thresholds from
 * the range cut) and their FP32 copies. Synchronous. Paper: the split of initialisation
 * and run time and the upload of physics data to the GPU (Sec. 2.2). */
int adept_build_tables(adept_ctx* ctx);

/* Buffer n tracks from host memory as one request (copied; the caller may reuse its
 * array on return). The request is admitted to the device at the next generation
 * boundary that has room for it. *request_id receives its id. n = 0 creates an empty
 * request that completes immediately. Thread-safe. Paper: buffering of particles
 * entering the GPU region (Sec. 4). */
int adept_submit(adept_ctx* ctx, const adept_track* host_tracks, size_t n, uint32_t* request_id);

/* Same, but the tracks are already in device memory (n records laid out as
 * adept_track) -- used to time transport with inputs resident in HBM. The records must be
 * written when the call is made (the library copies them back once, on a stream of its
 * own, for their event, pdg and energy fields) and must stay in place until the request has
 * been admitted, which happens at the start of a later adept_transport. Thread-safe. */
int adept_submit_device(adept_ctx* ctx, const void* dev_tracks, size_t n, uint32_t* request_id);

/* Run the stepping loop until every submitted request (including requests submitted
 * while it runs) has finished, or until timeout_us microseconds have passed
 * (ADEPT_ETIMEOUT; state is kept and a later call continues). 0 = no time limit.
 * Paper: the Flush that processes everything buffered (Sec. 4) and the per-step
 * population transport (Sec. 3). */
int adept_transport(adept_ctx* ctx, uint64_t timeout_us);

/* 1 if the request has finished, 0 if not, ADEPT_ENOTFOUND if unknown. */
int adept_poll(adept_ctx* ctx, uint32_t request_id);

/* Block until the request has finished (another thread drives adept_transport) or
 * timeout_us passes (ADEPT_ETIMEOUT). */
int adept_wait(adept_ctx* ctx, uint32_t request_id, uint64_t timeout_us);

/* Copy a finished request's deposits to host memory edep_out: n_events rows of n_bins
 * doubles (layer-major, material-minor), capacity n doubles, and fill *meta (may be
 * NULL). ADEPT_EBUSY if not finished; ADEPT_EINVAL if n is too small. The request's
 * results are released after a successful call. Paper: hits returned per event (Sec. 4). */
int adept_get_scoring(adept_ctx* ctx, uint32_t request_id, double* edep_out, size_t n,
                      adept_result* meta);

int adept_get_stats(adept_ctx* ctx, adept_stats* out);

/* Per-generation queue sizes (gamma, e-, e+) of generations since the last reset,
 * n_max rows of 3 uint32; returns the number of rows written (>= 0) or an error. */
int adept_get_generation_log(adept_ctx* ctx, uint32_t* host_out, size_t n_max);
int adept_reset_generation_log(adept_ctx* ctx);

/* Step-length histogram since adept_init (ADEPT_FLAG_STEP_HISTOGRAM): 3 x 64 counts, species
 * gamma, e-, e+, bin floor(log2(step / mm)) + 40 clamped to [0, 63]. The paper validates
 * step-length distributions against Geant4 (Sec. 2.1). */
int adept_get_step_histogram(adept_ctx* ctx, uint64_t* host_out);

/* Production thresholds chosen for material m (MeV). */
int adept_get_cuts(adept_ctx* ctx, int32_t m, double* e_cut, double* gamma_cut);

/* Device table of species s (0 gamma: compton, pair, photo; 1 e-: dedx, range, ioni,
 * brem; 2 e+: dedx, range, ioni, brem, annihilation), table t, material m, node
 * values in FP64 (prec 0) or FP32 widened to double (prec 1), 289 entries. */
int adept_get_table(adept_ctx* ctx, int32_t s, int32_t t, int32_t m, int32_t prec, double* host_out);

/* Device-side probes for parity tests: each runs the transport's own device functions
 * in a small kernel on host inputs and copies results back. Synchronous.
 *  - philox: n counters (4 words each) under one key -> 4 words each.
 *  - interp: table lookup at n energies (prec 0/1).
 *  - inverse_range: E(R) for n ranges.
 *  - distance: straight (field off) or helix (charge != 0 and field on) distance for n
 *    points: in pos[3n], dir[3n], vol[n], T[n], charge[n]; out s[n], next[n].
 *  - sample: n draws of sampler `which` (0 Compton, 1 pair, 2 Moller, 3 Bhabha, 4 brem,
 *    5 annihilation in flight, 6 at rest) at energy E in material m, stream i keyed
 *    (seed, event) with track id i+1 at step 0; 12 doubles per draw. */
int adept_probe_philox(adept_ctx* ctx, const uint32_t key[2], const uint32_t* host_ctr, size_t n,
                       uint32_t* host_out);
int adept_probe_interp(adept_ctx* ctx, int32_t s, int32_t t, int32_t m, int32_t prec,
                       const double* host_E, size_t n, double* host_out);
int adept_probe_inverse_range(adept_ctx* ctx, int32_t s, int32_t m, int32_t prec,
                              const double* host_R, size_t n, double* host_out);
int adept_probe_distance(adept_ctx* ctx, int32_t prec, const double* host_pos,
                         const double* host_dir, const int32_t* host_vol, const double* host_T,
                         const int32_t* host_charge, size_t n, double* host_s, int32_t* host_next);
int adept_probe_sample(adept_ctx* ctx, int32_t which, int32_t m, int32_t prec, double E,
                       uint32_t event, size_t n, double* host_out);
/*  - continuous: n draws of the optional along-step physics in material m at kinetic energy
 *    T over path s, stream i keyed (seed, event) with track id i+1 at step 0:
 *    which 0, the multiple-scattering deflection of the direction (0,0,1): 3 doubles per
 *    draw; which 1, the fluctuated loss of an e- (species 1) or e+ (species 2) and the mean
 *    loss it fluctuates about: 2 doubles per draw. */
int adept_probe_continuous(adept_ctx* ctx, int32_t which, int32_t species, int32_t m, int32_t prec,
                           double T, double s, uint32_t event, size_t n, double* host_out);
/*  - chord: one chord-propagated step (options field_max_iterations > 0) for n points: in
 *    pos[3n], dir[3n], vol[n], T[n], charge[n] (+-1), s_phys[n]; out 9 doubles per point:
 *    status (0 reached s_phys, 1 crossed, 2 iteration cap), path length, next volume,
 *    position (3), direction (3). */
int adept_probe_chord(adept_ctx* ctx, int32_t prec, const double* host_pos, const double* host_dir,
                      const int32_t* host_vol, const double* host_T, const int32_t* host_charge,
                      const double* host_s_phys, size_t n, double* host_out);

/* Ray-traced image of the geometry (paper Sec. 2.1: navigation validated on ray-traced
 * images, GPU against CPU and single against double precision). Orthographic camera
 * cam = {origin[3], view direction[3], up[3], width, height} (mm): the ray of pixel (i, j)
 * starts at origin + ((i+0.5)/nx - 0.5) width right + ((j+0.5)/ny - 0.5) height up' (right =
 * dir x up normalised, up' = right x dir) and runs along dir; it enters the world
 * analytically and crosses volume after volume with the transport's navigation, with FP64
 * (prec 0) or FP32 (prec 1) distances. out[2 (j nx + i) + {0, 1}] = mass thickness traversed
 * (g/cm^2) and volumes entered (0: the ray misses the world). out is host memory
 * (out_on_device 0; synchronous, the image is made and copied in bands) or caller-owned
 * device memory of 16 nx ny bytes (out_on_device 1; one launch on the context's stream, not
 * waited for). */
int adept_raytrace(adept_ctx* ctx, int32_t prec, const double cam[11], int32_t nx, int32_t ny, double* out,
                   int32_t out_on_device);

/* Table build without any allocation, for callers that cannot allocate device memory:
 * code that runs under a host framework which owns every device allocation (a fixed
 * device budget handed out by someone else), or that must not add an allocation, with its
 * latency and its failure mode, to its path. The paper has no counterpart.
 * Computes, for n_materials (1..ADEPT_NOALLOC_MAX_MATERIALS) materials and a range cut, the
 * same FP64 tables and production thresholds as adept_build_tables:
 *   dev_tables: caller-owned device memory, [n_materials][12][289] doubles: gamma (compton,
 *               pair, photo), e- (dedx, range, ioni, brem), e+ (dedx, range, ioni, brem,
 *               annihilation) at the 289 grid energies (zeros for vacuum);
 *   dev_cuts:   caller-owned device memory, [n_materials][2] doubles (e-/e+ cut, gamma cut).
 * Needs no context and allocates nothing: its working rows (ADEPT_NOALLOC_MAX_MATERIALS x
 * 17 x 289 doubles, 157 KB) are a static device array that every GPU loading the library
 * holds until exit. The first call on a device looks up that array's device address with the
 * device current; make that first call before any stream capture. Work is queued on stream
 * (a cudaStream_t; results are ready when the stream reaches it). Every call shares the
 * array, so calls that overlap on the GPU (other streams, other threads) race; serialise
 * them. Returns ADEPT_EINVAL for a null pointer, a bad material or a compound (single
 * elements only), a non-positive cut or n_materials outside 1..ADEPT_NOALLOC_MAX_MATERIALS,
 * ADEPT_ECUDA if the launch fails. */
#define ADEPT_NOALLOC_MAX_MATERIALS 4
int adept_build_tables_noalloc(const adept_material* materials, int32_t n_materials, double range_cut_mm,
                               double* dev_tables, double* dev_cuts, void* stream);

/* Message of the last failure on this context, from any thread. The pointer stays valid
 * until the next failure or adept_destroy. */
const char* adept_last_error(const adept_ctx* ctx);
void adept_destroy(adept_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* ADEPT_H */
