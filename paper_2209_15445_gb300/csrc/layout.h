// Memory layout shared by the host runtime (api.cu) and the kernels (kernels.cu):
// geometry and material views, physics tables, structure-of-arrays track queues,
// event slots and the device control block. All pointers are into the caller's arena.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace adept {

constexpr int kNNode = 289;   // 1 keV .. 1 TeV, 32 bins per decade
constexpr int kMaxMat = 8;
constexpr int kMaxVol = 1024;
constexpr int kNTabG = 3;     // gamma: compton, pair, photo
constexpr int kNTabE = 4;     // e-: dedx, range, ioni, brem
constexpr int kNTabP = 5;     // e+: dedx, range, ioni, brem, annihilation
constexpr int kMaxLogGen = 1 << 16;

struct GeoView {
  int kind;          // 0 slab, 1 tubes
  int n_vol;
  int n_bins;
  double half_xy, half_z;
  const double* bnd;     // slab: n_vol+1 planes; tubes: n_vol radii
  const int* vol_mat;    // material index or -1 (vacuum)
  const int* vol_bin;    // scoring bin or -1
};

// per-material constants derived on the device from (Z, A, rho, I)
constexpr int kMaxElem = 8;                    // elements of a compound
constexpr int kMatRec = 5 + 3 * kMaxElem;      // material record: Z, A, rho, I, n_elem, (Z, A, atoms) x n_elem

struct MatDev {
  double Z, A, rho, I;   // I in eV (a compound: its mean Z and A)
  int n_elem;            // elements: Z and atoms per mm^3
  double eZ[kMaxElem], en_at[kMaxElem];
  double ZoA;            // <Z/A> by mass
  double n_at, n_el;     // per mm^3
  double inv_x0;         // 1/mm
  double cbar, x0, x1, a_d;
  int vacuum;
  int pad;
};

struct TableView {
  // (value, slope) records: [mat][node][table]
  const double2* g64; const double2* e64; const double2* p64;
  const float2* g32; const float2* e32; const float2* p32;
  // range nodes for the inversion: [mat][node]
  const double* re64; const double* rp64;
  const float* re32; const float* rp32;
  // production thresholds per material
  const double* Tc; const double* kc;
};

// One species' queue. Plain form: one array per field. Split form: the 64-byte track in
// four arrays of 16-byte vectors (x,y | z,E | ux,uy,uz,nav | id lo,id hi,event,step), so
// that a warp moves a track with four coalesced 128-bit loads and stores.
struct TrackSoA {
  // plain form
  double *x, *y, *z;
  double *ux, *uy, *uz;
  double* E;
  unsigned long long* id;
  uint32_t* ev;    // event slot
  uint32_t* step;  // steps taken by this track
  uint32_t* nav;   // volume (low 16 bits) | consecutive vacuum steps (high 16 bits)
  // split form
  double2* xy;
  double2* zE;
  float4* un;      // direction and nav (bits)
  uint4* meta;     // id lo, id hi, event slot, step
};

// Device control block: queue sizes, generation counter, statistics and the done-event
// list of the last chunk. Written by kernels, read by the host after each chunk.
// Generation g reads the track buffers of parity g & 1 and the sizes count[g % 3], and
// appends to parity (g + 1) & 1 and count[(g + 1) % 3]. Three size slots let one thread of
// generation g empty count[(g + 2) % 3] (read by generation g - 1, appended to by g + 1)
// without a separate close step between generations.
// A queue size on a 128-byte line of its own: every warp of a generation reserves its slots
// with an atomic on one of these, and sizes sharing an L2 line would queue behind each other.
struct alignas(128) QCount {
  uint32_t n;
  uint32_t pad[31];
};
struct Ctrl {
  uint32_t gen;               // generations run before the current chunk (advanced at its end)
  QCount count[3][3];         // queue sizes [generation mod 3][species]
  uint32_t done_count[2];     // events found finished by the finish pass of a chunk (per buffer)
  uint32_t log_n;             // rows written to the generation log
  uint32_t error;             // first device-detected error code (0 = none)
  uint32_t tail_k;            // generations a tail chunk has run so far (see kGkDevice)
  uint32_t finish_ticket;     // blocks of the finish pass that have ended (the last one resets it)
  uint32_t pad[2];
  unsigned long long steps[3];
  unsigned long long created[3];
  unsigned long long overflow;
  unsigned long long generations;
  // outgoing particles: records appended (ring index = count mod capacity), records not
  // written because the host had not read far enough, and the host's read position when the
  // running chunk was launched (a record may go where the host has read)
  unsigned long long leak_count, leak_dropped, leak_floor;
};

// one outgoing particle, as it leaves the calorimeter (64 bytes)
struct LeakRec {
  int32_t pdg;
  uint32_t slot;
  double E;
  double pos[3];
  double dir[3];
};

struct EventView {
  uint32_t* key;       // RNG key word 1 (the caller's event number) per slot
  uint32_t* state;     // 0 free, 1 active, 2 done
  uint32_t* alive;     // last generation at which a live track of the slot was seen
  double* edep;        // [slot][n_bins]
  double* leaked;      // [slot]
  double* killed;      // [slot]
  uint32_t max_slots;
};

struct Params {
  GeoView geo;
  const MatDev* mat;
  TableView tab;
  TrackSoA q[2][3];     // [parity][species] (host copy; kernels index qd)
  const TrackSoA* qd;   // the same six descriptors in device memory, [3 * parity + species]
  uint32_t cap;         // tracks per species per buffer
  Ctrl* ctrl;
  EventView evt;
  uint32_t* gen_log;    // [max_log][3]
  uint32_t max_log;
  double field_T;
  double tcut;
  uint32_t seed, process_mask, max_steps, max_vac;
  unsigned long long* steplen;  // [3][64] step-length histogram (log2 bins), or null
  uint32_t physics;     // ADEPT_PHYS_* bits: multiple scattering, loss fluctuations
  double msc_f;         // multiple-scattering step limit: s <= max(msc_f R, 0.01 mm)
  LeakRec* leak;        // ring of outgoing particles
  uint32_t leak_cap;
  int chord_iter;       // 0: analytic helix; N > 0: chord propagation capped at N iterations
  double delta_chord;   // chord sagitta limit, mm
  double delta_int;     // intersection accuracy, mm
  uint32_t tail_exit;   // a tail chunk ends once this many tracks are live
  // the host's pinned, device-mapped status of the two chunk buffers: the copy of Ctrl and the
  // done list ([evt.max_slots]: slots found finished) that a chunk's finish pass writes, and the
  // outgoing-ring read position its first kernel reads (so no copy sits between two chunks)
  Ctrl* h_ctrl[2];
  uint32_t* h_done[2];
  const unsigned long long* h_floor[2];
};

// device view of one submitted particle; same layout as adept_track in adept.h
struct TrackIn {
  int32_t pdg;
  int32_t pad0;
  double E;
  double pos[3];
  double dir[3];
  uint32_t event;
  uint32_t pad1;
};

// ---- kernel launchers (kernels.cu) ----
struct BuildScratch {
  double* vals;     // [mat][16][kNNode] raw table values
  double* bins;     // [mat][4][kNNode] per-bin range integrals
};
cudaError_t launch_build_tables(const Params& P, const double* mat_in, int n_mat, double range_cut,
                                MatDev* mat, BuildScratch s, double2* g64, double2* e64, double2* p64,
                                float2* g32, float2* e32, float2* p32, double* re64, double* rp64,
                                float* re32, float* rp32, double* Tc, double* kc, cudaStream_t st);
// A tail chunk runs its generations as the body of a conditional (while) graph node, one
// generation per iteration, until the queues are empty or a cap is reached; its kernels are
// launched with gk = kGkDevice and read their place in the chunk from Ctrl::tail_k.
constexpr uint32_t kGkDevice = 0xFFFFFFFFu;
// generation gen + gk of one species (gk: its place in the chunk; the three species of a
// generation may run concurrently). pdl: launch with a programmatic dependency on the
// stream's preceding kernels (the previous generation's), see grid_dependency_wait.
cudaError_t launch_transport(const Params& P, uint32_t gk, int precision, int species, int minb, int grid, int block,
                             bool pdl, cudaStream_t st);
cudaError_t launch_admit(const Params& P, uint32_t slot_base, const uint32_t* keys, int n_slots,
                         cudaStream_t st);
// meta: per track (event index within the request, track id)
cudaError_t launch_init_primaries(const Params& P, const TrackIn* recs, const uint32_t* meta, int n,
                                  uint32_t slot_base, int precision, cudaStream_t st);
// start of a chunk in status buffer b: the host's outgoing-ring read position, done count 0
cudaError_t launch_open_chunk(const Params& P, int b, cudaStream_t st);
// end of a chunk of `gens` generations (kGkDevice: the count a tail chunk left in
// Ctrl::tail_k): log the last one, advance gen, find finished events, and write the status
// and the done list to the host's copy of buffer b
cudaError_t launch_finish(const Params& P, int buffer, uint32_t gens, cudaStream_t st);
// tail chunks: before the loop, tail_k = 0 and the condition = live tracks in the queues;
// after each generation, ++tail_k and the condition = live tracks and tail_k < max_gens
cudaError_t launch_tail_open(const Params& P, cudaGraphConditionalHandle h, cudaStream_t st);
cudaError_t launch_tail_step(const Params& P, cudaGraphConditionalHandle h, uint32_t max_gens, cudaStream_t st);
cudaError_t launch_probe_philox(const uint32_t* ctr, int n, uint32_t k0, uint32_t k1, uint32_t* out,
                                cudaStream_t st);
cudaError_t launch_probe_interp(const Params& P, int s, int t, int m, int prec, const double* E, int n,
                                double* out, cudaStream_t st);
cudaError_t launch_probe_inverse_range(const Params& P, int s, int m, int prec, const double* R, int n,
                                       double* out, cudaStream_t st);
cudaError_t launch_probe_distance(const Params& P, int prec, const double* pos, const double* dir,
                                  const int* vol, const double* T, const int* q, int n, double* s,
                                  int* next, cudaStream_t st);
cudaError_t launch_probe_sample(const Params& P, int which, int m, int prec, double E, uint32_t event,
                                int n, double* out, cudaStream_t st);
// variant: bit 0 chord propagation, bit 1 multiple scattering / loss fluctuations, bit 2 the
// step-length histogram, bit 3 the helix in the field
int transport_max_blocks_per_sm(int precision, int species, int minb, int block, int variant);
// resident blocks of `block` threads per SM for kernel fn, after asking for the smallest
// shared-memory carveout that still holds them (the rest of the SM's memory stays L1)
int max_blocks_small_carveout(const void* fn, int block);
// a variant (1..3, or 10: the optional physics in the field) of the e- (species 1) or e+ (2)
// kernel, 2 or 3 blocks/SM
const void* variant_transport_fn(int precision, int species, int minb, int variant);
// the default e- or e+ kernel with the helix (variant 8), 1..4 blocks/SM
const void* field_transport_fn(int precision, int species, int minb);
// a kernel with the step-length histogram (variant 4, or 6 with the optional physics for e-
// and e+, each + 8 in the field), any species, 2 or 3 blocks/SM; chords and the histogram
// are not combined
const void* hist_transport_fn(int precision, int species, int minb, int variant);
// the variant the options of P call for
inline int transport_variant(const Params& P) {
  // chords carry their own helix (chord_step)
  return (P.chord_iter > 0 ? 1 : 0) | (P.physics ? 2 : 0) | (P.steplen ? 4 : 0) |
         (P.field_T != 0.0 && P.chord_iter <= 0 ? 8 : 0);
}
// orthographic camera of the ray tracer: the image centre, the unit right, up and view vectors
struct RayCam {
  double o[3], right[3], up[3], d[3];
  double width, height;
};
// rows [row0, row0 + rows) of an nx x ny image into out (16 bytes per pixel)
cudaError_t launch_raytrace(const Params& P, int prec, const RayCam& cam, int nx, int ny, int row0, int rows,
                            double* out, cudaStream_t st);
cudaError_t launch_probe_chord(const Params& P, int prec, const double* pos, const double* dir, const int* vol,
                               const double* T, const int* q, const double* s_phys, int n, double* out, cudaStream_t st);
cudaError_t launch_probe_continuous(const Params& P, int which, int species, int m, int prec, double T, double s,
                                    uint32_t event, int n, double* out, cudaStream_t st);
// generation gen + gk of all species in one kernel
cudaError_t launch_fused_generation(const Params& P, uint32_t gk, int precision, int minb, int grid, int block,
                                    bool pdl, cudaStream_t st);
int fused_max_blocks_per_sm(int precision, int minb, int block, int variant);

}  // namespace adept
