// Host runtime behind the C ABI (include/adept.h): argument checking, the arena layout,
// request buffering and admission, the generation loop with CUDA graphs, completion
// tracking and result return. Every physics step runs in the kernels of kernels.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/adept.h"
#include "layout.h"

using namespace adept;

static_assert(sizeof(adept_track) == sizeof(TrackIn), "adept_track layout");
static_assert(offsetof(adept_track, E_kin_MeV) == offsetof(TrackIn, E), "adept_track layout");
static_assert(offsetof(adept_track, pos_mm) == offsetof(TrackIn, pos), "adept_track layout");
static_assert(offsetof(adept_track, dir) == offsetof(TrackIn, dir), "adept_track layout");
static_assert(offsetof(adept_track, event) == offsetof(TrackIn, event), "adept_track layout");

namespace {

using Clock = std::chrono::steady_clock;

// Host copy of a finished request's rows (deposits [event][bin], then leaked and killed per
// event): a pinned block from the context's pool, so that the copy out of device memory runs
// at the link's rate and reuses pages already mapped, or pageable memory if pinning fails.
struct ResultBuf {
  double* p = nullptr;
  size_t cap = 0;  // doubles
  bool pinned = false;
  std::vector<double> pageable;
};

struct Request {
  uint32_t id = 0;
  size_t n = 0;
  std::vector<adept_track> host;       // host submission (copied)
  const adept_track* dev = nullptr;    // device submission (caller-owned)
  std::vector<uint32_t> meta;          // [event index, track id] per track
  std::vector<uint32_t> keys;          // RNG key (caller's event number) per event
  double energy = 0.0;                 // primary energy incl. 2 m for positrons
  uint32_t slot_base = 0;
  uint32_t remaining = 0;              // events not finished
  int state = 0;                       // 0 pending, 1 in flight, 2 done
  Clock::time_point t_submit, t_done;
  ResultBuf res;                       // rows copied back at completion
  std::vector<adept_track> outgoing;   // particles that left the calorimeter
};

struct SlotAlloc {  // first-fit allocator of contiguous event-slot ranges
  std::map<uint32_t, uint32_t> free_;  // start -> length
  void init(uint32_t n) { free_.clear(); if (n) free_[0] = n; }
  bool alloc(uint32_t n, uint32_t* out) {
    if (n == 0) { *out = 0; return true; }
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        *out = it->first;
        const uint32_t s = it->first + n, l = it->second - n;
        free_.erase(it);
        if (l) free_[s] = l;
        return true;
      }
    }
    return false;
  }
  void release(uint32_t s, uint32_t n) {
    if (!n) return;
    auto it = free_.emplace(s, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) { it->second += nx->second; free_.erase(nx); }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) { pv->second += it->second; free_.erase(it); }
    }
  }
};

}  // namespace

struct adept_ctx {
  std::mutex err_mu;  // producers and the transport thread may both fail
  std::mutex submit_mu;  // device submissions share submit_stream
  std::string err;
  cudaStream_t stream = nullptr;
  adept_options opt{};
  int n_mat = 0;
  std::vector<adept_material> mats;
  double range_cut = 0.7;
  // geometry (host copy)
  int kind = 0, n_vol = 0, n_bins = 0;
  std::vector<double> bnd;
  std::vector<int> vol_mat, vol_bin;
  // arena
  char* arena = nullptr;
  size_t arena_bytes = 0, arena_used = 0;
  Params P{};
  MatDev* mat_dev = nullptr;
  double* mat_in = nullptr;
  std::vector<double> mat_rec;  // kMatRec doubles per material (elements of compounds copied)
  BuildScratch scratch{};
  double2 *g64 = nullptr, *e64 = nullptr, *p64 = nullptr;
  float2 *g32 = nullptr, *e32 = nullptr, *p32 = nullptr;
  double *re64 = nullptr, *rp64 = nullptr, *Tc = nullptr, *kc = nullptr;
  float *re32 = nullptr, *rp32 = nullptr;
  TrackIn* stage = nullptr;
  uint32_t* stage_meta = nullptr;
  uint32_t* stage_keys = nullptr;
  size_t stage_cap = 0;
  char* probe = nullptr;
  size_t probe_bytes = 0;
  bool built = false;
  // host pinned buffers
  Ctrl* h_ctrl[2] = {nullptr, nullptr};     // status of the two chunks that may be in flight
  unsigned long long* h_floor[2] = {nullptr, nullptr};  // outgoing-ring read position at each launch
  unsigned long long leak_read = 0, leak_dropped_seen = 0;  // host read position, drops seen
  LeakRec* h_leak = nullptr;  // pinned staging of the outgoing records read back at a status
  size_t h_leak_cap = 0;
  uint32_t* h_done[2] = {nullptr, nullptr};
  cudaEvent_t status_ev[2] = {nullptr, nullptr};
  cudaEvent_t stage_ev = nullptr;            // the last copy out of the pinned staging buffer
  cudaEvent_t out_ev = nullptr;              // the last copy of outgoing records into h_leak
  cudaStream_t copy_stream = nullptr;        // result copies, overlapping the next chunk
  cudaStream_t submit_stream = nullptr;      // device submissions' field reads (producer threads)
  char* h_stage = nullptr;
  size_t h_stage_bytes = 0;
  char* h_sub = nullptr;                     // device submissions' tracks read back (under submit_mu)
  size_t h_sub_bytes = 0;
  // pinned blocks for finished requests' rows: free ones, and all (freed at destroy)
  std::mutex pool_mu;
  std::vector<std::pair<double*, size_t>> pool_free;
  std::vector<double*> pool_all;
  // launch shape
  int grid[3] = {0, 0, 0}, block = 256, minb[3] = {1, 1, 1};  // per species
  int fgrid = 0, fminb = 0;  // fused generation kernel
  cudaGraphExec_t graph[2] = {nullptr, nullptr};  // one per status buffer (own timing events)
  int graph_gens = 0;
  // tail chunks (one per status buffer): a conditional while node runs one generation per
  // iteration until the queues are empty, so the end of a transport launches no empty
  // generations; chosen once the live tracks at the last status fall below kTailTracks
  cudaGraphExec_t tgraph[2] = {nullptr, nullptr};
  bool tail[2] = {false, false};  // the chunk queued in buffer b is a tail chunk
  uint64_t last_live = 0;         // live tracks at the end of the last chunk read back
  uint64_t peak_live = 0;         // most live tracks seen since the queues were last empty
  // estimated peak tracks (tracks_per_MeV x energy, plus the primaries) of the requests
  // admitted so far; its value when chunk b was launched; and the value behind last_live
  uint64_t admit_est = 0, admit_mark[2] = {0, 0}, admit_seen = 0;
  cudaStream_t bstream = nullptr; // captures the tail chunks' loop body
  std::vector<cudaEvent_t> ev;  // 4 per generation when timing: start, after e-, after e+, after gamma
  cudaStream_t side[2] = {nullptr, nullptr};     // the e+ and gamma kernels run on these
  cudaEvent_t fork = nullptr, join[2] = {nullptr, nullptr};
  // timing: the event-record nodes hang off the generation chain on their own stream, so
  // that nothing on the chain waits for them (kdone[sp]: species sp's kernel has ended)
  cudaStream_t tstream = nullptr;
  cudaEvent_t kdone[3] = {nullptr, nullptr, nullptr}, tjoin = nullptr;
  // requests
  std::mutex mu;
  std::condition_variable cv;
  uint32_t next_id = 1;
  std::deque<uint32_t> pending;
  std::unordered_map<uint32_t, std::unique_ptr<Request>> reqs;
  std::vector<Request*> slot_req;  // slot -> its request while that is in flight (else null)
  SlotAlloc slots;
  double energy_in_flight = 0.0;
  size_t in_flight = 0;
  adept_stats stats{};
  std::vector<uint32_t> gen_log_host;
  unsigned long long* steplen = nullptr;  // device histogram (always carved, filled on request)
};

static int fail(adept_ctx* c, int code, const char* fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    std::lock_guard<std::mutex> lk(c->err_mu);
    c->err = buf;
  }
  return code;
}

#define CK(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) return fail(c, ADEPT_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

static void* carve(adept_ctx* c, size_t bytes) {
  const size_t off = (c->arena_used + 255) & ~(size_t)255;
  if (off + bytes > c->arena_bytes) return nullptr;
  c->arena_used = off + bytes;
  return c->arena + off;
}

template <class T>
static bool carve_n(adept_ctx* c, T** out, size_t n) {
  *out = static_cast<T*>(carve(c, sizeof(T) * (n ? n : 1)));
  return *out != nullptr;
}

// an element with Z > 0 or a compound (Z = 0 and no elements: vacuum)
static bool is_matter(const adept_material& m) { return m.Z > 0 || m.n_elements > 0; }

// volumes of the calorimeter: slab planes, or tube radii with vacuum inside and between
static int build_geometry(adept_ctx* c, const adept_geometry* g) {
  if (g->kind != 0 && g->kind != 1) return fail(c, ADEPT_EINVAL, "geometry kind must be 0 or 1");
  if (g->n_layers < 1 || g->n_mat_per_layer < 1 || g->n_mat_per_layer > 16 || !g->layer_materials || !g->thickness_mm)
    return fail(c, ADEPT_EINVAL, "geometry needs n_layers >= 1 and 1..16 sublayers");
  double lt = 0.0;
  for (int s = 0; s < g->n_mat_per_layer; ++s) {
    if (g->layer_materials[s] < 0 || g->layer_materials[s] >= c->n_mat)
      return fail(c, ADEPT_EINVAL, "sublayer %d names material %d of %d", s, g->layer_materials[s], c->n_mat);
    if (!(g->thickness_mm[s] > 0.0)) return fail(c, ADEPT_EINVAL, "sublayer %d thickness must be > 0", s);
    lt += g->thickness_mm[s];
  }
  c->kind = g->kind;
  c->n_bins = g->n_layers * g->n_mat_per_layer;
  c->bnd.clear(); c->vol_mat.clear(); c->vol_bin.clear();
  auto mat_of = [&](int s) { return is_matter(c->mats[g->layer_materials[s]]) ? g->layer_materials[s] : -1; };
  if (g->kind == 0) {
    if (!(g->transverse_half_mm > 0.0)) return fail(c, ADEPT_EINVAL, "transverse_half_mm must be > 0");
    double z = 0.0;
    c->bnd.push_back(0.0);
    for (int l = 0; l < g->n_layers; ++l)
      for (int s = 0; s < g->n_mat_per_layer; ++s) {
        z += g->thickness_mm[s];
        c->bnd.push_back(z);
        const int m = mat_of(s);
        c->vol_mat.push_back(m);
        c->vol_bin.push_back(m >= 0 ? l * g->n_mat_per_layer + s : -1);
      }
  } else {
    if (!g->layer_inner_r_mm || !(g->half_length_mm > 0.0)) return fail(c, ADEPT_EINVAL, "tubes need radii and half length");
    for (int l = 0; l < g->n_layers; ++l) {
      if (!(g->layer_inner_r_mm[l] > 0.0)) return fail(c, ADEPT_EINVAL, "layer radius must be > 0");
      if (l + 1 < g->n_layers && !(g->layer_inner_r_mm[l] + lt <= g->layer_inner_r_mm[l + 1]))
        return fail(c, ADEPT_EINVAL, "layer %d overlaps the next one", l);
    }
    c->bnd.push_back(g->layer_inner_r_mm[0]);  // volume 0: vacuum inside the first layer
    c->vol_mat.push_back(-1);
    c->vol_bin.push_back(-1);
    for (int l = 0; l < g->n_layers; ++l) {
      double r = g->layer_inner_r_mm[l];
      for (int s = 0; s < g->n_mat_per_layer; ++s) {
        r += g->thickness_mm[s];
        c->bnd.push_back(r);
        const int m = mat_of(s);
        c->vol_mat.push_back(m);
        c->vol_bin.push_back(m >= 0 ? l * g->n_mat_per_layer + s : -1);
      }
      if (l + 1 < g->n_layers) {  // vacuum gap up to the next layer
        c->bnd.push_back(g->layer_inner_r_mm[l + 1]);
        c->vol_mat.push_back(-1);
        c->vol_bin.push_back(-1);
      }
    }
  }
  c->n_vol = (int)c->vol_mat.size();
  if (c->n_vol > kMaxVol || c->n_vol > 65535) return fail(c, ADEPT_EINVAL, "too many volumes (%d)", c->n_vol);
  return ADEPT_OK;
}

static size_t track_bytes(int precision) {
  return 3 * 8 + 3 * (precision ? 4 : 8) + 8 + 8 + 3 * 4;
}

static bool carve_queue(adept_ctx* c, TrackSoA* q, uint32_t cap) {
  *q = TrackSoA{};
  if (c->opt.precision)  // split form: four arrays of 16-byte vectors
    return carve_n(c, &q->xy, cap) && carve_n(c, &q->zE, cap) && carve_n(c, &q->un, cap) && carve_n(c, &q->meta, cap);
  return carve_n(c, &q->x, cap) && carve_n(c, &q->y, cap) && carve_n(c, &q->z, cap) && carve_n(c, &q->ux, cap) &&
         carve_n(c, &q->uy, cap) && carve_n(c, &q->uz, cap) && carve_n(c, &q->E, cap) && carve_n(c, &q->id, cap) &&
         carve_n(c, &q->ev, cap) && carve_n(c, &q->step, cap) && carve_n(c, &q->nav, cap);
}

extern "C" int adept_init(adept_ctx** out, const adept_geometry* geometry, const adept_material* materials,
                          int32_t n_materials, const adept_cuts* cuts, const adept_options* options, void* dev_arena,
                          size_t arena_bytes, void* stream) {
  if (!out || !geometry || !materials || !cuts || !dev_arena) return ADEPT_EINVAL;
  *out = nullptr;
  auto c = std::make_unique<adept_ctx>();
  if (n_materials < 1 || n_materials > kMaxMat) return ADEPT_EINVAL;
  if (reinterpret_cast<uintptr_t>(dev_arena) & 255) return ADEPT_EINVAL;
  c->n_mat = n_materials;
  c->mats.assign(materials, materials + n_materials);
  c->mat_rec.assign((size_t)kMatRec * kMaxMat, 0.0);
  for (int k = 0; k < n_materials; ++k) {
    adept_material& m = c->mats[k];
    double* r = c->mat_rec.data() + (size_t)kMatRec * k;
    if (m.n_elements < 0 || m.n_elements > kMaxElem) return ADEPT_EINVAL;
    if (m.n_elements > 0) {  // a compound: keep its elements (the caller's arrays are borrowed)
      if (!m.element_Z || !m.element_A || !m.element_atoms || !(m.density_g_cm3 > 0 && m.I_eV > 0))
        return ADEPT_EINVAL;
      for (int i = 0; i < m.n_elements; ++i) {
        if (m.element_Z[i] < 1 || m.element_Z[i] > 100 || !(m.element_A[i] > 0) || !(m.element_atoms[i] > 0))
          return ADEPT_EINVAL;
        r[5 + 3 * i] = m.element_Z[i];
        r[5 + 3 * i + 1] = m.element_A[i];
        r[5 + 3 * i + 2] = m.element_atoms[i];
      }
    } else if (m.Z < 0 || m.Z > 100 || (m.Z > 0 && !(m.A_g_mol > 0 && m.density_g_cm3 > 0 && m.I_eV > 0))) {
      return ADEPT_EINVAL;
    }
    r[0] = m.n_elements > 0 ? 0.0 : m.Z;
    r[1] = m.A_g_mol; r[2] = m.density_g_cm3; r[3] = m.I_eV; r[4] = m.n_elements;
    m.element_Z = nullptr; m.element_A = nullptr; m.element_atoms = nullptr;
  }
  if (!(cuts->range_cut_mm > 0.0) || !(cuts->tracking_cut_MeV >= 1e-3) || !(cuts->tracking_cut_MeV < 1e4))
    return ADEPT_EINVAL;
  if (options) c->opt = *options;
  adept_options& o = c->opt;
  if (o.precision != 0 && o.precision != 1) return ADEPT_EINVAL;
  if (o.flags & ~(ADEPT_FLAG_TIME_STEPS | ADEPT_FLAG_TIME_SPECIES | ADEPT_FLAG_STEP_HISTOGRAM)) return ADEPT_EINVAL;
  if (o.fused != 0 && o.fused != 1) return ADEPT_EINVAL;
  if (o.fused && (o.flags & ADEPT_FLAG_TIME_SPECIES)) return ADEPT_EINVAL;  // needs separate species kernels
  if (o.physics & ~(ADEPT_PHYS_MSC | ADEPT_PHYS_FLUCT)) return ADEPT_EINVAL;
  if (o.msc_range_factor < 0.0 || !(o.msc_range_factor < 1e30)) return ADEPT_EINVAL;
  if (o.msc_range_factor == 0.0) o.msc_range_factor = 0.04;
  if (o.field_max_iterations < 0) return ADEPT_EINVAL;
  // the fused kernel has no variant with chords, the optional physics or the step-length
  // histogram, and the histogram is not compiled together with chords
  if (o.fused && (o.field_max_iterations > 0 || o.physics)) return ADEPT_EINVAL;
  if ((o.flags & ADEPT_FLAG_STEP_HISTOGRAM) && (o.fused || o.field_max_iterations > 0)) return ADEPT_EINVAL;
  if (o.delta_chord_mm < 0.0 || o.delta_intersection_mm < 0.0) return ADEPT_EINVAL;
  if (o.delta_chord_mm == 0.0) o.delta_chord_mm = 0.25;
  if (o.delta_intersection_mm == 0.0) o.delta_intersection_mm = 0.001;
  if (!(o.delta_chord_mm < 1e6 && o.delta_intersection_mm < 1e6)) return ADEPT_EINVAL;
  if (o.block_size == 0) o.block_size = 256;
  if (o.block_size < 32 || o.block_size > 256 || (o.block_size & 31)) return ADEPT_EINVAL;
  if (o.graph_generations < -1 || o.graph_generations > 1024) return ADEPT_EINVAL;
  if (o.graph_generations == 0) o.graph_generations = 32;
  if (o.tail_tracks == 0) o.tail_tracks = 16384;
  if (o.seed == 0) o.seed = 1;
  if (o.max_steps == 0) o.max_steps = 100000;
  if (o.max_vacuum_steps == 0) o.max_vacuum_steps = 1000;
  if (o.max_vacuum_steps > 65535) return ADEPT_EINVAL;
  if (o.max_events == 0) o.max_events = 65536;
  if (o.max_generation_log == 0) o.max_generation_log = 4096;
  if (o.max_generation_log > (uint32_t)kMaxLogGen) o.max_generation_log = kMaxLogGen;
  if (o.max_outgoing == 0)  // a sixteenth of the arena (64 bytes a record), 2^16 .. 2^26 records
    o.max_outgoing = (uint32_t)std::min<size_t>(std::max<size_t>(arena_bytes / 1024, (size_t)1 << 16), (size_t)1 << 26);
  if (!(o.tracks_per_MeV > 0.0)) o.tracks_per_MeV = 0.25;
  c->range_cut = cuts->range_cut_mm;
  int rc = build_geometry(c.get(), geometry);
  if (rc) return rc;
  c->stream = static_cast<cudaStream_t>(stream);
  c->arena = static_cast<char*>(dev_arena);
  c->arena_bytes = arena_bytes;
  adept_ctx* cp = c.get();
  Params& P = c->P;
  bool ok = carve_n(cp, &P.ctrl, 1);
  double* bnd = nullptr; int *vm = nullptr, *vb = nullptr;
  ok = ok && carve_n(cp, &bnd, c->bnd.size()) && carve_n(cp, &vm, c->n_vol) && carve_n(cp, &vb, c->n_vol);
  ok = ok && carve_n(cp, &c->mat_dev, kMaxMat) && carve_n(cp, &c->mat_in, kMatRec * kMaxMat);
  const size_t nn = (size_t)kNNode * n_materials;
  ok = ok && carve_n(cp, &c->scratch.vals, 14 * nn) && carve_n(cp, &c->scratch.bins, 3 * nn);
  ok = ok && carve_n(cp, &c->g64, nn * kNTabG) && carve_n(cp, &c->e64, nn * kNTabE) && carve_n(cp, &c->p64, nn * kNTabP);
  ok = ok && carve_n(cp, &c->g32, nn * kNTabG) && carve_n(cp, &c->e32, nn * kNTabE) && carve_n(cp, &c->p32, nn * kNTabP);
  ok = ok && carve_n(cp, &c->re64, nn) && carve_n(cp, &c->rp64, nn) && carve_n(cp, &c->re32, nn) && carve_n(cp, &c->rp32, nn);
  ok = ok && carve_n(cp, &c->Tc, kMaxMat) && carve_n(cp, &c->kc, kMaxMat);
  EventView& E = P.evt;
  const uint32_t ms = o.max_events;
  ok = ok && carve_n(cp, &E.key, ms) && carve_n(cp, &E.state, ms) && carve_n(cp, &E.alive, ms) &&
       carve_n(cp, &E.edep, (size_t)ms * c->n_bins) && carve_n(cp, &E.leaked, ms) && carve_n(cp, &E.killed, ms);
  ok = ok && carve_n(cp, &P.gen_log, 3 * (size_t)o.max_generation_log);
  unsigned long long* steplen = nullptr;
  ok = ok && carve_n(cp, &steplen, 3 * 64);
  TrackSoA* qdesc = nullptr;
  ok = ok && carve_n(cp, &qdesc, 6);
  ok = ok && carve_n(cp, &P.leak, o.max_outgoing);
  P.leak_cap = o.max_outgoing;
  c->probe_bytes = (size_t)8 << 20;
  c->probe = static_cast<char*>(carve(cp, c->probe_bytes));
  ok = ok && c->probe;
  if (!ok) return ADEPT_ENOMEM;
  // the remainder: primary staging (1/16, at least room for 4096 tracks) and the queues
  const size_t per_track = track_bytes(o.precision);
  size_t rest = c->arena_bytes - ((c->arena_used + 255) & ~(size_t)255);
  size_t stage_cap = std::max<size_t>(4096, rest / 16 / (sizeof(TrackIn) + 12));
  stage_cap = std::min<size_t>(stage_cap, (size_t)1 << 22);
  ok = carve_n(cp, &c->stage, stage_cap) && carve_n(cp, &c->stage_meta, 2 * stage_cap) &&
       carve_n(cp, &c->stage_keys, stage_cap);
  if (!ok) return ADEPT_ENOMEM;
  c->stage_cap = stage_cap;
  rest = c->arena_bytes - ((c->arena_used + 255) & ~(size_t)255);
  // 6 queues x 11 arrays, each padded to 256 bytes
  uint64_t cap = rest > 6 * 11 * 256 ? (rest - 6 * 11 * 256) / (6 * per_track) : 0;
  if (o.track_capacity) {
    if (o.track_capacity > cap) return ADEPT_ENOMEM;
    cap = o.track_capacity;
  }
  cap = std::min<uint64_t>(cap, 0xFFFFFFF0ull);
  if (cap < 1024) return ADEPT_ENOMEM;
  o.track_capacity = cap;
  for (int par = 0; par < 2; ++par)
    for (int s = 0; s < 3; ++s)
      if (!carve_queue(cp, &P.q[par][s], (uint32_t)cap)) return ADEPT_ENOMEM;
  P.cap = (uint32_t)cap;
  P.qd = qdesc;
  // views
  P.geo.kind = c->kind; P.geo.n_vol = c->n_vol; P.geo.n_bins = c->n_bins;
  P.geo.half_xy = geometry->transverse_half_mm; P.geo.half_z = geometry->half_length_mm;
  P.geo.bnd = bnd; P.geo.vol_mat = vm; P.geo.vol_bin = vb;
  P.mat = c->mat_dev;
  P.tab = TableView{c->g64, c->e64, c->p64, c->g32, c->e32, c->p32, c->re64, c->rp64, c->re32, c->rp32, c->Tc, c->kc};
  E.max_slots = ms;
  P.max_log = o.max_generation_log;
  P.field_T = cuts->field_T;
  P.tcut = cuts->tracking_cut_MeV;
  P.seed = o.seed; P.process_mask = o.process_mask; P.max_steps = o.max_steps; P.max_vac = o.max_vacuum_steps;
  P.steplen = (o.flags & ADEPT_FLAG_STEP_HISTOGRAM) ? steplen : nullptr;
  P.physics = o.physics;
  P.msc_f = o.msc_range_factor;
  P.chord_iter = o.field_max_iterations;
  P.delta_chord = o.delta_chord_mm;
  P.delta_int = o.delta_intersection_mm;
  P.tail_exit = o.tail_tracks > 0 ? (uint32_t)std::min<uint64_t>(4ull * (uint64_t)o.tail_tracks, 0xFFFFFFFFull) : 0u;
  c->steplen = steplen;
  // device state
  adept_ctx* c_ = cp;
  {
    adept_ctx* c = c_;
    CK(cudaMemcpyAsync(bnd, c->bnd.data(), sizeof(double) * c->bnd.size(), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(vm, c->vol_mat.data(), sizeof(int) * c->n_vol, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(vb, c->vol_bin.data(), sizeof(int) * c->n_vol, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemsetAsync(P.ctrl, 0, sizeof(Ctrl), c->stream));
    CK(cudaMemcpyAsync(qdesc, &P.q[0][0], sizeof(TrackSoA) * 6, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemsetAsync(steplen, 0, sizeof(unsigned long long) * 3 * 64, c->stream));
    CK(cudaMemsetAsync(E.state, 0, sizeof(uint32_t) * ms, c->stream));
    // the chunk status buffers are mapped: the finish pass writes them and the chunk's first
    // kernel reads the floor, with no copy in the stream between two chunks
    for (int b = 0; b < 2; ++b) {
      CK(cudaHostAlloc(&c->h_ctrl[b], sizeof(Ctrl), cudaHostAllocMapped));
      CK(cudaHostAlloc(&c->h_floor[b], sizeof(unsigned long long), cudaHostAllocMapped));
      CK(cudaHostAlloc(&c->h_done[b], sizeof(uint32_t) * ms, cudaHostAllocMapped));
      memset(c->h_ctrl[b], 0, sizeof(Ctrl));
      *c->h_floor[b] = 0;
      void* d = nullptr;
      CK(cudaHostGetDevicePointer(&d, c->h_ctrl[b], 0));
      P.h_ctrl[b] = static_cast<Ctrl*>(d);
      CK(cudaHostGetDevicePointer(&d, c->h_done[b], 0));
      P.h_done[b] = static_cast<uint32_t*>(d);
      CK(cudaHostGetDevicePointer(&d, c->h_floor[b], 0));
      P.h_floor[b] = static_cast<const unsigned long long*>(d);
      CK(cudaEventCreateWithFlags(&c->status_ev[b], cudaEventDisableTiming));
    }
    CK(cudaEventCreateWithFlags(&c->stage_ev, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&c->out_ev, cudaEventDisableTiming));
    CK(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&c->submit_stream, cudaStreamNonBlocking));
    for (int j = 0; j < 2; ++j) {
      CK(cudaStreamCreateWithFlags(&c->side[j], cudaStreamNonBlocking));
      CK(cudaEventCreateWithFlags(&c->join[j], cudaEventDisableTiming));
    }
    CK(cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming));
    CK(cudaStreamCreateWithFlags(&c->tstream, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&c->bstream, cudaStreamNonBlocking));
    for (int j = 0; j < 3; ++j) CK(cudaEventCreateWithFlags(&c->kdone[j], cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&c->tjoin, cudaEventDisableTiming));
    CK(cudaStreamSynchronize(c->stream));
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // kernel variant per species: register cap for this many resident 256-thread blocks per SM
    c->block = o.block_size;
    for (int sp = 0; sp < 3; ++sp) {
      int mb = o.blocks_per_sm_species[sp] > 0 ? o.blocks_per_sm_species[sp] : o.blocks_per_sm;
      if (mb <= 0) mb = o.precision ? 3 : 2;
      c->minb[sp] = std::min(4, mb);
      int bps = transport_max_blocks_per_sm(o.precision, sp, c->minb[sp], o.block_size, transport_variant(P));
      c->grid[sp] = sms * (bps < 1 ? 1 : bps);
    }
    if (o.fused) {
      int mb = o.blocks_per_sm > 0 ? o.blocks_per_sm : (o.precision ? 2 : 1);
      c->fminb = std::min(4, mb);
      const int bps = fused_max_blocks_per_sm(o.precision, c->fminb, o.block_size, transport_variant(P));
      c->fgrid = sms * (bps < 1 ? 1 : bps);
    }
  }
  c->slots.init(ms);
  c->slot_req.assign(ms, nullptr);
  *out = c.release();
  return ADEPT_OK;
}

extern "C" int adept_build_tables(adept_ctx* c) {
  if (!c) return ADEPT_EINVAL;
  const std::vector<double>& in = c->mat_rec;
  CK(cudaMemcpyAsync(c->mat_in, in.data(), sizeof(double) * in.size(), cudaMemcpyHostToDevice, c->stream));
  CK(launch_build_tables(c->P, c->mat_in, c->n_mat, c->range_cut, c->mat_dev, c->scratch, c->g64, c->e64, c->p64,
                         c->g32, c->e32, c->p32, c->re64, c->rp64, c->re32, c->rp32, c->Tc, c->kc, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->stats.launches += 6;
  c->built = true;
  return ADEPT_OK;
}

// event numbering of a request: events in first-appearance order, tracks numbered 1, 2, ...
// within their event
template <class FE, class FP, class FX>
static int prepare_request(adept_ctx* c, Request& r, FE ev_at, FP pdg_at, FX e_at) {
  // (before the table below, whose size follows n: it must stay under half full)
  if (r.n > c->stage_cap)
    return fail(c, ADEPT_EINVAL, "request of %zu tracks exceeds the staging capacity %zu", r.n, c->stage_cap);
  // event number -> index into r.keys: open addressing in a power-of-two table of at least 2n
  // slots (tv holds index + 1, 0 = empty); consecutive tracks of one event skip the lookup
  int bits = 4;
  while (((size_t)1 << bits) < 2 * r.n && bits < 31) ++bits;
  const uint32_t tmask = (1u << bits) - 1u;
  std::vector<uint32_t> tk((size_t)1 << bits), tv((size_t)1 << bits, 0u);
  std::vector<uint32_t> count;
  r.meta.resize(2 * r.n);
  r.energy = 0.0;
  uint32_t last_ev = 0, last_k = 0xFFFFFFFFu;
  for (size_t i = 0; i < r.n; ++i) {
    const uint32_t ev = ev_at(i);
    uint32_t k;
    if (ev == last_ev && last_k != 0xFFFFFFFFu) {
      k = last_k;
    } else {
      uint32_t h = (ev * 2654435761u) >> (32 - bits);
      while (tv[h] != 0u && tk[h] != ev) h = (h + 1u) & tmask;
      if (tv[h] == 0u) {
        k = (uint32_t)r.keys.size();
        tk[h] = ev;
        tv[h] = k + 1u;
        r.keys.push_back(ev);
        count.push_back(0);
      } else {
        k = tv[h] - 1u;
      }
      last_ev = ev;
      last_k = k;
    }
    r.meta[2 * i] = k;
    r.meta[2 * i + 1] = ++count[k];
    const int32_t p = pdg_at(i);
    const double e = e_at(i);
    if (p != 22 && p != 11 && p != -11) return fail(c, ADEPT_EINVAL, "track %zu: pdg %d is not e-, e+ or gamma", i, p);
    if (!(e >= 0.0 && e <= 1e6)) return fail(c, ADEPT_EINVAL, "track %zu: energy %g outside [0, 1e6] MeV", i, e);
    r.energy += e + (p == -11 ? 2 * 0.51099895 : 0.0);
  }
  if (r.keys.size() > c->opt.max_events) return fail(c, ADEPT_EINVAL, "request has more events than event slots");
  return ADEPT_OK;
}

static int enqueue(adept_ctx* c, std::unique_ptr<Request> r, uint32_t* request_id) {
  std::lock_guard<std::mutex> lk(c->mu);
  r->id = c->next_id++;
  if (c->next_id == 0) c->next_id = 1;
  r->t_submit = Clock::now();
  *request_id = r->id;
  if (r->n == 0) {
    r->state = 2;
    r->t_done = r->t_submit;
    c->reqs.emplace(r->id, std::move(r));
    c->cv.notify_all();
    return ADEPT_OK;
  }
  c->pending.push_back(r->id);
  c->reqs.emplace(r->id, std::move(r));
  return ADEPT_OK;
}

extern "C" int adept_submit(adept_ctx* c, const adept_track* host_tracks, size_t n, uint32_t* request_id) {
  if (!c || !request_id || (n && !host_tracks)) return ADEPT_EINVAL;
  auto r = std::make_unique<Request>();
  r->n = n;
  r->host.assign(host_tracks, host_tracks + n);
  const adept_track* h = r->host.data();
  for (size_t i = 0; i < n; ++i) {
    const double* d = h[i].dir;
    const double nn = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (!(fabs(nn - 1.0) < 1e-6)) return fail(c, ADEPT_EINVAL, "track %zu: direction is not a unit vector", i);
  }
  int rc = prepare_request(
      c, *r, [&](size_t i) { return h[i].event; }, [&](size_t i) { return h[i].pdg; },
      [&](size_t i) { return h[i].E_kin_MeV; });
  if (rc) return rc;
  return enqueue(c, std::move(r), request_id);
}

extern "C" int adept_submit_device(adept_ctx* c, const void* dev_tracks, size_t n, uint32_t* request_id) {
  if (!c || !request_id || (n && !dev_tracks)) return ADEPT_EINVAL;
  auto r = std::make_unique<Request>();
  r->n = n;
  r->dev = static_cast<const adept_track*>(dev_tracks);
  std::vector<uint32_t> ev(n);
  std::vector<int32_t> pdg(n);
  std::vector<double> E(n);
  if (n) {
    // read back the tracks in one contiguous copy into pinned memory and keep the three fields
    // the host needs for numbering and admission (three strided copies of 4- and 8-byte rows
    // took 0.5 ms for 10^4 tracks); on a stream of its own: a producer must not wait for the
    // transport's queued work
    cudaStream_t ss = c->submit_stream;
    std::lock_guard<std::mutex> lk(c->submit_mu);
    const size_t bytes = sizeof(adept_track) * n;
    if (c->h_sub_bytes < bytes) {
      if (c->h_sub) CK(cudaFreeHost(c->h_sub));
      c->h_sub = nullptr;
      c->h_sub_bytes = 0;
      const size_t want = std::max(bytes, (size_t)1 << 20);
      CK(cudaHostAlloc(&c->h_sub, want, cudaHostAllocDefault));
      c->h_sub_bytes = want;
    }
    CK(cudaMemcpyAsync(c->h_sub, dev_tracks, bytes, cudaMemcpyDeviceToHost, ss));
    CK(cudaStreamSynchronize(ss));
    const adept_track* h = reinterpret_cast<const adept_track*>(c->h_sub);
    for (size_t i = 0; i < n; ++i) { ev[i] = h[i].event; pdg[i] = h[i].pdg; E[i] = h[i].E_kin_MeV; }
  }
  int rc = prepare_request(
      c, *r, [&](size_t i) { return ev[i]; }, [&](size_t i) { return pdg[i]; }, [&](size_t i) { return E[i]; });
  if (rc) return rc;
  return enqueue(c, std::move(r), request_id);
}

// ---------------------------------------------------------------- admission
static int ensure_host_stage(adept_ctx* c, size_t bytes) {
  if (c->h_stage_bytes >= bytes) return ADEPT_OK;
  if (c->h_stage) cudaFreeHost(c->h_stage);
  c->h_stage = nullptr;
  c->h_stage_bytes = 0;
  const size_t want = std::max(bytes, (size_t)1 << 20);
  CK(cudaHostAlloc(&c->h_stage, want, cudaHostAllocDefault));
  c->h_stage_bytes = want;
  return ADEPT_OK;
}

// Admit pending requests in arrival order while event slots, staging room and the
// track budget allow (an idle device always admits the next request).
static int admit(adept_ctx* c) {
  size_t used = 0;
  const double budget = (double)c->P.cap / c->opt.tracks_per_MeV;
  for (;;) {
    Request* r;
    {
      std::lock_guard<std::mutex> lk(c->mu);
      if (c->pending.empty()) return ADEPT_OK;
      r = c->reqs.at(c->pending.front()).get();
      if (used + r->n > c->stage_cap) return ADEPT_OK;
      if (c->in_flight > 0 && c->energy_in_flight + r->energy > budget) return ADEPT_OK;
      uint32_t base;
      if (!c->slots.alloc((uint32_t)r->keys.size(), &base)) return ADEPT_OK;
      r->slot_base = base;
      c->pending.pop_front();
      r->state = 1;
      r->remaining = (uint32_t)r->keys.size();
      for (uint32_t k = 0; k < r->remaining; ++k) c->slot_req[base + k] = r;
      c->energy_in_flight += r->energy;
      c->in_flight++;
      c->admit_est += (uint64_t)(r->energy * c->opt.tracks_per_MeV) + r->n;
    }
    const size_t nk = r->keys.size();
    // pinned staging: tracks (host submissions), meta, keys
    const size_t tb = r->dev ? 0 : sizeof(adept_track) * r->n;
    const size_t mb = sizeof(uint32_t) * 2 * r->n, kb = sizeof(uint32_t) * nk;
    int rc = ensure_host_stage(c, tb + mb + kb + 64);
    if (rc) return rc;
    CK(cudaEventSynchronize(c->stage_ev));  // the pinned buffer may still feed an earlier copy
    char* h = c->h_stage;
    if (tb) memcpy(h, r->host.data(), tb);
    memcpy(h + tb, r->meta.data(), mb);
    memcpy(h + tb + mb, r->keys.data(), kb);
    TrackIn* dst = c->stage + used;
    const TrackIn* src = r->dev ? reinterpret_cast<const TrackIn*>(r->dev) : dst;
    if (tb) CK(cudaMemcpyAsync(dst, h, tb, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->stage_meta + 2 * used, h + tb, mb, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->stage_keys, h + tb + mb, kb, cudaMemcpyHostToDevice, c->stream));
    CK(cudaEventRecord(c->stage_ev, c->stream));
    CK(launch_admit(c->P, r->slot_base, c->stage_keys, (int)nk, c->stream));
    CK(launch_init_primaries(c->P, src, c->stage_meta + 2 * used, (int)r->n, r->slot_base, c->opt.precision, c->stream));
    c->stats.launches += 2;
    used += r->n;
  }
}

// ---------------------------------------------------------------- generation chunks
static int ensure_events(adept_ctx* c, int n) {
  while ((int)c->ev.size() < n) {
    cudaEvent_t a;
    CK(cudaEventCreate(&a));
    c->ev.push_back(a);
  }
  return ADEPT_OK;
}

static bool timing(const adept_ctx* c) { return (c->opt.flags & (ADEPT_FLAG_TIME_STEPS | ADEPT_FLAG_TIME_SPECIES)) != 0; }
static bool timing_species(const adept_ctx* c) { return (c->opt.flags & ADEPT_FLAG_TIME_SPECIES) != 0; }

// the generations of one chunk; timing events of status buffer b are ev[4 G b ...]
// Timing events are recorded on tstream: the start one after the generation's fork, an end
// one after each kernel it times. tstream joins the chain only at the end of the chunk, so
// the records never delay the next generation.
static cudaError_t enqueue_generations(adept_ctx* c, int gens, int b, bool captured) {
  cudaError_t e = launch_open_chunk(c->P, b, c->stream);
  // inside a capture a timing record must be an external event node; outside, a plain record
  const unsigned rf = captured ? cudaEventRecordExternal : cudaEventRecordDefault;
  const bool T = timing(c), TS = timing_species(c);
  cudaEvent_t* ev = c->ev.empty() ? nullptr : c->ev.data() + 4 * gens * b;
  cudaStream_t ts = c->tstream;
  // record end event slot `at` on tstream once `done` (recorded on stream s) has happened
  auto time_end = [&](cudaStream_t s, cudaEvent_t done, int at) {
    if (e == cudaSuccess) e = cudaEventRecord(done, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ts, done, 0);
    if (e == cudaSuccess) e = cudaEventRecordWithFlags(ev[at], ts, rf);
  };
  for (int k = 0; k < gens && e == cudaSuccess; ++k) {
    e = cudaEventRecord(c->fork, c->stream);
    if (T) {
      if (e == cudaSuccess) e = cudaStreamWaitEvent(ts, c->fork, 0);
      if (e == cudaSuccess) e = cudaEventRecordWithFlags(ev[4 * k], ts, rf);
    }
    if (c->opt.fused) {  // one kernel per generation
      if (e == cudaSuccess)
        e = launch_fused_generation(c->P, (uint32_t)k, c->opt.precision, c->fminb, c->fgrid, c->block, k > 0,
                                    c->stream);
      if (T) time_end(c->stream, c->kdone[0], 4 * k + 1);
      continue;
    }
    // fork e- (main stream), e+ and gamma (side streams), join
    for (int j = 0; j < 2 && e == cudaSuccess; ++j) e = cudaStreamWaitEvent(c->side[j], c->fork, 0);
    cudaStream_t st[3] = {c->side[1], c->stream, c->side[0]};  // gamma, e-, e+
    // launch order gamma, e+, e-: on the 10 GeV showers 2.4 % faster than e-, e+, gamma with
    // the current kernels (e+ at 3 blocks per SM); the order mattered the other way round when
    // the e+ kernel ran at 2
    for (int sp : {0, 2, 1}) {
      if (e == cudaSuccess)
        e = launch_transport(c->P, (uint32_t)k, c->opt.precision, sp, c->minb[sp], c->grid[sp], c->block, k > 0,
                             st[sp]);
      if (TS) time_end(st[sp], c->kdone[sp], 4 * k + 1 + sp);
    }
    for (int j = 0; j < 2 && e == cudaSuccess; ++j) e = cudaEventRecord(c->join[j], c->side[j]);
    for (int j = 0; j < 2 && e == cudaSuccess; ++j) e = cudaStreamWaitEvent(c->stream, c->join[j], 0);
    // without the per-species split: one end event once all three kernels have ended
    if (T && !TS) time_end(c->stream, c->kdone[0], 4 * k + 1);
  }
  if (T && e == cudaSuccess) {
    e = cudaEventRecord(c->tjoin, ts);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, c->tjoin, 0);
  }
  if (e == cudaSuccess) e = launch_finish(c->P, b, gens, c->stream);
  return e;
}

// Below adept_options.tail_tracks live tracks a generation is dominated by its launch, and
// a tail chunk trades the programmatic launch between generations (about 5 us a generation
// on GB300) for stopping exactly when the last track dies (a fixed chunk runs to its end, and
// one more is queued behind it: at the end of a transport the rest of the one and all of the
// other run on empty queues). So tail chunks are
// kept for the decay at the end: fewer live tracks than tail_tracks and than a kTailDecay-th
// of the peak since the queues were last empty. A tail chunk runs at most
// graph_generations generations, like a fixed one, so the status is read as often.
constexpr uint64_t kTailDecay = 8;

// A tail chunk: open (condition = live tracks) -> while (condition) { one generation (the
// three species kernels, or the fused kernel) -> step (++tail_k, condition = live tracks,
// fewer than 4 tail_tracks, and tail_k < graph_generations) } -> end of chunk with the count
// the loop left. No timing records (event nodes are not allowed in a conditional body).
static int capture_tail_graph(adept_ctx* c, int b) {
  cudaGraph_t g = nullptr;
  cudaGraphConditionalHandle h;
  cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return fail(c, ADEPT_ECUDA, "tail capture: %s", cudaGetErrorString(e));
  cudaStreamCaptureStatus cs;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  e = launch_open_chunk(c->P, b, c->stream);
  if (e == cudaSuccess) e = cudaStreamGetCaptureInfo(c->stream, &cs, nullptr, &g, nullptr, nullptr, nullptr);
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault);
  if (e == cudaSuccess) e = launch_tail_open(c->P, h, c->stream);
  if (e == cudaSuccess) e = cudaStreamGetCaptureInfo(c->stream, &cs, nullptr, &g, &deps, nullptr, &ndeps);
  cudaGraphNode_t loop = nullptr;
  cudaGraph_t body = nullptr;
  if (e == cudaSuccess) {
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    e = cudaGraphAddNode(&loop, g, deps, nullptr, ndeps, &cp);
    if (e == cudaSuccess) body = cp.conditional.phGraph_out[0];
  }
  if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(c->stream, &loop, nullptr, 1, cudaStreamSetCaptureDependencies);
  // the loop body: one generation, captured on a stream of its own
  if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(c->bstream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaStream_t s0 = c->bstream;
    if (c->opt.fused) {
      e = launch_fused_generation(c->P, kGkDevice, c->opt.precision, c->fminb, c->fgrid, c->block, false, s0);
    } else {
      e = cudaEventRecord(c->fork, s0);
      for (int j = 0; j < 2 && e == cudaSuccess; ++j) e = cudaStreamWaitEvent(c->side[j], c->fork, 0);
      cudaStream_t st[3] = {c->side[1], s0, c->side[0]};  // gamma, e-, e+
      for (int sp : {0, 2, 1})
        if (e == cudaSuccess) e = launch_transport(c->P, kGkDevice, c->opt.precision, sp, c->minb[sp], c->grid[sp], c->block, false, st[sp]);
      for (int j = 0; j < 2 && e == cudaSuccess; ++j) e = cudaEventRecord(c->join[j], c->side[j]);
      for (int j = 0; j < 2 && e == cudaSuccess; ++j) e = cudaStreamWaitEvent(s0, c->join[j], 0);
    }
    if (e == cudaSuccess) e = launch_tail_step(c->P, h, (uint32_t)c->opt.graph_generations, s0);
    cudaGraph_t bg = nullptr;
    const cudaError_t e3 = cudaStreamEndCapture(s0, &bg);
    if (e == cudaSuccess) e = e3;
  }
  if (e == cudaSuccess) e = launch_finish(c->P, b, kGkDevice, c->stream);
  cudaGraph_t out = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(c->stream, &out);
  if (e != cudaSuccess) {
    if (out) cudaGraphDestroy(out);
    return fail(c, ADEPT_ECUDA, "tail graph capture: %s", cudaGetErrorString(e));
  }
  if (e2 != cudaSuccess) return fail(c, ADEPT_ECUDA, "tail graph capture end: %s", cudaGetErrorString(e2));
  e = cudaGraphInstantiate(&c->tgraph[b], out, 0);
  cudaGraphDestroy(out);
  if (e != cudaSuccess) return fail(c, ADEPT_ECUDA, "tail graph instantiate: %s", cudaGetErrorString(e));
  return ADEPT_OK;
}

static int capture_graph(adept_ctx* c, int gens, int b) {
  cudaGraph_t g;
  CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = enqueue_generations(c, gens, b, true);
  cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
  if (e != cudaSuccess) return fail(c, ADEPT_ECUDA, "graph capture: %s", cudaGetErrorString(e));
  if (e2 != cudaSuccess) return fail(c, ADEPT_ECUDA, "graph capture end: %s", cudaGetErrorString(e2));
  e = cudaGraphInstantiate(&c->graph[b], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(c, ADEPT_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
  c->graph_gens = gens;
  return ADEPT_OK;
}

// Queue one chunk of generations and the copy of its status into buffer b; returns at once.
static int launch_chunk(adept_ctx* c, int b) {
  const int G = c->opt.graph_generations;
  const int gens = G > 0 ? G : 1;
  // the outgoing ring may be written up to the host's read position plus its capacity (read
  // by the chunk's first kernel from this pinned word)
  *c->h_floor[b] = c->leak_read;
  if (timing(c)) {
    int rc = ensure_events(c, 8 * gens);
    if (rc) return rc;
  }
  const uint64_t live = c->last_live + (c->admit_est - c->admit_seen);
  c->tail[b] = G > 0 && c->opt.tail_tracks > 0 && live < (uint64_t)c->opt.tail_tracks &&
               live * kTailDecay < c->peak_live;
  c->admit_mark[b] = c->admit_est;
  if (c->tail[b]) {
    if (!c->tgraph[b]) {
      int rc = capture_tail_graph(c, b);
      if (rc) return rc;
    }
    CK(cudaGraphLaunch(c->tgraph[b], c->stream));
    c->stats.launches += 5;  // chunk open, loop open, end of chunk, mark, finish; the loop's kernels once read back
  } else if (G > 0) {
    if (!c->graph[b]) {
      int rc = capture_graph(c, G, b);
      if (rc) return rc;
    }
    CK(cudaGraphLaunch(c->graph[b], c->stream));
    c->stats.launches += (c->opt.fused ? 1 : 3) * gens + 4;  // and chunk open, end, mark, finish
  } else {
    CK(enqueue_generations(c, 1, b, false));
    c->stats.launches += (c->opt.fused ? 1 : 3) * gens + 4;  // and chunk open, end, mark, finish
  }
  // the chunk's finish pass has written its status and done list to h_ctrl[b] and h_done[b]
  CK(cudaEventRecord(c->status_ev[b], c->stream));
  return ADEPT_OK;
}

// Wait for chunk b and account its timing events.
static int wait_chunk(adept_ctx* c, int b) {
  CK(cudaEventSynchronize(c->status_ev[b]));
  if (c->tail[b]) {  // the loop's generations: the species kernels (or the fused one) and a step kernel
    c->stats.launches += (uint64_t)c->h_ctrl[b]->tail_k * ((c->opt.fused ? 1 : 3) + 1);
    return ADEPT_OK;
  }
  if (timing(c)) {
    const int G = c->opt.graph_generations;
    const int gens = G > 0 ? G : 1;
    const cudaEvent_t* ev = c->ev.data() + 4 * gens * b;
    // concurrent species kernels: each one's time from the generation's fork to its end;
    // the generation's time is the longest of the three
    for (int k = 0; k < gens; ++k) {
      if (!timing_species(c)) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, ev[4 * k], ev[4 * k + 1]));
        c->stats.step_kernel_ms += ms;
        continue;
      }
      float mx = 0.f;
      for (int sp = 0; sp < 3; ++sp) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, ev[4 * k], ev[4 * k + 1 + sp]));
        c->stats.species_ms[sp] += ms;
        mx = ms > mx ? ms : mx;
      }
      c->stats.step_kernel_ms += mx;
    }
    c->stats.step_launches += gens;
  }
  return ADEPT_OK;
}

// Outgoing particles recorded up to the end of chunk b, in two halves, so that the host can
// relaunch the chunk's buffer in between: start_outgoing copies the new ring entries into
// pinned staging on copy_stream (then out_ev) and advances the host's read position, which the
// next launch hands the device as its floor; finish_outgoing waits for the copy and gives each
// particle to its request. Records the device could not write (ring full) are counted; they
// make the transport fail with ADEPT_ENOMEM like a queue overflow.
static int start_outgoing(adept_ctx* c, const Ctrl& h, int b, size_t* n_out) {
  *n_out = 0;
  const unsigned long long cap = c->P.leak_cap;
  const unsigned long long end = std::min<unsigned long long>(h.leak_count, *c->h_floor[b] + cap);
  if (end > c->leak_read) {
    const size_t n = (size_t)(end - c->leak_read);
    // pinned staging, grown by doubling (pageable memory would take the copy through a bounce
    // buffer)
    if (c->h_leak_cap < n) {
      const size_t want = std::max<size_t>(n, std::max<size_t>(2 * c->h_leak_cap, (size_t)1 << 16));
      if (c->h_leak) CK(cudaFreeHost(c->h_leak));
      c->h_leak = nullptr;
      c->h_leak_cap = 0;
      CK(cudaHostAlloc(reinterpret_cast<void**>(&c->h_leak), sizeof(LeakRec) * want, cudaHostAllocDefault));
      c->h_leak_cap = want;
    }
    const size_t start = (size_t)(c->leak_read % cap);
    const size_t first = std::min<size_t>(n, (size_t)cap - start);
    CK(cudaMemcpyAsync(c->h_leak, c->P.leak + start, sizeof(LeakRec) * first, cudaMemcpyDeviceToHost, c->copy_stream));
    if (first < n)
      CK(cudaMemcpyAsync(c->h_leak + first, c->P.leak, sizeof(LeakRec) * (n - first), cudaMemcpyDeviceToHost,
                         c->copy_stream));
    CK(cudaEventRecord(c->out_ev, c->copy_stream));
    *n_out = n;
  }
  c->leak_read = std::max<unsigned long long>(c->leak_read, h.leak_count);
  return ADEPT_OK;
}

static int finish_outgoing(adept_ctx* c, const Ctrl& h, size_t n, int* stop_rc) {
  if (n) {
    CK(cudaEventSynchronize(c->out_ev));
    // runs of consecutive records of one request: one capacity check per run (about 5 ns a
    // record: with tens of thousands a chunk, this is why it runs after the relaunch)
    std::lock_guard<std::mutex> lk(c->mu);
    for (size_t i = 0; i < n;) {
      Request* r = c->slot_req[c->h_leak[i].slot];
      size_t j = i + 1;
      while (j < n && c->slot_req[c->h_leak[j].slot] == r) ++j;
      if (r) {
        const size_t need = r->outgoing.size() + (j - i);
        if (r->outgoing.capacity() < need) r->outgoing.reserve(std::max(2 * r->outgoing.capacity(), need));
        for (size_t k = i; k < j; ++k) {
          const LeakRec& x = c->h_leak[k];
          adept_track t;
          t.pdg = x.pdg;
          t.E_kin_MeV = x.E;
          t.pos_mm[0] = x.pos[0]; t.pos_mm[1] = x.pos[1]; t.pos_mm[2] = x.pos[2];
          t.dir[0] = x.dir[0]; t.dir[1] = x.dir[1]; t.dir[2] = x.dir[2];
          t.event = r->keys[x.slot - r->slot_base];
          r->outgoing.push_back(t);
        }
      }
      i = j;
    }
  }
  if (h.leak_dropped > c->leak_dropped_seen && *stop_rc == ADEPT_OK)
    *stop_rc = fail(c, ADEPT_ENOMEM, "%llu outgoing particles exceeded the ring of %u (max_outgoing); results are "
                    "incomplete", h.leak_dropped - c->leak_dropped_seen, c->P.leak_cap);
  c->leak_dropped_seen = h.leak_dropped;
  return ADEPT_OK;
}

// a host block of at least `need` doubles for a finished request's rows: the smallest free
// pinned block that holds them, else a new pinned one, else pageable memory
static void acquire_result(adept_ctx* c, ResultBuf& rb, size_t need) {
  {
    std::lock_guard<std::mutex> lk(c->pool_mu);
    size_t best = c->pool_free.size();
    for (size_t i = 0; i < c->pool_free.size(); ++i)
      if (c->pool_free[i].second >= need && (best == c->pool_free.size() || c->pool_free[i].second < c->pool_free[best].second))
        best = i;
    if (best < c->pool_free.size()) {
      rb.p = c->pool_free[best].first;
      rb.cap = c->pool_free[best].second;
      rb.pinned = true;
      c->pool_free.erase(c->pool_free.begin() + (std::ptrdiff_t)best);
      return;
    }
  }
  const size_t cap = std::max<size_t>(need, 8192);
  double* p = nullptr;
  if (cudaHostAlloc(reinterpret_cast<void**>(&p), sizeof(double) * cap, cudaHostAllocDefault) == cudaSuccess) {
    std::lock_guard<std::mutex> lk(c->pool_mu);
    c->pool_all.push_back(p);
    rb.p = p;
    rb.cap = cap;
    rb.pinned = true;
    return;
  }
  (void)cudaGetLastError();  // a failed pinned allocation leaves no error behind
  rb.pageable.resize(need);
  rb.p = rb.pageable.data();
  rb.cap = need;
  rb.pinned = false;
}

static void release_result(adept_ctx* c, ResultBuf& rb) {
  if (rb.pinned) {
    std::lock_guard<std::mutex> lk(c->pool_mu);
    c->pool_free.emplace_back(rb.p, rb.cap);
  }
  rb.p = nullptr;
  rb.cap = 0;
  rb.pinned = false;
  std::vector<double>().swap(rb.pageable);
}

// copy a finished request's rows back and release its slots
static int complete(adept_ctx* c, Request* r) {
  const size_t nk = r->keys.size(), nb = c->n_bins;
  if (nk) {
    acquire_result(c, r->res, nk * nb + 2 * nk);
    double* h = r->res.p;
    // the rows are final: the host has waited for the chunk that finished the request (its
    // status event may since have been recorded again by a relaunch of the chunk's buffer);
    // copy them while the next chunk computes
    cudaStream_t cs = c->copy_stream;
    CK(cudaMemcpyAsync(h, c->P.evt.edep + (size_t)r->slot_base * nb, sizeof(double) * nk * nb, cudaMemcpyDeviceToHost, cs));
    CK(cudaMemcpyAsync(h + nk * nb, c->P.evt.leaked + r->slot_base, sizeof(double) * nk, cudaMemcpyDeviceToHost, cs));
    CK(cudaMemcpyAsync(h + nk * nb + nk, c->P.evt.killed + r->slot_base, sizeof(double) * nk, cudaMemcpyDeviceToHost,
                       cs));
    // a finished slot is never read again by the finish pass (state 2 or 0 are both inert)
    CK(cudaMemsetAsync(c->P.evt.state + r->slot_base, 0, sizeof(uint32_t) * nk, cs));
    CK(cudaStreamSynchronize(cs));
  }
  std::lock_guard<std::mutex> lk(c->mu);
  for (size_t k = 0; k < nk; ++k) c->slot_req[r->slot_base + k] = nullptr;
  c->slots.release(r->slot_base, (uint32_t)nk);
  c->energy_in_flight -= r->energy;
  if (c->energy_in_flight < 0) c->energy_in_flight = 0;
  c->in_flight--;
  r->state = 2;
  r->t_done = Clock::now();
  r->dev = nullptr;
  std::vector<adept_track>().swap(r->host);
  std::vector<uint32_t>().swap(r->meta);
  c->stats.requests_done++;
  c->cv.notify_all();
  return ADEPT_OK;
}

// The host keeps at most two chunks queued: while chunk b runs, chunk b^1 is already
// behind it in the stream, so the GPU does not idle while the host reads b's status; once b
// has ended, its buffer is relaunched before the host processes that status (below). A
// speculative chunk that finds empty queues costs only empty launches.
extern "C" int adept_transport(adept_ctx* c, uint64_t timeout_us) {
  if (!c) return ADEPT_EINVAL;
  if (!c->built) return fail(c, ADEPT_ESTATE, "adept_build_tables has not run");
  const auto t0 = Clock::now();
  std::vector<uint32_t> done;
  std::vector<Request*> finished;
  int idle_chunks = 0;
  bool queued[2] = {false, false};
  int b = 0;
  int stop_rc = ADEPT_OK;  // set on timeout or overflow: launch nothing more, drain, return it
  for (;;) {
    bool work = false;
    if (stop_rc == ADEPT_OK) {
      int rc = admit(c);
      if (rc) return rc;
      std::lock_guard<std::mutex> lk(c->mu);
      work = c->in_flight > 0 || !c->pending.empty();
    }
    if (work) {
      for (int k : {b, b ^ 1}) {
        if (!queued[k]) {
          int rc = launch_chunk(c, k);
          if (rc) return rc;
          queued[k] = true;
        }
      }
    }
    if (!queued[b]) {
      if (!queued[b ^ 1]) return stop_rc == ADEPT_OK ? ADEPT_OK : stop_rc;
      b ^= 1;
      continue;
    }
    int rc = wait_chunk(c, b);
    if (rc) return rc;
    queued[b] = false;
    // copies of the chunk's status and done list: a relaunch of buffer b rewrites both
    const Ctrl h = *c->h_ctrl[b];
    for (int k = 0; k < 3; ++k) { c->stats.steps[k] = h.steps[k]; c->stats.secondaries[k] = h.created[k]; }
    c->stats.generations = h.generations;
    c->stats.overflow = h.overflow;
    size_t n_out = 0;
    rc = start_outgoing(c, h, b, &n_out);
    if (rc) return rc;
    const uint32_t nd = std::min<uint32_t>(h.done_count[b], (uint32_t)c->slot_req.size());
    done.assign(c->h_done[b], c->h_done[b] + nd);
    const uint32_t live = h.count[h.gen % 3][0].n + h.count[h.gen % 3][1].n + h.count[h.gen % 3][2].n;
    c->last_live = live;
    c->admit_seen = c->admit_mark[b];
    c->peak_live = live ? std::max<uint64_t>(c->peak_live, live) : 0;
    // While tracks are live and no request waits for admission, relaunch buffer b at once, so
    // that the host's processing of this status (outgoing particles, finished events) overlaps
    // the next chunk instead of delaying the launch of the one after it: on the 10 GeV showers
    // it took up to 0.5 ms, longer than the short chunks near the end. The relaunched chunk's
    // outgoing-ring floor counts this chunk's records as read, so it waits for their copy.
    // With requests waiting, completions free their slots first and the launch follows the
    // admission at the top of the loop.
    bool early = false;
    if (stop_rc == ADEPT_OK && live > 0) {
      std::lock_guard<std::mutex> lk(c->mu);
      early = c->pending.empty();
    }
    if (early) {
      if (n_out) CK(cudaStreamWaitEvent(c->stream, c->out_ev, 0));
      rc = launch_chunk(c, b);
      if (rc) return rc;
      queued[b] = true;
    }
    rc = finish_outgoing(c, h, n_out, &stop_rc);
    if (rc) return rc;
    // the finished events: each slot's request directly, under one lock for the whole list
    // (a lookup and a lock per slot took longer than the next chunk ran once thousands of
    // events finished in one chunk, and the GPU waited for the chunk after it)
    finished.clear();
    {
      std::lock_guard<std::mutex> lk(c->mu);
      for (uint32_t s : done) {
        Request* r = s < c->slot_req.size() ? c->slot_req[s] : nullptr;
        if (r && r->state == 1 && r->remaining > 0 && --r->remaining == 0) finished.push_back(r);
      }
    }
    for (Request* r : finished) {
      rc = complete(c, r);
      if (rc) return rc;
    }
    idle_chunks = (live == 0 && done.empty()) ? idle_chunks + 1 : 0;
    if (idle_chunks > 8) {
      std::lock_guard<std::mutex> lk(c->mu);
      if (c->in_flight > 0) return fail(c, ADEPT_ESTATE, "requests in flight but no live tracks (internal error)");
    }
    if (h.overflow && stop_rc == ADEPT_OK)
      stop_rc = fail(c, ADEPT_ENOMEM, "%llu tracks exceeded the queue capacity %u; results are incomplete",
                     (unsigned long long)h.overflow, c->P.cap);
    if (timeout_us && stop_rc == ADEPT_OK) {
      const auto us = std::chrono::duration_cast<std::chrono::microseconds>(Clock::now() - t0).count();
      if ((uint64_t)us >= timeout_us)
        stop_rc = fail(c, ADEPT_ETIMEOUT, "transport stopped after %llu us", (unsigned long long)us);
    }
    b ^= 1;
  }
}

// ---------------------------------------------------------------- results
extern "C" int adept_poll(adept_ctx* c, uint32_t id) {
  if (!c) return ADEPT_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  auto it = c->reqs.find(id);
  if (it == c->reqs.end()) return ADEPT_ENOTFOUND;
  return it->second->state == 2 ? 1 : 0;
}

extern "C" int adept_wait(adept_ctx* c, uint32_t id, uint64_t timeout_us) {
  if (!c) return ADEPT_EINVAL;
  std::unique_lock<std::mutex> lk(c->mu);
  auto pred = [&] {
    auto it = c->reqs.find(id);
    return it == c->reqs.end() || it->second->state == 2;
  };
  if (timeout_us == 0) c->cv.wait(lk, pred);
  else if (!c->cv.wait_for(lk, std::chrono::microseconds(timeout_us), pred)) return ADEPT_ETIMEOUT;
  return c->reqs.count(id) ? ADEPT_OK : ADEPT_ENOTFOUND;
}

// copy s[lo, hi) to d[lo, hi) and return its sum, with eight partial sums
static double copy_sum(const double* s, double* d, size_t lo, size_t hi) {
  double a[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  size_t i = lo;
  for (; i + 8 <= hi; i += 8)
    for (int j = 0; j < 8; ++j) {
      const double v = s[i + j];
      d[i + j] = v;
      a[j] += v;
    }
  for (; i < hi; ++i) {
    d[i] = s[i];
    a[0] += s[i];
  }
  return ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
}

extern "C" int adept_get_scoring(adept_ctx* c, uint32_t id, double* edep_out, size_t n, adept_result* meta) {
  if (!c) return ADEPT_EINVAL;
  std::unique_ptr<Request> r;
  {
    std::lock_guard<std::mutex> lk(c->mu);
    auto it = c->reqs.find(id);
    if (it == c->reqs.end()) return ADEPT_ENOTFOUND;
    if (it->second->state != 2) return ADEPT_EBUSY;
    const size_t need = it->second->keys.size() * (size_t)c->n_bins;
    if (need && (!edep_out || n < need)) return fail(c, ADEPT_EINVAL, "edep_out holds %zu doubles, %zu needed", n, need);
    r = std::move(it->second);
    c->reqs.erase(it);
  }
  // copy the rows out and sum them in one pass, with eight partial sums (one dependent chain
  // of 10^6 additions took about a millisecond); a large request in up to four parts on as
  // many threads (one pass over 8 MB took 0.5 ms of a 36 ms headline step on one core). The
  // parts depend only on the request's size and their sums combine in a fixed order, so the
  // result does not depend on how many threads could be started.
  const size_t nk = r->keys.size(), m = nk * (size_t)c->n_bins;
  double d = 0, l = 0, k = 0;
  if (nk) {
    const double* s = r->res.p;
    constexpr size_t kPart = (size_t)1 << 17;  // doubles (1 MB) a part at least
    const size_t np = std::min<size_t>(4, std::max<size_t>(1, m / kPart));
    const size_t step = (m + np - 1) / np;
    double part[4] = {0, 0, 0, 0};
    auto run = [&](size_t t) { part[t] = copy_sum(s, edep_out, std::min(m, t * step), std::min(m, (t + 1) * step)); };
    std::thread th[3];
    size_t started = 0;
    try {
      for (size_t t = 1; t < np; ++t) {
        th[t - 1] = std::thread(run, t);
        ++started;
      }
    } catch (...) {  // no thread to spare: the parts not started run here
    }
    run(0);
    for (size_t t = started + 1; t < np; ++t) run(t);
    for (size_t t = 0; t < started; ++t) th[t].join();
    d = (part[0] + part[1]) + (part[2] + part[3]);
    for (size_t e = 0; e < nk; ++e) {
      l += s[m + e];
      k += s[m + nk + e];
    }
    release_result(c, r->res);
  }
  if (meta) {
    meta->request = r->id;
    meta->n_events = (uint32_t)nk;
    meta->n_bins = (uint32_t)c->n_bins;
    meta->deposited_MeV = d;
    meta->leaked_MeV = l;
    meta->killed_MeV = k;
    meta->latency_us = std::chrono::duration<double, std::micro>(r->t_done - r->t_submit).count();
  }
  return ADEPT_OK;
}

extern "C" int adept_get_leaked(adept_ctx* c, uint32_t id, adept_track* out, size_t n_max, size_t* n_out) {
  if (!c || !n_out || (n_max && !out)) return ADEPT_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  auto it = c->reqs.find(id);
  if (it == c->reqs.end()) return ADEPT_ENOTFOUND;
  const Request& r = *it->second;
  if (r.state != 2) return ADEPT_EBUSY;
  *n_out = r.outgoing.size();
  const size_t n = std::min(n_max, r.outgoing.size());
  if (n) memcpy(out, r.outgoing.data(), sizeof(adept_track) * n);
  return ADEPT_OK;
}

extern "C" int adept_get_stats(adept_ctx* c, adept_stats* out) {
  if (!c || !out) return ADEPT_EINVAL;
  *out = c->stats;
  return ADEPT_OK;
}

extern "C" int adept_get_generation_log(adept_ctx* c, uint32_t* host_out, size_t n_max) {
  if (!c || (n_max && !host_out)) return ADEPT_EINVAL;
  Ctrl h;
  CK(cudaMemcpyAsync(&h, c->P.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  const size_t n = std::min<size_t>(h.log_n, n_max);
  if (n) {
    CK(cudaMemcpyAsync(host_out, c->P.gen_log, sizeof(uint32_t) * 3 * n, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  return (int)n;
}

extern "C" int adept_reset_generation_log(adept_ctx* c) {
  if (!c) return ADEPT_EINVAL;
  CK(cudaMemsetAsync(&c->P.ctrl->log_n, 0, sizeof(uint32_t), c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return ADEPT_OK;
}

extern "C" int adept_get_step_histogram(adept_ctx* c, uint64_t* host_out) {
  if (!c || !host_out) return ADEPT_EINVAL;
  CK(cudaMemcpyAsync(host_out, c->steplen, sizeof(uint64_t) * 3 * 64, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return ADEPT_OK;
}

extern "C" int adept_get_cuts(adept_ctx* c, int32_t m, double* e_cut, double* gamma_cut) {
  if (!c || !e_cut || !gamma_cut || m < 0 || m >= c->n_mat) return ADEPT_EINVAL;
  if (!c->built) return fail(c, ADEPT_ESTATE, "tables not built");
  CK(cudaMemcpy(e_cut, c->Tc + m, sizeof(double), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(gamma_cut, c->kc + m, sizeof(double), cudaMemcpyDeviceToHost));
  return ADEPT_OK;
}

static int ntab(int s) { return s == 0 ? kNTabG : (s == 1 ? kNTabE : kNTabP); }

extern "C" int adept_get_table(adept_ctx* c, int32_t s, int32_t t, int32_t m, int32_t prec, double* host_out) {
  if (!c || !host_out || s < 0 || s > 2 || t < 0 || t >= ntab(s) || m < 0 || m >= c->n_mat || (prec != 0 && prec != 1))
    return ADEPT_EINVAL;
  if (!c->built) return fail(c, ADEPT_ESTATE, "tables not built");
  const int nt = ntab(s);
  const size_t off = ((size_t)m * kNNode) * nt;
  if (prec == 0) {
    std::vector<double2> rec((size_t)kNNode * nt);
    const double2* src = (s == 0 ? c->g64 : (s == 1 ? c->e64 : c->p64)) + off;
    CK(cudaMemcpy(rec.data(), src, sizeof(double2) * rec.size(), cudaMemcpyDeviceToHost));
    for (int i = 0; i < kNNode; ++i) host_out[i] = rec[(size_t)i * nt + t].x;
  } else {
    std::vector<float2> rec((size_t)kNNode * nt);
    const float2* src = (s == 0 ? c->g32 : (s == 1 ? c->e32 : c->p32)) + off;
    CK(cudaMemcpy(rec.data(), src, sizeof(float2) * rec.size(), cudaMemcpyDeviceToHost));
    for (int i = 0; i < kNNode; ++i) host_out[i] = rec[(size_t)i * nt + t].x;
  }
  return ADEPT_OK;
}

// ---------------------------------------------------------------- probes
template <class F>
static int probe_run(adept_ctx* c, size_t in_bytes_per, size_t out_bytes_per, size_t n, F fn) {
  const size_t per = in_bytes_per + out_bytes_per + 64;
  const size_t chunk = std::max<size_t>(1, c->probe_bytes / per / 2);
  for (size_t b = 0; b < n; b += chunk) {
    const size_t k = std::min(chunk, n - b);
    int rc = fn(b, k);
    if (rc) return rc;
  }
  return ADEPT_OK;
}

extern "C" int adept_probe_philox(adept_ctx* c, const uint32_t key[2], const uint32_t* host_ctr, size_t n,
                                  uint32_t* host_out) {
  if (!c || !key || (n && (!host_ctr || !host_out))) return ADEPT_EINVAL;
  return probe_run(c, 16, 16, n, [&](size_t b, size_t k) {
    uint32_t* din = reinterpret_cast<uint32_t*>(c->probe);
    uint32_t* dout = din + 4 * k;
    CK(cudaMemcpyAsync(din, host_ctr + 4 * b, 16 * k, cudaMemcpyHostToDevice, c->stream));
    CK(launch_probe_philox(din, (int)k, key[0], key[1], dout, c->stream));
    CK(cudaMemcpyAsync(host_out + 4 * b, dout, 16 * k, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return ADEPT_OK;
  });
}

extern "C" int adept_probe_interp(adept_ctx* c, int32_t s, int32_t t, int32_t m, int32_t prec, const double* host_E,
                                  size_t n, double* host_out) {
  if (!c || s < 0 || s > 2 || t < 0 || t >= ntab(s) || m < 0 || m >= c->n_mat || (prec != 0 && prec != 1) ||
      (n && (!host_E || !host_out)))
    return ADEPT_EINVAL;
  if (!c->built) return fail(c, ADEPT_ESTATE, "tables not built");
  return probe_run(c, 8, 8, n, [&](size_t b, size_t k) {
    double* din = reinterpret_cast<double*>(c->probe);
    double* dout = din + k;
    CK(cudaMemcpyAsync(din, host_E + b, 8 * k, cudaMemcpyHostToDevice, c->stream));
    CK(launch_probe_interp(c->P, s, t, m, prec, din, (int)k, dout, c->stream));
    CK(cudaMemcpyAsync(host_out + b, dout, 8 * k, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return ADEPT_OK;
  });
}

extern "C" int adept_probe_inverse_range(adept_ctx* c, int32_t s, int32_t m, int32_t prec, const double* host_R,
                                         size_t n, double* host_out) {
  if (!c || s < 1 || s > 2 || m < 0 || m >= c->n_mat || (prec != 0 && prec != 1) || (n && (!host_R || !host_out)))
    return ADEPT_EINVAL;
  if (!c->built) return fail(c, ADEPT_ESTATE, "tables not built");
  return probe_run(c, 8, 8, n, [&](size_t b, size_t k) {
    double* din = reinterpret_cast<double*>(c->probe);
    double* dout = din + k;
    CK(cudaMemcpyAsync(din, host_R + b, 8 * k, cudaMemcpyHostToDevice, c->stream));
    CK(launch_probe_inverse_range(c->P, s, m, prec, din, (int)k, dout, c->stream));
    CK(cudaMemcpyAsync(host_out + b, dout, 8 * k, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return ADEPT_OK;
  });
}

extern "C" int adept_probe_distance(adept_ctx* c, int32_t prec, const double* host_pos, const double* host_dir,
                                    const int32_t* host_vol, const double* host_T, const int32_t* host_charge, size_t n,
                                    double* host_s, int32_t* host_next) {
  if (!c || (prec != 0 && prec != 1)) return ADEPT_EINVAL;
  if (n && (!host_pos || !host_dir || !host_vol || !host_T || !host_charge || !host_s || !host_next)) return ADEPT_EINVAL;
  for (size_t i = 0; i < n; ++i)
    if (host_vol[i] < 0 || host_vol[i] >= c->n_vol) return fail(c, ADEPT_EINVAL, "point %zu: volume out of range", i);
  return probe_run(c, 64, 16, n, [&](size_t b, size_t k) {
    char* p = c->probe;
    double* dpos = reinterpret_cast<double*>(p);
    double* ddir = dpos + 3 * k;
    double* dT = ddir + 3 * k;
    double* ds = dT + k;
    int* dvol = reinterpret_cast<int*>(ds + k);
    int* dq = dvol + k;
    int* dnx = dq + k;
    CK(cudaMemcpyAsync(dpos, host_pos + 3 * b, 24 * k, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(ddir, host_dir + 3 * b, 24 * k, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(dT, host_T + b, 8 * k, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(dvol, host_vol + b, 4 * k, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(dq, host_charge + b, 4 * k, cudaMemcpyHostToDevice, c->stream));
    CK(launch_probe_distance(c->P, prec, dpos, ddir, dvol, dT, dq, (int)k, ds, dnx, c->stream));
    CK(cudaMemcpyAsync(host_s + b, ds, 8 * k, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(host_next + b, dnx, 4 * k, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return ADEPT_OK;
  });
}

extern "C" int adept_probe_sample(adept_ctx* c, int32_t which, int32_t m, int32_t prec, double E, uint32_t event,
                                  size_t n, double* host_out) {
  if (!c || which < 0 || which > 6 || m < 0 || m >= c->n_mat || (prec != 0 && prec != 1) || (n && !host_out))
    return ADEPT_EINVAL;
  if (!c->built) return fail(c, ADEPT_ESTATE, "tables not built");
  if (n > c->probe_bytes / 96) return fail(c, ADEPT_EINVAL, "at most %zu draws per call", c->probe_bytes / 96);
  double* dout = reinterpret_cast<double*>(c->probe);
  CK(launch_probe_sample(c->P, which, m, prec, E, event, (int)n, dout, c->stream));
  CK(cudaMemcpyAsync(host_out, dout, 96 * n, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return ADEPT_OK;
}

extern "C" int adept_raytrace(adept_ctx* c, int32_t prec, const double cam[11], int32_t nx, int32_t ny, double* out,
                              int32_t out_on_device) {
  if (!c || !cam || (prec != 0 && prec != 1) || nx < 0 || ny < 0 || (nx && ny && !out)) return ADEPT_EINVAL;
  if ((long long)nx * ny > (1ll << 31)) return fail(c, ADEPT_EINVAL, "at most 2^31 pixels");
  // the camera frame, as the CPU reference builds it
  RayCam k{};
  double d[3] = {cam[3], cam[4], cam[5]}, up[3] = {cam[6], cam[7], cam[8]};
  auto norm = [](double* v) {
    const double n = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    v[0] /= n; v[1] /= n; v[2] /= n;
    return n > 0.0 && std::isfinite(n);
  };
  if (!norm(d)) return fail(c, ADEPT_EINVAL, "camera view direction is zero");
  double rt[3] = {d[1] * up[2] - d[2] * up[1], d[2] * up[0] - d[0] * up[2], d[0] * up[1] - d[1] * up[0]};
  if (!norm(rt)) return fail(c, ADEPT_EINVAL, "camera up vector is parallel to the view direction");
  for (int a = 0; a < 3; ++a) { k.o[a] = cam[a]; k.d[a] = d[a]; k.right[a] = rt[a]; }
  k.up[0] = rt[1] * d[2] - rt[2] * d[1];
  k.up[1] = rt[2] * d[0] - rt[0] * d[2];
  k.up[2] = rt[0] * d[1] - rt[1] * d[0];
  k.width = cam[9];
  k.height = cam[10];
  if (!nx || !ny) return ADEPT_OK;
  if (out_on_device) {
    CK(launch_raytrace(c->P, prec, k, nx, ny, 0, ny, out, c->stream));
    return ADEPT_OK;
  }
  // host output: bands of rows through the probe buffer
  if (16 * (size_t)nx > c->probe_bytes)
    return fail(c, ADEPT_EINVAL, "rows wider than %zu pixels need device output", c->probe_bytes / 16);
  double* dout = reinterpret_cast<double*>(c->probe);
  const int rows = (int)std::max<size_t>(1, c->probe_bytes / (16 * (size_t)nx));
  for (int j0 = 0; j0 < ny; j0 += rows) {
    const int nr = std::min(rows, ny - j0);
    CK(launch_raytrace(c->P, prec, k, nx, ny, j0, nr, dout, c->stream));
    CK(cudaMemcpyAsync(out + 2 * (size_t)j0 * nx, dout, 16 * (size_t)nx * nr, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  return ADEPT_OK;
}

extern "C" int adept_probe_chord(adept_ctx* c, int32_t prec, const double* pos, const double* dir, const int32_t* vol,
                                 const double* T, const int32_t* q, const double* s_phys, size_t n, double* out) {
  if (!c || (prec != 0 && prec != 1) || (n && (!pos || !dir || !vol || !T || !q || !s_phys || !out)))
    return ADEPT_EINVAL;
  if (c->P.chord_iter <= 0) return fail(c, ADEPT_ESTATE, "the context uses the analytic helix (field_max_iterations = 0)");
  for (size_t i = 0; i < n; ++i)
    if (vol[i] < 0 || vol[i] >= c->n_vol || (q[i] != 1 && q[i] != -1) || !(T[i] > 0.0) || !(s_phys[i] >= 0.0))
      return fail(c, ADEPT_EINVAL, "point %zu: bad volume, charge, energy or step", i);
  // in: pos 24, dir 24, vol 4, T 8, q 4, s 8 bytes; out 72 bytes
  const size_t per = 24 + 24 + 8 + 8 + 8 + 8 + 72;
  if (n > c->probe_bytes / per) return fail(c, ADEPT_EINVAL, "at most %zu points per call", c->probe_bytes / per);
  char* b = c->probe;
  double* dpos = reinterpret_cast<double*>(b); b += 24 * n;
  double* ddir = reinterpret_cast<double*>(b); b += 24 * n;
  double* dT = reinterpret_cast<double*>(b); b += 8 * n;
  double* ds = reinterpret_cast<double*>(b); b += 8 * n;
  double* dout = reinterpret_cast<double*>(b); b += 72 * n;
  int* dvol = reinterpret_cast<int*>(b); b += 8 * n;
  int* dq = reinterpret_cast<int*>(b);
  CK(cudaMemcpyAsync(dpos, pos, 24 * n, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(ddir, dir, 24 * n, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(dT, T, 8 * n, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(ds, s_phys, 8 * n, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(dvol, vol, 4 * n, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(dq, q, 4 * n, cudaMemcpyHostToDevice, c->stream));
  CK(launch_probe_chord(c->P, prec, dpos, ddir, dvol, dT, dq, ds, (int)n, dout, c->stream));
  CK(cudaMemcpyAsync(out, dout, 72 * n, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return ADEPT_OK;
}

extern "C" int adept_probe_continuous(adept_ctx* c, int32_t which, int32_t species, int32_t m, int32_t prec, double T,
                                      double s, uint32_t event, size_t n, double* host_out) {
  if (!c || which < 0 || which > 1 || (species != 1 && species != 2) || m < 0 || m >= c->n_mat ||
      (prec != 0 && prec != 1) || (n && !host_out) || !(T >= 1e-3 && T <= 1e6) || !(s >= 0.0))
    return ADEPT_EINVAL;
  if (!is_matter(c->mats[m])) return fail(c, ADEPT_EINVAL, "material %d is vacuum", m);
  if (!c->built) return fail(c, ADEPT_ESTATE, "tables not built");
  const size_t per = which == 0 ? 24 : 16;
  if (n > c->probe_bytes / per) return fail(c, ADEPT_EINVAL, "at most %zu draws per call", c->probe_bytes / per);
  double* dout = reinterpret_cast<double*>(c->probe);
  CK(launch_probe_continuous(c->P, which, species, m, prec, T, s, event, (int)n, dout, c->stream));
  CK(cudaMemcpyAsync(host_out, dout, per * n, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return ADEPT_OK;
}

extern "C" const char* adept_last_error(const adept_ctx* c) {
  if (!c) return "null context";
  std::lock_guard<std::mutex> lk(const_cast<adept_ctx*>(c)->err_mu);
  return c->err.c_str();
}

extern "C" void adept_destroy(adept_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (int b = 0; b < 2; ++b) {
    if (c->graph[b]) cudaGraphExecDestroy(c->graph[b]);
    if (c->tgraph[b]) cudaGraphExecDestroy(c->tgraph[b]);
  }
  for (auto e : c->ev) cudaEventDestroy(e);
  for (int j = 0; j < 2; ++j) {
    if (c->side[j]) { cudaStreamSynchronize(c->side[j]); cudaStreamDestroy(c->side[j]); }
    if (c->join[j]) cudaEventDestroy(c->join[j]);
  }
  if (c->submit_stream) { cudaStreamSynchronize(c->submit_stream); cudaStreamDestroy(c->submit_stream); }
  if (c->fork) cudaEventDestroy(c->fork);
  if (c->tstream) { cudaStreamSynchronize(c->tstream); cudaStreamDestroy(c->tstream); }
  if (c->bstream) cudaStreamDestroy(c->bstream);
  for (int j = 0; j < 3; ++j)
    if (c->kdone[j]) cudaEventDestroy(c->kdone[j]);
  if (c->tjoin) cudaEventDestroy(c->tjoin);
  for (int b = 0; b < 2; ++b) {
    if (c->h_ctrl[b]) cudaFreeHost(c->h_ctrl[b]);
    if (c->h_floor[b]) cudaFreeHost(c->h_floor[b]);
    if (c->h_done[b]) cudaFreeHost(c->h_done[b]);
    if (c->status_ev[b]) cudaEventDestroy(c->status_ev[b]);
  }
  if (c->stage_ev) cudaEventDestroy(c->stage_ev);
  if (c->out_ev) cudaEventDestroy(c->out_ev);
  if (c->copy_stream) { cudaStreamSynchronize(c->copy_stream); cudaStreamDestroy(c->copy_stream); }
  if (c->h_stage) cudaFreeHost(c->h_stage);
  if (c->h_sub) cudaFreeHost(c->h_sub);
  if (c->h_leak) cudaFreeHost(c->h_leak);
  for (double* p : c->pool_all) cudaFreeHost(p);
  delete c;
}
