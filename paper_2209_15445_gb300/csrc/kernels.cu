// Kernels of the shower transport: table build, the per-generation step kernel over
// the three species queues, primary injection, event completion, and parity probes.
#include <cuda_runtime.h>

#include "device.cuh"
#include "layout.h"
#include "physics_init.cuh"
#include "transport.cuh"

namespace adept {

// ======================================================================== table build
// raw value rows in BuildScratch::vals
enum { V_MUC, V_MUP, V_MUPH, V_SFULL, V_SE, V_IE, V_BE, V_SP, V_IP, V_BP, V_AP, V_RFULL, V_RE, V_RP, V_NROW };
enum { B_RFULL, B_RE, B_RP };

using init::bin_integral;
using init::node_E;

__global__ void k_materials(const double* in, int n, MatDev* out) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m < n) init::setup_material(in + kMatRec * m, out + m);
}

__device__ inline double s_full(const MatDev& M, double T) {
  return init::dedx_col(M, T, T, false) + init::dedx_rad(M, T, T);
}
__device__ inline double s_restr(const MatDev& M, double T, double Tc, double kc, bool pos) {
  return init::dedx_col(M, T, Tc, pos) + init::dedx_rad(M, T, kc);
}

__global__ void k_gamma_full(const MatDev* mats, int n_mat, BuildScratch s) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_mat * kNNode) return;
  const int m = idx / kNNode, i = idx % kNNode;
  const MatDev M = mats[m];
  if (M.vacuum) return;
  double* v = s.vals + (size_t)m * V_NROW * kNNode;
  const double E = node_E(i);
  v[V_MUC * kNNode + i] = init::mu_compton(M, E);
  v[V_MUP * kNNode + i] = init::mu_pair(M, E);
  v[V_MUPH * kNNode + i] = init::mu_photo(M, E);
  v[V_SFULL * kNNode + i] = s_full(M, E);
  if (i < kNNode - 1)
    s.bins[((size_t)m * 3 + B_RFULL) * kNNode + i] = bin_integral(i, [&](double T) { return s_full(M, T); });
}

// production thresholds: e+- from the unrestricted range, gamma from 5 mean free paths
__global__ void k_cuts(const MatDev* mats, int n_mat, double range_cut, BuildScratch s, double* Tc, double* kc) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n_mat) return;
  if (mats[m].vacuum) { Tc[m] = 0.0; kc[m] = 0.0; return; }
  double* v = s.vals + (size_t)m * V_NROW * kNNode;
  double* Rf = v + V_RFULL * kNNode;
  init::prefix_range(v + V_SFULL * kNNode, s.bins + ((size_t)m * 3 + B_RFULL) * kNNode, Rf);
  auto mu = [&](int i) { return v[V_MUC * kNNode + i] + v[V_MUP * kNNode + i] + v[V_MUPH * kNNode + i]; };
  Tc[m] = init::clamp_cut(init::range_threshold(Rf, range_cut));
  kc[m] = init::clamp_cut(init::gamma_threshold(mu, range_cut));
}

__global__ void k_charged(const MatDev* mats, int n_mat, BuildScratch s, const double* Tc, const double* kc) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_mat * kNNode) return;
  const int m = idx / kNNode, i = idx % kNNode;
  const MatDev M = mats[m];
  if (M.vacuum) return;
  const double tc = Tc[m], kk = kc[m];
  double* v = s.vals + (size_t)m * V_NROW * kNNode;
  const double T = node_E(i);
  v[V_SE * kNNode + i] = s_restr(M, T, tc, kk, false);
  v[V_IE * kNNode + i] = init::lambda_ioni(M, T, tc, false);
  v[V_BE * kNNode + i] = init::lambda_brem(M, T, kk);
  v[V_SP * kNNode + i] = s_restr(M, T, tc, kk, true);
  v[V_IP * kNNode + i] = init::lambda_ioni(M, T, tc, true);
  v[V_BP * kNNode + i] = init::lambda_brem(M, T, kk);
  v[V_AP * kNNode + i] = init::lambda_annih(M, T);
  if (i < kNNode - 1) {
    s.bins[((size_t)m * 3 + B_RE) * kNNode + i] = bin_integral(i, [&](double x) { return s_restr(M, x, tc, kk, false); });
    s.bins[((size_t)m * 3 + B_RP) * kNNode + i] = bin_integral(i, [&](double x) { return s_restr(M, x, tc, kk, true); });
  }
}

__global__ void k_ranges(const MatDev* mats, int n_mat, BuildScratch s) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 2 * n_mat) return;
  const int m = idx >> 1, pos = idx & 1;
  if (mats[m].vacuum) return;
  double* v = s.vals + (size_t)m * V_NROW * kNNode;
  init::prefix_range(v + (pos ? V_SP : V_SE) * kNNode, s.bins + ((size_t)m * 3 + (pos ? B_RP : B_RE)) * kNNode,
               v + (pos ? V_RP : V_RE) * kNNode);
}

struct PackOut {
  double2 *g64, *e64, *p64;
  float2 *g32, *e32, *p32;
  double *re64, *rp64;
  float *re32, *rp32;
};

__device__ inline void put(double2* d64, float2* d32, size_t at, const double* row, int i) {
  const double a = row[i];
  const double b = (i + 1 < kNNode) ? row[i + 1] : row[i];
  d64[at] = make_double2(a, b - a);
  d32[at] = make_float2((float)a, (float)(b - a));
}

// Packs the raw rows into (value, slope) records. A process switched off by the process mask
// (tests of one process at a time) gets a zero cross-section table, so that the step needs
// no test of the mask: its lookup gives exactly 0, as a skipped one did.
__global__ void k_pack(const MatDev* mats, int n_mat, BuildScratch s, PackOut o, uint32_t mask) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_mat * kNNode) return;
  const int m = idx / kNNode, i = idx % kNNode;
  const size_t r = (size_t)m * kNNode + i;
  if (mats[m].vacuum) {
    for (int t = 0; t < kNTabG; ++t) { o.g64[r * kNTabG + t] = make_double2(0, 0); o.g32[r * kNTabG + t] = make_float2(0, 0); }
    for (int t = 0; t < kNTabE; ++t) { o.e64[r * kNTabE + t] = make_double2(0, 0); o.e32[r * kNTabE + t] = make_float2(0, 0); }
    for (int t = 0; t < kNTabP; ++t) { o.p64[r * kNTabP + t] = make_double2(0, 0); o.p32[r * kNTabP + t] = make_float2(0, 0); }
    o.re64[r] = o.rp64[r] = 0.0;
    o.re32[r] = o.rp32[r] = 0.0f;
    return;
  }
  const double* v = s.vals + (size_t)m * V_NROW * kNNode;
  const int grow[kNTabG] = {V_MUC, V_MUP, V_MUPH};
  const int erow[kNTabE] = {V_SE, V_RE, V_IE, V_BE};
  const int prow[kNTabP] = {V_SP, V_RP, V_IP, V_BP, V_AP};
  for (int t = 0; t < kNTabG; ++t) put(o.g64, o.g32, r * kNTabG + t, v + grow[t] * kNNode, i);
  for (int t = 0; t < kNTabE; ++t) put(o.e64, o.e32, r * kNTabE + t, v + erow[t] * kNNode, i);
  for (int t = 0; t < kNTabP; ++t) put(o.p64, o.p32, r * kNTabP + t, v + prow[t] * kNNode, i);
  if (mask) {
    // process bits: gamma Compton, pair, photo (tables 0-2); e- ionisation, brems (tables
    // 2-3); e+ ionisation, brems, annihilation (tables 2-4)
    auto off = [&](double2* d64, float2* d32, size_t at) { d64[at] = make_double2(0, 0); d32[at] = make_float2(0, 0); };
    for (int t = 0; t < 3; ++t)
      if (!(mask & (1u << t))) off(o.g64, o.g32, r * kNTabG + t);
    for (int t = 2; t < 4; ++t)
      if (!(mask & (1u << (t + 1)))) off(o.e64, o.e32, r * kNTabE + t);
    for (int t = 2; t < 5; ++t)
      if (!(mask & (1u << (t + 3)))) off(o.p64, o.p32, r * kNTabP + t);
  }
  o.re64[r] = v[V_RE * kNNode + i];
  o.rp64[r] = v[V_RP * kNNode + i];
  o.re32[r] = (float)v[V_RE * kNNode + i];
  o.rp32[r] = (float)v[V_RP * kNNode + i];
}

cudaError_t launch_build_tables(const Params& P, const double* mat_in, int n_mat, double range_cut, MatDev* mat,
                                BuildScratch s, double2* g64, double2* e64, double2* p64, float2* g32,
                                float2* e32, float2* p32, double* re64, double* rp64, float* re32, float* rp32,
                                double* Tc, double* kc, cudaStream_t st) {
  const int nn = n_mat * kNNode;
  const int B = 128;
  k_materials<<<1, 32, 0, st>>>(mat_in, n_mat, mat);
  k_gamma_full<<<(nn + B - 1) / B, B, 0, st>>>(mat, n_mat, s);
  k_cuts<<<1, 32, 0, st>>>(mat, n_mat, range_cut, s, Tc, kc);
  k_charged<<<(nn + B - 1) / B, B, 0, st>>>(mat, n_mat, s, Tc, kc);
  k_ranges<<<1, 32, 0, st>>>(mat, n_mat, s);
  PackOut o{g64, e64, p64, g32, e32, p32, re64, rp64, re32, rp32};
  k_pack<<<(nn + B - 1) / B, B, 0, st>>>(mat, n_mat, s, o, P.process_mask);
  return cudaGetLastError();
}

// Each species kernel is compiled for 1..4 resident blocks of 256 threads per SM
// (register caps 255, 128, 85, 64); the choice trades occupancy against spills.
template <class R, int S>
static const void* transport_fn(int minb) {
  switch (minb) {
    case 1: return (const void*)k_transport<R, S, 1>;
    case 2: return (const void*)k_transport<R, S, 2>;
    case 3: return (const void*)k_transport<R, S, 3>;
    default: return (const void*)k_transport<R, S, 4>;
  }
}

template <class R>
static const void* transport_fn(int species, int minb) {
  return species == 0 ? transport_fn<R, 0>(minb) : (species == 1 ? transport_fn<R, 1>(minb) : transport_fn<R, 2>(minb));
}

// the kernel of species `species` for this variant: photons have no optional parts and
// move straight in any field
static const void* pick_transport(int precision, int species, int minb, int variant) {
  if (variant & 4) return hist_transport_fn(precision, species, minb, variant);
  if (species != 0 && (variant & 3)) return variant_transport_fn(precision, species, minb, variant);
  if (species != 0 && (variant & 8)) return field_transport_fn(precision, species, minb);
  return precision ? transport_fn<float>(species, minb) : transport_fn<double>(species, minb);
}

// The driver's default carveout kept 132 KiB of shared memory for the 99 KiB that three FP32
// blocks need (launch__shared_mem_config_size); asking for the share they need, rounded down
// (the driver then takes the next size that fits), gives 100 KiB and leaves L1 32 KiB more
// (+0.3 % on the 10 GeV showers). The preference is dropped if it would cost a block.
int max_blocks_small_carveout(const void* fn, int block) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, block, 0) != cudaSuccess || n < 1) return 0;
  cudaFuncAttributes fa;
  int dev = 0, smem_sm = 0, reserved = 0;
  if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
      smem_sm <= 0)
    return n;
  const int pct = (int)(100.0 * n * ((double)fa.sharedSizeBytes + reserved) / smem_sm);
  if (cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, pct) != cudaSuccess) return n;
  int m = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m, fn, block, 0) != cudaSuccess || m < n)
    cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, -1);  // back to the default
  return n;
}

int transport_max_blocks_per_sm(int precision, int species, int minb, int block, int variant) {
  return max_blocks_small_carveout(pick_transport(precision, species, minb, variant), block);
}

cudaError_t launch_transport(const Params& P, uint32_t gk, int precision, int species, int minb, int grid, int block,
                             bool pdl, cudaStream_t st) {
  void* args[] = {const_cast<Params*>(&P), &gk};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelExC(&cfg, pick_transport(precision, species, minb, transport_variant(P)), args);
}

// ======================================================================== admission
// The request's deposit rows are one contiguous range of slots, zeroed by a grid-stride loop
// over its doubles (coalesced; a row per thread wrote 32 rows per warp store).
__global__ void k_admit(Params P, uint32_t slot_base, const uint32_t* keys, int n) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) {
    const uint32_t s = slot_base + j;
    P.evt.key[s] = keys[j];
    P.evt.state[s] = 1u;
    P.evt.alive[s] = 0xFFFFFFFFu;
    P.evt.leaked[s] = 0.0;
    P.evt.killed[s] = 0.0;
  }
  double* rows = P.evt.edep + (size_t)slot_base * P.geo.n_bins;
  const size_t m = (size_t)n * P.geo.n_bins;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (size_t)gridDim.x * blockDim.x)
    rows[i] = 0.0;
}

cudaError_t launch_admit(const Params& P, uint32_t slot_base, const uint32_t* keys, int n, cudaStream_t st) {
  if (n > 0) k_admit<<<(n + 127) / 128, 128, 0, st>>>(P, slot_base, keys, n);
  return cudaGetLastError();
}

// S12: unpack primaries into the current queues (paper Sec. 4: particles entering the
// GPU region); a primary outside the calorimeter leaks at once
template <class R>
__global__ void k_init_primaries(Params P, const TrackIn* recs, const uint32_t* meta, int n, uint32_t slot_base) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const TrackIn r = recs[i];
  const uint32_t slot = slot_base + meta[2 * i];
  const uint32_t id = meta[2 * i + 1];
  const int sp = r.pdg == 22 ? 0 : (r.pdg == 11 ? 1 : 2);
  const double rest = sp == 2 ? 2.0 * kMe : 0.0;
  const int vol = locate(P.geo, r.pos[0], r.pos[1], r.pos[2], r.dir[0], r.dir[1], r.dir[2]);
  if (vol < 0) {
    atomicAdd(P.evt.leaked + slot, r.E + rest);
    record_leak(P, r.pdg, slot, r.E, r.pos[0], r.pos[1], r.pos[2], r.dir[0], r.dir[1], r.dir[2]);
    return;
  }
  const uint32_t gen = __ldcg(&P.ctrl->gen);
  const int p = gen & 1;
  const uint32_t d = atomicAdd(&P.ctrl->count[gen % 3][sp].n, 1u);
  if (d >= P.cap) {
    atomicAdd(&P.ctrl->overflow, 1ull);
    atomicAdd(P.evt.killed + slot, r.E + rest);
    return;
  }
  store_track<R>(P.q[p][sp], d, r.pos[0], r.pos[1], r.pos[2], (R)r.dir[0], (R)r.dir[1], (R)r.dir[2], r.E,
                 (unsigned long long)id, slot, 0u, (uint32_t)vol);
}

cudaError_t launch_init_primaries(const Params& P, const TrackIn* recs, const uint32_t* meta, int n, uint32_t slot_base,
                                  int precision, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (precision) k_init_primaries<float><<<(n + 255) / 256, 256, 0, st>>>(P, recs, meta, n, slot_base);
  else k_init_primaries<double><<<(n + 255) / 256, 256, 0, st>>>(P, recs, meta, n, slot_base);
  return cudaGetLastError();
}

// ======================================================================== completion
// End of a chunk of `gens` generations: log the sizes its last generation left, and advance
// gen and the generation count. One thread.
__global__ void k_end_chunk(Params P, uint32_t gens) {
  if (threadIdx.x != 0) return;
  volatile Ctrl* c = P.ctrl;
  if (gens == kGkDevice) gens = c->tail_k;
  if (gens == 0) return;  // a tail chunk that found the queues empty ran nothing
  const uint32_t gen = c->gen + gens;
  const uint32_t ln = c->log_n;
  if (ln < P.max_log) {
    for (int k = 0; k < 3; ++k) P.gen_log[3 * ln + k] = min(c->count[gen % 3][k].n, P.cap);
    c->log_n = ln + 1;
  }
  c->generations = c->generations + gens;
  c->gen = gen;
}

// An event is finished when no live track of it is left in the current queues: mark
// the slots that still have tracks with the current generation, then every active slot
// not marked is done and goes to the done list.
__global__ void k_mark(Params P) {
  const uint32_t gen = __ldcg(&P.ctrl->gen);
  const int p = gen & 1, cr = gen % 3;
  const uint32_t n0 = min(__ldcg(&P.ctrl->count[cr][0].n), P.cap), n1 = min(__ldcg(&P.ctrl->count[cr][1].n), P.cap),
                 n2 = min(__ldcg(&P.ctrl->count[cr][2].n), P.cap);
  const uint32_t total = n0 + n1 + n2;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int sp = i < n0 ? 0 : (i < n0 + n1 ? 1 : 2);
    const uint32_t j = sp == 0 ? i : (sp == 1 ? i - n0 : i - n0 - n1);
    const TrackSoA& q = P.q[p][sp];
    const uint32_t ev = q.meta ? q.meta[j].z : q.ev[j];
    if (P.evt.alive[ev] != gen) P.evt.alive[ev] = gen;
  }
}

// The same marks with per-block deduplication: a block sets one bit per event slot seen among
// its share of the live tracks in a shared-memory bitmap, then writes the marks of the slots
// it saw in slot order (coalesced). All live tracks writing their event's mark, about ten
// thousand events on a few hundred L2 lines, was bound by the contention on those lines.
// Used while the bitmap fits 48 KB (evt.max_slots up to 393,216); with few live tracks, whose
// marks contend little, it marks directly (the bitmap's zeroing and scan cost the one-shower
// batches 4 us a chunk).
constexpr uint32_t kMarkBitsMaxSlots = 48u * 1024u * 8u;
constexpr uint32_t kMarkDirectTracks = 16384u;  // below this many live tracks, no bitmap
__global__ void k_mark_bits(Params P) {
  extern __shared__ uint32_t seen[];  // [ceil(max_slots / 32)]
  const uint32_t gen = __ldcg(&P.ctrl->gen);
  const int p = gen & 1, cr = gen % 3;
  const uint32_t n0 = min(__ldcg(&P.ctrl->count[cr][0].n), P.cap), n1 = min(__ldcg(&P.ctrl->count[cr][1].n), P.cap),
                 n2 = min(__ldcg(&P.ctrl->count[cr][2].n), P.cap);
  const uint32_t total = n0 + n1 + n2;
  if (blockIdx.x * blockDim.x >= total) return;  // a block with no tracks has nothing to mark
  if (total <= kMarkDirectTracks) {  // few tracks contend little: mark directly, as k_mark does
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
      const int sp = i < n0 ? 0 : (i < n0 + n1 ? 1 : 2);
      const uint32_t j = sp == 0 ? i : (sp == 1 ? i - n0 : i - n0 - n1);
      const TrackSoA& q = P.q[p][sp];
      const uint32_t ev = q.meta ? q.meta[j].z : q.ev[j];
      if (P.evt.alive[ev] != gen) P.evt.alive[ev] = gen;
    }
    return;
  }
  const uint32_t nw = (P.evt.max_slots + 31u) / 32u;
  for (uint32_t w = threadIdx.x; w < nw; w += blockDim.x) seen[w] = 0u;
  __syncthreads();
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int sp = i < n0 ? 0 : (i < n0 + n1 ? 1 : 2);
    const uint32_t j = sp == 0 ? i : (sp == 1 ? i - n0 : i - n0 - n1);
    const TrackSoA& q = P.q[p][sp];
    const uint32_t ev = q.meta ? q.meta[j].z : q.ev[j];
    if (ev < P.evt.max_slots) atomicOr(&seen[ev >> 5], 1u << (ev & 31u));
  }
  __syncthreads();
  for (uint32_t s = threadIdx.x; s < P.evt.max_slots; s += blockDim.x)
    if ((seen[s >> 5] >> (s & 31u)) & 1u) P.evt.alive[s] = gen;
}

// The done list (at most one entry per event slot) goes straight to the host's pinned copy of
// buffer b; the last block to end then writes the whole Ctrl there. The host reads both once
// the chunk has ended, and no copy runs between two chunks (two device-to-host copies and one
// host-to-device copy a chunk boundary before, and a synchronous one for long lists).
__global__ void k_finish(Params P, int b) {
  const uint32_t gen = __ldcg(&P.ctrl->gen);
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < P.evt.max_slots; s += gridDim.x * blockDim.x) {
    if (P.evt.state[s] == 1u && P.evt.alive[s] != gen) {
      P.evt.state[s] = 2u;
      P.h_done[b][atomicAdd(&P.ctrl->done_count[b], 1u)] = s;
    }
  }
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(&P.ctrl->finish_ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (threadIdx.x == 0) P.ctrl->finish_ticket = 0;
  const uint32_t* src = reinterpret_cast<const uint32_t*>(P.ctrl);
  uint32_t* dst = reinterpret_cast<uint32_t*>(P.h_ctrl[b]);
  for (uint32_t i = threadIdx.x; i < sizeof(Ctrl) / 4; i += blockDim.x) dst[i] = __ldcg(src + i);
  __threadfence_system();
}

// Start of a chunk: the outgoing-ring read position the host left in its pinned copy of
// buffer b, and an empty done count for the chunk's finish pass. One thread.
__global__ void k_open_chunk(Params P, int b) {
  if (threadIdx.x != 0) return;
  P.ctrl->leak_floor = *reinterpret_cast<const volatile unsigned long long*>(P.h_floor[b]);
  P.ctrl->done_count[b] = 0;
}

cudaError_t launch_open_chunk(const Params& P, int b, cudaStream_t st) {
  k_open_chunk<<<1, 32, 0, st>>>(P, b);
  return cudaGetLastError();
}

// Tail chunks (conditional while node): the condition that runs the next generation. Live
// tracks are the sizes of the generation slot the next generation reads.
__device__ __forceinline__ uint32_t live_tracks(const Params& P, uint32_t gen) {
  const uint32_t cr = gen % 3;
  return min(__ldcg(&P.ctrl->count[cr][0].n), P.cap) + min(__ldcg(&P.ctrl->count[cr][1].n), P.cap) +
         min(__ldcg(&P.ctrl->count[cr][2].n), P.cap);
}
__global__ void k_tail_open(Params P, cudaGraphConditionalHandle h) {
  if (threadIdx.x != 0) return;
  P.ctrl->tail_k = 0;
  cudaGraphSetConditional(h, live_tracks(P, __ldcg(&P.ctrl->gen)) > 0 ? 1u : 0u);
}
__global__ void k_tail_step(Params P, cudaGraphConditionalHandle h, uint32_t max_gens) {
  if (threadIdx.x != 0) return;
  const uint32_t k = __ldcg(&P.ctrl->tail_k) + 1;
  P.ctrl->tail_k = k;
  const uint32_t live = live_tracks(P, __ldcg(&P.ctrl->gen) + k);
  cudaGraphSetConditional(h, (k < max_gens && live > 0 && live < P.tail_exit) ? 1u : 0u);
}
cudaError_t launch_tail_open(const Params& P, cudaGraphConditionalHandle h, cudaStream_t st) {
  k_tail_open<<<1, 32, 0, st>>>(P, h);
  return cudaGetLastError();
}
cudaError_t launch_tail_step(const Params& P, cudaGraphConditionalHandle h, uint32_t max_gens, cudaStream_t st) {
  k_tail_step<<<1, 32, 0, st>>>(P, h, max_gens);
  return cudaGetLastError();
}

cudaError_t launch_finish(const Params& P, int b, uint32_t gens, cudaStream_t st) {
  k_end_chunk<<<1, 32, 0, st>>>(P, gens);
  if (P.evt.max_slots <= kMarkBitsMaxSlots)
    k_mark_bits<<<304, 512, sizeof(uint32_t) * ((P.evt.max_slots + 31) / 32), st>>>(P);
  else
    k_mark<<<1216, 256, 0, st>>>(P);
  k_finish<<<(P.evt.max_slots + 255) / 256 < 1216 ? (P.evt.max_slots + 255) / 256 : 1216, 256, 0, st>>>(P, b);
  return cudaGetLastError();
}

// ======================================================================== probes
__global__ void k_probe_philox(const uint32_t* ctr, int n, uint32_t k0, uint32_t k1, uint32_t* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const U4 r = philox(U4{ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]}, k0, k1);
  out[4 * i] = r.a; out[4 * i + 1] = r.b; out[4 * i + 2] = r.c; out[4 * i + 3] = r.d;
}

cudaError_t launch_probe_philox(const uint32_t* ctr, int n, uint32_t k0, uint32_t k1, uint32_t* out, cudaStream_t st) {
  if (n > 0) k_probe_philox<<<(n + 127) / 128, 128, 0, st>>>(ctr, n, k0, k1, out);
  return cudaGetLastError();
}

template <class R>
__global__ void k_probe_interp(Params P, int s, int t, int m, const double* E, int n, double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int bin;
  R tt;
  grid_pos<R>(E[i], &bin, &tt);
  const size_t r = (size_t)m * kNNode + bin;
  R v;
  if (s == 0) v = lerp_rec<R>(tab_g<R>(P.tab) + r * kNTabG, t, tt);
  else if (s == 1) v = lerp_rec<R>(tab_e<R>(P.tab) + r * kNTabE, t, tt);
  else v = lerp_rec<R>(tab_p<R>(P.tab) + r * kNTabP, t, tt);
  out[i] = (double)v;
}

cudaError_t launch_probe_interp(const Params& P, int s, int t, int m, int prec, const double* E, int n, double* out,
                                cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (prec) k_probe_interp<float><<<(n + 127) / 128, 128, 0, st>>>(P, s, t, m, E, n, out);
  else k_probe_interp<double><<<(n + 127) / 128, 128, 0, st>>>(P, s, t, m, E, n, out);
  return cudaGetLastError();
}

template <class R>
__global__ void k_probe_inverse_range(Params P, int s, int m, const double* Rv, int n, double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[i] = inverse_range<R>(range_nodes<R>(P.tab, s == 2) + (size_t)m * kNNode, (R)Rv[i], kNNode - 2);
}

cudaError_t launch_probe_inverse_range(const Params& P, int s, int m, int prec, const double* R, int n, double* out,
                                       cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (prec) k_probe_inverse_range<float><<<(n + 127) / 128, 128, 0, st>>>(P, s, m, R, n, out);
  else k_probe_inverse_range<double><<<(n + 127) / 128, 128, 0, st>>>(P, s, m, R, n, out);
  return cudaGetLastError();
}

template <class R>
__global__ void k_probe_distance(Params P, const double* pos, const double* dir, const int* vol, const double* T,
                                 const int* q, int n, double* s, int* next) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const R u[3] = {(R)dir[3 * i], (R)dir[3 * i + 1], (R)dir[3 * i + 2]};
  int nx;
  const double d = (q[i] != 0 && P.field_T != 0.0)
                       ? helix_distance<R>(P.geo, P.field_T, T[i], q[i], pos[3 * i], pos[3 * i + 1], pos[3 * i + 2], u,
                                           vol[i], &nx)
                       : straight_distance<R>(P.geo, pos[3 * i], pos[3 * i + 1], pos[3 * i + 2], u, vol[i], &nx);
  s[i] = d;
  next[i] = nx;
}

cudaError_t launch_probe_distance(const Params& P, int prec, const double* pos, const double* dir, const int* vol,
                                  const double* T, const int* q, int n, double* s, int* next, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (prec) k_probe_distance<float><<<(n + 127) / 128, 128, 0, st>>>(P, pos, dir, vol, T, q, n, s, next);
  else k_probe_distance<double><<<(n + 127) / 128, 128, 0, st>>>(P, pos, dir, vol, T, q, n, s, next);
  return cudaGetLastError();
}

// out per point: status, path, next, x, y, z, ux, uy, uz, iterations unused (9 doubles used)
template <class R>
__global__ void k_probe_chord(Params P, const double* pos, const double* dir, const int* vol, const double* T,
                              const int* q, const double* s_phys, int n, double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  R u[3] = {(R)dir[3 * i], (R)dir[3 * i + 1], (R)dir[3 * i + 2]};
  double x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
  int nx = vol[i];
  R sd = 0;
  const int rc = chord_step<R>(P.geo, P.field_T, T[i], q[i], (R)s_phys[i], P.chord_iter, (R)P.delta_chord,
                               (R)P.delta_int, &x, &y, &z, u, vol[i], &nx, &sd);
  double* o = out + 9 * (size_t)i;
  o[0] = rc; o[1] = sd; o[2] = nx;
  o[3] = x; o[4] = y; o[5] = z;
  o[6] = u[0]; o[7] = u[1]; o[8] = u[2];
}

cudaError_t launch_probe_chord(const Params& P, int prec, const double* pos, const double* dir, const int* vol,
                               const double* T, const int* q, const double* s_phys, int n, double* out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (prec) k_probe_chord<float><<<(n + 127) / 128, 128, 0, st>>>(P, pos, dir, vol, T, q, s_phys, n, out);
  else k_probe_chord<double><<<(n + 127) / 128, 128, 0, st>>>(P, pos, dir, vol, T, q, s_phys, n, out);
  return cudaGetLastError();
}

template <class R>
__global__ void k_probe_sample(Params P, int which, int m, double E, uint32_t event, int n, double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  Stream<R> st(P.seed, event, (unsigned long long)(i + 1), 0u);
  const R u[3] = {(R)0, (R)0, (R)1};
  Ixn<R> r;
  r.happened = false; r.parent_alive = false; r.n = 0; r.parent_E = 0.0;
  r.pd[0] = r.pd[1] = r.pd[2] = (R)0;
  const double Tc = P.tab.Tc[m], kc = P.tab.kc[m];
  switch (which) {
    case 0: compton<R>(st, E, u, r); break;
    case 1: pair<R>(st, E, u, r); break;
    case 2: moller<R>(st, E, Tc, u, r); break;
    case 3: bhabha<R>(st, E, Tc, u, r); break;
    case 4: brem<R>(st, E, kc, u, r); break;
    case 5: annihilate<R>(st, E, u, r); break;
    default: annihilate_at_rest<R>(st, r); break;
  }
  double* o = out + 12 * (size_t)i;
  o[0] = r.happened ? 1.0 : 0.0;
  o[1] = r.parent_alive ? r.parent_E : -1.0;
  o[2] = r.pd[0]; o[3] = r.pd[1]; o[4] = r.pd[2];
  o[5] = r.n > 0 ? r.E[0] : -1.0;
  o[6] = r.n > 0 ? (double)r.d[0][0] : 0.0;
  o[7] = r.n > 0 ? (double)r.d[0][1] : 0.0;
  o[8] = r.n > 0 ? (double)r.d[0][2] : 0.0;
  o[9] = r.n > 1 ? r.E[1] : -1.0;
  o[10] = r.n > 1 ? (double)r.d[1][2] : 0.0;
  o[11] = r.n > 1 ? (double)(r.d[1][0] * r.d[0][0] + r.d[1][1] * r.d[0][1] + r.d[1][2] * r.d[0][2]) : 0.0;
}

cudaError_t launch_probe_sample(const Params& P, int which, int m, int prec, double E, uint32_t event, int n,
                                double* out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (prec) k_probe_sample<float><<<(n + 127) / 128, 128, 0, st>>>(P, which, m, E, event, n, out);
  else k_probe_sample<double><<<(n + 127) / 128, 128, 0, st>>>(P, which, m, E, event, n, out);
  return cudaGetLastError();
}

template <class R>
__global__ void k_probe_continuous(Params P, int which, int species, int m, double T, double s, uint32_t event, int n,
                                   double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  Stream<R> st(P.seed, event, (unsigned long long)(i + 1), 0u);
  const MatDev& md = P.mat[m];
  if (which == 0) {
    R u[3] = {(R)0, (R)0, (R)1};
    msc_deflect<R>(st, msc_theta0<R>((R)T, (R)md.inv_x0, (R)s), u);
    out[3 * (size_t)i] = u[0]; out[3 * (size_t)i + 1] = u[1]; out[3 * (size_t)i + 2] = u[2];
    return;
  }
  // the mean loss as in the step: through the range table of the species
  int bin;
  R tt;
  grid_pos<R>(T, &bin, &tt);
  const auto* rec = (species == 2 ? tab_p<R>(P.tab) + ((size_t)m * kNNode + bin) * kNTabP
                                  : tab_e<R>(P.tab) + ((size_t)m * kNNode + bin) * kNTabE);
  const R Rr = lerp_rec<R>(rec, 1, tt);
  R Epr = 0;
  if ((R)s < Rr) Epr = inverse_range<R>(range_nodes<R>(P.tab, species == 2) + (size_t)m * kNNode, Rr - (R)s, bin + 1);
  const double Ep = (Epr > (R)T) ? T : to_d<R>(Epr);
  const R xi = (R)(kTwoPiRe2Me * md.n_el);
  const R sig = M<R>::sqrt(fluct_sigma2<R>((R)T, xi, (R)P.tab.Tc[m], (R)s, species == 2));
  out[2 * (size_t)i] = fluct_loss<R>(st, T - Ep, sig);
  out[2 * (size_t)i + 1] = T - Ep;
}

cudaError_t launch_probe_continuous(const Params& P, int which, int species, int m, int prec, double T, double s,
                                    uint32_t event, int n, double* out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (prec) k_probe_continuous<float><<<(n + 127) / 128, 128, 0, st>>>(P, which, species, m, T, s, event, n, out);
  else k_probe_continuous<double><<<(n + 127) / 128, 128, 0, st>>>(P, which, species, m, T, s, event, n, out);
  return cudaGetLastError();
}

}  // namespace adept
