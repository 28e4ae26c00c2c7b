// Device side of one transport step, shared by the per-species generation kernels
// (kernels.cu, variants.cu) and the one-kernel-per-generation form (fused.cu): track load
// and store, phase A (S1-S8), phase B (S9), scoring (S10), warp-aggregated appends and
// the per-warp ring of deferred interactions.
//
// Queue descriptors are read from P.qd (device memory) with a runtime parity index:
// indexing the kernel-parameter copy P.q that way makes the compiler copy the parameter
// block to local memory once several species paths share a kernel.
#pragma once
#include <cuda_runtime.h>

#include "device.cuh"
#include "layout.h"

namespace adept {

template <class R> struct Trk {
  double x, y, z;
  R u[3];
  double E;
  unsigned long long id;
  uint32_t ev, step, nav;
};

// Queue loads are streaming (ld.global.cs): each slot is read once per generation.
template <class R>
__device__ __forceinline__ void load_track(const TrackSoA& q, uint32_t i, Trk<R>& t);
template <>
__device__ __forceinline__ void load_track<double>(const TrackSoA& q, uint32_t i, Trk<double>& t) {
  t.x = __ldcs(q.x + i); t.y = __ldcs(q.y + i); t.z = __ldcs(q.z + i);
  t.u[0] = __ldcs(q.ux + i); t.u[1] = __ldcs(q.uy + i); t.u[2] = __ldcs(q.uz + i);
  t.E = __ldcs(q.E + i);
  t.id = __ldcs(q.id + i);
  t.ev = __ldcs(q.ev + i);
  t.step = __ldcs(q.step + i);
  t.nav = __ldcs(q.nav + i);
}
template <>
__device__ __forceinline__ void load_track<float>(const TrackSoA& q, uint32_t i, Trk<float>& t) {
  const double2 a = __ldcs(q.xy + i), b = __ldcs(q.zE + i);
  const float4 c = __ldcs(q.un + i);
  const uint4 d = __ldcs(q.meta + i);
  t.x = a.x; t.y = a.y; t.z = b.x; t.E = b.y;
  t.u[0] = c.x; t.u[1] = c.y; t.u[2] = c.z;
  t.nav = __float_as_uint(c.w);
  t.id = (unsigned long long)d.x | ((unsigned long long)d.y << 32);
  t.ev = d.z;
  t.step = d.w;
}

template <class R>
__device__ __forceinline__ void store_track(const TrackSoA& q, uint32_t i, double x, double y, double z, R ux,
                                            R uy, R uz, double E, unsigned long long id, uint32_t ev,
                                            uint32_t step, uint32_t nav);
template <>
__device__ __forceinline__ void store_track<double>(const TrackSoA& q, uint32_t i, double x, double y, double z,
                                                    double ux, double uy, double uz, double E, unsigned long long id,
                                                    uint32_t ev, uint32_t step, uint32_t nav) {
  q.x[i] = x; q.y[i] = y; q.z[i] = z;
  q.ux[i] = ux; q.uy[i] = uy; q.uz[i] = uz;
  q.E[i] = E;
  q.id[i] = id;
  q.ev[i] = ev;
  q.step[i] = step;
  q.nav[i] = nav;
}
template <>
__device__ __forceinline__ void store_track<float>(const TrackSoA& q, uint32_t i, double x, double y, double z,
                                                   float ux, float uy, float uz, double E, unsigned long long id,
                                                   uint32_t ev, uint32_t step, uint32_t nav) {
  q.xy[i] = make_double2(x, y);
  q.zE[i] = make_double2(z, E);
  q.un[i] = make_float4(ux, uy, uz, __uint_as_float(nav));
  q.meta[i] = make_uint4((uint32_t)id, (uint32_t)(id >> 32), ev, step);
}

// an outgoing particle (paper Sec. 4: the GPU region hands back the particles that leave it)
__device__ __forceinline__ void record_leak(const Params& P, int pdg, uint32_t slot, double E, double x, double y,
                                            double z, double ux, double uy, double uz) {
  const unsigned long long i = atomicAdd(&P.ctrl->leak_count, 1ull);
  if (i - __ldcg(&P.ctrl->leak_floor) >= P.leak_cap) {
    atomicAdd(&P.ctrl->leak_dropped, 1ull);
    return;
  }
  LeakRec& r = P.leak[i % P.leak_cap];
  r.pdg = pdg; r.slot = slot; r.E = E;
  r.pos[0] = x; r.pos[1] = y; r.pos[2] = z;
  r.dir[0] = ux; r.dir[1] = uy; r.dir[2] = uz;
}

template <class R> __device__ __forceinline__ const typename Pair2<R>::T* tab_g(const TableView& T);
template <> __device__ __forceinline__ const double2* tab_g<double>(const TableView& T) { return T.g64; }
template <> __device__ __forceinline__ const float2* tab_g<float>(const TableView& T) { return T.g32; }
template <class R> __device__ __forceinline__ const typename Pair2<R>::T* tab_e(const TableView& T);
template <> __device__ __forceinline__ const double2* tab_e<double>(const TableView& T) { return T.e64; }
template <> __device__ __forceinline__ const float2* tab_e<float>(const TableView& T) { return T.e32; }
template <class R> __device__ __forceinline__ const typename Pair2<R>::T* tab_p(const TableView& T);
template <> __device__ __forceinline__ const double2* tab_p<double>(const TableView& T) { return T.p64; }
template <> __device__ __forceinline__ const float2* tab_p<float>(const TableView& T) { return T.p32; }
template <class R> __device__ __forceinline__ const R* range_nodes(const TableView& T, bool pos);
template <> __device__ __forceinline__ const double* range_nodes<double>(const TableView& T, bool pos) { return pos ? T.rp64 : T.re64; }
template <> __device__ __forceinline__ const float* range_nodes<float>(const TableView& T, bool pos) { return pos ? T.rp32 : T.re32; }

enum Outcome { kDead = 0, kAlive = 1, kInteract = 2 };

// Phase A of one step of one track of species S (0 gamma, 1 e-, 2 e+) -- paper Sec. 3:
// every live track advances by one step per generation. Cross sections and range at the
// pre-step energy (S2), sampled interaction length (S3), step limit (S4), boundary
// distance (S5/S6), move, continuous loss (S7) and boundary crossing (S8). A step that
// ends in a discrete interaction returns kInteract with the chosen process; the
// interaction itself (S9) runs later on a full warp. dep is the energy to score in
// dep_bin. A positron that stops also returns kInteract (process 3): its annihilation at
// rest runs with the interactions, from the same random stream, so that phase A emits no
// secondaries (its appends take the one-ballot path, and the e+ kernel needs fewer
// registers: 3 blocks per SM measured +2.4 % over 2). So does a track that leaves the world
// (process 4), recorded there with its exit state (+0.9 %). The variant V compiles
// in the optional parts, kept out of the kernels that do not use them: bit 0 the chord
// propagator of the field (P.chord_iter > 0), bit 1 multiple scattering and loss
// fluctuations (P.physics), bit 2 the validation histogram of step lengths (P.steplen;
// its never-taken branch cost the default kernels 1.6 %), bit 3 the helix of a charged
// track in the uniform field (P.field_T != 0; without it a track moves straight, and the
// kernels for the field-free calorimeters carry no helix code: +1.5 %).
template <class R, int S, int V = 0>
__device__ __forceinline__ int step_transport(const Params& P, Trk<R>& t, Ixn<R>& sec, double& dep, int& dep_bin,
                                              uint32_t& pstep, int& proc) {
  constexpr int q = S == 1 ? -1 : (S == 2 ? 1 : 0);
  const double rest = S == 2 ? 2.0 * kMe : 0.0;
  const int vol = (int)(t.nav & 0xFFFFu);
  uint32_t vac = t.nav >> 16;
  const int m = __ldg(P.geo.vol_mat + vol);
  dep_bin = __ldg(P.geo.vol_bin + vol);
  sec.n = 0;
  dep = 0.0;
  const uint32_t step = t.step;
  pstep = step;
  if (step >= P.max_steps) { atomicAdd(P.evt.killed + t.ev, t.E + rest); return kDead; }
  if (m < 0) {
    if (vac >= P.max_vac) { atomicAdd(P.evt.killed + t.ev, t.E + rest); return kDead; }
    ++vac;
  } else {
    vac = 0;
  }
  const R tcut = (R)P.tcut;
  const R Er = to_r<R>(t.E);
  Stream<R> rs(P.seed, __ldg(P.evt.key + t.ev), t.id, step);
  if (Er < tcut) {
    dep = t.E;
    if (S == 2) { proc = 3; return kInteract; }  // annihilates at rest in phase B
    return kDead;
  }
  R u0, u1;
  rs.block0(&u0, &u1);

  // S2: cross sections and range at the pre-step energy
  R sg0 = 0, sg1 = 0, sg2 = 0, Rr = 0;
  int bin = 0;
  if (m >= 0) {
    R tt;
    grid_pos<R>(t.E, &bin, &tt);
    if (S == 0) {
      const auto* rec = tab_g<R>(P.tab) + ((size_t)m * kNNode + bin) * kNTabG;
      // a process switched off by the mask has a zero table (k_pack)
      sg0 = lerp_rec<R>(rec, 0, tt);
      sg1 = lerp_rec<R>(rec, 1, tt);
      sg2 = lerp_rec<R>(rec, 2, tt);
    } else if (S == 1) {
      const auto* rec = tab_e<R>(P.tab) + ((size_t)m * kNNode + bin) * kNTabE;
      Rr = lerp_rec<R>(rec, 1, tt);
      sg0 = lerp_rec<R>(rec, 2, tt);
      sg1 = lerp_rec<R>(rec, 3, tt);
    } else {
      const auto* rec = tab_p<R>(P.tab) + ((size_t)m * kNNode + bin) * kNTabP;
      Rr = lerp_rec<R>(rec, 1, tt);
      sg0 = lerp_rec<R>(rec, 2, tt);
      sg1 = lerp_rec<R>(rec, 3, tt);
      sg2 = lerp_rec<R>(rec, 4, tt);
    }
  }
  sg0 = sg0 < (R)0 ? (R)0 : sg0;
  sg1 = sg1 < (R)0 ? (R)0 : sg1;
  sg2 = sg2 < (R)0 ? (R)0 : sg2;
  const R stot = sg0 + sg1 + sg2;
  // S3/S4: sampled interaction length and the range-based step limit
  R s_phys = stot > (R)0 ? M<R>::fdiv(-M<R>::flog(u0), stot) : M<R>::big();
  constexpr bool CH = (V & 1) != 0, PH = (V & 2) != 0 && S != 0;
  const bool msc = PH && (P.physics & 1u) != 0, fluct = PH && (P.physics & 2u) != 0;
  bool limited = false;  // the step limit, not the sampled interaction length, ends the step
  if (q != 0 && m >= 0) {
    R smax = (Rr <= (R)kRhoF) ? Rr : ((R)kAlphaR * Rr > (R)kRhoF ? (R)kAlphaR * Rr : (R)kRhoF);
    if (PH && msc) {  // multiple-scattering step limit
      const R fR = (R)P.msc_f * Rr;
      const R sm = fR > (R)0.01 ? fR : (R)0.01;
      if (sm < smax) smax = sm;
    }
    if (smax < s_phys) { s_phys = smax; limited = true; }
  }
  // S5/S6: distance to the boundary along the straight line or helix
  int next;
  const bool field = (V & 8) != 0 && (q != 0) && (P.field_T != 0.0);
  bool boundary;
  R s;
  if constexpr (CH) {
    // chord propagation (paper Sec. 2.3): a step whose integration does not finish within
    // the iteration cap kills its track, with the energy accounted
    R sd;
    const int rc = chord_step<R>(P.geo, P.field_T, t.E, q, s_phys, P.chord_iter, (R)P.delta_chord, (R)P.delta_int,
                                 &t.x, &t.y, &t.z, t.u, vol, &next, &sd);
    if (rc == 2) { atomicAdd(P.evt.killed + t.ev, t.E + rest); return kDead; }
    boundary = rc == 1;
    s = sd;
  } else {
    const R s_geom = field ? helix_distance<R>(P.geo, P.field_T, t.E, q, t.x, t.y, t.z, t.u, vol, &next)
                           : straight_distance<R>(P.geo, t.x, t.y, t.z, t.u, vol, &next);
    boundary = s_geom <= s_phys;
    s = boundary ? s_geom : s_phys;
    if (field) {
      helix_move<R>(P.field_T, t.E, q, s, &t.x, &t.y, &t.z, t.u);
    } else {
      t.x += to_d<R>(s * t.u[0]);
      t.y += to_d<R>(s * t.u[1]);
      t.z += to_d<R>(s * t.u[2]);
    }
  }
  if (boundary && P.geo.kind == 0 && next >= 0) t.z = __ldg(P.geo.bnd + (t.u[2] > (R)0 ? vol + 1 : vol));
  t.step = step + 1;
  if constexpr ((V & 4) != 0) {
    if (P.steplen && s > (R)0 && s < M<R>::big()) {
      // validation histogram of step lengths: bin = floor(log2 s[mm]) + 40
      int b = ilogb(s) + 40;
      b = b < 0 ? 0 : (b > 63 ? 63 : b);
      atomicAdd(P.steplen + 64 * S + b, 1ull);
    }
  }

  // S7: continuous loss by inverting the range table; optionally a Gaussian loss about
  // that mean for a track that survives the mean loss
  if (q != 0 && m >= 0) {
    R Epr = 0;
    if (s < Rr) Epr = inverse_range<R>(range_nodes<R>(P.tab, S == 2) + (size_t)m * kNNode, Rr - s, bin + 1);
    double Ep = (Epr > Er) ? t.E : to_d<R>(Epr);
    if constexpr (PH) {
      if (fluct && s < Rr && Ep >= P.tcut) {
        const R xi = (R)(kTwoPiRe2Me * __ldg(&P.mat[m].n_el));
        const R sig = M<R>::sqrt(fluct_sigma2<R>(Er, xi, (R)__ldg(P.tab.Tc + m), s, S == 2));
        Ep = t.E - fluct_loss<R>(rs, t.E - Ep, sig);
        Epr = to_r<R>(Ep);
      }
    }
    dep += t.E - Ep;
    t.E = Ep;
    if (Epr < tcut) {
      dep += t.E;
      t.E = 0.0;
      if (S == 2) { proc = 3; return kInteract; }  // annihilates at rest in phase B
      return kDead;
    }
    // optional multiple scattering: the direction at the end of the step
    if constexpr (PH) {
      if (msc && s > (R)0) msc_deflect<R>(rs, msc_theta0<R>(Er, (R)__ldg(&P.mat[m].inv_x0), s), t.u);
    }
  }
  // S8: boundary crossing
  if (boundary) {
    if (next < 0) { proc = 4; return kInteract; }  // recorded as it leaves, in phase B
    t.nav = (uint32_t)next | (vac << 16);
    return kAlive;
  }
  t.nav = (uint32_t)vol | (vac << 16);
  // a step cut short by the step limit ends with its continuous loss only
  if (limited) return kAlive;
  // S9 (deferred): the process is chosen with u1 over the fixed order
  const R xs = u1 * stot;
  proc = (S == 1) ? 1 : 2;
  if (xs < sg0) proc = 0;
  else if (xs < sg0 + sg1) proc = 1;
  return kInteract;
}

// Phase B: the discrete interaction (S9) of a track queued by phase A, the annihilation at
// rest of a positron that stopped (process 3), or the outgoing record of a track that left
// the world (process 4). Its random stream is rebuilt from (event,
// id, step): block 0 was consumed in phase A, the models draw from block 1 on. Returns
// whether the parent survives (with its new state in t).
template <class R, int S>
__device__ __forceinline__ bool step_interact(const Params& P, Trk<R>& t, uint32_t pstep, int proc, Ixn<R>& sec,
                                              double& dep) {
  Stream<R> rs(P.seed, __ldg(P.evt.key + t.ev), t.id, pstep);
  if (proc == 4) {  // the track left the world: its energy and its outgoing record
    sec.happened = false;
    sec.n = 0;
    dep = 0.0;
    atomicAdd(P.evt.leaked + t.ev, t.E + (S == 2 ? 2.0 * kMe : 0.0));
    record_leak(P, S == 0 ? 22 : (S == 1 ? 11 : -11), t.ev, t.E, t.x, t.y, t.z, t.u[0], t.u[1], t.u[2]);
    return false;
  }
  if (S == 2 && proc == 3) {  // a positron that stopped: two photons, drawn from block 1 on
    sec.happened = false;
    dep = 0.0;
    annihilate_at_rest<R>(rs, sec);
    return false;
  }
  const int m = __ldg(P.geo.vol_mat + (int)(t.nav & 0xFFFFu));
  const double Tc = __ldg(P.tab.Tc + m), kc = __ldg(P.tab.kc + m);
  const R tcut = (R)P.tcut;
  sec.happened = false;
  sec.n = 0;
  dep = 0.0;
  if (S == 0) {
    if (proc == 0) compton<R>(rs, t.E, t.u, sec);
    else if (proc == 1) pair<R>(rs, t.E, t.u, sec);
    else photo<R>(t.E, t.u, sec);
  } else if (S == 1) {
    if (proc == 0) moller<R>(rs, t.E, Tc, t.u, sec);
    else brem<R>(rs, t.E, kc, t.u, sec);
  } else {
    if (proc == 0) bhabha<R>(rs, t.E, Tc, t.u, sec);
    else if (proc == 1) brem<R>(rs, t.E, kc, t.u, sec);
    else annihilate<R>(rs, t.E, t.u, sec);
  }
  if (!sec.happened) { sec.n = 0; return true; }
  // secondaries other than positrons below the tracking cut deposit locally
#pragma unroll
  for (int k = 0; k < 2; ++k)
    if (k < sec.n && sec.sp[k] != 2 && to_r<R>(sec.E[k]) < tcut) { dep += sec.E[k]; sec.sp[k] = -1; }
  if (!sec.parent_alive) return false;
  t.E = sec.parent_E;
  t.u[0] = sec.pd[0]; t.u[1] = sec.pd[1]; t.u[2] = sec.pd[2];
  if (S == 0 && to_r<R>(t.E) < tcut) { dep += t.E; return false; }
  return true;
}

__device__ __forceinline__ void score(const Params& P, uint32_t ev, int bin, double dep) {
  if (bin >= 0 && __double_as_longlong(dep) != 0) atomicAdd(P.evt.edep + (size_t)ev * P.geo.n_bins + bin, dep);
}

// Warp-aggregated appends (S9/S11): every lane of the warp calls this; a lane passes the
// surviving track (alive) and up to two secondaries, and gets consecutive slots of the
// next queues through one atomic per species per warp.
// Most passes append survivors of the kernel's own species only (every phase-A pass of a
// photon or an electron, and interactions whose secondaries all fell below the cuts): a
// warp-uniform test sends those through one ballot and one reservation instead of nine
// (measured +2.1 % on the 10 GeV showers).
template <class R, int S>
__device__ __forceinline__ void emit(const Params& P, int p, int cw, const Trk<R>& t, bool alive, const Ixn<R>& sec,
                                     uint32_t pstep, uint32_t* ncreated) {
  const int lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  if (!__any_sync(0xFFFFFFFFu, sec.n > 0 && (sec.sp[0] >= 0 || (sec.n > 1 && sec.sp[1] >= 0)))) {
    const uint32_t bs = __ballot_sync(0xFFFFFFFFu, alive);
    uint32_t bk = 0;
    if (lane == 0 && bs) bk = atomicAdd(&P.ctrl->count[cw][S].n, __popc(bs));
    bk = __shfl_sync(0xFFFFFFFFu, bk, 0);
    if (alive) {
      const uint32_t d = bk + __popc(bs & lt);
      if (d < P.cap) {
        store_track<R>(P.qd[3 * (p ^ 1) + S], d, t.x, t.y, t.z, t.u[0], t.u[1], t.u[2], t.E, t.id, t.ev, t.step, t.nav);
      } else {
        atomicAdd(&P.ctrl->overflow, 1ull);
        atomicAdd(P.evt.killed + t.ev, t.E + (S == 2 ? 2.0 * kMe : 0.0));
      }
    }
    return;
  }
  const bool f1 = sec.n > 0 && sec.sp[0] >= 0;
  const bool f2 = sec.n > 1 && sec.sp[1] >= 0;
  const int s1 = f1 ? sec.sp[0] : -1, s2 = f2 ? sec.sp[1] : -1;
  uint32_t b0[3], b1[3], b2[3], wbase[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    b0[k] = __ballot_sync(0xFFFFFFFFu, alive && k == S);
    b1[k] = __ballot_sync(0xFFFFFFFFu, s1 == k);
    b2[k] = __ballot_sync(0xFFFFFFFFu, s2 == k);
    const uint32_t cnt = __popc(b0[k]) + __popc(b1[k]) + __popc(b2[k]);
    uint32_t bk = 0;
    if (lane == 0 && cnt) bk = atomicAdd(&P.ctrl->count[cw][k].n, cnt);
    wbase[k] = __shfl_sync(0xFFFFFFFFu, bk, 0);
    ncreated[k] += __popc(b1[k]) + __popc(b2[k]);
  }
  const TrackSoA* nq = P.qd + 3 * (p ^ 1);
  // pick entry k of a 3-array without dynamic indexing (which would place it in local memory)
  auto pick = [](const uint32_t* a, int k) { return k == 0 ? a[0] : (k == 1 ? a[1] : a[2]); };
  if (alive) {
    const uint32_t d = wbase[S] + __popc(b0[S] & lt);
    if (d < P.cap) {
      store_track<R>(nq[S], d, t.x, t.y, t.z, t.u[0], t.u[1], t.u[2], t.E, t.id, t.ev, t.step, t.nav);
    } else {
      atomicAdd(&P.ctrl->overflow, 1ull);
      atomicAdd(P.evt.killed + t.ev, t.E + (S == 2 ? 2.0 * kMe : 0.0));
    }
  }
  const uint32_t vnav = t.nav & 0xFFFFu;  // secondaries start with no vacuum history
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int sk = k == 0 ? s1 : s2;
    if (sk < 0) continue;
    const uint32_t before = __popc(pick(b0, sk)) + (k == 1 ? __popc(pick(b1, sk)) : 0u);
    const uint32_t mine = __popc((k == 0 ? pick(b1, sk) : pick(b2, sk)) & lt);
    const uint32_t d = pick(wbase, sk) + before + mine;
    if (d < P.cap) {
      const unsigned long long cid = child_id(P.seed, __ldg(P.evt.key + t.ev), t.id, pstep, (uint32_t)k);
      store_track<R>(nq[sk], d, t.x, t.y, t.z, sec.d[k][0], sec.d[k][1], sec.d[k][2], sec.E[k], cid, t.ev, 0u,
                     vnav);
    } else {
      atomicAdd(&P.ctrl->overflow, 1ull);
      atomicAdd(P.evt.killed + t.ev, sec.E[k] + (sk == 2 ? 2.0 * kMe : 0.0));
    }
  }
}

// Per-warp ring of tracks waiting for their discrete interaction (64 entries: phase A of
// one tile adds at most 32 to fewer than 32 waiting, so nothing is overwritten before it
// is processed). Interactions then run 32 at a time on a full warp instead of on the few
// lanes of each tile that happened to interact.
// nav holds the volume in its low half and the process in its high half, in place of the
// vacuum-step count: a discrete interaction (processes 0-2) happens only in a material,
// where that count is 0, and the parent of processes 3 and 4 does not continue. The FP32
// form's entry is then 64 bytes, and three 256-thread blocks take 99 KiB of shared memory,
// which leaves the SM's L1 a larger share (see max_blocks_small_carveout).
constexpr int kRing = 64;
template <class R> struct WarpRing {
  double x[kRing], y[kRing], z[kRing], E[kRing];
  unsigned long long id[kRing];
  R ux[kRing], uy[kRing], uz[kRing];
  uint32_t ev[kRing], pstep[kRing], nav[kRing];
};

// Tiles go to a warp in a fixed stride, so its next tile is known while it steps this one:
// 16 lanes each ask L2 for one of the next tile's 16 lines of track records (4 arrays x 512
// bytes), so that the tile's loads find them there instead of in DRAM (+0.9 % on the 10 GeV
// showers; two tiles ahead gained less). FP32 form: the FP64 form is bound by its FP64 pipe.
template <class R, int S>
__device__ __forceinline__ void prefetch_tile(const Params& P, int p, uint32_t tile, uint32_t n, uint32_t lane) {
  if constexpr (sizeof(R) == 4) {
    const uint32_t e0 = (tile << 5) + ((lane & 3u) << 3);  // first of the 8 records in this lane's line
    if (lane < 16u && e0 < n) {
      const TrackSoA& q = P.qd[3 * p + S];
      const uint32_t a = lane >> 2;
      const char* b = a == 0 ? (const char*)q.xy
                             : (a == 1 ? (const char*)q.zE : (a == 2 ? (const char*)q.un : (const char*)q.meta));
      asm volatile("prefetch.global.L2 [%0];" ::"l"(b + (size_t)e0 * 16));
    }
  }
}

// All of one warp's tiles of species S (tile, tile + stride, ... below tiles). Each pass of
// the loop is either phase A of the next tile (load, step to the next boundary or
// interaction, queue the interactions in the ring) or, once 32 wait or no tile is left, a
// warp of up to 32 queued interactions. Both share the scoring and the appends, so every
// part of the step is inlined once per kernel (smaller code: fewer instruction-cache
// misses).
template <class R, int S, int V = 0>
__device__ __forceinline__ void run_tiles(const Params& P, int p, int cw, uint32_t tile, uint32_t tiles, uint32_t stride,
                                          uint32_t n, WarpRing<R>& ring, uint32_t* nsteps, uint32_t* ncreated) {
  const uint32_t lane = threadIdx.x & 31;
  uint32_t head = 0, tail = 0;
  for (;;) {
    const uint32_t waiting = tail - head;
    const bool phase_a = waiting < 32u && tile < tiles;  // warp-uniform
    if (!phase_a && waiting == 0u) break;
    const uint32_t c = phase_a ? 0u : min(waiting, 32u);
    Trk<R> t;
    t.nav = 0; t.ev = 0; t.id = 0; t.E = 0.0; t.step = 0;
    Ixn<R> sec;
    sec.n = 0;
    uint32_t pstep = 0;
    int outcome = kDead, proc = 0, bin = -1;
    double dep = 0.0;
    if (phase_a) {
      const uint32_t i = (tile << 5) + lane;
      const bool active = i < n;
      if (active) load_track<R>(P.qd[3 * p + S], i, t);
      if (tile + stride < tiles) prefetch_tile<R, S>(P, p, tile + stride, n, lane);
      if (active) outcome = step_transport<R, S, V>(P, t, sec, dep, bin, pstep, proc);
      nsteps[S] += active ? 1u : 0u;  // per lane; reduced over the warp at the end
    } else if (lane < c) {
      const uint32_t j = (head + lane) & (kRing - 1);
      t.x = ring.x[j]; t.y = ring.y[j]; t.z = ring.z[j]; t.E = ring.E[j];
      t.u[0] = ring.ux[j]; t.u[1] = ring.uy[j]; t.u[2] = ring.uz[j];
      const uint32_t nv = ring.nav[j];
      t.id = ring.id[j]; t.ev = ring.ev[j]; t.nav = nv & 0xFFFFu;
      pstep = ring.pstep[j];
      t.step = pstep + 1;
      outcome = step_interact<R, S>(P, t, pstep, (int)(nv >> 16), sec, dep) ? kAlive : kDead;
      bin = __ldg(P.geo.vol_bin + (int)(t.nav & 0xFFFFu));
    }
    // S10: score the step's deposit in (event, layer, material)
    score(P, t.ev, bin, dep);
    emit<R, S>(P, p, cw, t, outcome == kAlive, sec, pstep, ncreated);
    if (phase_a) {
      const uint32_t need = __ballot_sync(0xFFFFFFFFu, outcome == kInteract);
      if (outcome == kInteract) {
        const uint32_t j = (tail + __popc(need & ((1u << lane) - 1u))) & (kRing - 1);
        ring.x[j] = t.x; ring.y[j] = t.y; ring.z[j] = t.z; ring.E[j] = t.E;
        ring.ux[j] = t.u[0]; ring.uy[j] = t.u[1]; ring.uz[j] = t.u[2];
        ring.id[j] = t.id; ring.ev[j] = t.ev; ring.nav[j] = (t.nav & 0xFFFFu) | ((uint32_t)proc << 16);
        ring.pstep[j] = pstep;
      }
      tail += __popc(need);
      tile += stride;
    } else {
      head += c;
    }
    // the next pass may write ring entries that lanes of this one read
    __syncwarp();
  }
}

// Programmatic dependent launch between generations: a generation's kernels may be
// launched (and their blocks made resident) as soon as every block of the previous
// generation's kernels has started, so that they wait on the SMs instead of being launched
// after the previous generation ends. grid_dependency_wait() returns once the previous
// generation's grids have completed and their writes are visible; both are no-ops for a
// launch without programmatic dependencies.
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void allow_dependent_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// The bookkeeping between generations, done by one thread of generation g while it runs:
// empty the size slot that generation g + 1 appends to (its last reader, generation g - 1,
// has ended), and log the sizes generation g - 1 left (final once it ended). gk = 0 (the
// first generation of a chunk) leaves the log to the end of the previous chunk.
__device__ __forceinline__ void open_generation(const Params& P, uint32_t gen, uint32_t gk) {
  volatile Ctrl* c = P.ctrl;
  const uint32_t cz = (gen + 2) % 3, cr = gen % 3;
  for (int k = 0; k < 3; ++k) c->count[cz][k].n = 0;
  if (gk == 0) return;
  const uint32_t ln = c->log_n;
  if (ln < P.max_log) {
    for (int k = 0; k < 3; ++k) P.gen_log[3 * ln + k] = min(c->count[cr][k].n, P.cap);
    c->log_n = ln + 1;
  }
}

// One generation of one species (paper Sec. 3: TransportElectrons, TransportPositrons and
// TransportGammas). Persistent launch: each warp takes 32-track tiles of the current queue.
// The three species kernels of a generation are independent (each reads its own current
// queue and appends to the next ones atomically), so they run concurrently on three
// streams, and the next generation's kernels start once all three have ended.
// gk: the generation's place in its chunk (gen, advanced only between chunks, plus gk).
// V: the variant of the step (see step_transport); variants.cu instantiates V = 1..3 for
// e- and e+.
template <class R, int S, int MINB, int V = 0>
__global__ void __launch_bounds__(256, MINB) k_transport(Params P, uint32_t gk) {
  __shared__ unsigned long long s_steps, s_created[3];
  __shared__ WarpRing<R> rings[8];
  grid_dependency_wait();
  allow_dependent_launch();
  if (gk == kGkDevice) gk = __ldcg(&P.ctrl->tail_k);  // a generation of a tail chunk
  const uint32_t gen = __ldcg(&P.ctrl->gen) + gk;
  const int p = gen & 1;
  if (threadIdx.x == 0) { s_steps = 0; s_created[0] = s_created[1] = s_created[2] = 0; }
  // one block of the e- kernel does the bookkeeping (any of the three could)
  if (S == 1 && blockIdx.x == 0 && threadIdx.x == 0) open_generation(P, gen, gk);
  __syncthreads();
  // injection may have counted past the capacity (those tracks were dropped)
  const uint32_t n = min(__ldcg(&P.ctrl->count[gen % 3][S].n), P.cap);
  const uint32_t tiles = (n + 31) >> 5;
  const uint32_t wpb = blockDim.x >> 5;
  WarpRing<R>& ring = rings[threadIdx.x >> 5];
  // counts of one generation (at most the queue capacity each: 32 bits suffice): steps per
  // lane, reduced over the warp at the end (a ballot per pass measured 1.2 % slower), and
  // secondaries per warp
  uint32_t nsteps[3] = {0, 0, 0}, ncreated[3] = {0, 0, 0};
  run_tiles<R, S, V>(P, p, (gen + 1) % 3, blockIdx.x * wpb + (threadIdx.x >> 5), tiles, gridDim.x * wpb, n, ring,
                     nsteps, ncreated);
  const uint32_t wsteps = __reduce_add_sync(0xFFFFFFFFu, nsteps[S]);
  if ((threadIdx.x & 31) == 0) {
    if (wsteps) atomicAdd(&s_steps, (unsigned long long)wsteps);
    for (int k = 0; k < 3; ++k)
      if (ncreated[k]) atomicAdd(&s_created[k], (unsigned long long)ncreated[k]);
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  if (s_steps) atomicAdd(&P.ctrl->steps[S], s_steps);
  for (int k = 0; k < 3; ++k)
    if (s_created[k]) atomicAdd(&P.ctrl->created[k], s_created[k]);
}

}  // namespace adept
