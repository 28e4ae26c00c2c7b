#!/usr/bin/env python
"""Throughput of the GB300 shower transport on its headline workload.

Workload: 10,000 primary 10 GeV electrons at normal incidence on the 50-layer Pb/lAr
sampling calorimeter (40 x 40 cm, 0.7 mm production cut, no field), split precision
(FP32 physics, FP64 positions/boundary distances/energy), all events batched into one
persistent-kernel transport with CUDA-graph chunks of generations. One bench step is the
complete transport of that batch: injection, every generation until the last track
dies, and the per-event scoring returned to the host.

Prints one JSON line (rank 0): tracked steps/s for the whole job, 10 GeV showers/s,
the step kernel's achieved HBM bandwidth against the measured peak, the FP64 CPU oracle
timed on this host's cores, an end-to-end number through the C ABI with host buffers,
and the SM clocks seen during the timed region.

``--impl reference`` times the FP64 CPU oracle (the reference of this build) instead.
Multi-GPU (torchrun): every rank transports its own independent batch of events (the
path shards by event with no exchange), the timed region is bracketed by barriers and
the slowest rank's time is used.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "tracked steps/sec and 10 GeV e- showers/sec on 1 GB300; HBM GB/s vs peak"
UNIT = "tracked steps/s"
WORKLOAD = ("10,000 x 10 GeV e- showers, 50-layer Pb 2.3 mm + lAr 5.7 mm slab calorimeter, 0.7 mm cut, "
            "no field; split precision, batched persistent launch with CUDA graphs")
TRACK_BYTES_SPLIT = 64  # x,y,z f64 + direction 3 f32 + E f64 + id u64 + event, step, nav u32
# DRAM bytes (read + write) per tracked step of the three concurrent transport kernels, from
# the ncu captures of generation 60 (profiles/transport_kernels_10gev_e_showers_gen60_full.md
# for the split form, profiles/transport_kernels_10gev_e_showers_fp64_gen60_full.md for the
# plain FP64 form); valid while the kernel sources hash to NCU_SRC_HASH, null otherwise
NCU_BYTES_PER_STEP = {1: 107.9, 0: 132.1}
NCU_SRC_HASH = "0364c2f2c0239b1f"


def kernel_src_hash() -> str:
    h = hashlib.sha256()
    for f in ("kernels.cu", "transport.cuh", "device.cuh", "layout.h"):
        with open(os.path.join(ROOT, "paper_2209_15445_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def args_parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--events", type=int, default=10000)
    ap.add_argument("--energy", type=float, default=1e4)
    ap.add_argument("--precision", type=int, default=1)
    ap.add_argument("--graph", type=int, default=0, help="generations per CUDA graph (0 = tuned)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 form on the same workload")
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--fp64-warmup", type=int, default=1)
    ap.add_argument("--one-events", type=int, default=20,
                    help="events of the FP64 one-event-per-launch sample in fp64_form")
    ap.add_argument("--arena-gb", type=float, default=10.0)
    ap.add_argument("--bps", type=int, default=0, help="transport-kernel blocks/SM variant (0 = library default)")
    ap.add_argument("--bps-species", type=str, default="", help="per-species variants gamma,e-,e+")
    ap.add_argument("--block", type=int, default=0, help="threads per transport block (0 = tuned)")
    ap.add_argument("--workload", default="c2", choices=["c1", "c2", "c3", "c4", "c5", "rt", "batch"],
                    help="c2 (default) is the headline line; the others are the configuration studies")
    ap.add_argument("--seconds", type=float, default=20.0, help="serving workload duration")
    ap.add_argument("--genlog", default="", help="write the per-generation queue sizes of the last step here")
    ap.add_argument("--no-kernel-timing", action="store_true", help="no CUDA events around the transport kernels")
    ap.add_argument("--species-timing", action="store_true", help="also time each species kernel")
    ap.add_argument("--physics", type=int, default=0, choices=[0, 1, 2, 3],
                    help="optional continuous physics: 1 multiple scattering, 2 loss fluctuations, 3 both "
                         "(0: the paper's process list, the headline)")
    ap.add_argument("--field-iter", type=int, default=0,
                    help="c3/c4: chord propagation in the field with this iteration cap (0: analytic helix)")
    ap.add_argument("--fused", type=int, default=-1, choices=[-1, 0, 1],
                    help="1: one kernel per generation for all species; 0: concurrent species kernels; -1: tuned")
    return ap.parse_args()


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p:
            time.sleep(0.25)
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
                self.out, _ = self.p.communicate()

    def summary(self):
        rows = [r for r in csv.reader(io.StringIO(self.out or "")) if len(r) >= 9]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].strip().lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def oracle_rate(n_events, energy, threads=None, physics=0):
    """FP64 oracle (as it stands) on n_events of the workload; returns (steps/s, steps, s, cores)."""
    import oracle
    from paper_2209_15445_gb300 import workloads as W
    o = oracle.Oracle(W.slab_calorimeter())
    prim = W.electrons(n_events, energy, first_event=777000)
    cores = threads or os.cpu_count() or 1
    t0 = time.perf_counter()
    r = o.transport(prim, n_threads=cores, physics=physics)
    dt = time.perf_counter() - t0
    steps = int(r["steps"].sum())
    return steps / dt, steps, dt, cores


def cpu_baseline(energy, target_s=12.0, physics=0):
    rate, steps, dt, cores = oracle_rate(8, energy, physics=physics)
    per_event = steps / 8
    n = max(8, min(10000, int(target_s * rate / per_event)))
    rate, steps, dt, cores = oracle_rate(n, energy, physics=physics)
    return {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} of the 10,000 events ({steps} steps, {dt:.1f} s), FP64 C oracle on {cores} threads",
            "showers_per_s": n / dt}


def run_reference(a):
    ws, rank, _ = dist_info()
    if rank != 0:
        return
    rate, steps, dt, cores = oracle_rate(8, a.energy)
    per_event = steps / 8
    per_step_s = max(2.0, min(20.0, 120.0 / max(1, a.steps + a.warmup)))
    n = max(8, min(10000, int(per_step_s * rate / per_event)))
    for _ in range(a.warmup):
        oracle_rate(max(2, n // 8), a.energy)
    tot_steps, tot_t = 0, 0.0
    for _ in range(a.steps):
        r, s, d, cores = oracle_rate(n, a.energy)
        tot_steps += s
        tot_t += d
    value = tot_steps / tot_t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * tot_t / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "events_per_step": n, "precision": "fp64 cpu oracle"},
            "showers_per_s": n * a.steps / tot_t,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{n} events of 10 GeV e- per step on {cores} host threads"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def reduce_over_ranks(t, steps, device):
    """Whole-job timing over replicas: the slowest rank's time and the sum of all ranks'
    tracked steps (device None: a single process)."""
    if device is None:
        return t, steps
    import torch
    import torch.distributed as dist
    v = torch.tensor([float(t), float(steps)], dtype=torch.float64, device=device)
    vmax = v.clone()
    dist.all_reduce(vmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(v, op=dist.ReduceOp.SUM)
    return float(vmax[0]), int(v[1])


def run_ours(a):
    import numpy as np
    import torch

    from paper_2209_15445_gb300 import adept as A
    from paper_2209_15445_gb300 import build as B
    from paper_2209_15445_gb300 import workloads as W

    ws, rank, local = dist_info()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl", init_method="env://")
    torch.cuda.set_device(local)
    B.build()
    dev = torch.device("cuda", local)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    n, E = a.events, a.energy
    geom = W.slab_calorimeter()
    prim = W.electrons(n, E, first_event=rank * n)  # each rank: its own events
    host = A.tracks_array(prim)
    dev_tracks = torch.from_numpy(host.view(np.uint8).copy()).to(dev)
    # launch settings: the autotuned ones (tuning.json) unless given on the command line
    launch_opts = {}
    if a.bps:
        launch_opts["blocks_per_sm"] = a.bps
    if a.bps_species:
        launch_opts["blocks_per_sm_species"] = (A.C.c_int32 * 3)(*[int(x) for x in a.bps_species.split(",")])
    if a.graph:
        launch_opts["graph_generations"] = a.graph
    if a.block:
        launch_opts["block_size"] = a.block
    if a.fused >= 0:
        launch_opts["fused"] = a.fused
    if a.physics:
        launch_opts["physics"] = a.physics
    tr = A.Transport(geom, precision=a.precision, arena_bytes=int(a.arena_gb * (1 << 30)),
                     flags=0 if a.no_kernel_timing else (A.FLAG_TIME_SPECIES if a.species_timing else A.FLAG_TIME_STEPS),
                     max_events=max(65536, n), **launch_opts)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB of L2

    out_rows = np.empty((n, tr.n_bins))  # the caller's result buffer, reused every step

    def step_device():
        rid = tr.submit_device(dev_tracks, n)
        tr.transport()
        out, meta = tr.result(rid, n, out=out_rows)
        return meta

    for _ in range(a.warmup):
        step_device()
    if a.genlog:
        A.adept_reset_generation_log(tr.h)
    s0 = tr.stats()
    barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
    clk = Clocks(local)
    with clk:
        for k in range(a.steps):
            flush.zero_()
            torch.cuda.synchronize()
            ev[k][0].record(tr.stream)
            meta = step_device()
            ev[k][1].record(tr.stream)
        barrier()
    s1 = tr.stats()
    if a.genlog:
        nlog, log = A.adept_get_generation_log(tr.h)
        np.savetxt(a.genlog, log, fmt="%d", header="gamma e- e+ queue sizes after each generation")
    t_ms = sum(e0.elapsed_time(e1) for e0, e1 in ev)
    steps = sum(s1.steps) - sum(s0.steps)
    launches = s1.launches - s0.launches
    kern_ms = s1.step_kernel_ms - s0.step_kernel_ms
    kern_n = s1.step_launches - s0.step_launches
    species_ms = [s1.species_ms[k] - s0.species_ms[k] for k in range(3)]
    edep_ok = abs(meta.deposited_MeV + meta.leaked_MeV + meta.killed_MeV - n * E) <= 1e-9 * n * E
    t_ms_max, steps_all = reduce_over_ranks(t_ms, steps, dev if ws > 1 else None)
    value = steps_all / (t_ms_max / 1e3)
    showers = ws * n * a.steps / (t_ms_max / 1e3)

    # roofline of the step kernel: algorithmic track-state bytes per launch / its mean duration
    tb = TRACK_BYTES_SPLIT if a.precision else 76
    alg_bytes = tb * (2 * steps - a.steps * n)
    peak, peak_kind = peaks()
    achieved = alg_bytes / (kern_ms / 1e3) / 1e9 if kern_ms > 0 else None
    traffic = None
    # the ncu figures were taken on the concurrent species kernels; the fused mode reports none
    if a.precision in NCU_BYTES_PER_STEP and not tr.options.fused and NCU_SRC_HASH == kernel_src_hash() and kern_n:
        traffic = NCU_BYTES_PER_STEP[a.precision] * steps / kern_n
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": (achieved / peak) if achieved else None, "traffic": traffic,
            "kernel": ("k_fused_generation<%s> (one launch = one generation, all species)" if tr.options.fused else
                       "k_transport<%s, species> x3, concurrent (one launch = one generation: gamma, e+, e-)")
                      % ("float" if a.precision else "double"),
            "alg_bytes_per_launch": alg_bytes / kern_n if kern_n else None,
            "mean_launch_us": 1e3 * kern_ms / kern_n if kern_n else None,
            "launches": kern_n, "peak_kind": f"{peak_kind} (hbm_gbs burst copy)",
            "kernel_share_of_step_time": kern_ms / t_ms if t_ms else None,
            "species_ms_per_step": [round(x / a.steps, 3) for x in species_ms] if a.species_timing else None}

    # end to end through the C ABI with host buffers: submit copies host tracks to the device
    e2e = None
    if not a.no_e2e:
        barrier()
        e0 = tr.stats()
        t0 = time.perf_counter()
        for _ in range(max(1, a.steps // 2)):
            rid = tr.submit(host)
            tr.transport()
            out, m2 = tr.result(rid, n, out=out_rows)
        barrier()
        dt = time.perf_counter() - t0
        e1 = tr.stats()
        k2 = max(1, a.steps // 2)
        st2 = sum(e1.steps) - sum(e0.steps)
        dt, st2 = reduce_over_ranks(dt, st2, dev if ws > 1 else None)
        e2e = {"value": st2 / dt, "unit": UNIT, "h2d_bytes_per_step": int(n * (72 + 8) + 4 * n),
               "d2h_bytes_per_step": int(n * (geom.n_bins + 2) * 8), "steps": k2,
               "showers_per_s": ws * n * k2 / dt}

    # the plain FP64 form on the same workload and GPU, in the same process (the comparison
    # the split form is built for): FP64 physics, one array per field, its own tuned launch
    fp64 = None
    topt = tr.options
    if a.precision and not a.no_fp64:
        tr.close()
        tr = None
        del dev_tracks
        torch.cuda.empty_cache()
        dev64 = torch.from_numpy(host.view(np.uint8).copy()).to(dev)
        t64 = A.Transport(geom, precision=0, arena_bytes=int(a.arena_gb * (1 << 30)), flags=A.FLAG_TIME_STEPS,
                          max_events=max(65536, n))

        out64 = np.empty((n, t64.n_bins))

        def step64():
            rid = t64.submit_device(dev64, n)
            t64.transport()
            return t64.result(rid, n, out=out64)[1]

        for _ in range(a.fp64_warmup):
            step64()
        f0 = t64.stats()
        barrier()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.fp64_steps)]
        for k in range(a.fp64_steps):
            flush.zero_()
            torch.cuda.synchronize()
            evs[k][0].record(t64.stream)
            m64 = step64()
            evs[k][1].record(t64.stream)
        barrier()
        f1 = t64.stats()
        ms64 = sum(e0.elapsed_time(e1) for e0, e1 in evs)
        st64 = sum(f1.steps) - sum(f0.steps)
        km64 = f1.step_kernel_ms - f0.step_kernel_ms
        kn64 = f1.step_launches - f0.step_launches
        ok64 = abs(m64.deposited_MeV + m64.leaked_MeV + m64.killed_MeV - n * E) <= 1e-9 * n * E
        fp64 = {"value": st64 / (ms64 / 1e3), "unit": UNIT, "showers_per_s": n * a.fp64_steps / (ms64 / 1e3),
                "ms_per_step": ms64 / a.fp64_steps, "steps": a.fp64_steps, "warmup": a.fp64_warmup,
                "steps_per_shower": st64 / (a.fp64_steps * n), "energy_conserved": bool(ok64),
                "blocks_per_sm_species": list(t64.options.blocks_per_sm_species),
                "kernel_share_of_step_time": km64 / ms64 if ms64 else None,
                "algorithmic_GBs": 76 * (2 * st64 - a.fp64_steps * n) / (km64 / 1e3) / 1e9 if km64 else None,
                "mean_launch_us": 1e3 * km64 / kn64 if kn64 else None,
                "traffic": (NCU_BYTES_PER_STEP[0] * st64 / kn64
                            if kn64 and NCU_SRC_HASH == kernel_src_hash() else None),
                "split_over_fp64": value / (st64 / (ms64 / 1e3))}
        t64.close()
        del dev64
        # the plain FP64 form one event per transport, one generation per launch with the
        # queue sizes read back after each (no graphs), on a sample of the same events
        t1 = A.Transport(geom, precision=0, arena_bytes=1 << 30, graph_generations=-1, max_events=1024)
        one = [A.tracks_array(prim.take([i])) for i in range(a.one_events + 1)]
        rid = t1.submit(one[-1]); t1.transport(); t1.result(rid, 1)  # warm-up
        g0 = t1.stats()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(a.one_events):
            rid = t1.submit(one[k]); t1.transport(); t1.result(rid, 1)
        torch.cuda.synchronize()
        dt1 = time.perf_counter() - t0
        g1 = t1.stats()
        t1.close()
        st1 = sum(g1.steps) - sum(g0.steps)
        fp64["one_event_per_launch"] = {"value": st1 / dt1, "unit": UNIT, "showers_per_s": a.one_events / dt1,
                                        "events": a.one_events, "ms_per_event": 1e3 * dt1 / a.one_events,
                                        "gpu_launches_per_event": (g1.launches - g0.launches) / a.one_events,
                                        "split_over_this": value / (st1 / dt1)}

    base = None
    if rank == 0 and ws == 1 and not a.no_cpu_baseline:
        base = cpu_baseline(E, physics=a.physics)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": a.steps,
                "warmup": a.warmup, "ms_per_step": t_ms_max / a.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f32/f64" if a.precision else "f64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "events": n, "E_MeV": E, "precision": "split" if a.precision else "fp64",
                           "graph_generations": topt.graph_generations,
                           "block": topt.block_size or 256,
                           "fused": int(topt.fused),
                           "physics": {0: "paper process list", 1: "+ multiple scattering", 2: "+ loss fluctuations",
                                       3: "+ multiple scattering + loss fluctuations"}[a.physics],
                           "blocks_per_sm": int(topt.blocks_per_sm),
                           "blocks_per_sm_species": list(topt.blocks_per_sm_species) if not a.bps else [a.bps] * 3,
                           "l2": "track queues (GBs) exceed L2; 256 MB buffer written between steps"},
                "showers_per_s": showers, "steps_per_shower": steps / (a.steps * n),
                "generations_per_step": (s1.generations - s0.generations) / a.steps,
                "energy_conserved": bool(edep_ok), "roofline": roof, "fp64_form": fp64, "cpu_baseline": base, "e2e": e2e,
                "gpu_launches": int(launches), "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    if tr is not None:
        tr.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def _line(a, workload, value, t_s, extra):
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": 1e3 * t_s / max(1, a.steps), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32/f64" if a.precision else "f64", "data": "synthetic",
            "config": {"workload": workload, **extra.pop("config", {})}, **extra}


def run_study(a):
    """Configuration studies (not the headline line): c1 plain FP64 one event per launch,
    c3 batched mixed primaries in 1 T, c4 barrel in 3.8 T, c5 serving with 16 producers."""
    import threading

    import numpy as np
    import torch

    from paper_2209_15445_gb300 import adept as A
    from paper_2209_15445_gb300 import build as B
    from paper_2209_15445_gb300 import workloads as W

    B.build()
    torch.cuda.set_device(0)
    if a.workload == "rt":
        # ray-traced images of the barrel (paper Sec. 2.1: single against double precision
        # navigation), 4096 x 4096 side view into device memory, and the CPU oracle on a
        # 256 x 256 image of the same view
        import oracle
        geom = W.barrel_calorimeter()
        cam = [-4000.0, 0.0, 0.0, 1.0, 0.05, 0.02, 0, 0, 1, 3800.0, 6500.0]
        nx = ny = 4096
        tr = A.Transport(geom, precision=1, field_T=3.8, arena_bytes=1 << 30)
        dev = torch.empty(nx * ny * 2, dtype=torch.float64, device="cuda")
        res = {}
        for prec in (0, 1):
            for _ in range(max(1, a.warmup)):
                A.adept_raytrace_device(tr.h, prec, cam, nx, ny, dev.data_ptr())
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            tr.stream.synchronize()
            e0.record(tr.stream)
            for _ in range(a.steps):
                assert A.adept_raytrace_device(tr.h, prec, cam, nx, ny, dev.data_ptr()) == 0
            e1.record(tr.stream)
            tr.stream.synchronize()
            ms = e0.elapsed_time(e1) / a.steps
            crossings = float(dev.view(ny, nx, 2)[..., 1].sum())
            res["fp32" if prec else "fp64"] = {"ms": ms, "rays_per_s": nx * ny / (ms / 1e3),
                                                "crossings_per_s": crossings / (ms / 1e3)}
        tr.close()
        o = oracle.Oracle(geom, field_T=3.8)
        t0 = time.perf_counter()
        o.raytrace(cam, 256, 256)
        cpu = 256 * 256 / (time.perf_counter() - t0)
        line = {"metric": "ray-traced pixels/s (geometry validation)", "value": res["fp32"]["rays_per_s"],
                "unit": "pixels/s", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
                "ms_per_step": res["fp32"]["ms"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32 distances / f64 positions", "data": "synthetic",
                "config": {"workload": "4096 x 4096 orthographic side view of the 20-layer barrel"},
                "fp64": res["fp64"], "fp32": res["fp32"], "fp32_over_fp64": res["fp32"]["rays_per_s"] / res["fp64"]["rays_per_s"],
                "cpu_baseline": {"value": cpu, "unit": "pixels/s", "cores": 1, "kind": "oracle",
                                 "sample": "256 x 256 image of the same view, FP64 C oracle, one thread"}}
        print(json.dumps(line))
        return
    if a.workload == "batch":
        # throughput against the number of 10 GeV e- showers transported together (paper
        # Sec. 5: batching primaries keeps the GPU busy); one line per batch size
        geom = W.slab_calorimeter()
        tr = A.Transport(geom, precision=1, arena_bytes=int(a.arena_gb * (1 << 30)), max_events=65536)
        rows = []
        for nb in (1, 10, 100, 1000, 10000, 30000):
            arr = A.tracks_array(W.electrons(nb, 1e4))
            ob = np.empty((nb, tr.n_bins))  # the caller's result buffer, reused
            rid = tr.submit(arr); tr.transport(); tr.result(rid, nb, out=ob)
            s0 = tr.stats(); torch.cuda.synchronize(); t0 = time.perf_counter()
            reps = max(1, min(a.steps, int(30000 / nb)))
            for _ in range(reps):
                rid = tr.submit(arr); tr.transport(); tr.result(rid, nb, out=ob)
            torch.cuda.synchronize(); dt = time.perf_counter() - t0; s1 = tr.stats()
            st = sum(s1.steps) - sum(s0.steps)
            rows.append({"showers_per_batch": nb, "steps_per_s": st / dt, "showers_per_s": nb * reps / dt,
                         "ms_per_batch": 1e3 * dt / reps})
        tr.close()
        print(json.dumps(_line(a, "10 GeV e- showers in batches of 1 to 30,000 (slab, split, end to end through the "
                                  "C ABI with host buffers)", rows[-2]["steps_per_s"], rows[-2]["ms_per_batch"] / 1e3,
                               {"batches": rows})))
        return
    if a.workload == "c1":
        # plain FP64, one event per transport, one generation per launch with the queue
        # sizes read back after each (the paper's small-batch form)
        tr = A.Transport(W.slab_calorimeter(), precision=0, arena_bytes=1 << 30, graph_generations=-1)
        prim = W.electrons(100, 1000.0)
        arrs = [A.tracks_array(prim.take([i])) for i in range(100)]
        for k in range(a.warmup):
            rid = tr.submit(arrs[k]); tr.transport(); tr.result(rid, 1)
        s0 = tr.stats(); t0 = time.perf_counter()
        for k in range(100):
            rid = tr.submit(arrs[k]); tr.transport(); tr.result(rid, 1)
        dt = time.perf_counter() - t0; s1 = tr.stats()
        st = sum(s1.steps) - sum(s0.steps)
        a.precision = 0
        print(json.dumps(_line(a, "100 x 1 GeV e-, slab, plain FP64, one event per transport, one generation per launch",
                               st / dt, dt, {"showers_per_s": 100 / dt, "steps": 1, "gpu_launches": int(s1.launches - s0.launches)})))
        return
    if a.workload in ("c3", "c4"):
        if a.workload == "c3":
            geom, field, prim = W.slab_calorimeter(), 1.0, W.mixed(20000, seed=3)
            name = "20,000 primaries 0.1-100 GeV, 50% gamma / 40% e- / 10% e+, slab, 1 T; split, batched"
            chunks, arena = 1, 12 << 30
        else:
            geom, field, prim = W.barrel_calorimeter(), 3.8, W.barrel_primaries(100000, seed=4)
            name = "100,000 e-/gamma 1-50 GeV, |eta|<1.5, 20-layer barrel, 3.8 T; split, batched in 100 requests"
            chunks, arena = 100, 40 << 30
        fo = {"fused": a.fused} if a.fused >= 0 else {}
        if a.field_iter:
            fo["field_max_iterations"] = a.field_iter
        tr = A.Transport(geom, precision=a.precision, field_T=field, arena_bytes=arena, graph_generations=a.graph,
                         flags=A.FLAG_TIME_STEPS if a.fused == 1 else A.FLAG_TIME_SPECIES, max_events=200000,
                         tracks_per_MeV=0.1, **fo)
        n = len(prim)
        parts = [prim.take(np.arange(k * n // chunks, (k + 1) * n // chunks)) for k in range(chunks)]
        arrs = [A.tracks_array(pp) for pp in parts]

        def once():
            ids = [tr.submit(x) for x in arrs]
            tr.transport()
            k = 0.0
            for rid, pp in zip(ids, parts):
                k += tr.result(rid, len(pp))[1].killed_MeV
            return k
        once()
        s0 = tr.stats(); torch.cuda.synchronize(); t0 = time.perf_counter()
        killed = 0.0
        for _ in range(a.steps):
            killed += once()
        torch.cuda.synchronize(); dt = time.perf_counter() - t0; s1 = tr.stats()
        st = sum(s1.steps) - sum(s0.steps)
        print(json.dumps(_line(a, name, st / dt, dt / a.steps,
                               {"showers_per_s": n * a.steps / dt, "steps_per_primary": st / (n * a.steps),
                                "field": f"chords, at most {a.field_iter} iterations per step" if a.field_iter
                                else "analytic helix",
                                "killed_fraction": killed / (a.steps * float((prim.E + np.where(prim.pdg == -11,
                                                                                                 2 * 0.51099895, 0.0)).sum())),
                                "species_ms_per_step": [round((s1.species_ms[k] - s0.species_ms[k]) / a.steps, 2) for k in range(3)],
                                "gpu_launches": int(s1.launches - s0.launches)})))
        return
    # c5: serving -- 16 producers in a closed loop, one driver thread running the transport
    geom = W.barrel_calorimeter()
    # serving keeps few tracks per generation in flight: one fused kernel per generation
    # (less launch latency per generation) serves it faster than concurrent species kernels
    fo = {"fused": a.fused if a.fused >= 0 else 1}
    tr = A.Transport(geom, precision=a.precision, field_T=3.8, arena_bytes=24 << 30,
                     graph_generations=a.graph or 8, max_events=65536, tracks_per_MeV=0.1, **fo)
    stop = threading.Event()
    lat, done_steps, errors = [], [0], []
    lock = threading.Lock()

    def driver():
        while not stop.is_set():
            rc = A.adept_transport(tr.h, 20000)
            if rc not in (A.OK, A.ETIMEOUT):
                errors.append(A.adept_last_error(tr.h)); return
            if rc == A.OK:
                time.sleep(5e-5)

    def producer(k):
        rng = np.random.default_rng(1000 + k)
        ev = 1_000_000 * (k + 1)
        while not stop.is_set():
            nb = W.serving_batch_size(rng)
            batch = W.serving_batch(nb, seed=int(rng.integers(1 << 30)), event=ev)
            ev += 1
            rid = tr.submit(batch)
            while A.adept_wait(tr.h, rid, 200000) == A.ETIMEOUT:
                if stop.is_set():
                    return
            out, meta = tr.result(rid, 1)
            with lock:
                lat.append(meta.latency_us)

    th = [threading.Thread(target=driver)] + [threading.Thread(target=producer, args=(k,)) for k in range(16)]
    s0 = tr.stats(); t0 = time.perf_counter()
    for t in th:
        t.start()
    time.sleep(a.seconds)
    stop.set()
    for t in th:
        t.join()
    dt = time.perf_counter() - t0; s1 = tr.stats()
    st = sum(s1.steps) - sum(s0.steps)
    l = np.array(lat) if lat else np.zeros(1)
    print(json.dumps(_line(a, "serving: 16 producers, batches of 10-10,000 e-/e+/gamma (E^-2, 10 MeV-20 GeV) on the barrel inner face, 3.8 T",
                           st / dt, dt, {"requests": len(lat), "latency_us": {"p50": float(np.percentile(l, 50)),
                                                                              "p99": float(np.percentile(l, 99)),
                                                                              "mean": float(l.mean())},
                                         "errors": errors})))


def main():
    a = args_parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.workload != "c2":
        run_study(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
