"""Autotuner for the transport launch configuration.

Measures tracked steps/s of a workload on the current GPU for candidate launch settings
and keeps the fastest: the CUDA-graph chunk length, the block size, and per species the
register-cap variant of its transport kernel (how many 256-thread blocks per SM it is
compiled for, which trades occupancy against spills). Search: coordinate descent from
the library defaults, then the fused one-kernel-per-generation mode with its variants. The result is written to tuning.json next to this file, keyed by
"<geometry kind>/<precision>", and `adept.Transport` applies it to options the caller
leaves at zero.

    python -m paper_2209_15445_gb300.autotune            # slab split + FP64, barrel split
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
TUNING = os.path.join(HERE, "tuning.json")


def key(kind: int, precision: int) -> str:
    return f"{'slab' if kind == 0 else 'tubes'}/{'split' if precision else 'fp64'}"


def load() -> dict:
    try:
        with open(TUNING) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def measure(geom, prim, precision, field_T, cfg, repeat=2):
    """tracked steps/s of transporting prim with launch settings cfg (dict of options)"""
    import torch

    from . import adept as A

    bps = cfg.get("blocks_per_sm_species", [0, 0, 0])
    extra = {"fused": 1, "blocks_per_sm": cfg["blocks_per_sm"]} if cfg.get("fused") else \
        {"blocks_per_sm_species": (A.C.c_int32 * 3)(*bps)}
    tr = A.Transport(geom, precision=precision, field_T=field_T, arena_bytes=cfg.get("arena_bytes", 10 << 30),
                     graph_generations=cfg["graph_generations"], block_size=cfg["block_size"],
                     max_events=max(65536, len(prim)), tuned=False, **extra)
    arr = A.tracks_array(prim)
    n_ev = len(np.unique(prim.event))
    rid = tr.submit(arr); tr.transport(); tr.result(rid, n_ev)  # warm-up (graph capture)
    s0 = tr.stats()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(repeat):
        rid = tr.submit(arr); tr.transport(); tr.result(rid, n_ev)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    steps = sum(tr.stats().steps) - sum(s0.steps)
    tr.close()
    return steps / dt


def tune(geom, prim, precision, field_T=0.0, log=print):
    cfg = {"graph_generations": 32, "block_size": 256, "blocks_per_sm_species": [3, 3, 3] if precision else [2, 2, 2]}
    best = measure(geom, prim, precision, field_T, cfg)
    log(f"  start {cfg}: {best:.3e}")
    trials = [("graph_generations", v) for v in (16, 64)]
    trials += [("block_size", v) for v in (64, 128)]  # 256 is the kernels' launch bound
    for sp in range(3):
        for v in (1, 2, 3, 4):
            trials.append((("blocks_per_sm_species", sp), v))
    for what, v in trials:
        c = json.loads(json.dumps(cfg))
        if isinstance(what, tuple):
            if c[what[0]][what[1]] == v:
                continue
            c[what[0]][what[1]] = v
        else:
            if c[what] == v:
                continue
            c[what] = v
        try:
            r = measure(geom, prim, precision, field_T, c)
        except Exception as e:  # an invalid combination (e.g. out of memory) is skipped
            log(f"  {what}={v}: failed ({e})")
            continue
        log(f"  {what}={v}: {r:.3e}")
        if r > best * 1.005:
            best, cfg = r, c
    # the fused mode: one kernel per generation, one register-cap variant for all species
    for v in ((2, 3) if precision else (1, 2)):
        c = dict(cfg, fused=1, blocks_per_sm=v)
        c.pop("blocks_per_sm_species", None)
        try:
            r = measure(geom, prim, precision, field_T, c)
        except Exception as e:
            log(f"  fused blocks_per_sm={v}: failed ({e})")
            continue
        log(f"  fused blocks_per_sm={v}: {r:.3e}")
        if r > best * 1.005:
            best, cfg = r, c
    cfg["steps_per_s"] = best
    return cfg


def main(argv=None):
    from . import build
    from . import workloads as W

    build.build()
    out = load()
    jobs = [(W.slab_calorimeter(), W.electrons(10000, 1e4), 1, 0.0),
            (W.slab_calorimeter(), W.electrons(10000, 1e4), 0, 0.0),
            (W.barrel_calorimeter(), W.barrel_primaries(10000, seed=4), 1, 3.8)]
    for geom, prim, precision, field in jobs:
        k = key(geom.kind, precision)
        print(f"tuning {k} on {len(prim)} primaries", flush=True)
        cfg = tune(geom, prim, precision, field)
        cfg["gpu"] = __import__("torch").cuda.get_device_name(0)
        out[k] = cfg
        print(f"  best {cfg}", flush=True)
    with open(TUNING, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
    print("wrote", TUNING)


if __name__ == "__main__":
    main(sys.argv[1:])
