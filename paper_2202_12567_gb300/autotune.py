"""Autotuner of the library's launch shapes (lt_tuning) for a workload.

Each tunable value is tried over its candidates with the others fixed
(coordinate descent, in the order of CANDIDATES), timing the frame stage the value
acts on with CUDA events on the context's stream (median of `reps` frames after a
warm frame).  Results are cached in a JSON file keyed by the workload:
(config name, rank, power-of-two bucket of the median slice rows m', and of the
median coarsened cut n').  `apply` loads a cached entry or tunes and stores one.
"""
from __future__ import annotations

import json
import os
import statistics

import numpy as np
import torch

from . import lt

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_CACHE = os.path.join(HERE, "tuning_cache.json")

# value -> (candidates, frame stage it acts on)
# (a kernel form comes before the launch shapes that act under it)
CANDIDATES = {
    "eval_ctas_per_sm": ([4, 8, 16, 32], "eval"),
    "p1_form": ([0, 1], "pass1"),       # pass-1 levels: a launch per step, or one persistent walk
    "ray_ctas_per_sm": ([4, 8, 16, 32], "pass1"),
    "als_form": ([0, 1], "complete"),   # lane-group SIMT Gram or the tensor-core (tcgen05) Gram
    "als_lane_entries": ([48, 64, 96, 128, 192], "complete"),
}


def bucket(x: float) -> int:
    """Power-of-two bucket (the largest power of two <= x, at least 1)."""
    x = max(float(x), 1.0)
    return 1 << int(np.floor(np.log2(x)))


def workload_key(name: str, rank: int, slice_rows, ncol) -> str:
    return f"{name}|r{int(rank)}|m{bucket(np.median(slice_rows))}|n{bucket(np.median(ncol))}"


def stage_times(R, seed: int) -> dict:
    """ms of each stage of one plain frame (events on the current stream)."""
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    ev[0].record()
    R.pass1(seed)
    ev[1].record()
    R.pass2(seed)
    ev[2].record()
    R.evaluate()
    ev[3].record()
    R.complete(seed)
    ev[4].record()
    R.render_image()
    ev[5].record()
    torch.cuda.synchronize()
    names = ["pass1", "pass2", "eval", "complete", "render"]
    return {n: ev[i].elapsed_time(ev[i + 1]) for i, n in enumerate(names)}


def tune(R, reps: int = 3, seed: int = 7, log=None) -> dict:
    """Coordinate descent over CANDIDATES on renderer R (set up); leaves R's context
    tuned and returns the chosen values with the measured stage times."""
    ctx = R.ctx
    best = lt.lt_get_tuning(ctx)
    report = {}
    for name, (cands, stage) in CANDIDATES.items():
        times = {}
        for v in cands:
            lt.lt_set_tuning(ctx, **{name: v})
            stage_times(R, seed)  # warm (scratch sized for this value)
            times[v] = statistics.median(stage_times(R, seed + 1 + k)[stage] for k in range(reps))
            if log:
                log(f"{name}={v}: {stage} {times[v]:.4f} ms")
        v_best = min(cands, key=lambda v: (times[v], cands.index(v)))
        best[name] = v_best
        lt.lt_set_tuning(ctx, **{name: v_best})
        report[name] = {str(k): round(t, 4) for k, t in times.items()}
    lt.lt_sync(ctx)
    return dict(values=best, stage_ms=report)


def apply(R, name: str, path: str = DEFAULT_CACHE, retune: bool = False, log=None) -> tuple[str, dict, bool]:
    """Tuning for R's workload from the cache, else tuned now and stored.
    Returns (key, values, from_cache)."""
    ncol = R.smp.ncol.cpu().numpy() if int(R.smp.ncol.sum()) > 0 else None
    if ncol is None:  # n' is known after a pass 1
        R.pass1(R.cfg["frame_seed"])
        ncol = R.smp.ncol.cpu().numpy()
    key = workload_key(name, R.cfg["rank"], R.frame.sizes, ncol)
    cache = {}
    if os.path.exists(path):
        with open(path) as f:
            cache = json.load(f)
    if key in cache and not retune:
        lt.lt_set_tuning(R.ctx, **cache[key]["values"])
        return key, cache[key]["values"], True
    res = tune(R, log=log)
    cache[key] = res
    with open(path, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    return key, res["values"], False
