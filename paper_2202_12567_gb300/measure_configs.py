"""Quality and speed of the renderer on a workload preset, over a sweep of its
parameters: ms/frame of the batched form (the frame as one captured CUDA graph) and
rel-RMSE against the brute-force column sum over all VPLs, both on the GPU.

    python -m paper_2202_12567_gb300.measure_configs --workload room256_vpl16k_200box \\
        --sweep rate=0.05,0.1 --sweep tau=0.02,0.0005 [--set d_min=0.1] [--subset-rows 16384] \\
        [--scene-cache DIR] [--frames 5]

Every combination of the --sweep values (with the --set overrides) is one JSON line:
the parameters, ms/frame (median of the graph replays), the plain form's ms/frame,
setup ms, rel-RMSE, the global cut size, mean coarsened columns per slice, observed
entries and shadow-ray entries per pixel.  --subset-rows N compares on N seeded
pixels only (the brute force over all VPLs of a 1024x1024 image takes tens of
seconds); the line says which.
"""
from __future__ import annotations

import argparse
import itertools
import json
import statistics
import time

import numpy as np
import torch

from ltinputs import get_config, load_or_make_scene

from . import lt
from .renderer import Renderer


def _value(v: str):
    if ":" in v:  # a pair such as slice_bounds=128:4096
        return tuple(_value(x) for x in v.split(":"))
    for cast in (int, float):
        try:
            return cast(v)
        except ValueError:
            pass
    return v


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", required=True)
    ap.add_argument("--set", action="append", default=[], help="key=value override of the preset")
    ap.add_argument("--sweep", action="append", default=[], help="key=v1,v2,... swept values")
    ap.add_argument("--subset-rows", type=int, default=0)
    ap.add_argument("--scene-cache", default=None)
    ap.add_argument("--frames", type=int, default=5)
    return ap.parse_args(argv)


class _Reference:
    """The brute-force image (or the pixels of a seeded subset), per d_min."""

    def __init__(self, scene, subset_rows: int, dev):
        self.scene, self.dev, self.cache = scene, dev, {}
        self.idx = None
        if subset_rows and subset_rows < scene.m:
            self.idx = np.sort(np.random.default_rng(20240).choice(scene.m, subset_rows, replace=False))
        self.pts = torch.from_numpy(np.ascontiguousarray(scene.points if self.idx is None
                                                         else scene.points[:, self.idx])).to(dev)
        self.vpls = torch.from_numpy(np.ascontiguousarray(scene.vpls)).to(dev)

    def get(self, ctx, d_min):
        if d_min not in self.cache:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            img = lt.lt_bruteforce(ctx, self.pts, self.vpls, d_min)
            torch.cuda.synchronize()
            self.cache[d_min] = (img.double(), (time.perf_counter() - t0) * 1e3)
        return self.cache[d_min]

    def pick(self, img):
        return img.double() if self.idx is None else img.double()[torch.from_numpy(self.idx).to(img.device)]


def run(args) -> list[dict]:
    base = get_config(args.workload, **{k: _value(v) for k, v in (s.split("=", 1) for s in args.set)})
    scene = load_or_make_scene(base, args.scene_cache)
    dev = torch.device("cuda", 0)
    ref = _Reference(scene, args.subset_rows, dev)
    keys = [s.split("=", 1)[0] for s in args.sweep]
    vals = [[_value(v) for v in s.split("=", 1)[1].split(",")] for s in args.sweep]
    out = []
    for combo in itertools.product(*vals) if keys else [()]:
        cfg = dict(base, **dict(zip(keys, combo)))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        R = Renderer(scene, cfg, device=0).setup()
        torch.cuda.synchronize()
        setup_ms = (time.perf_counter() - t0) * 1e3
        R.render(seed=cfg["frame_seed"])
        plain = []
        for k in range(max(1, args.frames // 2)):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            R.render(seed=cfg["frame_seed"] + 1 + k, sync=False)
            b.record()
            torch.cuda.synchronize()
            plain.append(a.elapsed_time(b))
        R.capture()
        R.render_graph(cfg["frame_seed"] + 50)
        ms = []
        for k in range(args.frames):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            R.render_graph(cfg["frame_seed"] + 100 + k, sync=False)
            b.record()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        lt.lt_sync(R.ctx)
        bf, bf_ms = ref.get(R.ctx, cfg["d_min"])
        img = ref.pick(R.img)
        rel = float(torch.linalg.norm(img - bf) / torch.linalg.norm(bf))
        ncol = R.smp.ncol.double()
        line = dict(workload=args.workload, params={k: cfg[k] for k in keys} | {s.split("=", 1)[0]: cfg[s.split("=", 1)[0]]
                                                                                for s in args.set},
                    ms_per_frame=round(statistics.median(ms), 3), plain_ms=round(statistics.median(plain), 3),
                    setup_ms=round(setup_ms, 1), rel_rmse=round(rel, 5),
                    reference=("full image" if ref.idx is None else f"{ref.idx.size} seeded pixels"),
                    bruteforce_ms=round(bf_ms, 1), global_cut=int(R.frame.C),
                    mean_columns=round(float(ncol.mean()), 1), slices=int(R.frame.S),
                    slice_rows=[int(x) for x in (np.diff(R.slice_off.cpu().numpy()).min(),
                                                 np.diff(R.slice_off.cpu().numpy()).max())],
                    entries=int(R.smp.cnt.sum().item()), entries_per_pixel=round(R.rays() / R.frame.m, 2),
                    points=int(scene.m), vpls=int(scene.n), boxes=int(scene.nb))
        print(json.dumps(line), flush=True)
        out.append(line)
        R.graph.close()
        R.ctx.close()
        del R
        torch.cuda.empty_cache()
    return out


if __name__ == "__main__":
    run(parse())
