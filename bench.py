"""Benchmark: ms per frame of the sparse sampling + completion renderer on one GB300.

A step is one frame of the method's hot path (pass 1 + coarsening, pass 2, entry
evaluation, masked-ALS completion of every slice, factorised render) on the
256x256-point, 16384-VPL room scene with two boxes (the scene family of the
learned-proposal experiments, held-out seed 5000), 64 slices, 15% sampling, rank 16.
The timed form is the batched one: the whole frame is one captured CUDA graph.  Its
pass-2 pdf (the paper's g, or the shipped learned proposal mixed with g) and rate
come from an equal-error study on held-out scenes of the same family: each form at
the lowest rate where the held-out mean and this scene reach rel-RMSE <= 2%, the
faster of the two.  Next to it: the other form, the plain form (the same calls one
by one, with their host synchronisations) and the brute-force sum.
Setup (light tree, global cut, slices) is timed separately and reported.  Quality
is the rel-RMSE of the frame against the brute-force column sum over all VPLs
(computed on the GPU by the library's brute-force kernel, which the tests check
against the CPU oracle).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun: one frame is split by slices over the ranks (no
collective on the data path; the pixel blocks are gathered once for the quality
check; strong scaling).
--impl reference times the CPU oracle (the plain float64 restatement of the method)
on the host cores on a bounded sample of the same frame.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "room256_vpl16k_2box"
ISO_SCENES = 10                                    # held-out scenes of the equal-error study
ISO_RATES = (0.10, 0.12, 0.14, 0.16, 0.18, 0.20, 0.22, 0.24)  # pass-2 rates of the study
METRIC = "ms/frame at rel-RMSE<=2% vs full-matrix render; speedup vs plain GPU form"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-iso", action="store_true", help="skip the equal-error study of the two pass-2 pdfs")
    ap.add_argument("--frames-only", type=int, default=0,
                    help="for profilers: set up, render this many plain frames and as many graph replays, print no line")
    ap.add_argument("--rate", type=float, default=0.0,
                    help="with --frames-only: the pass-2 rate (the headline's, as the equal-error study chose it)")
    ap.add_argument("--form", default="learned", choices=["learned", "g"],
                    help="with --frames-only: the pass-2 pdf of the graph replays")
    return ap.parse_args()


# ------------------------------------------------------------------ CPU oracle leg
# The oracle runs slice by slice (slices are independent after setup), one slice per
# process of a spawn pool over the host cores, each process single-threaded numpy.
_ORACLE = {}


def _oracle_init(sc, st, cfg):
    _ORACLE.update(sc=sc, st=st, cfg=cfg)


def _oracle_noop(_):
    return os.getpid()


def _oracle_slice(s, seed):
    from oracle import pipeline
    t0 = time.perf_counter()
    pipeline.run_slice(_ORACLE["st"], _ORACLE["sc"], _ORACLE["cfg"], s, seed)
    return s, time.perf_counter() - t0


def _oracle_pool(sc, st, cfg, cores):
    """A warmed spawn pool of `cores` single-threaded oracle processes."""
    import multiprocessing
    keep = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS",
                                           "CUDA_VISIBLE_DEVICES")}
    os.environ.update(OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="")
    try:
        pool = multiprocessing.get_context("spawn").Pool(cores, initializer=_oracle_init, initargs=(sc, st, cfg))
        pool.map(_oracle_noop, range(4 * cores), chunksize=1)  # every worker started and initialised
    finally:
        for k, v in keep.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return pool


def host_cores() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return max(1, os.cpu_count() or 1)


def oracle_sample(workload: str, setup=None) -> dict:
    """cpu_baseline: the CPU oracle on one wave of slices, one slice per host core,
    the slices spread over the frame's size range, timed wall-clock; ms/frame =
    wall x m / (rows of the wave).  `setup` = (cut, row_perm, slice_off) of the GPU's
    setup, so the oracle skips its own (untimed either way)."""
    import numpy as np
    from ltinputs import get_config, make_scene
    from oracle import pipeline
    cfg = get_config(workload)
    sc = make_scene(cfg)
    if setup is None:
        st = pipeline.setup(sc, cfg)
    else:
        cut, perm, off = setup
        st = pipeline.setup(sc, cfg, cut=cut, slicing=(perm, off))
    off = np.asarray(st["slice_off"])
    sizes = np.diff(off)
    S = sizes.size
    cores = host_cores()
    k = min(S, cores)
    order = np.argsort(sizes, kind="stable")
    pick = sorted({int(order[int(round(q * (S - 1)))]) for q in np.linspace(0.0, 1.0, k)})
    pool = _oracle_pool(sc, st, cfg, cores)
    try:
        t0 = time.perf_counter()
        res = pool.starmap(_oracle_slice, [(s, cfg["frame_seed"]) for s in pick], chunksize=1)
        wall = time.perf_counter() - t0
    finally:
        pool.close()
        pool.join()
    rows = int(sizes[pick].sum())
    cpu_s = sum(t for _, t in res)
    ms_frame = wall * 1e3 * sc.m / rows
    return dict(value=round(ms_frame, 1), unit="ms/frame", cores=cores, kind="oracle",
                sample=f"{len(pick)} of {S} slices ({rows} of {sc.m} rows, sizes {int(sizes[pick].min())}-"
                       f"{int(sizes[pick].max())}) run at once, one per process on {cores} host cores: "
                       f"{wall:.1f} s wall, {cpu_s:.1f} s CPU; ms/frame = wall x m / rows of the sample; "
                       f"setup (tree, cut, slices) not timed")


def run_reference(args):
    """The reference arm: the CPU oracle as it stands on the host cores.  Step k is
    one slice (spread over the frame) run by one single-threaded process; the K steps
    run concurrently on a spawn pool over the host cores.  A step's ms/frame is its
    slice time scaled to the frame's rows on all cores, t_k x m / (m'_k x cores);
    the line reports their median, and ms_per_step is the wall time of the whole
    timed run divided by K."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np
    from ltinputs import get_config, make_scene
    from oracle import pipeline
    cfg = get_config(args.workload)
    sc = make_scene(cfg)
    t_setup = time.perf_counter()
    st = pipeline.setup(sc, cfg)  # untimed: the frame metric excludes setup on both arms
    t_setup = time.perf_counter() - t_setup
    sizes = np.diff(np.asarray(st["slice_off"]))
    S = sizes.size
    K = max(1, args.steps)
    cores = host_cores()
    pick = [int(k * S // K) % S for k in range(K)]
    pool = _oracle_pool(sc, st, cfg, min(cores, K))
    try:
        t0 = time.perf_counter()
        res = pool.starmap(_oracle_slice, [(s, cfg["frame_seed"]) for s in pick], chunksize=1)
        wall = time.perf_counter() - t0
    finally:
        pool.close()
        pool.join()
    per = [t * 1e3 * sc.m / (int(sizes[s]) * cores) for s, t in res]
    value = float(np.median(per))
    sample = (f"{K} steps, step k = slice {pick[0]}, {pick[1] if K > 1 else ''}... (one slice each, "
              f"{int(sizes[pick].min())}-{int(sizes[pick].max())} rows) run concurrently on {min(cores, K)} "
              f"single-threaded processes of {cores} host cores; step ms/frame = slice time x m / (rows x "
              f"{cores} cores), median over steps; timed run {wall:.1f} s wall; oracle setup {t_setup:.1f} s "
              f"untimed; warm-up steps: none run (no caches or compilation on the CPU path)")
    line = dict(impl="reference", metric=METRIC, value=round(value, 1), unit="ms/frame",
                n_gpus=args.gpus, steps=K, warmup=args.warmup, ms_per_step=round(wall * 1e3 / K, 1),
                higher_is_better=False, scaling="strong", vs_baseline=None, dtype="f64", data="synthetic",
                config=dict(workload=args.workload),
                cpu_baseline=dict(value=round(value, 1), unit="ms/frame", cores=cores, kind="oracle",
                                  sample=sample),
                e2e=dict(value=round(value, 1), unit="ms/frame", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ clocks
class ClockSampler:
    def __init__(self, index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"])
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.f.name)
        return dict(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=max(mx) if mx else None,
                    reasons=sorted(reasons), samples=len(sm))


# ------------------------------------------------------------------ roofline
# Algorithmic FP32 operations of one evaluated entry (counted from the source of
# the entry model and the traversal): shading of the unoccluded value 40, ray set-up
# and grid clipping 40 per shadow ray, 6 per grid cell visited, 24 per box slab test.
OPS_ENTRY, OPS_RAY, OPS_CELL, OPS_BOX = 40, 40, 6, 24
SMS, FP32_LANES, MAX_SM_MHZ = 152, 128, 2070.0

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch from one ncu
# capture of each kernel on room256_vpl16k_2box at the headline's pass-2 rate (18%,
# learned pdf), the median over the captured launches; profiles/traffic_room256_vpl16k_2box.md
# gives the command.  A kernel changed since its capture has no entry here.
MEASURED_TRAFFIC = {
    "k_render": 7_067_392,
    "k_als_line": 49_546_240,  # U-steps and V-steps of the captured frames
}


def fp32_peak(clk) -> dict:
    """FP32 peak from the unit counts (152 SMs x 128 lanes x 2 flops per FMA) at the
    maximum SM clock and at the median SM clock sampled during the timed region."""
    at_max = SMS * FP32_LANES * 2 * MAX_SM_MHZ * 1e6 / 1e12
    mhz = clk.get("sm_mhz") or MAX_SM_MHZ
    return dict(peak=round(at_max, 2), peak_at_sampled_clock=round(SMS * FP32_LANES * 2 * mhz * 1e6 / 1e12, 2),
                peak_source=f"152 SMs x 128 FP32 lanes x 2 (FMA) x {MAX_SM_MHZ:.0f} MHz max SM clock (derived; "
                            f"no measured FP32 peak); at the sampled median {mhz:.0f} MHz in peak_at_sampled_clock")


def eval_roofline(lt, ctx, R, eval_ms, clk):
    """ALU roofline of the entry-evaluation kernel (the shadow-ray kernel)."""
    st = lt.lt_eval_stats(ctx, R.frame, R.smp, R.cfg["d_min"])
    ops = OPS_ENTRY * st["entries"] + OPS_RAY * st["rays"] + OPS_CELL * st["cells"] + OPS_BOX * st["boxes"]
    secs = eval_ms * 1e-3
    achieved = ops / secs / 1e12 if secs > 0 else 0.0
    pk = fp32_peak(clk)
    return dict(bound="alu", kernel="k_eval_entries", achieved=round(achieved, 3), unit="TFLOP/s",
                frac=round(achieved / pk["peak"], 4), traffic=MEASURED_TRAFFIC.get("k_eval_entries"),
                launch_ms=round(eval_ms, 4), **pk,
                work=dict(entries=st["entries"], rays=st["rays"], cells=st["cells"], boxes=st["boxes"],
                          ops_per_launch=int(ops)))


def als_roofline(lt, ctx, R, half_ms, clk):
    """FP32 roofline of the lane-group ALS half-step (k_als_line): per observed entry
    r(r+1)/2 + r FMAs (Gram lower triangle and right-hand side), per line a Cholesky
    (r^3/3 flops) and two triangular solves (2 r^2 flops)."""
    r = R.cfg["rank"]
    E = int(R.smp.cnt.sum())
    lines = (R.frame.m + int(R.smp.ncol.sum())) / 2.0
    flops = 2.0 * E * (r * (r + 1) / 2 + r) + lines * (r ** 3 / 3.0 + 2.0 * r * r)
    achieved = flops / (half_ms * 1e-3) / 1e12
    pk = fp32_peak(clk)
    return dict(bound="alu", kernel="k_als_line (ALS half-step)", achieved=round(achieved, 3), unit="TFLOP/s",
                frac=round(achieved / pk["peak"], 4),
                traffic=MEASURED_TRAFFIC.get("k_als_line") if R.cfg["rank"] == 16 else None,
                launch_ms=round(half_ms, 4), **pk,
                work=dict(entries=E, lines_per_half_step=lines, flops_per_launch=int(flops)))


def bruteforce_roofline(lt, ctx, R, bf_ms, clk):
    """ALU roofline of the brute-force column sum (the baseline of the speed-up): the
    entry-model operations of all m n entries, their shadow rays, cells and boxes."""
    st = lt.lt_bruteforce_stats(ctx, R.pts, R.vpls, R.cfg["d_min"])
    ops = OPS_ENTRY * st["entries"] + OPS_RAY * st["rays"] + OPS_CELL * st["cells"] + OPS_BOX * st["boxes"]
    achieved = ops / (bf_ms * 1e-3) / 1e12
    pk = fp32_peak(clk)
    return dict(bound="alu", kernel="k_bruteforce", achieved=round(achieved, 3), unit="TFLOP/s",
                frac=round(achieved / pk["peak"], 4), launch_ms=round(bf_ms, 3), **pk,
                work=dict(entries=st["entries"], rays=st["rays"], cells=st["cells"], boxes=st["boxes"],
                          ops_per_launch=int(ops)))


def render_roofline(R, render_ms, peaks):
    """HBM roofline of the render kernel: it reads U (4 r m bytes), V of every slice's
    columns (4 r sum n'), the row permutation (4 m) and writes the image (4 m)."""
    r = R.uv.r
    byts = 4 * r * (R.frame.m + int(R.smp.ncol.sum())) + 8 * R.frame.m
    achieved = byts / (render_ms * 1e-3) / 1e9
    peak = peaks.get("hbm_gbs", 6800.0)
    return dict(bound="hbm", kernel="k_render", achieved=round(achieved, 1), peak=peak, unit="GB/s",
                frac=round(achieved / peak, 4), traffic=MEASURED_TRAFFIC.get("k_render"),
                launch_ms=round(render_ms, 4), bytes_per_launch=int(byts),
                peak_source="measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)" if "hbm_gbs" in peaks
                else "fallback 6.8 TB/s")


def timed(fn, reps, flush=None):
    """Median device time (ms) of fn() on the current stream, L2 flushed before each."""
    import torch
    xs = []
    for _ in range(reps):
        if flush is not None:
            flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        xs.append(a.elapsed_time(b))
    return statistics.median(xs)


# ------------------------------------------------------------------ GPU leg
def rgb_leg(args, device: int, flush) -> dict | None:
    """The colour form of the workload (channels stacked as rows of each slice), plain
    calls on a context of its own: ms/frame and rel-RMSE against the RGB brute force."""
    import torch

    from ltinputs import CONFIGS, get_config, make_scene
    from paper_2202_12567_gb300 import lt
    from paper_2202_12567_gb300.renderer import Renderer
    name = args.workload + "_rgb"
    if name not in CONFIGS:
        return None
    cfg = get_config(name)
    sc = make_scene(cfg)
    R = Renderer(sc, cfg, device=device).setup()
    R.setup_rgb()
    for k in range(2):
        R.render_rgb(seed=cfg["frame_seed"] + k)
    ts, tc = [], []
    for k in range(max(3, args.steps // 4)):
        flush.zero_()
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        seed = cfg["frame_seed"] + 100 + k
        evs[0].record()
        R.pass1(seed)
        R.pass2(seed)
        R.evaluate()
        lt.lt_expand_rgb(R.ctx, R.frame, R.smp, R.rgb)
        evs[1].record()
        lt.lt_complete_rgb(R.ctx, R.rgb, cfg["als_iters"], cfg["lam_rel"], seed)
        lt.lt_render_rgb(R.ctx, R.rgb)
        evs[2].record()
        torch.cuda.synchronize()
        ts.append(evs[0].elapsed_time(evs[2]))
        tc.append(evs[1].elapsed_time(evs[2]))
    img = R.rgb.img.view(-1, 3).double()
    ref = R.bruteforce_rgb().double()
    rel = float(torch.linalg.norm(img - ref) / torch.linalg.norm(ref))
    out = dict(workload=f"{name}: RGB face albedos, light colour {tuple(cfg['light_rgb'])}, 3 channels stacked "
                        f"as rows of each slice (3m' x n', one V)",
               ms_per_frame=round(statistics.median(ts), 3), stacked_completion_ms=round(statistics.median(tc), 3),
               rel_rmse_vs_rgb_bruteforce=round(rel, 5), pixel_entries=int(R.smp.cnt.sum().item()),
               stacked_entries=int(R.rgb.cnt.sum().item()))
    lt.lt_sync(R.ctx)
    return out


def temporal_leg(R, bf, flush, frames: int = 6) -> dict:
    """Temporal coherence across frames (plain calls on the headline renderer): a chain
    of frames of the static scene with new seeds, each completion started from the
    previous frame's factors (lt_complete_warm) with fewer sweeps, against frames started
    cold with the workload's sweeps: completion ms and rel-RMSE of the chain's last frame
    against the brute force."""
    import torch

    cfg = R.cfg
    nbf = torch.linalg.norm(bf.double())
    out = {}
    for name, warm, iters in (("cold", False, cfg["als_iters"]), ("warm_5", True, 5), ("warm_3", True, 3),
                              ("warm_2", True, 2), ("warm_1", True, 1)):
        R._prev = None
        if warm:
            R.render(seed=cfg["frame_seed"] + 300, warm=True)  # the chain's first frame, started cold
        tc, tf = [], []
        for k in range(frames):
            flush.zero_()
            seed = cfg["frame_seed"] + 301 + k
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            ev[0].record()
            R.pass1(seed)
            R.pass2(seed)
            R.evaluate()
            ev[1].record()
            R.complete(seed, warm=warm, iters=iters)
            R.render_image()
            ev[2].record()
            torch.cuda.synchronize()
            tc.append(ev[1].elapsed_time(ev[2]))
            tf.append(ev[0].elapsed_time(ev[2]))
        rel = float(torch.linalg.norm(R.img.double() - bf.double()) / nbf)
        out[name] = dict(sweeps=iters, completion_ms=round(statistics.median(tc), 3),
                         frame_ms=round(statistics.median(tf), 3), rel_rmse=round(rel, 5))
    R._prev = None
    out["chain"] = (f"{frames} frames of the same scene with new seeds, plain calls, pass-2 pdf g at the "
                    f"headline's rate; warm: each completion started from the previous frame's factors")
    return out


def mesh_leg(args, device: int, flush) -> dict | None:
    """The workload with triangle-mesh occluders (icospheres through a BVH) besides the
    boxes, plain calls on a context of its own: ms/frame and rel-RMSE against the GPU
    brute force of the same scene."""
    import torch

    from ltinputs import CONFIGS, get_config, make_scene
    from paper_2202_12567_gb300 import lt
    from paper_2202_12567_gb300.renderer import Renderer
    name = args.workload.replace("_2box", "_mesh")
    if name == args.workload or name not in CONFIGS:
        return None
    cfg = get_config(name)
    sc = make_scene(cfg)
    R = Renderer(sc, cfg, device=device).setup()
    for k in range(2):
        R.render(seed=cfg["frame_seed"] + k)
    ts = []
    for k in range(max(3, args.steps // 4)):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        R.render(seed=cfg["frame_seed"] + 100 + k, sync=False)
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    img = R.img.double()
    ref = R.bruteforce().double()
    rel = float(torch.linalg.norm(img - ref) / torch.linalg.norm(ref))
    lt.lt_sync(R.ctx)
    return dict(workload=f"{name}: {sc.tris.shape[0]} triangles ({cfg['n_meshes']} icospheres) and "
                         f"{sc.nb} boxes as occluders",
                ms_per_frame=round(statistics.median(ts), 3), rel_rmse_vs_bruteforce=round(rel, 5),
                rays_per_pixel=round(float(R.rays()) / R.frame.m, 2))


def run_sharded(args, world: int, rank: int, local: int):
    """N > 1: one frame split by slices over the ranks (strong scaling).  Every rank
    sets up the frame, renders its longest-processing-time share of the slices as a
    captured graph (each slice with its index in the whole frame, so the pixels are
    the whole frame's), and the frame time is the slowest rank's; the pixel blocks are
    gathered once on rank 0 for the quality check."""
    import torch
    import torch.distributed as dist

    from ltinputs import get_config, make_scene
    from paper_2202_12567_gb300 import lt, shard
    from paper_2202_12567_gb300.renderer import Renderer

    # the ranks exchange only host values (frame times, the final pixel blocks): gloo
    dist.init_process_group("gloo", init_method="env://")
    local = local % torch.cuda.device_count()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cfg = get_config(args.workload)
    sc = make_scene(cfg)
    R = Renderer(sc, cfg, device=local).setup()
    parts = shard.lpt_partition(shard.slice_costs(R.slice_off.cpu().numpy(), C=R.frame.C), world)
    sub = shard.shard_renderer(R, parts[rank])
    seed0 = cfg["frame_seed"]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    if sub is not None:
        sub.capture()
        for i in range(args.warmup):
            sub.render_graph(seed0 + 100 + i)
    dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    launches0 = lt.lt_launch_count(R.ctx)
    ms = []
    for k in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        if sub is not None:
            lt.lt_frame_graph_launch(sub.graph, seed0 + 1000 + k)
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    clk = clocks.stop()
    launches = lt.lt_launch_count(R.ctx) - launches0
    med = shard.max_over_ranks(float(statistics.median(ms)))
    total = shard.max_over_ranks(float(sum(ms)))
    dist.barrier()
    # end to end: this rank's points in from pinned memory, its graph, its pixels out
    e2e = []
    if sub is not None:
        pts_h = sub.pts_s.cpu().pin_memory()
        out_h = torch.empty(sub.pixels.numel(), dtype=torch.float32).pin_memory()
    for k in range(max(3, args.steps // 2) + 1):
        flush.zero_()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        if sub is not None:
            sub.pts_s.copy_(pts_h, non_blocking=True)
            lt.lt_frame_graph_launch(sub.graph, seed0 + 5000 + k)
            out_h.copy_(sub.img[sub.pixels], non_blocking=True)
        b.record()
        torch.cuda.synchronize()
        if k > 0:
            e2e.append(a.elapsed_time(b))
    e2e_ms = shard.max_over_ranks(float(statistics.median(e2e)))
    h2d = int(sub.pts_s.numel() * 4) if sub is not None else 0
    d2h = int(sub.pixels.numel() * 4) if sub is not None else 0
    h2d = int(shard.max_over_ranks(h2d))
    d2h = int(shard.max_over_ranks(d2h))
    # quality of the last timed frame, gathered on rank 0
    if sub is not None:
        lt.lt_frame_graph_launch(sub.graph, seed0 + 1000 + args.steps - 1)
        lt.lt_sync(R.ctx)
        pixels, values = sub.pixels.cpu(), sub.img[sub.pixels].cpu()
    else:
        pixels, values = torch.zeros(0, dtype=torch.int64), torch.zeros(0)
    img = shard.gather_image(pixels, values, sc.m)
    if rank == 0:
        bf = R.bruteforce().double().cpu()
        rel = float(torch.linalg.norm(img.double() - bf) / torch.linalg.norm(bf))
        line = dict(metric=METRIC, value=round(med, 4), unit="ms/frame", n_gpus=world, steps=args.steps,
                    warmup=args.warmup, ms_per_step=round(total / args.steps, 4), higher_is_better=False,
                    scaling="strong", vs_baseline=None, dtype="f32", data="synthetic",
                    config=dict(workload=f"{args.workload}: one frame split by slices over {world} GPUs "
                                         f"(longest-processing-time on m' n'; slices per rank "
                                         f"{[len(p) for p in parts]}), each rank's share as one captured graph",
                                l2="flushed (256 MB write) between timed frames",
                                rel_rmse_vs_bruteforce=round(rel, 5)),
                    e2e=dict(value=round(e2e_ms, 4), unit="ms/frame", h2d_bytes_per_step=h2d,
                             d2h_bytes_per_step=d2h),
                    gpu_launches=int(launches), clocks=clk)
        print(json.dumps(line), flush=True)
    dist.barrier()
    dist.destroy_process_group()


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from ltinputs import get_config, make_scene
    from paper_2202_12567_gb300 import lt
    from paper_2202_12567_gb300.renderer import Renderer

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        return run_sharded(args, world, rank, local)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    peaks = {}
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        peaks = json.load(open(pk))

    cfg = get_config(args.workload)
    ctx = lt.Context(local)
    from paper_2202_12567_gb300 import autotune, proposal
    theta = proposal.load_theta(device=local) if os.path.exists(proposal.DEFAULT_THETA) else None
    # Which pass-2 pdf and rate the headline takes: each form at the lowest rate where
    # the held-out scenes' mean rel-RMSE and this scene's own are <= 2% (equal error),
    # the faster of the two; without a study, the preset's rate and the learned form.
    iso, headline = None, ("learned" if theta is not None else "g")
    if args.frames_only:
        headline = args.form if theta is not None else "g"
        if args.rate > 0:
            cfg["rate"] = args.rate
    if theta is not None and not args.frames_only and not args.no_iso:
        iso = proposal.iso_error(ctx, cfg, theta, [cfg["scene_seed"] + k for k in range(ISO_SCENES)], ISO_RATES,
                                 timing_scene=cfg["scene_seed"])
        ok = {f: iso[f] for f in ("g", "learned")
              if iso[f].get("iso_rate") is not None and iso[f]["rel_rmse_timing_scene"] <= 0.02}
        if ok:
            headline = min(ok, key=lambda f: ok[f]["ms_per_frame"])
            cfg["rate"] = ok[headline]["iso_rate"]
    sc = make_scene(cfg)
    R = Renderer(sc, cfg, device=local, ctx=ctx)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    R.setup()
    torch.cuda.synchronize()
    setup_ms = (time.perf_counter() - t0) * 1e3

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)
    seed0 = cfg["frame_seed"]

    def frame(i, stage_events=None):
        seed = seed0 + i
        ev = stage_events
        if ev:
            ev[0].record()
        R.pass1(seed)
        if ev:
            ev[1].record()
        R.pass2(seed)
        if ev:
            ev[2].record()
        R.evaluate()
        if ev:
            ev[3].record()
        R.complete(seed)
        if ev:
            ev[4].record()
        R.render_image()
        if ev:
            ev[5].record()

    # launch shapes for this workload: the shipped tuning cache, else tuned now
    tune_key, tune_values, tune_cached = autotune.apply(R, args.workload)

    for i in range(args.warmup):
        frame(i)
    lt.lt_sync(ctx)
    if args.frames_only:
        for i in range(args.frames_only):
            frame(100 + i)
        if headline == "learned":
            g_only = lt.lt_frame_graph_capture(ctx, R.frame, lt.params(cfg, proposal=theta, mix=0.8), R.smp, R.uv,
                                               R.row_perm, R.img, keep=(theta,))
        else:
            g_only = lt.lt_frame_graph_capture(ctx, R.frame, lt.params(cfg), R.smp, R.uv, R.row_perm, R.img)
        for i in range(args.frames_only):
            lt.lt_frame_graph_launch(g_only, seed0 + 200 + i)
        lt.lt_sync(ctx)
        torch.cuda.synchronize()
        return
    # the batched form: the whole frame as one CUDA graph, pass 2 from the learned
    # proposal (or from g when no trained network is shipped)
    prm_g = lt.params(cfg)
    graph_g = lt.lt_frame_graph_capture(ctx, R.frame, prm_g, R.smp, R.uv, R.row_perm, R.img)
    graph_l = None
    if theta is not None:
        prm_l = lt.params(cfg, proposal=theta, mix=0.8)
        graph_l = lt.lt_frame_graph_capture(ctx, R.frame, prm_l, R.smp, R.uv, R.row_perm, R.img, keep=(theta,))
    graph = graph_l if headline == "learned" else graph_g
    for i in range(args.warmup):
        for gr in (graph_g, graph_l):
            if gr is not None:
                lt.lt_frame_graph_launch(gr, seed0 + 100 + i)
    lt.lt_sync(ctx)

    def replay(g, k0):
        ms = []
        for k in range(args.steps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            lt.lt_frame_graph_launch(g, seed0 + k0 + k)
            b.record()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return ms

    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    launches0 = lt.lt_launch_count(ctx)
    per = replay(graph, 1000)
    torch.cuda.synchronize()
    launches = lt.lt_launch_count(ctx) - launches0
    lt.lt_sync(ctx)
    total_ms = float(sum(per))
    ms_frame = float(statistics.median(per))  # median replay
    img = R.img.clone()
    # the other form's graph (seeds as above: the same pass-1 draws)
    if headline == "learned":
        per_l, img_l = per, img
        per_g = replay(graph_g, 1000)
        img_g = R.img.clone()
    else:
        per_g, img_g = per, img
        per_l, img_l = (replay(graph_l, 1000), R.img.clone()) if graph_l is not None else (None, None)
    g_graph_ms = statistics.median(per_g)

    # the plain form (the same calls one by one, with the two size read-backs),
    # with events between the stages for the breakdown
    plain = []
    stages = []
    for k in range(args.steps):
        flush.zero_()
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        frame(1000 + k, evs)
        torch.cuda.synchronize()
        plain.append(evs[0].elapsed_time(evs[5]))
        stages.append([evs[j].elapsed_time(evs[j + 1]) for j in range(5)])
    stage_ms = np.median(np.array(stages), axis=0)
    plain_ms = statistics.median(plain)
    same_as_graph = bool(torch.equal(R.img, img_g))
    # ALS half-step on the launching stream: complete at K sweeps minus at 0 sweeps
    c_ms = {}
    for iters in (0, cfg["als_iters"]):
        xs = []
        for k in range(max(3, args.steps // 4)):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            lt.lt_complete(ctx, R.frame, R.smp, R.uv, iters, cfg["lam_rel"], seed0)
            b.record()
            torch.cuda.synchronize()
            xs.append(a.elapsed_time(b))
        c_ms[iters] = statistics.median(xs[1:])
    half_ms = (c_ms[cfg["als_iters"]] - c_ms[0]) / (2 * cfg["als_iters"])
    img_als = torch.empty_like(R.img)
    lt.lt_render(ctx, R.frame, R.smp, R.uv, R.row_perm, img_als)
    # the nonnegative ADM completion of App. A on the same samples (one launch runs
    # every iteration; the start alone is timed as 0 iterations)
    a_ms = {}
    for iters in (0, cfg["adm_iters"]):
        xs = []
        for k in range(4):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            lt.lt_complete_adm(ctx, R.frame, R.smp, R.uv, iters, cfg["adm_alpha_rel"], cfg["adm_gamma"], seed0)
            b.record()
            torch.cuda.synchronize()
            xs.append(a.elapsed_time(b))
        a_ms[iters] = statistics.median(xs[1:])
    img_adm = torch.empty_like(R.img)
    lt.lt_render(ctx, R.frame, R.smp, R.uv, R.row_perm, img_adm)
    clk = clocks.stop()
    lt.lt_sync(ctx)

    # quality: the last frames against the brute-force column sum over all VPLs
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    bf = torch.empty_like(img)
    R.bruteforce(bf)  # warm
    flush.zero_()
    e0.record()
    R.bruteforce(bf)
    e1.record()
    torch.cuda.synchronize()
    bf_ms = e0.elapsed_time(e1)
    nbf = torch.linalg.norm(bf.double())
    rel = float(torch.linalg.norm(img.double() - bf.double()) / nbf)
    rel_g = float(torch.linalg.norm(img_g.double() - bf.double()) / nbf)
    rel_l = float(torch.linalg.norm(img_l.double() - bf.double()) / nbf) if img_l is not None else None
    rays_per_px = float(R.rays()) / R.frame.m
    adm = dict(iters=cfg["adm_iters"], alpha_rel=cfg["adm_alpha_rel"], gamma=cfg["adm_gamma"],
               completion_ms=round(a_ms[cfg["adm_iters"]], 3),
               ms_per_iteration=round((a_ms[cfg["adm_iters"]] - a_ms[0]) / max(cfg["adm_iters"], 1), 4),
               rel_rmse=round(float(torch.linalg.norm(img_adm.double() - bf.double()) / nbf), 5),
               als_completion_ms=round(c_ms[cfg["als_iters"]], 3),
               als_rel_rmse_same_samples=round(float(torch.linalg.norm(img_als.double() - bf.double()) / nbf), 5))

    # end to end through the C ABI from pinned host buffers: points and VPLs in, image out
    pts_h = torch.from_numpy(sc.points).pin_memory()
    vpl_h = torch.from_numpy(sc.vpls).pin_memory()
    img_h = torch.empty(R.frame.m, dtype=torch.float32).pin_memory()
    e2e = []
    for k in range(max(3, args.steps // 2) + 1):
        flush.zero_()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        R.pts.copy_(pts_h, non_blocking=True)
        R.vpls.copy_(vpl_h, non_blocking=True)
        R.pts_s.copy_(lt.lt_permute_points(ctx, R.pts, R.row_perm))
        lt.lt_frame_graph_launch(graph, seed0 + 5000 + k)
        img_h.copy_(R.img, non_blocking=True)
        b.record()
        torch.cuda.synchronize()
        if k > 0:
            e2e.append(a.elapsed_time(b))
    e2e_ms = statistics.median(e2e)
    h2d = sc.points.nbytes + sc.vpls.nbytes
    d2h = img_h.numel() * 4

    roof = als_roofline(lt, ctx, R, half_ms, clk)
    eval_ms = timed(lambda: lt.lt_eval_entries(ctx, R.frame, R.smp, cfg["d_min"]), max(5, args.steps // 2), flush)
    roof_eval = eval_roofline(lt, ctx, R, eval_ms, clk)
    render_ms = timed(lambda: lt.lt_render(ctx, R.frame, R.smp, R.uv, R.row_perm, img_als), max(5, args.steps // 2),
                      flush)
    roof_render = render_roofline(R, render_ms, peaks)
    roof_bf = bruteforce_roofline(lt, ctx, R, bf_ms, clk)
    # the colour and mesh forms run on contexts of their own after the headline; a
    # failure there is reported in the line instead of losing it
    try:
        colour = rgb_leg(args, local, flush)
    except RuntimeError as e:
        colour = dict(error=str(e))
    try:
        meshes = mesh_leg(args, local, flush)
    except RuntimeError as e:
        meshes = dict(error=str(e))
    try:
        temporal = temporal_leg(R, bf, flush)
    except RuntimeError as e:
        temporal = dict(error=str(e))

    line = dict(metric=METRIC, value=round(ms_frame, 4), unit="ms/frame", n_gpus=world, steps=args.steps,
                warmup=args.warmup, ms_per_step=round(total_ms / args.steps, 4), higher_is_better=False,
                scaling="strong", vs_baseline=None, dtype="f32", data="synthetic",
                config=dict(workload=f"{args.workload}: {sc.width}x{sc.height} points, {sc.n} VPLs, {sc.nb} boxes, "
                                     f"{cfg['n_slices']} slices, {100 * cfg['rate']:g}% sampling, rank {cfg['rank']}, "
                                     f"{cfg['als_iters']} ALS sweeps, cut <= {cfg['max_cut']}, tau {cfg['tau']}",
                            l2="flushed (256 MB write) between timed frames", global_cut=int(R.frame.C),
                            rel_rmse_vs_bruteforce=round(rel, 5), rays_per_pixel=round(rays_per_px, 2),
                            bruteforce_gpu_ms=round(bf_ms, 3), speedup_vs_bruteforce=round(bf_ms / ms_frame, 2),
                            form=("batched + learned proposal: the frame as one captured CUDA graph "
                                  f"({graph.kernels} kernels per replay), pass 2 from 0.8 softmax(MLP) + 0.2 g"
                                  if headline == "learned" else
                                  f"batched: the frame as one captured CUDA graph ({graph.kernels} kernels per "
                                  f"replay), pass 2 from the paper's pdf g"),
                            headline_form=headline,
                            forms=dict(g=dict(ms_per_frame=round(g_graph_ms, 4), rel_rmse=round(rel_g, 5)),
                                       learned=(dict(ms_per_frame=round(statistics.median(per_l), 4),
                                                     rel_rmse=round(rel_l, 5)) if per_l is not None else None)),
                            iso_error=iso,
                            paper_pdf_graph_ms=round(g_graph_ms, 4),
                            rel_rmse_paper_pdf=round(rel_g, 5),
                            plain_form_ms=round(plain_ms, 4), speedup_vs_plain_form=round(plain_ms / ms_frame, 3),
                            plain_equals_graph_bitwise=same_as_graph,
                            tuning=dict(key=tune_key, values=tune_values, from_cache=tune_cached),
                            eval_roofline=roof_eval,
                            render_roofline=roof_render,
                            bruteforce_roofline=roof_bf,
                            adm_completion=adm,
                            rgb=colour,
                            mesh=meshes,
                            temporal=temporal,
                            setup_ms=round(setup_ms, 1),
                            setup_breakdown_ms=R.setup_ms,
                            setup_plus_one_plain_frame_ms=round(setup_ms + plain_ms, 2),
                            stage_ms=dict(zip(["pass1", "pass2", "eval", "complete", "render"],
                                              [round(x, 4) for x in stage_ms.tolist()]))),
                e2e=dict(value=round(e2e_ms, 4), unit="ms/frame", h2d_bytes_per_step=int(h2d),
                         d2h_bytes_per_step=int(d2h)),
                gpu_launches=int(launches), clocks=clk, roofline=roof)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            line["cpu_baseline"] = oracle_sample(args.workload, setup=(R.frame.cut.cpu().numpy(),
                                                                      R.row_perm.cpu().numpy(),
                                                                      R.slice_off.cpu().numpy()))
        except Exception as e:  # report, do not hide
            line["cpu_baseline"] = dict(value=None, unit="ms/frame", cores=host_cores(), kind="oracle",
                                        sample=f"failed: {e}")
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
