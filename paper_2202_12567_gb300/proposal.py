"""Training and evaluation of the learned pass-2 proposal through liblt.

Every computation runs in the library's kernels; this module only orders the calls
and owns the tensors.  Training data are the method's own matrices on seeded
scenes: for each scene, pass 1 on the GPU, the 32 features of every (slice,
column), the full slice matrices and their leverage targets (include/lt.h).  One
Adam step per scene batch (the scene's slices are the softmax groups).

    python -m paper_2202_12567_gb300.proposal --scenes 200 --epochs 30 --out proposal_theta.npy
"""
from __future__ import annotations

import argparse
import os
import time

import numpy as np
import torch

from . import lt
from .renderer import Renderer

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_THETA = os.path.join(HERE, "proposal_theta.npy")
TRAIN_SEED0 = 1000      # training scenes 1000 + k
TARGET_ITERS = 30       # subspace-iteration rounds of the leverage targets


def scene_batch(ctx: lt.Context, cfg: dict, scene_seed: int, frame_seed: int | None = None):
    """Features, targets and groups of one scene (all slices), on the device."""
    from ltinputs import make_scene
    frame_seed = cfg["frame_seed"] if frame_seed is None else frame_seed
    R = Renderer(make_scene(cfg, scene_seed), cfg, device=ctx.device, ctx=ctx).setup()
    R.pass1(frame_seed)
    feat, goff = lt.lt_proposal_features(ctx, R.frame, R.smp)
    ncol = R.smp.ncol.cpu().numpy().astype(np.int64)
    cap = int(np.sum(R.frame.sizes * ncol))
    M, moff = lt.lt_slice_matrices(ctx, R.frame, R.smp, cfg["d_min"], cap)
    tgt = lt.lt_leverage_targets(ctx, R.frame, R.smp, M, moff, goff, cfg["rank"], TARGET_ITERS, frame_seed)
    n = int(ncol.sum())
    lt.lt_sync(ctx)
    return dict(feat=feat[:n].clone(), target=tgt[:n].clone(), goff=goff.clone(), ngroups=R.frame.S, n=n)


def train(ctx: lt.Context, cfg: dict, scene_seeds, epochs: int = 30, lr: float = 3e-3, init_seed: int = 1,
          batches=None, verbose: bool = False):
    """Train from scratch; returns (theta, per-epoch mean loss)."""
    t0 = time.perf_counter()
    if batches is None:
        batches = [scene_batch(ctx, cfg, s) for s in scene_seeds]
    if verbose:
        print(f"data: {len(batches)} scenes, {sum(b['n'] for b in batches)} rows, {time.perf_counter() - t0:.1f} s",
              flush=True)
    dev = torch.device("cuda", ctx.device)
    theta = lt.lt_proposal_init(ctx, init_seed)
    m = torch.zeros_like(theta)
    v = torch.zeros_like(theta)
    grad = torch.zeros_like(theta)
    losses = torch.zeros(epochs * len(batches), dtype=torch.float32, device=dev)
    rng = np.random.default_rng(init_seed)
    step = 0
    for ep in range(epochs):
        for i in rng.permutation(len(batches)):
            b = batches[i]
            lt.lt_proposal_grad(ctx, theta, b["feat"], b["target"], b["goff"], b["ngroups"], b["n"], grad,
                                losses[step:step + 1])
            step += 1
            lt.lt_proposal_adam(ctx, theta, m, v, grad, step, lr)
        if verbose:
            print(f"epoch {ep}: loss {float(losses[step - len(batches):step].mean()):.5f}", flush=True)
    lt.lt_sync(ctx)
    hist = losses.view(epochs, len(batches)).mean(1).cpu().numpy()
    return theta, hist


def loss_of(ctx: lt.Context, theta, batches) -> float:
    """Mean proposal loss over scene batches (no update)."""
    grad = torch.zeros_like(theta)
    out = torch.zeros(len(batches), dtype=torch.float32, device=theta.device)
    for i, b in enumerate(batches):
        lt.lt_proposal_grad(ctx, theta, b["feat"], b["target"], b["goff"], b["ngroups"], b["n"], grad, out[i:i + 1])
    return float(out.mean())


def load_theta(path: str = DEFAULT_THETA, device: int = 0):
    return torch.from_numpy(np.load(path).astype(np.float32)).to(torch.device("cuda", device))


def ab_compare(ctx: lt.Context, cfg: dict, theta, scene_seeds, mix: float = 0.8, seed: int | None = None):
    """rel-RMSE against the brute-force image at equal sample count: pass 2 from the
    pass-1 estimate g (the paper) versus from the learned proposal."""
    from ltinputs import make_scene
    out = []
    for s in scene_seeds:
        R = Renderer(make_scene(cfg, s), cfg, device=ctx.device, ctx=ctx).setup()
        ref = R.bruteforce().double()
        nref = float(torch.linalg.norm(ref))
        img_g = R.render_frame(seed=seed).double()
        cnt_g = int(R.smp.cnt.sum())
        prm = lt.params(R.cfg, proposal=theta, mix=mix)
        lt.lt_render_frame(ctx, R.frame, prm, R.cfg["frame_seed"] if seed is None else seed, R.smp, R.uv,
                           R.row_perm, R.img)
        lt.lt_sync(ctx)
        img_p = R.img.double()
        cnt_p = int(R.smp.cnt.sum())
        out.append(dict(scene=int(s), rel_g=float(torch.linalg.norm(img_g - ref)) / nref,
                        rel_learned=float(torch.linalg.norm(img_p - ref)) / nref, entries_g=cnt_g,
                        entries_learned=cnt_p))
    return out


def iso_error(ctx: lt.Context, cfg: dict, theta, scene_seeds, rates, target: float = 0.02, mix: float = 0.8,
              timing_scene: int | None = None, replays: int = 10):
    """The two pass-2 pdfs at equal error instead of equal sample count: for every
    rate, the mean rel-RMSE over the held-out scenes of the frame with g (the paper)
    and with the learned proposal; each form's iso rate is the lowest rate whose mean
    is <= target, and its ms/frame is the median replay of the captured frame at that
    rate on `timing_scene` (L2 flushed between replays)."""
    from ltinputs import make_scene
    rates = sorted(float(r) for r in rates)
    top = dict(cfg, rate=rates[-1])
    err = {"g": np.zeros(len(rates)), "learned": np.zeros(len(rates))}
    for s in scene_seeds:
        R = Renderer(make_scene(top, s), top, device=ctx.device, ctx=ctx).setup()
        ref = R.bruteforce().double()
        nref = float(torch.linalg.norm(ref))
        for k, rate in enumerate(rates):
            R.cfg["rate"] = rate
            for form in ("g", "learned"):
                prm = lt.params(R.cfg, proposal=theta if form == "learned" else None, mix=mix)
                lt.lt_render_frame(ctx, R.frame, prm, R.cfg["frame_seed"], R.smp, R.uv, R.row_perm, R.img)
                lt.lt_sync(ctx)
                err[form][k] += float(torch.linalg.norm(R.img.double() - ref)) / nref / len(scene_seeds)
        del R
    out = dict(target=target, rates=rates, scenes=len(scene_seeds),
               mean_rel_rmse={f: [round(float(x), 5) for x in v] for f, v in err.items()})
    scene = make_scene(top, scene_seeds[0] if timing_scene is None else timing_scene)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=torch.device("cuda", ctx.device))
    for form in ("g", "learned"):
        ok = [k for k in range(len(rates)) if err[form][k] <= target]
        if not ok:
            out[form] = dict(iso_rate=None)
            continue
        rate = rates[ok[0]]
        R = Renderer(scene, dict(top, rate=rate), device=ctx.device, ctx=ctx).setup()
        g = lt.lt_frame_graph_capture(ctx, R.frame, lt.params(R.cfg, proposal=theta if form == "learned" else None,
                                                              mix=mix), R.smp, R.uv, R.row_perm, R.img,
                                      keep=(theta,))
        for k in range(3):
            lt.lt_frame_graph_launch(g, 9000 + k)
        ms = []
        for k in range(replays):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            lt.lt_frame_graph_launch(g, 9100 + k)
            b.record()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        ref = R.bruteforce().double()
        lt.lt_frame_graph_launch(g, R.cfg["frame_seed"])
        lt.lt_sync(ctx)
        rel = float(torch.linalg.norm(R.img.double() - ref) / torch.linalg.norm(ref))
        out[form] = dict(iso_rate=rate, ms_per_frame=round(float(np.median(ms)), 4),
                         rel_rmse_timing_scene=round(rel, 5), entries=int(R.smp.cnt.sum()))
        g.close()
        del R
    return out


def main():
    from ltinputs import get_config
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="room256_vpl16k_2box")
    ap.add_argument("--scenes", type=int, default=200)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--out", default=DEFAULT_THETA)
    ap.add_argument("--heldout", type=int, default=20)
    args = ap.parse_args()
    cfg = get_config(args.workload)
    ctx = lt.Context(0)
    theta, hist = train(ctx, cfg, [TRAIN_SEED0 + k for k in range(args.scenes)], args.epochs, args.lr, verbose=True)
    np.save(args.out, theta.cpu().numpy())
    print("saved", args.out, "loss", hist[0], "->", hist[-1])
    if args.heldout:
        res = ab_compare(ctx, cfg, theta, [cfg["scene_seed"] + k for k in range(args.heldout)])
        for r in res:
            print(r)
        g = np.mean([r["rel_g"] for r in res])
        p = np.mean([r["rel_learned"] for r in res])
        print(f"held-out mean rel-RMSE: g {g:.5f}  learned {p:.5f}")


if __name__ == "__main__":
    main()
