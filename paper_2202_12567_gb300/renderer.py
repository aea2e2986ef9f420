"""One scene, one camera: setup (tree, global cut, forest, slices) and frames.

A frame is the hot path of the method: pass 1 with coarsening (Sec. 4), pass 2
(Sec. 5), evaluation of the pass-2 entries, completion of every slice and the
factorised render (Sec. 3 step 5).  Every step is a liblt call; this class only
owns the tensors.
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import lt


def test_rows(width: int, height: int, block: int = 8) -> np.ndarray:
    """One pixel per block x block tile (offset block/2): the rows that drive the global cut."""
    ys = np.arange(block // 2, height, block)
    xs = np.arange(block // 2, width, block)
    if ys.size == 0:
        ys = np.array([height // 2])
    if xs.size == 0:
        xs = np.array([width // 2])
    gy, gx = np.meshgrid(ys, xs, indexing="ij")
    return (gy * width + gx).ravel()


class Renderer:
    def __init__(self, scene, cfg: dict, device: int = 0, ctx: lt.Context | None = None):
        self.cfg = dict(cfg)
        self.scene = scene
        self.dev = torch.device("cuda", device)
        self.ctx = ctx if ctx is not None else lt.Context(device)
        self.pts = torch.from_numpy(np.ascontiguousarray(scene.points)).to(self.dev)
        self.vpls = torch.from_numpy(np.ascontiguousarray(scene.vpls)).to(self.dev)
        self.boxes = torch.from_numpy(np.ascontiguousarray(scene.boxes)).to(self.dev).reshape(-1, 6)
        lt.lt_scene_upload(self.ctx, self.boxes)
        if getattr(scene, "tris", None) is not None:  # triangle occluders of a mesh scene
            self.tris = torch.from_numpy(np.ascontiguousarray(scene.tris, dtype=np.float32)).to(self.dev)
            lt.lt_mesh_upload(self.ctx, self.tris)
        self.frame = None

    # ---------------------------------------------------------------- setup (a0)
    def setup(self, cut=None, row_perm=None, slice_off=None):
        """Tree, global cut, forest and slices; ``cut``/``row_perm``/``slice_off`` may be
        given (e.g. from another implementation) instead of being computed."""
        cfg = self.cfg
        ctx = self.ctx
        times = {}
        mark = [time.perf_counter()]

        def lap(name):  # host time of the stage just finished (the stream is synchronised)
            torch.cuda.synchronize(self.dev)
            now = time.perf_counter()
            times[name] = round((now - mark[0]) * 1e3, 3)
            mark[0] = now

        self.tree = lt.lt_build_tree(ctx, self.vpls)
        lap("light_tree")
        if cut is None:
            rows = torch.from_numpy(test_rows(self.scene.width, self.scene.height).astype(np.int32)).to(self.dev)
            cut = lt.lt_build_global_cut(ctx, self.tree, self.pts, self.vpls, rows, cfg["eps_cut"], cfg["max_cut"],
                                         cfg.get("cut_growth", 0.5), cfg["d_min"])
        else:
            cut = torch.as_tensor(np.asarray(cut), dtype=torch.int32).to(self.dev)
        self.cut = cut
        lap("global_cut")
        forest, level_off, level_nodes, H = lt.lt_cut_forest(ctx, self.tree, cut)
        lap("cut_forest")
        if row_perm is None and cfg.get("slicing", "kmeans") == "split6d":  # the paper's recursive split
            row_perm, slice_off = lt.lt_make_slices_split(ctx, self.pts, cfg["slice_size"],
                                                          cfg["slice_feature_normal_weight"])
        elif row_perm is None:
            row_perm, slice_off = lt.lt_make_slices(ctx, self.pts, cfg["n_slices"], cfg["kmeans_iters"],
                                                    cfg["slice_feature_normal_weight"])
            if cfg.get("slice_bounds"):  # uneven slices held between two row counts
                lo, hi = cfg["slice_bounds"]
                row_perm, slice_off = lt.lt_bound_slices(ctx, self.pts, row_perm, slice_off, lo, hi,
                                                         cfg["slice_feature_normal_weight"])
        else:
            row_perm = torch.as_tensor(np.asarray(row_perm), dtype=torch.int32).to(self.dev)
            slice_off = torch.as_tensor(np.asarray(slice_off), dtype=torch.int32).to(self.dev)
        self.row_perm, self.slice_off = row_perm, slice_off
        lap("slices")
        self.pts_s = lt.lt_permute_points(ctx, self.pts, row_perm)
        self.frame = lt.Frame(self.pts_s, self.vpls, slice_off, self.tree, cut, forest, level_off, level_nodes, H)
        self.smp = lt.Samples(self.frame, cfg["rate"], cfg["rate1"])
        self.uv = lt.Factors(self.frame, cfg["rank"], per_slice=int(cfg.get("rank_cols", 0)) > 0)
        self.img = torch.zeros(self.frame.m, dtype=torch.float32, device=self.dev)
        lt.lt_sync(ctx)
        lap("points_and_buffers")
        self.setup_ms = times
        return self

    # ---------------------------------------------------------------- frame stages
    def pass1(self, seed):
        c = self.cfg
        if int(c.get("target_cut", 0)) > 0:  # coarsen to a target cut size (Sec. 4)
            lt.lt_sample_pass1_target(self.ctx, self.frame, self.smp, c["rate1"], c["target_cut"], c["d_min"], seed)
        else:
            lt.lt_sample_pass1(self.ctx, self.frame, self.smp, c["rate1"], c["tau"], c["d_min"], seed)

    def pass2(self, seed, weights=None):
        lt.lt_sample_pass2(self.ctx, self.frame, self.smp, self.cfg["rate"], seed, weights)

    def evaluate(self):
        lt.lt_eval_entries(self.ctx, self.frame, self.smp, self.cfg["d_min"])

    def complete(self, seed, warm=False, iters=None):
        """warm: start from the previous warm frame's factors (lt_complete_warm) and keep
        this frame's for the next; iters: sweeps instead of the workload's."""
        c = self.cfg
        iters = c["als_iters"] if iters is None else int(iters)
        if int(c.get("rank_cols", 0)) > 0:  # per-slice ranks from the coarsened cut
            lt.lt_slice_ranks(self.ctx, self.frame, self.smp, c["rank"], c["rank_cols"], self.uv.rank)
        if c.get("completion", "als") == "adm":  # nonnegative completion (App. A)
            lt.lt_complete_adm(self.ctx, self.frame, self.smp, self.uv, c["adm_iters"], c["adm_alpha_rel"],
                               c["adm_gamma"], seed)
            return
        prev = getattr(self, "_prev", None)
        if warm and prev is not None:  # temporal coherence: the previous frame's factors
            lt.lt_complete_warm(self.ctx, self.frame, self.smp, self.uv, iters, c["lam_rel"], seed, *prev)
        else:
            lt.lt_complete(self.ctx, self.frame, self.smp, self.uv, iters, c["lam_rel"], seed)
        if warm:
            self._prev = (self.smp.col_node.clone(), self.smp.ncol.clone(), self.uv.V.clone())

    def render_image(self, w=None):
        lt.lt_render(self.ctx, self.frame, self.smp, self.uv, self.row_perm, self.img, w)

    def render(self, seed=None, weights=None, sync=True, warm=False, iters=None):
        """One frame: pass 1, pass 2, entry evaluation, completion, image (warm, iters:
        see complete)."""
        seed = self.cfg["frame_seed"] if seed is None else seed
        self.pass1(seed)
        self.pass2(seed, weights)
        self.evaluate()
        self.complete(seed, warm=warm, iters=iters)
        self.render_image()
        if sync:
            lt.lt_sync(self.ctx)
        return self.img

    def render_frame(self, seed=None, weights=None, sync=True):
        """The same frame through the single C entry point lt_render_frame."""
        seed = self.cfg["frame_seed"] if seed is None else seed
        self._prm = lt.params(self.cfg, weights)
        lt.lt_render_frame(self.ctx, self.frame, self._prm, seed, self.smp, self.uv, self.row_perm, self.img)
        if sync:
            lt.lt_sync(self.ctx)
        return self.img

    def capture(self, weights=None):
        """Capture the frame as a CUDA graph (lt_frame_graph_capture); replay with render_graph."""
        if getattr(self, "graph", None) is not None:
            self.graph.close()
        self.graph = lt.lt_frame_graph_capture(self.ctx, self.frame, lt.params(self.cfg, weights), self.smp, self.uv,
                                               self.row_perm, self.img, keep=(weights,))
        return self.graph

    def render_graph(self, seed=None, sync=True):
        seed = self.cfg["frame_seed"] if seed is None else seed
        lt.lt_frame_graph_launch(self.graph, seed)
        if sync:
            lt.lt_sync(self.ctx)
        return self.img

    # ---------------------------------------------------------------- colour
    def setup_rgb(self):
        """Colour tables and the stacked frame of an RGB scene (scene.rgb)."""
        rgb = self.scene.rgb
        m, n = self.scene.m, self.scene.n
        pa = np.zeros((m, 4), dtype=np.float32)
        pa[:, :3] = rgb["point_albedo"]
        vp = np.zeros((n, 4), dtype=np.float32)
        vp[:, :3] = rgb["vpl_flux"].astype(np.float64) * rgb["vpl_albedo"]
        self.rgb = lt.RGB(self.frame, self.smp, self.cfg["rank"], per_slice=int(self.cfg.get("rank_cols", 0)) > 0)
        self._rgb_in = (torch.from_numpy(pa).to(self.dev), torch.from_numpy(vp).to(self.dev))
        lt.lt_rgb_setup(self.ctx, self.frame, self.rgb, self._rgb_in[0], self._rgb_in[1], self.row_perm)
        return self

    def render_rgb(self, seed=None, weights=None, sync=True):
        """One colour frame: scalar sampling and evaluation, the three channels of every
        sample, completion of the stacked slices, image [m][3]."""
        c = self.cfg
        seed = c["frame_seed"] if seed is None else seed
        self.pass1(seed)
        self.pass2(seed, weights)
        self.evaluate()
        lt.lt_expand_rgb(self.ctx, self.frame, self.smp, self.rgb)
        if self.rgb.rank is not None:
            lt.lt_slice_ranks(self.ctx, self.frame, self.smp, c["rank"], c["rank_cols"], self.rgb.rank)
        adm = (c["adm_iters"], c["adm_alpha_rel"], c["adm_gamma"]) if c.get("completion", "als") == "adm" else None
        lt.lt_complete_rgb(self.ctx, self.rgb, c["als_iters"], c["lam_rel"], seed, adm)
        lt.lt_render_rgb(self.ctx, self.rgb)
        if sync:
            lt.lt_sync(self.ctx)
        return self.rgb.img.view(-1, 3)

    def bruteforce_rgb(self):
        """The full image over all VPLs per channel [m][3] (k_bruteforce per channel)."""
        rgb = self.scene.rgb
        out = torch.zeros((self.scene.m, 3), dtype=torch.float32, device=self.dev)
        for k in range(3):
            pts = self.pts.clone()
            pts[0, :, 3] = torch.from_numpy(np.ascontiguousarray(rgb["point_albedo"][:, k])).to(self.dev)
            vpl = self.vpls.clone()
            vpl[0, :, 3] = torch.from_numpy(np.ascontiguousarray(rgb["vpl_albedo"][:, k])).to(self.dev)
            vpl[2, :, 3] = torch.from_numpy(np.ascontiguousarray(rgb["vpl_flux"][:, k])).to(self.dev)
            img = torch.empty(self.scene.m, dtype=torch.float32, device=self.dev)
            lt.lt_bruteforce(self.ctx, pts, vpl, self.cfg["d_min"], img)
            out[:, k] = img
        return out

    def bruteforce(self, out=None):
        return lt.lt_bruteforce(self.ctx, self.pts, self.vpls, self.cfg["d_min"], out)

    def rays(self) -> int:
        """Shadow-ray-bearing entries of the last frame (pass-1 tests are counted in pass 1)."""
        return int(self.smp.cnt.sum().item())
