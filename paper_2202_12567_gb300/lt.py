"""Thin Python binding of liblt (include/lt.h): argument marshalling only.

Every function here has the name of the C entry point it wraps and does no
computation of its own: device memory comes from PyTorch tensors, whose raw
pointers are handed to the library, and every step runs in the library's CUDA
kernels.  The first context (or an explicit load()) loads liblt.so and fails
loudly when it is missing; there is no fallback path.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblt.so")

LT_OK, LT_EINVAL, LT_ENOMEM, LT_ECUDA, LT_ELIMIT, LT_ENUMERIC = 0, 1, 2, 3, 4, 5


class LtError(RuntimeError):
    def __init__(self, fn, code, msg):
        super().__init__(f"{fn} failed with status {code}: {msg}")
        self.code = code


_lib = None
_p = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_f32 = ctypes.c_float
_u64 = ctypes.c_uint64


class lt_tree(ctypes.Structure):
    _fields_ = [("n", _i64), ("order", _p), ("child", _p), ("parent", _p), ("range", _p), ("rep", _p),
                ("I", _p), ("B", _p), ("aabb", _p)]


class lt_frame(ctypes.Structure):
    _fields_ = [("pts", _p), ("m", _i64), ("vpls", _p), ("n", _i64), ("slice_off", _p), ("S", _i32),
                ("max_rows", _i32), ("tree", lt_tree), ("C", _i32), ("forest", _p), ("level_off", _p),
                ("level_nodes", _p), ("H", _i32), ("slice_id", _p)]


class lt_samples(ctypes.Structure):
    _fields_ = [("ncol", _p), ("col_node", _p), ("g", _p), ("off", _p), ("key", _p), ("val", _p), ("n1", _p),
                ("cnt", _p)]


class lt_factors(ctypes.Structure):
    _fields_ = [("r", _i32), ("U", _p), ("V", _p), ("rank", _p)]


class lt_rgb(ctypes.Structure):
    _fields_ = [("pt_ratio", _p), ("node_ratio", _p), ("slice_off3", _p), ("row_perm3", _p)]


class lt_params(ctypes.Structure):
    _fields_ = [("rate1", _f32), ("tau", _f32), ("d_min", _f32), ("rate", _f32), ("als_iters", _i32),
                ("lam_rel", _f32), ("weights", _p), ("proposal", _p), ("mix", _f32), ("rank_cols", _i32),
                ("completion", _i32), ("adm_iters", _i32), ("adm_alpha_rel", _f32), ("adm_gamma", _f32),
                ("target_cut", _i32)]


COMPLETE_ALS, COMPLETE_ADM = 0, 1


MLP_FEATURES, MLP_HIDDEN, MLP_PARAMS = 32, 64, 10497


class lt_tuning(ctypes.Structure):
    _fields_ = [("eval_ctas_per_sm", _i32), ("ray_ctas_per_sm", _i32), ("als_lane_entries", _i32),
                ("als_form", _i32), ("p1_form", _i32)]


_SIGS = {
    "lt_status_str": (ctypes.c_char_p, [_i32]),
    "lt_last_error": (ctypes.c_char_p, [_p]),
    "lt_create": (_i32, [ctypes.POINTER(_p), ctypes.c_int, _p]),
    "lt_destroy": (_i32, [_p]),
    "lt_sync": (_i32, [_p]),
    "lt_status_word": (_p, [_p]),
    "lt_launch_count": (_i64, [_p]),
    "lt_debug_scratch": (_i32, [_p, _i32, ctypes.POINTER(_p), ctypes.POINTER(_i64)]),
    "lt_set_scratch_limit": (_i32, [_p, _i64]),
    "lt_scene_upload": (_i32, [_p, _p, _i64, _i32]),
    "lt_shadow_test": (_i32, [_p, _p, _p, _i64, _p]),
    "lt_eval_pairs": (_i32, [_p, _p, _i64, _p, _i64, _p, _p, _p, _i64, _f32, _p]),
    "lt_bruteforce": (_i32, [_p, _p, _i64, _p, _i64, _f32, _p]),
    "lt_bruteforce_stats": (_i32, [_p, _p, _i64, _p, _i64, _f32, _p]),
    "lt_build_tree": (_i32, [_p, _p, _i64, ctypes.POINTER(lt_tree)]),
    "lt_build_global_cut": (_i32, [_p, ctypes.POINTER(lt_tree), _p, _i64, _p, _p, _i64, _f32, _i32, _f32, _f32,
                                   _p, ctypes.POINTER(_i32)]),
    "lt_cut_errors": (_i32, [_p, ctypes.POINTER(lt_tree), _p, _i64, _p, _p, _i64, _p, _i32, _f32, _p]),
    "lt_complete_fp64_lines": (_i32, [_p, ctypes.POINTER(_i64)]),
    "lt_als_gram": (_i32, [_p, ctypes.POINTER(lt_frame), ctypes.POINTER(lt_samples), ctypes.POINTER(lt_factors),
                           _i32, _p]),
    "lt_cut_forest": (_i32, [_p, ctypes.POINTER(lt_tree), _p, _i32, _p, _p, _i32, _p, ctypes.POINTER(_i32)]),
    "lt_make_slices": (_i32, [_p, _p, _i64, _i32, _i32, _f32, _p, _p]),
    "lt_permute_points": (_i32, [_p, _p, _i64, _p, _p]),
    "lt_bound_slices": (_i32, [_p, _p, _i64, _p, _p, _i32, _i32, _i32, _f32, _i32, _p, _p, ctypes.POINTER(_i32)]),
    "lt_sample_pass1": (_i32, [_p, ctypes.POINTER(lt_frame), _f32, _f32, _f32, _u64, ctypes.POINTER(lt_samples)]),
    "lt_sample_pass1_target": (_i32, [_p, ctypes.POINTER(lt_frame), _f32, _i32, _f32, _u64,
                                      ctypes.POINTER(lt_samples)]),
    "lt_sample_pass2": (_i32, [_p, ctypes.POINTER(lt_frame), _p, _f32, _u64, ctypes.POINTER(lt_samples)]),
    "lt_eval_entries": (_i32, [_p, ctypes.POINTER(lt_frame), _f32, ctypes.POINTER(lt_samples)]),
    "lt_eval_stats": (_i32, [_p, ctypes.POINTER(lt_frame), _f32, ctypes.POINTER(lt_samples), _p]),
    "lt_eval_entries_noalloc": (_i32, [_p, ctypes.POINTER(lt_frame), _f32, ctypes.POINTER(lt_samples)]),
    "lt_complete": (_i32, [_p, ctypes.POINTER(lt_frame), ctypes.POINTER(lt_samples), _i32, _f32, _u64,
                           ctypes.POINTER(lt_factors)]),
    "lt_complete_warm": (_i32, [_p, ctypes.POINTER(lt_frame), ctypes.POINTER(lt_samples), _i32, _f32, _u64, _p, _p,
                                _p, ctypes.POINTER(lt_factors)]),
    "lt_complete_adm": (_i32, [_p, ctypes.POINTER(lt_frame), ctypes.POINTER(lt_samples), _i32, _f32, _f32, _u64,
                               ctypes.POINTER(lt_factors)]),
    "lt_mesh_upload": (_i32, [_p, _p, _i64]),
    "lt_mesh_bvh": (_i32, [_p, _p, _p, _p]),
    "lt_split_slice_count": (_i32, [_i64, _i32]),
    "lt_make_slices_split": (_i32, [_p, _p, _i64, _i32, _f32, _p, _p]),
    "lt_rgb_setup": (_i32, [_p, ctypes.POINTER(lt_frame), _p, _p, _p, ctypes.POINTER(lt_rgb)]),
    "lt_expand_rgb": (_i32, [_p, ctypes.POINTER(lt_frame), ctypes.POINTER(lt_samples), ctypes.POINTER(lt_rgb),
                             ctypes.POINTER(lt_samples)]),
    "lt_render": (_i32, [_p, ctypes.POINTER(lt_frame), ctypes.POINTER(lt_samples), ctypes.POINTER(lt_factors), _p,
                         _p, _p]),
    "lt_render_frame": (_i32, [_p, ctypes.POINTER(lt_frame), ctypes.POINTER(lt_params), _u64,
                               ctypes.POINTER(lt_samples), ctypes.POINTER(lt_factors), _p, _p]),
    "lt_frame_graph_capture": (_i32, [_p, ctypes.POINTER(lt_frame), ctypes.POINTER(lt_params),
                                      ctypes.POINTER(lt_samples), ctypes.POINTER(lt_factors), _p, _p,
                                      ctypes.POINTER(_p)]),
    "lt_frame_graph_launch": (_i32, [_p, _u64]),
    "lt_get_tuning": (_i32, [_p, ctypes.POINTER(lt_tuning)]),
    "lt_slice_ranks": (_i32, [_p, ctypes.POINTER(lt_frame), ctypes.POINTER(lt_samples), _i32, _i32, _p]),
    "lt_set_tuning": (_i32, [_p, ctypes.POINTER(lt_tuning)]),
    "lt_proposal_features": (_i32, [_p, ctypes.POINTER(lt_frame), ctypes.POINTER(lt_samples), _p, _p]),
    "lt_proposal_forward": (_i32, [_p, _p, _p, _i64, _p, _p]),
    "lt_proposal_weights": (_i32, [_p, ctypes.POINTER(lt_frame), ctypes.POINTER(lt_samples), _p, _p, _f32, _p]),
    "lt_slice_matrices": (_i32, [_p, ctypes.POINTER(lt_frame), ctypes.POINTER(lt_samples), _f32, _p, _i64, _p]),
    "lt_leverage_targets": (_i32, [_p, ctypes.POINTER(lt_frame), ctypes.POINTER(lt_samples), _p, _p, _p, _i32, _i32,
                                   _u64, _p]),
    "lt_proposal_init": (_i32, [_p, _u64, _p]),
    "lt_proposal_grad": (_i32, [_p, _p, _p, _p, _p, _i32, _i64, _p, _p]),
    "lt_proposal_adam": (_i32, [_p, _p, _p, _p, _p, _i32, _f32]),
    "lt_frame_graph_kernels": (_i64, [_p]),
    "lt_frame_graph_destroy": (_i32, [_p]),
}

EXPORTED = sorted(_SIGS)


def load(path: str = LIB_PATH):
    """Load liblt.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(f"liblt.so not found at {path}: run __graft_entry__.build() first")
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _ptr(t):
    if t is None:
        return None
    assert isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous(), "expected a contiguous CUDA tensor"
    return ctypes.c_void_p(t.data_ptr())


class Context:
    """An lt_ctx handle on one device; calls run on ``stream`` (default: the current torch stream)."""

    def __init__(self, device: int = 0, stream: torch.cuda.Stream | None = None):
        self.lib = load()
        self.device = device
        torch.cuda.set_device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        h = _p()
        self._check("lt_create", self.lib.lt_create(ctypes.byref(h), device, _p(self.stream.cuda_stream)))
        self.h = h

    def _check(self, fn, code):
        if code != LT_OK:
            msg = self.lib.lt_last_error(self.h).decode() if getattr(self, "h", None) else ""
            raise LtError(fn, code, msg)

    def close(self):
        if getattr(self, "h", None):
            self.lib.lt_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lt_launch_count(ctx: Context) -> int:
    return int(ctx.lib.lt_launch_count(ctx.h))


class _DevBuf:
    def __init__(self, ptr, nbytes):
        self.__cuda_array_interface__ = dict(shape=(nbytes,), typestr="|u1", data=(ptr, False), version=3)


def lt_debug_scratch(ctx: Context, slot: int) -> torch.Tensor:
    """A uint8 view of scratch slot ``slot`` (debugging aid)."""
    ptr, size = _p(), _i64()
    ctx._check("lt_debug_scratch", ctx.lib.lt_debug_scratch(ctx.h, slot, ctypes.byref(ptr), ctypes.byref(size)))
    if not ptr.value:
        return torch.zeros(0, dtype=torch.uint8, device="cuda")
    return torch.as_tensor(_DevBuf(ptr.value, size.value), device="cuda")


def lt_set_scratch_limit(ctx: Context, nbytes: int):
    ctx._check("lt_set_scratch_limit", ctx.lib.lt_set_scratch_limit(ctx.h, int(nbytes)))


def lt_sync(ctx: Context):
    ctx._check("lt_sync", ctx.lib.lt_sync(ctx.h))


def lt_scene_upload(ctx: Context, boxes: torch.Tensor, grid_res: int = 0):
    boxes = boxes.contiguous()
    ctx._boxes = boxes
    ctx._check("lt_scene_upload", ctx.lib.lt_scene_upload(ctx.h, _ptr(boxes) if boxes.numel() else None,
                                                          boxes.shape[0], grid_res))


def lt_shadow_test(ctx: Context, org: torch.Tensor, end: torch.Tensor) -> torch.Tensor:
    k = org.shape[0]
    out = torch.empty(k, dtype=torch.uint8, device=org.device)
    ctx._check("lt_shadow_test", ctx.lib.lt_shadow_test(ctx.h, _ptr(org), _ptr(end), k, _ptr(out)))
    return out


def lt_eval_pairs(ctx: Context, pts, vpls, rows, vpl, scale=None, d_min=0.01) -> torch.Tensor:
    out = torch.empty(rows.shape[0], dtype=torch.float32, device=pts.device)
    ctx._check("lt_eval_pairs", ctx.lib.lt_eval_pairs(ctx.h, _ptr(pts), pts.shape[1], _ptr(vpls), vpls.shape[1],
                                                      _ptr(rows), _ptr(vpl), _ptr(scale), rows.shape[0], d_min,
                                                      _ptr(out)))
    return out


def lt_bruteforce(ctx: Context, pts, vpls, d_min=0.01, out=None) -> torch.Tensor:
    m = pts.shape[1]
    img = torch.empty(m, dtype=torch.float32, device=pts.device) if out is None else out
    ctx._check("lt_bruteforce", ctx.lib.lt_bruteforce(ctx.h, _ptr(pts), m, _ptr(vpls), vpls.shape[1], d_min,
                                                      _ptr(img)))
    return img


def lt_bruteforce_stats(ctx: Context, pts, vpls, d_min=0.01) -> dict:
    out = (ctypes.c_int64 * 4)()
    ctx._check("lt_bruteforce_stats", ctx.lib.lt_bruteforce_stats(ctx.h, _ptr(pts), pts.shape[1], _ptr(vpls),
                                                                  vpls.shape[1], d_min, ctypes.cast(out, _p)))
    return dict(entries=out[0], rays=out[1], cells=out[2], boxes=out[3])


class Tree:
    """Device arrays of a light tree (see lt_tree)."""

    def __init__(self, n: int, device):
        N = 2 * n - 1
        i32 = dict(dtype=torch.int32, device=device)
        f32 = dict(dtype=torch.float32, device=device)
        self.n = n
        self.order = torch.empty(n, **i32)
        self.child = torch.empty(N, 2, **i32)
        self.parent = torch.empty(N, **i32)
        self.range = torch.empty(N, 2, **i32)
        self.rep = torch.empty(N, **i32)
        self.I = torch.empty(N, **f32)
        self.B = torch.empty(N, **f32)
        self.aabb = torch.empty(N, 6, **f32)

    def struct(self) -> lt_tree:
        return lt_tree(self.n, _ptr(self.order), _ptr(self.child), _ptr(self.parent), _ptr(self.range),
                       _ptr(self.rep), _ptr(self.I), _ptr(self.B), _ptr(self.aabb))


def lt_build_tree(ctx: Context, vpls: torch.Tensor) -> Tree:
    n = vpls.shape[1]
    t = Tree(n, vpls.device)
    s = t.struct()
    ctx._check("lt_build_tree", ctx.lib.lt_build_tree(ctx.h, _ptr(vpls), n, ctypes.byref(s)))
    return t


def lt_build_global_cut(ctx: Context, tree: Tree, pts, vpls, rows, eps, max_cut, growth=0.5, d_min=0.01):
    cut = torch.empty(max_cut, dtype=torch.int32, device=pts.device)
    size = _i32(0)
    s = tree.struct()
    ctx._check("lt_build_global_cut", ctx.lib.lt_build_global_cut(
        ctx.h, ctypes.byref(s), _ptr(pts), pts.shape[1], _ptr(vpls), _ptr(rows), rows.shape[0], eps, max_cut,
        growth, d_min, _ptr(cut), ctypes.byref(size)))
    return cut[:size.value].clone()


def lt_cut_errors(ctx: Context, tree: Tree, pts, vpls, rows, cut, d_min=0.01) -> torch.Tensor:
    err = torch.empty(cut.shape[0], dtype=torch.float32, device=cut.device)
    ctx._check("lt_cut_errors", ctx.lib.lt_cut_errors(ctx.h, ctypes.byref(tree.struct()), _ptr(pts), pts.shape[1],
                                                      _ptr(vpls), _ptr(rows), rows.shape[0], _ptr(cut),
                                                      cut.shape[0], d_min, _ptr(err)))
    return err


def lt_cut_forest(ctx: Context, tree: Tree, cut: torch.Tensor, max_levels: int = 256):
    C = cut.shape[0]
    dev = cut.device
    forest = torch.empty((2 * C - 1) * 8, dtype=torch.int32, device=dev)
    level_off = torch.zeros(max_levels + 2, dtype=torch.int32, device=dev)
    level_nodes = torch.empty(max(C - 1, 1), dtype=torch.int32, device=dev)
    H = _i32(0)
    s = tree.struct()
    ctx._check("lt_cut_forest", ctx.lib.lt_cut_forest(ctx.h, ctypes.byref(s), _ptr(cut), C, _ptr(forest),
                                                      _ptr(level_off), max_levels, _ptr(level_nodes),
                                                      ctypes.byref(H)))
    return forest, level_off, level_nodes, H.value


def lt_make_slices(ctx: Context, pts, S, iters=10, normal_weight=0.3):
    m = pts.shape[1]
    perm = torch.empty(m, dtype=torch.int32, device=pts.device)
    off = torch.empty(S + 1, dtype=torch.int32, device=pts.device)
    ctx._check("lt_make_slices", ctx.lib.lt_make_slices(ctx.h, _ptr(pts), m, S, iters, normal_weight, _ptr(perm),
                                                        _ptr(off)))
    return perm, off


def lt_permute_points(ctx: Context, pts, row_perm):
    out = torch.empty_like(pts)
    ctx._check("lt_permute_points", ctx.lib.lt_permute_points(ctx.h, _ptr(pts), pts.shape[1], _ptr(row_perm),
                                                              _ptr(out)))
    return out


class Frame:
    """The fixed inputs of a frame (lt_frame) and the tensors behind its pointers."""

    def __init__(self, pts_s, vpls, slice_off, tree: Tree, cut, forest, level_off, level_nodes, H, slice_id=None):
        self.pts_s, self.vpls, self.slice_off, self.tree, self.cut = pts_s, vpls, slice_off, tree, cut
        self.forest, self.level_off, self.level_nodes, self.H = forest, level_off, level_nodes, H
        self.slice_id = slice_id  # [S] int32 device tensor: each slice's index in the whole frame, or None
        self.slice_off_host = slice_off.cpu().numpy().astype(np.int64)
        self.sizes = np.diff(self.slice_off_host)
        self.S = len(self.sizes)
        self.C = int(cut.shape[0])
        self.m = pts_s.shape[1]
        self._s = lt_frame(_ptr(pts_s), self.m, _ptr(vpls), vpls.shape[1], _ptr(slice_off), self.S,
                           int(self.sizes.max()) if self.S else 0, tree.struct(), self.C, _ptr(forest),
                           _ptr(level_off), _ptr(level_nodes), H, _ptr(slice_id))

    def struct(self) -> lt_frame:
        return self._s


class Samples:
    """Per-slice observed entries (lt_samples) with a capacity layout for ``rate``."""

    def __init__(self, frame: Frame, rate: float, rate1: float):
        S, C = frame.S, frame.C
        dev = frame.pts_s.device
        caps = []
        for ms in frame.sizes:
            kappa = max(2.0, rate1 * ms)
            k_sum = min(64, ms) * C if ms else 0
            k_sum = min(k_sum, int(1.001 * (kappa * C + 2.5 * C)) + 16)
            caps.append(2 * k_sum + int(math.ceil(rate * ms * C)) + 64)
        off = np.concatenate([[0], np.cumsum(caps)]).astype(np.int64)
        i32 = dict(dtype=torch.int32, device=dev)
        self.ncol = torch.zeros(S, **i32)
        self.col_node = torch.zeros(S * C, **i32)
        self.g = torch.zeros(S * C, dtype=torch.float32, device=dev)
        self.off = torch.from_numpy(off).to(dev)
        self.key = torch.zeros(int(off[-1]), dtype=torch.int32, device=dev)
        self.val = torch.zeros(int(off[-1]), dtype=torch.float32, device=dev)
        self.n1 = torch.zeros(S, **i32)
        self.cnt = torch.zeros(S, **i32)
        self.off_host = off
        self._s = lt_samples(_ptr(self.ncol), _ptr(self.col_node), _ptr(self.g), _ptr(self.off), _ptr(self.key),
                             _ptr(self.val), _ptr(self.n1), _ptr(self.cnt))

    def struct(self) -> lt_samples:
        return self._s

    def slice(self, s: int):
        """Host copies (rows, cols, vals, col_node, g) of slice s."""
        o = int(self.off_host[s])
        c = int(self.cnt[s].item())
        n = int(self.ncol[s].item())
        C = self.col_node.shape[0] // self.ncol.shape[0]
        key = self.key[o:o + c].cpu().numpy().astype(np.uint32)
        return (key >> 16).astype(np.int64), (key & 0xFFFF).astype(np.int64), self.val[o:o + c].cpu().numpy(), \
            self.col_node[s * C:s * C + n].cpu().numpy(), self.g[s * C:s * C + n].cpu().numpy()


class RGB:
    """Colour tables of a frame (lt_rgb) and the stacked frame, samples, factors and
    image: slice s of m' pixels becomes 3m' rows, row 3i + k = channel k of pixel i."""

    def __init__(self, frame: Frame, smp: Samples, r: int, per_slice: bool = False):
        dev = frame.pts_s.device
        n = frame.vpls.shape[1]
        self.pt_ratio = torch.zeros(frame.m * 4, dtype=torch.float32, device=dev)
        self.node_ratio = torch.zeros((2 * n - 1) * 4, dtype=torch.float32, device=dev)
        self.slice_off3 = torch.zeros(frame.S + 1, dtype=torch.int32, device=dev)
        self.row_perm3 = torch.zeros(3 * frame.m, dtype=torch.int32, device=dev)
        self._s = lt_rgb(_ptr(self.pt_ratio), _ptr(self.node_ratio), _ptr(self.slice_off3), _ptr(self.row_perm3))
        f = frame.struct()
        self._f3 = lt_frame(f.pts, 3 * frame.m, f.vpls, f.n, _ptr(self.slice_off3), f.S, 3 * f.max_rows, f.tree,
                            f.C, f.forest, f.level_off, f.level_nodes, f.H, f.slice_id)
        # stacked samples: three times the capacity of every slice
        i32 = dict(dtype=torch.int32, device=dev)
        self.off_host = 3 * smp.off_host
        self.off = torch.from_numpy(self.off_host).to(dev)
        self.key = torch.zeros(int(self.off_host[-1]), **i32)
        self.val = torch.zeros(int(self.off_host[-1]), dtype=torch.float32, device=dev)
        self.ncol = torch.zeros(frame.S, **i32)
        self.n1 = torch.zeros(frame.S, **i32)
        self.cnt = torch.zeros(frame.S, **i32)
        self.col_node, self.g = smp.col_node, smp.g
        self._smp3 = lt_samples(_ptr(self.ncol), _ptr(smp.col_node), _ptr(smp.g), _ptr(self.off), _ptr(self.key),
                                _ptr(self.val), _ptr(self.n1), _ptr(self.cnt))
        self.r = r
        self.U = torch.zeros(3 * frame.m * r, dtype=torch.float32, device=dev)
        self.V = torch.zeros(frame.S * frame.C * r, dtype=torch.float32, device=dev)
        self.rank = torch.full((frame.S,), r, dtype=torch.int32, device=dev) if per_slice else None
        self._uv3 = lt_factors(r, _ptr(self.U), _ptr(self.V), _ptr(self.rank))
        self.img = torch.zeros(3 * frame.m, dtype=torch.float32, device=dev)
        self.C = frame.C

    def struct(self) -> lt_rgb:
        return self._s

    def frame3(self) -> lt_frame:
        return self._f3

    def samples3(self) -> lt_samples:
        return self._smp3

    def factors3(self) -> lt_factors:
        return self._uv3

    def slice(self, s: int):
        """Host copies (rows, cols, vals) of stacked slice s."""
        o = int(self.off_host[s])
        c = int(self.cnt[s].item())
        key = self.key[o:o + c].cpu().numpy().astype(np.uint32)
        return (key >> 16).astype(np.int64), (key & 0xFFFF).astype(np.int64), self.val[o:o + c].cpu().numpy()


class Factors:
    """U, V with row stride r; per_slice=True adds the per-slice rank array [S]."""

    def __init__(self, frame: Frame, r: int, per_slice: bool = False):
        dev = frame.pts_s.device
        self.r = r
        self.U = torch.zeros(frame.m * r, dtype=torch.float32, device=dev)
        self.V = torch.zeros(frame.S * frame.C * r, dtype=torch.float32, device=dev)
        self.rank = torch.full((frame.S,), r, dtype=torch.int32, device=dev) if per_slice else None
        self._s = lt_factors(r, _ptr(self.U), _ptr(self.V), _ptr(self.rank))

    def struct(self) -> lt_factors:
        return self._s


def lt_sample_pass1(ctx: Context, frame: Frame, smp: Samples, rate, tau, d_min, seed):
    ctx._check("lt_sample_pass1", ctx.lib.lt_sample_pass1(ctx.h, ctypes.byref(frame.struct()), rate, tau, d_min,
                                                          seed, ctypes.byref(smp.struct())))


def lt_sample_pass1_target(ctx: Context, frame: Frame, smp: Samples, rate1, target, d_min, seed):
    ctx._check("lt_sample_pass1_target", ctx.lib.lt_sample_pass1_target(ctx.h, ctypes.byref(frame.struct()), rate1,
                                                                        int(target), d_min, seed,
                                                                        ctypes.byref(smp.struct())))


def lt_sample_pass2(ctx: Context, frame: Frame, smp: Samples, rate, seed, weights=None):
    ctx._check("lt_sample_pass2", ctx.lib.lt_sample_pass2(ctx.h, ctypes.byref(frame.struct()), _ptr(weights), rate,
                                                          seed, ctypes.byref(smp.struct())))


def lt_eval_entries(ctx: Context, frame: Frame, smp: Samples, d_min):
    ctx._check("lt_eval_entries", ctx.lib.lt_eval_entries(ctx.h, ctypes.byref(frame.struct()), d_min,
                                                          ctypes.byref(smp.struct())))


def lt_eval_entries_noalloc(ctx: Context, frame: Frame, smp: Samples, d_min):
    """lt_eval_entries for hosts that forbid library allocations (see include/lt.h)."""
    ctx._check("lt_eval_entries_noalloc", ctx.lib.lt_eval_entries_noalloc(ctx.h, ctypes.byref(frame.struct()), d_min,
                                                                          ctypes.byref(smp.struct())))


def lt_eval_stats(ctx: Context, frame: Frame, smp: Samples, d_min) -> dict:
    out = (ctypes.c_int64 * 4)()
    ctx._check("lt_eval_stats", ctx.lib.lt_eval_stats(ctx.h, ctypes.byref(frame.struct()), d_min,
                                                      ctypes.byref(smp.struct()), ctypes.cast(out, _p)))
    return dict(entries=out[0], rays=out[1], cells=out[2], boxes=out[3])


def lt_complete(ctx: Context, frame: Frame, smp: Samples, uv: Factors, iters, lam_rel, seed):
    ctx._check("lt_complete", ctx.lib.lt_complete(ctx.h, ctypes.byref(frame.struct()), ctypes.byref(smp.struct()),
                                                  iters, lam_rel, seed, ctypes.byref(uv.struct())))


def lt_complete_warm(ctx: Context, frame: Frame, smp: Samples, uv: Factors, iters, lam_rel, seed, prev_col_node,
                     prev_ncol, prev_V):
    """lt_complete started from a previous frame's columns and V (device tensors the
    caller keeps; prev_V is not uv.V)."""
    ctx._check("lt_complete_warm", ctx.lib.lt_complete_warm(ctx.h, ctypes.byref(frame.struct()),
                                                            ctypes.byref(smp.struct()), iters, lam_rel, seed,
                                                            _ptr(prev_col_node), _ptr(prev_ncol), _ptr(prev_V),
                                                            ctypes.byref(uv.struct())))


def lt_als_gram(ctx: Context, frame: Frame, smp: Samples, uv: Factors, side: int):
    """Gram matrices and right-hand sides of one ALS half-step from the tensor-core
    contraction: [lines][r (r + 3) / 2] float32 (side 0: m slice-ordered rows, side 1:
    S C columns; lines past n'_s stay NaN)."""
    r = uv.r
    lines = frame.m if side == 0 else frame.S * frame.C
    out = torch.full((lines, r * (r + 3) // 2), float("nan"), dtype=torch.float32, device=uv.U.device)
    ctx._check("lt_als_gram", ctx.lib.lt_als_gram(ctx.h, ctypes.byref(frame.struct()), ctypes.byref(smp.struct()),
                                                  ctypes.byref(uv.struct()), int(side), _ptr(out)))
    return out


def lt_complete_fp64_lines(ctx: Context) -> int:
    n = _i64(0)
    ctx._check("lt_complete_fp64_lines", ctx.lib.lt_complete_fp64_lines(ctx.h, ctypes.byref(n)))
    return int(n.value)


def lt_complete_adm(ctx: Context, frame: Frame, smp: Samples, uv: Factors, iters, alpha_rel, gamma, seed):
    ctx._check("lt_complete_adm", ctx.lib.lt_complete_adm(ctx.h, ctypes.byref(frame.struct()),
                                                          ctypes.byref(smp.struct()), iters, alpha_rel, gamma, seed,
                                                          ctypes.byref(uv.struct())))


def lt_mesh_upload(ctx: Context, tris):
    """tris: device float32 [nt, 9] (or [nt, 3, 3]); nt = 0 clears the triangles."""
    t = tris.reshape(-1, 9).contiguous() if tris is not None and tris.numel() else None
    ctx._check("lt_mesh_upload", ctx.lib.lt_mesh_upload(ctx.h, _ptr(t), 0 if t is None else t.shape[0]))
    ctx._mesh = t  # the caller's buffer is only read during the call


def lt_mesh_bvh(ctx: Context, nt: int, device):
    aabb = torch.empty((2 * nt - 1, 6), dtype=torch.float32, device=device)
    child = torch.empty((max(nt - 1, 1), 2), dtype=torch.int32, device=device)
    leaf = torch.empty(nt, dtype=torch.int32, device=device)
    ctx._check("lt_mesh_bvh", ctx.lib.lt_mesh_bvh(ctx.h, _ptr(aabb), _ptr(child), _ptr(leaf)))
    return aabb, child[:nt - 1], leaf


def lt_make_slices_split(ctx: Context, pts, target: int, normal_weight: float):
    """Recursive 6-D binary split into slices of at most `target` points; returns
    (row_perm [m], slice_off [S+1]) device int32 tensors."""
    m = pts.shape[1]
    S = int(ctx.lib.lt_split_slice_count(m, int(target)))
    if S < 1:
        raise RuntimeError("lt_split_slice_count: bad arguments")
    row_perm = torch.empty(m, dtype=torch.int32, device=pts.device)
    slice_off = torch.empty(S + 1, dtype=torch.int32, device=pts.device)
    ctx._check("lt_make_slices_split", ctx.lib.lt_make_slices_split(ctx.h, _ptr(pts), m, int(target),
                                                                    float(normal_weight), _ptr(row_perm),
                                                                    _ptr(slice_off)))
    return row_perm, slice_off


def lt_bound_slices(ctx: Context, pts, row_perm, slice_off, min_rows: int, max_rows: int, normal_weight: float):
    """Slices held between min_rows and max_rows rows; returns new (row_perm [m],
    slice_off [S'+1]) device int32 tensors."""
    m = pts.shape[1]
    S = slice_off.numel() - 1
    cap = S + m // max(1, (int(max_rows) + 1) // 2) + 1
    out_perm = torch.empty(m, dtype=torch.int32, device=pts.device)
    out_off = torch.empty(cap + 1, dtype=torch.int32, device=pts.device)
    n = _i32(0)
    ctx._check("lt_bound_slices", ctx.lib.lt_bound_slices(ctx.h, _ptr(pts), m, _ptr(row_perm), _ptr(slice_off), S,
                                                          int(min_rows), int(max_rows), float(normal_weight), cap,
                                                          _ptr(out_perm), _ptr(out_off), ctypes.byref(n)))
    return out_perm, out_off[:n.value + 1].clone()


def lt_rgb_setup(ctx: Context, frame: Frame, rgb: RGB, pt_albedo, vpl_power, row_perm):
    """pt_albedo [m, 4] (image order) and vpl_power [n, 4] device float32 tensors."""
    ctx._check("lt_rgb_setup", ctx.lib.lt_rgb_setup(ctx.h, ctypes.byref(frame.struct()), _ptr(pt_albedo),
                                                    _ptr(vpl_power), _ptr(row_perm), ctypes.byref(rgb.struct())))


def lt_expand_rgb(ctx: Context, frame: Frame, smp: Samples, rgb: RGB):
    ctx._check("lt_expand_rgb", ctx.lib.lt_expand_rgb(ctx.h, ctypes.byref(frame.struct()), ctypes.byref(smp.struct()),
                                                      ctypes.byref(rgb.struct()), ctypes.byref(rgb.samples3())))


def lt_complete_rgb(ctx: Context, rgb: RGB, iters, lam_rel, seed, adm=None):
    """Completion of the stacked slices: lt_complete, or lt_complete_adm when adm =
    (iters, alpha_rel, gamma)."""
    f3, s3, uv3 = rgb.frame3(), rgb.samples3(), rgb.factors3()
    if adm is None:
        ctx._check("lt_complete", ctx.lib.lt_complete(ctx.h, ctypes.byref(f3), ctypes.byref(s3), iters, lam_rel, seed,
                                                      ctypes.byref(uv3)))
    else:
        ctx._check("lt_complete_adm", ctx.lib.lt_complete_adm(ctx.h, ctypes.byref(f3), ctypes.byref(s3), adm[0],
                                                              adm[1], adm[2], seed, ctypes.byref(uv3)))


def lt_render_rgb(ctx: Context, rgb: RGB):
    """The stacked image into rgb.img ([m][3], image order)."""
    ctx._check("lt_render", ctx.lib.lt_render(ctx.h, ctypes.byref(rgb.frame3()), ctypes.byref(rgb.samples3()),
                                              ctypes.byref(rgb.factors3()), None, _ptr(rgb.row_perm3), _ptr(rgb.img)))


def lt_render(ctx: Context, frame: Frame, smp: Samples, uv: Factors, row_perm, img, w=None):
    ctx._check("lt_render", ctx.lib.lt_render(ctx.h, ctypes.byref(frame.struct()), ctypes.byref(smp.struct()),
                                              ctypes.byref(uv.struct()), _ptr(w), _ptr(row_perm), _ptr(img)))


def params(cfg: dict, weights=None, proposal=None, mix: float = 0.8) -> lt_params:
    """lt_params of a configuration dict (rate1, tau, d_min, rate, als_iters, lam_rel,
    rank_cols: 0 or absent = one rank per frame; completion "als" (default) or "adm"
    with adm_iters, adm_alpha_rel, adm_gamma)."""
    adm = cfg.get("completion", "als") == "adm"
    return lt_params(cfg["rate1"], cfg["tau"], cfg["d_min"], cfg["rate"], cfg["als_iters"], cfg["lam_rel"],
                     _ptr(weights), _ptr(proposal), mix, int(cfg.get("rank_cols", 0)),
                     COMPLETE_ADM if adm else COMPLETE_ALS, int(cfg.get("adm_iters", 100)),
                     float(cfg.get("adm_alpha_rel", 0.3)), float(cfg.get("adm_gamma", 1.0)),
                     int(cfg.get("target_cut", 0)))


def lt_slice_ranks(ctx: Context, frame: Frame, smp: Samples, R: int, cols: int, rank=None):
    if rank is None:
        rank = torch.zeros(frame.S, dtype=torch.int32, device=frame.pts_s.device)
    ctx._check("lt_slice_ranks", ctx.lib.lt_slice_ranks(ctx.h, ctypes.byref(frame.struct()), ctypes.byref(smp.struct()),
                                                        int(R), int(cols), _ptr(rank)))
    return rank


def lt_render_frame(ctx: Context, frame: Frame, prm: lt_params, seed, smp: Samples, uv: Factors, row_perm, img):
    ctx._check("lt_render_frame", ctx.lib.lt_render_frame(ctx.h, ctypes.byref(frame.struct()), ctypes.byref(prm),
                                                          seed, ctypes.byref(smp.struct()), ctypes.byref(uv.struct()),
                                                          _ptr(row_perm), _ptr(img)))


class Graph:
    """A captured frame (lt_graph); holds every object whose memory the graph uses."""

    def __init__(self, ctx: Context, frame: Frame, prm: lt_params, smp: Samples, uv: Factors, row_perm, img,
                 keep=()):
        self.ctx = ctx
        self._keep = (frame, prm, smp, uv, row_perm, img, *keep)
        h = _p()
        ctx._check("lt_frame_graph_capture",
                   ctx.lib.lt_frame_graph_capture(ctx.h, ctypes.byref(frame.struct()), ctypes.byref(prm),
                                                  ctypes.byref(smp.struct()), ctypes.byref(uv.struct()),
                                                  _ptr(row_perm), _ptr(img), ctypes.byref(h)))
        self.h = h
        self.kernels = int(ctx.lib.lt_frame_graph_kernels(h))

    def close(self):
        if getattr(self, "h", None):
            self.ctx.lib.lt_frame_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lt_frame_graph_capture(ctx: Context, frame: Frame, prm: lt_params, smp: Samples, uv: Factors, row_perm, img,
                           keep=()) -> Graph:
    return Graph(ctx, frame, prm, smp, uv, row_perm, img, keep)


def lt_frame_graph_launch(g: Graph, seed):
    g.ctx._check("lt_frame_graph_launch", g.ctx.lib.lt_frame_graph_launch(g.h, seed))


def lt_frame_graph_kernels(g: Graph) -> int:
    return int(g.ctx.lib.lt_frame_graph_kernels(g.h))


def lt_frame_graph_destroy(g: Graph):
    g.close()


# ------------------------------------------------------------------ learned proposal
def lt_proposal_features(ctx: Context, frame: Frame, smp: Samples, feat=None, group_off=None):
    """(feat [S*C][32] float32, group_off [S+1] int32) after pass 1."""
    dev = frame.pts_s.device
    if feat is None:
        feat = torch.zeros(frame.S * frame.C, MLP_FEATURES, dtype=torch.float32, device=dev)
    if group_off is None:
        group_off = torch.zeros(frame.S + 1, dtype=torch.int32, device=dev)
    ctx._check("lt_proposal_features", ctx.lib.lt_proposal_features(ctx.h, ctypes.byref(frame.struct()),
                                                                    ctypes.byref(smp.struct()), _ptr(feat),
                                                                    _ptr(group_off)))
    return feat, group_off


def lt_proposal_forward(ctx: Context, theta, feat, n_max=None, n_dev=None, z=None):
    n_max = feat.shape[0] if n_max is None else n_max
    if z is None:
        z = torch.zeros(n_max, dtype=torch.float32, device=feat.device)
    ctx._check("lt_proposal_forward", ctx.lib.lt_proposal_forward(ctx.h, _ptr(theta), _ptr(feat), n_max, _ptr(n_dev),
                                                                  _ptr(z)))
    return z


def lt_proposal_weights(ctx: Context, frame: Frame, smp: Samples, group_off, z, mix=0.8, w=None):
    if w is None:
        w = torch.zeros(frame.S * frame.C, dtype=torch.float32, device=z.device)
    ctx._check("lt_proposal_weights", ctx.lib.lt_proposal_weights(ctx.h, ctypes.byref(frame.struct()),
                                                                  ctypes.byref(smp.struct()), _ptr(group_off),
                                                                  _ptr(z), mix, _ptr(w)))
    return w


def lt_slice_matrices(ctx: Context, frame: Frame, smp: Samples, d_min, cap: int):
    """(M [cap] float32, moff [S+1] int64): the full matrix of every slice over its coarsened columns."""
    dev = frame.pts_s.device
    M = torch.zeros(max(int(cap), 1), dtype=torch.float32, device=dev)
    moff = torch.zeros(frame.S + 1, dtype=torch.int64, device=dev)
    ctx._check("lt_slice_matrices", ctx.lib.lt_slice_matrices(ctx.h, ctypes.byref(frame.struct()),
                                                              ctypes.byref(smp.struct()), d_min, _ptr(M), int(cap),
                                                              _ptr(moff)))
    return M, moff


def lt_leverage_targets(ctx: Context, frame: Frame, smp: Samples, M, moff, group_off, r, iters, seed, target=None):
    if target is None:
        target = torch.zeros(frame.S * frame.C, dtype=torch.float32, device=M.device)
    ctx._check("lt_leverage_targets", ctx.lib.lt_leverage_targets(ctx.h, ctypes.byref(frame.struct()),
                                                                  ctypes.byref(smp.struct()), _ptr(M), _ptr(moff),
                                                                  _ptr(group_off), r, iters, seed, _ptr(target)))
    return target


def lt_proposal_init(ctx: Context, seed, device=None):
    device = torch.device("cuda", ctx.device) if device is None else device
    theta = torch.zeros(MLP_PARAMS, dtype=torch.float32, device=device)
    ctx._check("lt_proposal_init", ctx.lib.lt_proposal_init(ctx.h, seed, _ptr(theta)))
    return theta


def lt_proposal_grad(ctx: Context, theta, feat, target, group_off, ngroups, n, grad=None, loss=None):
    if grad is None:
        grad = torch.zeros(MLP_PARAMS, dtype=torch.float32, device=theta.device)
    if loss is None:
        loss = torch.zeros(1, dtype=torch.float32, device=theta.device)
    ctx._check("lt_proposal_grad", ctx.lib.lt_proposal_grad(ctx.h, _ptr(theta), _ptr(feat), _ptr(target),
                                                            _ptr(group_off), int(ngroups), int(n), _ptr(grad),
                                                            _ptr(loss)))
    return grad, loss


def lt_proposal_adam(ctx: Context, theta, m, v, grad, step, lr):
    ctx._check("lt_proposal_adam", ctx.lib.lt_proposal_adam(ctx.h, _ptr(theta), _ptr(m), _ptr(v), _ptr(grad),
                                                            int(step), lr))


# ------------------------------------------------------------------ launch tuning
def lt_get_tuning(ctx: Context) -> dict:
    t = lt_tuning()
    ctx._check("lt_get_tuning", ctx.lib.lt_get_tuning(ctx.h, ctypes.byref(t)))
    return {name: int(getattr(t, name)) for name, _ in lt_tuning._fields_}


def lt_set_tuning(ctx: Context, **values):
    """Set some tuning values (names of lt_tuning); the others keep their current value."""
    cur = lt_get_tuning(ctx)
    unknown = set(values) - set(cur)
    if unknown:
        raise KeyError(f"unknown tuning values: {sorted(unknown)}")
    cur.update({k: int(v) for k, v in values.items()})
    t = lt_tuning(*[cur[name] for name, _ in lt_tuning._fields_])
    ctx._check("lt_set_tuning", ctx.lib.lt_set_tuning(ctx.h, ctypes.byref(t)))
