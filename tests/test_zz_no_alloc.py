"""The allocation-free entry evaluation (lt_eval_entries_noalloc) through the C ABI.

It serves hosts that own the device-memory budget and cannot let the library call
cudaMalloc.  Its output must equal that of lt_eval_entries on the same sampled
entries, on two calls in a row (the second call reuses the fixed prefix array left
by the first).  The file is named to be collected last.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from ltinputs import get_config, make_scene

pytestmark = pytest.mark.gpu

ENTRY_RTOL = 1e-5


def _pass2_values(R, lt):
    out = []
    for s in range(R.frame.S):
        o = int(R.smp.off_host[s])
        n1, c = int(R.smp.n1[s].item()), int(R.smp.cnt[s].item())
        out.append(R.smp.val[o + n1:o + c].clone())
    return torch.cat(out).cpu().numpy()


def _clear_pass2_values(R):
    for s in range(R.frame.S):
        o = int(R.smp.off_host[s])
        n1, c = int(R.smp.n1[s].item()), int(R.smp.cnt[s].item())
        R.smp.val[o + n1:o + c] = -1.0


def test_noalloc_eval_matches_eval_entries_twice():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2202_12567_gb300 import lt
    from paper_2202_12567_gb300.renderer import Renderer

    cfg = get_config("room64_vpl1k_2box", max_cut=256, rate=0.2)
    sc = make_scene(cfg)
    R = Renderer(sc, cfg, device=0).setup()
    seed = cfg["frame_seed"]
    R.pass1(seed)
    R.pass2(seed)
    lt.lt_eval_entries(R.ctx, R.frame, R.smp, cfg["d_min"])
    lt.lt_sync(R.ctx)
    ref = _pass2_values(R, lt)
    assert ref.size > 1000 and np.all(ref >= 0)
    for call in range(2):
        _clear_pass2_values(R)
        lt.lt_eval_entries_noalloc(R.ctx, R.frame, R.smp, cfg["d_min"])
        lt.lt_sync(R.ctx)
        got = _pass2_values(R, lt)
        assert got.shape == ref.shape
        assert np.all(np.abs(got - ref) <= ENTRY_RTOL * np.abs(ref) + 1e-12), f"call {call}"


@pytest.fixture(scope="module")
def one_pixel_slices():
    """The tiny scene's generator at 256x128 pixels cut into 4096 slices of 8 pixels
    (the recursive split): the most slices the allocation-free call accepts; no
    coarsening (tau = 0), so pass 1 leaves room for pass-2 draws at 50% sampling."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2202_12567_gb300.renderer import Renderer
    cfg = get_config("room64_vpl1k_2box", width=256, height=128, max_cut=64, rate=0.5, slicing="split6d",
                     slice_size=8, tau=0.0)
    sc = make_scene(cfg)
    R = Renderer(sc, cfg, device=0).setup()
    assert R.frame.S == 4096
    return cfg, R


def test_noalloc_eval_at_the_slice_limit(one_pixel_slices):
    """4096 slices: the per-slice prefix takes several scan chunks and more than the
    default 48 KB of shared memory, and the count is exactly the limit."""
    from paper_2202_12567_gb300 import lt
    cfg, R = one_pixel_slices
    seed = cfg["frame_seed"]
    R.pass1(seed)
    R.pass2(seed)
    lt.lt_eval_entries(R.ctx, R.frame, R.smp, cfg["d_min"])
    lt.lt_sync(R.ctx)
    ref = _pass2_values(R, lt)
    assert ref.size > 4096
    for call in range(2):
        _clear_pass2_values(R)
        lt.lt_eval_entries_noalloc(R.ctx, R.frame, R.smp, cfg["d_min"])
        lt.lt_sync(R.ctx)
        got = _pass2_values(R, lt)
        assert np.all(np.abs(got - ref) <= ENTRY_RTOL * np.abs(ref) + 1e-12), f"call {call}"


def test_noalloc_refuses_more_slices_without_launching(one_pixel_slices):
    """A frame of 4097 slices is refused with LT_EINVAL before anything is launched."""
    import ctypes
    from paper_2202_12567_gb300 import lt
    cfg, R = one_pixel_slices
    f = lt.lt_frame.from_buffer_copy(R.frame.struct())
    f.S = 4097
    before = lt.lt_launch_count(R.ctx)
    code = R.ctx.lib.lt_eval_entries_noalloc(R.ctx.h, ctypes.byref(f), cfg["d_min"], ctypes.byref(R.smp.struct()))
    assert code == 1  # LT_EINVAL
    assert "4096" in R.ctx.lib.lt_last_error(R.ctx.h).decode()
    assert lt.lt_launch_count(R.ctx) == before


_CAPTURE_CHILD = r"""
import sys, ctypes
sys.path.insert(0, sys.argv[1])
import torch
from ltinputs import get_config, make_scene
from paper_2202_12567_gb300 import lt
from paper_2202_12567_gb300.renderer import Renderer
cfg = get_config("room64_vpl1k_2box", max_cut=64)
sc = make_scene(cfg)
stream = torch.cuda.Stream()
with torch.cuda.stream(stream):
    ctx = lt.Context(0, stream=stream)
    R = Renderer(sc, cfg, device=0, ctx=ctx).setup()
    R.pass1(cfg["frame_seed"])
    R.pass2(cfg["frame_seed"])
    lt.lt_sync(ctx)
    g = torch.cuda.CUDAGraph()
    g.capture_begin()
    code = ctx.lib.lt_eval_entries_noalloc(ctx.h, ctypes.byref(R.frame.struct()), cfg["d_min"],
                                           ctypes.byref(R.smp.struct()))
    msg = ctx.lib.lt_last_error(ctx.h).decode()
    g.capture_end()
print("CODE", code, msg)
"""


def test_noalloc_first_call_inside_a_capture_is_refused():
    """In a fresh process, a first call made while the stream is captured cannot look
    the array up and returns LT_EINVAL, asking for one call before capturing."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "-c", _CAPTURE_CHILD, root], capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = [x for x in out.stdout.splitlines() if x.startswith("CODE")][-1]
    assert line.split()[1] == "1", line
    assert "before capturing" in line
