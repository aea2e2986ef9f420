"""The frame as one C call and as a captured CUDA graph (the batched form).

The graph replays the same kernels with sizes recorded by a warm run and the seed
read from device memory, so for every seed its image must equal the one of the
plain sequence of launches."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from ltinputs import get_config, make_scene

pytestmark = pytest.mark.gpu


def _renderer(name="room64_vpl1k_2box", **kw):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2202_12567_gb300.renderer import Renderer
    cfg = get_config(name, **kw)
    return Renderer(make_scene(cfg), cfg, device=0).setup()


def test_render_frame_equals_staged_calls():
    R = _renderer(max_cut=256)
    a = R.render(seed=7).clone()
    b = R.render_frame(seed=7).clone()
    assert torch.equal(a, b)


@pytest.mark.parametrize("name,kw", [("room64_vpl1k_2box", dict(max_cut=256)),
                                     ("room256_vpl16k_200box", dict(max_cut=1024, n_slices=32))])
def test_graph_replay_equals_plain_frame(name, kw):
    from paper_2202_12567_gb300 import lt
    R = _renderer(name, **kw)
    plain = {}
    for seed in (7, 11, 12345):
        plain[seed] = R.render_frame(seed=seed).clone()
    assert not torch.equal(plain[7], plain[11])
    g = R.capture()
    assert g.kernels > 10
    n0 = lt.lt_launch_count(R.ctx)
    for seed in (11, 7, 12345, 7):
        img = R.render_graph(seed=seed)
        assert torch.equal(img, plain[seed]), f"seed {seed}"
    assert lt.lt_launch_count(R.ctx) - n0 == 4 * (g.kernels + 1)
    # the factors and samples written by the replay are those of the plain frame too
    R.render_frame(seed=11)
    U_plain = R.uv.U.clone()
    R.render_graph(seed=11)
    assert torch.equal(R.uv.U, U_plain)


def test_graph_guards_the_scene_and_context():
    from paper_2202_12567_gb300 import lt
    R = _renderer(max_cut=256)
    g = R.capture()
    with pytest.raises(lt.LtError):
        lt.lt_scene_upload(R.ctx, R.boxes)
    g.close()
    R.graph = None
    lt.lt_scene_upload(R.ctx, R.boxes)  # allowed again once the graph is gone
    img = R.render_frame(seed=7).clone()
    assert torch.isfinite(img).all() and float(img.sum()) > 0
