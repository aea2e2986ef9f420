"""Failure detection through the C ABI, made on the host or with undersized inputs (no
GPU fault is provoked): every device loop and capacity bound latches a status that
lt_sync returns, scratch growth beyond a caller's budget fails with LT_ENOMEM before
allocating, non-finite inputs latch LT_ENUMERIC, and the degenerate cases of the
method (an all-zero pass-2 pdf, a rank above the samples of a row) give defined
results.  After each error the context keeps working."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from ltinputs import get_config, make_scene
from oracle import pass2 as o_pass2

pytestmark = pytest.mark.gpu

LT_ENOMEM, LT_ELIMIT, LT_ENUMERIC = 2, 4, 5


@pytest.fixture(scope="module")
def tiny():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    cfg = get_config("room64_vpl1k_2box", max_cut=256)
    return cfg, make_scene(cfg)


def _renderer(cfg, sc):
    from paper_2202_12567_gb300.renderer import Renderer
    return Renderer(sc, cfg, device=0).setup()


def test_undersized_capacity_latches_elimit(tiny):
    """Sample capacities far below the pass-1 entries: the kernels keep within them,
    latch LT_ELIMIT, and the next lt_sync reports it; with the capacities restored the
    same context renders a finite frame."""
    from paper_2202_12567_gb300 import lt
    cfg, sc = tiny
    R = _renderer(cfg, sc)
    full = R.smp.off.clone()
    small = torch.arange(0, 8 * (R.frame.S + 1), 8, dtype=torch.int64, device=full.device)
    R.smp.off.copy_(small)
    with pytest.raises(lt.LtError) as e:
        R.pass1(cfg["frame_seed"])
        lt.lt_sync(R.ctx)
    assert e.value.code == LT_ELIMIT
    lt.lt_sync(R.ctx)  # the status was cleared by the failing sync
    R.smp.off.copy_(full)
    img = R.render().cpu().numpy()
    assert np.all(np.isfinite(img)) and img.max() > 0


def test_scratch_budget_gives_enomem(tiny):
    """With a scratch cap at what the context already holds, a call that needs more
    returns LT_ENOMEM at once (nothing is allocated); lifting the cap lets it run."""
    from paper_2202_12567_gb300 import lt
    cfg, sc = tiny
    R = _renderer(cfg, sc)
    lt.lt_set_scratch_limit(R.ctx, 1)
    with pytest.raises(lt.LtError) as e:
        R.pass1(cfg["frame_seed"])
    assert e.value.code == LT_ENOMEM
    assert "scratch limit" in str(e.value)
    lt.lt_set_scratch_limit(R.ctx, 0)
    img = R.render().cpu().numpy()
    assert np.all(np.isfinite(img)) and img.max() > 0
    with pytest.raises(lt.LtError):
        lt.lt_set_scratch_limit(R.ctx, -1)


def test_non_finite_input_latches_enumeric(tiny):
    """A slice whose shading points carry a NaN albedo: its entries are not finite,
    the evaluation latches LT_ENUMERIC, and the pixels of the other slices stay
    finite (slices are completed independently)."""
    from paper_2202_12567_gb300 import lt
    cfg, sc = tiny
    R = _renderer(cfg, sc)
    off = R.slice_off.cpu().numpy()
    a, b = int(off[0]), int(off[1])
    R.pts_s[0, a:b, 3] = float("nan")
    with pytest.raises(lt.LtError) as e:
        R.render()
    assert e.value.code == LT_ENUMERIC
    img = R.img.cpu().numpy()
    perm = R.row_perm.cpu().numpy()
    others = perm[b:]
    assert np.all(np.isfinite(img[others])) and img[others].max() > 0


def test_all_zero_pdf_draws_uniformly(tiny):
    """All pass-2 weights zero (no column has any importance): every column gets the
    same integer weight, as in the oracle, the draws equal the oracle's and the
    slice reaches its target count."""
    from paper_2202_12567_gb300 import lt
    cfg, sc = tiny
    R = _renderer(cfg, sc)
    seed = cfg["frame_seed"]
    R.pass1(seed)
    w = torch.zeros(R.frame.S * R.frame.C, dtype=torch.float32, device=R.smp.g.device)
    lt.lt_sample_pass2(R.ctx, R.frame, R.smp, cfg["rate"], seed, w)
    lt.lt_sync(R.ctx)
    off = R.slice_off.cpu().numpy()
    for s in range(R.frame.S):
        rows, cols, _, col_node, _ = R.smp.slice(s)
        n1 = int(R.smp.n1[s].item())
        m_s, n_s = int(off[s + 1] - off[s]), col_node.size
        r2, c2, _, cap = o_pass2.draw_pass2(seed, s, m_s, np.zeros(n_s), rows[:n1] * n_s + cols[:n1], cfg["rate"])
        assert np.array_equal(rows[n1:], r2) and np.array_equal(cols[n1:], c2), s
        assert cap or rows.size == max(n1, o_pass2.target_count(cfg["rate"], m_s, n_s))


def test_rank_above_the_samples_of_a_row_is_finite():
    """Rank 32 at 2% sampling: most rows are observed in fewer entries than the rank;
    the ridge keeps every solve defined and the frame is finite."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    cfg = get_config("room64_vpl1k_2box", max_cut=256, rate=0.02, rank=32)
    R = _renderer(cfg, make_scene(cfg))
    img = R.render().cpu().numpy()
    assert np.all(np.isfinite(img)) and img.max() > 0
