"""The tensor-core form of the ALS half-step (lt_complete with als_form 1): the Gram
matrices and right-hand sides that the dense masked products on the tensor cores
produce, against float64 sums over the same samples and factors, and the two forms
of the completion against each other.

For a line with observed entries (j, A_j) and factor rows x_j (Sec. 5):
G = sum_j x_j x_j^T and b = sum_j A_j x_j.  Tolerance: every Gram element within
1e-5 of sum_j |x_j|^2 (a bound on |G|), every b element within 1e-5 of
sum_j |A_j| max|x_j| -- float32 accumulation of 22-bit products over a few hundred
terms stays two orders of magnitude inside it.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from ltinputs import get_config, make_scene

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _renderer(workload, **over):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2202_12567_gb300.renderer import Renderer
    cfg = get_config(workload, **over)
    R = Renderer(make_scene(cfg), cfg, device=0).setup()
    R.render()
    return cfg, R


def _check_slice(G, b, lines, idx_line, idx_src, vals, X, r, what):
    """float64 Gram / b of `lines` lines from entries (idx_line, idx_src, vals) and
    source rows X, against the device's G [lines][r(r+1)/2] and b [lines][r]."""
    nt = r * (r + 1) // 2
    ia, ic = np.tril_indices(r)
    order = np.lexsort((ic, ia))
    ia, ic = ia[order], ic[order]  # packed order: (a, c), c <= a, at a (a + 1) / 2 + c
    Xe = X[idx_src]
    W = Xe[:, ia] * Xe[:, ic]
    G64 = np.zeros((lines, nt))
    np.add.at(G64, idx_line, W)
    b64 = np.zeros((lines, r))
    np.add.at(b64, idx_line, vals[:, None] * Xe)
    bound_g = np.zeros(lines)
    np.add.at(bound_g, idx_line, np.sum(Xe * Xe, axis=1))
    bound_b = np.zeros(lines)
    np.add.at(bound_b, idx_line, np.abs(vals) * np.max(np.abs(Xe), axis=1))
    eg = np.max(np.abs(G - G64), axis=1)
    eb = np.max(np.abs(b - b64), axis=1)
    assert np.all(eg <= TOL * bound_g + 1e-30), (what, float(np.max(eg / np.maximum(bound_g, 1e-30))))
    assert np.all(eb <= TOL * bound_b + 1e-30), (what, float(np.max(eb / np.maximum(bound_b, 1e-30))))
    return float(np.max(eg / np.maximum(bound_g, 1e-30)))


@pytest.mark.parametrize("workload,over", [
    ("room64_vpl1k_2box", dict(max_cut=256)),
    ("room64_vpl1k_2box", dict(max_cut=256, rank=16)),
    ("room64_vpl1k_2box", dict(max_cut=256, rank=5)),
    ("room256_vpl16k_2box", {}),
])
def test_tc_gram_matches_float64(workload, over):
    """Both sides (rows of U from V, columns of V from U) on every slice of the tiny
    workload and on three slices of the bench workload (several 128-line tiles, a
    ragged last tile and K blocks, ranks 5, 8 and 16)."""
    from paper_2202_12567_gb300 import lt
    cfg, R = _renderer(workload, **over)
    r, S, C = cfg["rank"], R.frame.S, R.frame.C
    U = R.uv.U.cpu().numpy().reshape(-1, r).astype(np.float64)
    V = R.uv.V.cpu().numpy().reshape(S, C, r).astype(np.float64)
    g0 = lt.lt_als_gram(R.ctx, R.frame, R.smp, R.uv, 0).cpu().numpy().astype(np.float64)
    g1 = lt.lt_als_gram(R.ctx, R.frame, R.smp, R.uv, 1).cpu().numpy().astype(np.float64)
    lt.lt_sync(R.ctx)
    nt = r * (r + 1) // 2
    off = R.slice_off.cpu().numpy()
    sizes = np.diff(off)
    slices = range(S) if S <= 16 else sorted({0, S // 2, int(np.argmax(sizes))})
    worst = 0.0
    for s in slices:
        rows, cols, vals, col_node, _ = R.smp.slice(s)
        vals = vals.astype(np.float64)
        m_s, n_s = int(sizes[s]), col_node.size
        a = int(off[s])
        worst = max(worst, _check_slice(g0[a:a + m_s, :nt], g0[a:a + m_s, nt:], m_s, rows, cols, vals, V[s, :n_s], r,
                                        f"slice {s} rows"))
        q = g1[s * C:s * C + n_s]
        worst = max(worst, _check_slice(q[:, :nt], q[:, nt:], n_s, cols, rows, vals, U[a:a + m_s], r,
                                        f"slice {s} columns"))
    print(f"{workload} r={r}: largest Gram error / bound {worst:.2e}")


def test_tc_and_simt_forms_agree_on_the_bench_frame():
    """The same samples completed by both forms: images within 1e-3, completed
    factors' images within 1e-3 of each other per slice."""
    from paper_2202_12567_gb300 import lt
    cfg, R = _renderer("room256_vpl16k_2box")
    seed = cfg["frame_seed"]
    imgs = {}
    for form in (0, 1):
        lt.lt_set_tuning(R.ctx, als_form=form)
        R.complete(seed)
        R.render_image()
        lt.lt_sync(R.ctx)
        imgs[form] = R.img.cpu().numpy().astype(np.float64)
    rel = np.linalg.norm(imgs[1] - imgs[0]) / np.linalg.norm(imgs[0])
    print(f"tensor-core vs SIMT image: rel {rel:.2e}")
    assert rel <= 1e-3
