"""The multi-process path on CPU (gloo, world size 2): a frame sharded by slices.

Each rank renders the slices the longest-processing-time split gives it (here with
the oracle, which stands in for one GPU per rank), the pixel blocks are gathered on
rank 0 and must equal the single-process frame exactly; the timing reduction is
the maximum over ranks."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2202_12567_gb300 import shard  # noqa: E402


def test_lpt_partition_balances_and_covers():
    costs = np.array([9, 1, 7, 3, 3, 8, 2, 5])
    parts = shard.lpt_partition(costs, 3)
    flat = sorted(s for p in parts for s in p)
    assert flat == list(range(8))
    loads = [int(costs[p].sum()) for p in parts]
    assert max(loads) - min(loads) <= costs.max()
    assert shard.lpt_partition(costs, 1) == [list(range(8))]
    # more ranks than slices: the extra ranks get nothing
    parts = shard.lpt_partition(np.array([4, 2]), 4)
    assert sorted(len(p) for p in parts) == [0, 0, 1, 1]


def test_rows_of_slices():
    off = np.array([0, 3, 3, 7, 10])
    assert shard.rows_of(off, [0, 2]).tolist() == [0, 1, 2, 3, 4, 5, 6]
    assert shard.rows_of(off, [1]).size == 0 and shard.rows_of(off, []).size == 0
    assert shard.slice_costs(off, ncol=[2, 5, 1, 0]).tolist() == [6, 0, 4, 3]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out, extra=None):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from ltinputs import get_config, make_scene
        from oracle import pipeline
        cfg = get_config("room64_vpl1k_2box", max_cut=64, n_slices=8, **(extra or {}))
        sc = make_scene(cfg)
        st = pipeline.setup(sc, cfg)
        parts = shard.lpt_partition(shard.slice_costs(st["slice_off"], C=len(st["cut"])), world)
        mine = parts[rank]
        img_part, results = pipeline.render_frame(sc, cfg, st, slices=mine)
        rows = shard.rows_of(st["slice_off"], mine)
        pix = torch.from_numpy(st["row_perm"][rows].astype(np.int64))
        vals = torch.from_numpy(img_part[pix.numpy()])
        img = shard.gather_image(pix, vals, sc.m)
        t = shard.max_over_ranks(10.0 + rank)
        if rank == 0:
            np.save(out, img.numpy())
            with open(out + ".t", "w") as f:
                f.write(str(t))
    finally:
        dist.destroy_process_group()


@pytest.mark.slow
def test_two_ranks_render_the_single_process_frame(tmp_path):
    from ltinputs import get_config, make_scene
    from oracle import pipeline
    out = str(tmp_path / "img.npy")
    mp.start_processes(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    cfg = get_config("room64_vpl1k_2box", max_cut=64, n_slices=8)
    sc = make_scene(cfg)
    want, _ = pipeline.render_frame(sc, cfg)
    got = np.load(out)
    assert np.array_equal(got, want)
    assert float(open(out + ".t").read()) == 11.0


@pytest.mark.slow
def test_two_ranks_with_bounded_slices(tmp_path):
    """The same with slices held between 450 and 900 rows (8 k-means slices become 6:
    small ones merged, none above the bound), so the split runs over the bounded
    slice count."""
    from ltinputs import get_config, make_scene
    from oracle import pipeline
    extra = dict(slice_bounds=(450, 900))
    out = str(tmp_path / "img.npy")
    mp.start_processes(_rank_main, args=(2, _free_port(), out, extra), nprocs=2, join=True, start_method="spawn")
    cfg = get_config("room64_vpl1k_2box", max_cut=64, n_slices=8, **extra)
    sc = make_scene(cfg)
    st = pipeline.setup(sc, cfg)
    assert len(st["slice_off"]) - 1 == 6
    want, _ = pipeline.render_frame(sc, cfg, st)
    assert np.array_equal(np.load(out), want)


def _rank_main_rgb(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from ltinputs import get_config, make_scene
        from oracle import pipeline, rgb
        cfg = get_config("room64_vpl1k_2box", width=32, height=32, n_vpl=256, max_cut=64, n_slices=6, rgb=True)
        sc = make_scene(cfg)
        st = pipeline.setup(sc, cfg)
        mine = shard.lpt_partition(shard.slice_costs(st["slice_off"], C=len(st["cut"])), world)[rank]
        img_part, _ = rgb.render_frame(sc, cfg, st, slices=mine)
        rows = shard.rows_of(st["slice_off"], mine)
        pix = torch.from_numpy(st["row_perm"][rows].astype(np.int64))
        vals = torch.from_numpy(img_part[pix.numpy()])
        img = shard.gather_image(pix, vals, sc.m)
        if rank == 0:
            np.save(out, img.numpy())
    finally:
        dist.destroy_process_group()


@pytest.mark.slow
def test_two_ranks_gather_a_colour_frame(tmp_path):
    """Colour pixel blocks [k, 3] gathered over two gloo ranks give the whole image."""
    from ltinputs import get_config, make_scene
    from oracle import pipeline, rgb
    out = str(tmp_path / "rgb.npy")
    mp.start_processes(_rank_main_rgb, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    cfg = get_config("room64_vpl1k_2box", width=32, height=32, n_vpl=256, max_cut=64, n_slices=6, rgb=True)
    sc = make_scene(cfg)
    want, _ = rgb.render_frame(sc, cfg, pipeline.setup(sc, cfg))
    got = np.load(out)
    assert got.shape == (sc.m, 3) and np.array_equal(got, want)
