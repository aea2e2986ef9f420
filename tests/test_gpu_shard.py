"""One frame split by slices over two processes through the library (two ranks that
share the one GPU here; their kernels never wait on one another).  Every rank sets
up the frame, takes its longest-processing-time share of the slices, renders them
with their indices in the whole frame (lt_frame.slice_id), and the pixel blocks are
gathered over gloo on rank 0: the image equals the single-process frame bit for
bit, for the calls one by one and for the captured graph."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

pytestmark = pytest.mark.gpu


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, workload, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        from ltinputs import get_config, make_scene
        from paper_2202_12567_gb300 import lt, shard
        from paper_2202_12567_gb300.renderer import Renderer
        cfg = get_config(workload)
        sc = make_scene(cfg)
        R = Renderer(sc, cfg, device=0).setup()
        parts = shard.lpt_partition(shard.slice_costs(R.slice_off.cpu().numpy(), C=R.frame.C), world)
        sub = shard.shard_renderer(R, parts[rank])
        seeds = (cfg["frame_seed"], cfg["frame_seed"] + 11)
        got = []
        for k, seed in enumerate(seeds):
            if sub is not None:
                if k == 0:
                    sub.render(seed)
                else:
                    sub.capture()
                    sub.render_graph(seed)
                pixels, values = sub.pixels.cpu(), sub.img[sub.pixels].cpu()
            else:
                pixels, values = torch.zeros(0, dtype=torch.int64), torch.zeros(0)
            got.append(shard.gather_image(pixels, values, sc.m))
        if rank == 0:
            ref = [R.render(seeds[0]).cpu().clone()]
            R.capture()
            ref.append(R.render_graph(seeds[1]).cpu().clone())
            out.put(dict(equal=[bool(torch.equal(g, r)) for g, r in zip(got, ref)],
                         parts=[len(p) for p in parts], S=int(R.frame.S),
                         maxdiff=[float((g - r).abs().max()) for g, r in zip(got, ref)]))
        lt.lt_sync(R.ctx)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("workload", ["room64_vpl1k_2box", "room256_vpl16k_2box"])
def test_sharded_frame_equals_the_whole_frame(workload):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, workload, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = out.get(timeout=900)
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    assert sum(res["parts"]) == res["S"] and min(res["parts"]) > 0
    assert res["equal"] == [True, True], res
