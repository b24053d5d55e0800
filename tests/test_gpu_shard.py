"""Beam sharding with the library on the GPU: whole beams partitioned across
ranks by bytes, each rank cleaning its share with rfim_clean, results gathered
host-side.  The sharded result must equal one unsharded rfim_clean_batch of
all beams bit for bit.  The ranks' kernels are independent (no rank waits on
another's device work); with one GPU per box, both ranks of the world-size-2
run share cuda:0."""
import os
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SHAPES = [(384, 1000), (768, 2500), (1536, 1333), (4096, 1200), (384, 3001), (768, 1021), (1536, 777)]
TD = dict(k=3.0, iterations=2, replace="median")
FD = dict(k=3.0, iterations=2, replace="median", bin=32)


def _clean_fn(ctx, rfim):
    import torch

    def fn(x):
        xin = torch.from_numpy(x).to("cuda:0")[None]
        C, T = x.shape
        out = torch.empty_like(xin)
        mask = torch.zeros(rfim.mask_words(C, T), dtype=torch.int32, device="cuda:0")
        ctx.clean(ctx.block(xin, out, mask, "bct", "bits"), rfim.make_cut(**TD), rfim.make_cut(**FD))
        torch.cuda.synchronize()
        return out.cpu().numpy()[0], mask.cpu().numpy()

    return fn


def _unsharded(beams):
    import torch

    from paper_2001_03389_gb300 import rfim

    ctx = rfim.Context(0)
    xs = [torch.from_numpy(b).to("cuda:0") for b in beams]
    outs = [torch.empty_like(x) for x in xs]
    masks = [torch.zeros(rfim.mask_words(*x.shape), dtype=torch.int32, device="cuda:0") for x in xs]
    blks = [rfim.Context.block(x[None], o[None], m, "bct", "bits") for x, o, m in zip(xs, outs, masks)]
    ctx.clean_batch(blks, rfim.make_cut(**TD), rfim.make_cut(**FD))
    torch.cuda.synchronize()
    res = [(o.cpu().numpy(), m.cpu().numpy()) for o, m in zip(outs, masks)]
    ctx.close()
    return res


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run(rank, world, port, out_dir):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2001_03389_gb300 import build

        build.build()
        from paper_2001_03389_gb300 import rfim, shard, synth

        beams = [synth.ragged_beam(j, C, T) for j, (C, T) in enumerate(SHAPES)]
        ctx = rfim.Context(0)
        res = shard.clean_sharded(beams, _clean_fn(ctx, rfim))
        ctx.close()
        if rank == 0:
            want = _unsharded(beams)
            ok = all(np.array_equal(o, wo) and np.array_equal(m, wm) for (o, m), (wo, wm) in zip(res, want))
            with open(os.path.join(out_dir, "result"), "w") as fh:
                fh.write("ok" if ok else "mismatch")
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [1, 2])
def test_sharded_library_equals_unsharded(tmp_path, world):
    import torch.multiprocessing as mp

    port = _free_port()
    mp.start_processes(_run, args=(world, port, str(tmp_path)), nprocs=world, start_method="spawn", join=True)
    assert (tmp_path / "result").read_text() == "ok"
