"""Beam sharding (the multi-GPU partition) on CPU: the partition's invariants,
and a world_size-2 gloo run whose ranks clean their shares with the oracle and
reproduce the single-process result exactly."""
import os
import socket

import numpy as np
import pytest


def test_partition_invariants():
    from paper_2001_03389_gb300.shard import partition_beams

    rng = np.random.default_rng(0)
    for world in (1, 2, 3, 8):
        sizes = rng.integers(1000, 100000, 57).tolist()
        shares = partition_beams(sizes, world)
        flat = sorted(i for s in shares for i in s)
        assert flat == list(range(57))
        loads = [sum(sizes[i] for i in s) for s in shares]
        assert max(loads) - min(loads) <= max(sizes)
        assert shares == partition_beams(sizes, world)  # deterministic
    assert partition_beams([5, 5], 4) == [[0], [1], [], []]
    with pytest.raises(ValueError):
        partition_beams([1], 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import oracle
        from paper_2001_03389_gb300 import shard, synth

        shapes = [(48, 300), (96, 120), (24, 999), (48, 257), (64, 64), (96, 333), (32, 500)]
        beams = [synth.ragged_beam(j, C, T) for j, (C, T) in enumerate(shapes)]
        td = dict(k=3.0, iterations=2, replace="median")
        fd = dict(k=3.0, iterations=2, replace="median", bin=16)
        res = shard.clean_sharded(beams, lambda b: oracle.clean(b[None], "bct", tdsc=td, fdsc=fd))
        if rank == 0:
            ok = True
            for b, (out, fl) in zip(beams, res):
                want, wf = oracle.clean(b[None], "bct", tdsc=td, fdsc=fd)
                ok &= bool(np.array_equal(out, want) and np.array_equal(fl, wf))
            with open(os.path.join(out_dir, "result"), "w") as fh:
                fh.write("ok" if ok else "mismatch")
    finally:
        dist.destroy_process_group()


def test_gloo_two_ranks_reproduce_single_process(tmp_path):
    import torch.multiprocessing as mp

    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn", join=True)
    assert (tmp_path / "result").read_text() == "ok"
