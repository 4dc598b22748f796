"""Multi-rank path on CPU (gloo, world size 2): channel ownership covers every
channel exactly once, per-rank results gathered equal the single-process
result, and the timing reduction takes the slowest rank. The per-rank compute
here is the FP64 oracle; on GPUs each rank runs the CUDA path on its own
device with no collective."""
import os
import socket

import numpy as np
import pytest

from paper_1702_00844_gb300.shard import channel_range, job_throughput


def test_channel_ranges_partition():
    for n in (0, 1, 7, 480):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                lo, hi = channel_range(n, world, r)
                assert 0 <= lo <= hi <= n
                seen.extend(range(lo, hi))
            assert seen == list(range(n))
    with pytest.raises(ValueError):
        channel_range(4, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist

    import oracle
    import synth
    from paper_1702_00844_gb300.shard import channel_range, max_over_ranks

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    d = synth.tiny()
    lo, hi = channel_range(d["C"], world, rank)
    vis = oracle.correlate(d["x"][lo:hi])
    gathered = [None] * world
    dist.all_gather_object(gathered, (lo, hi, vis))
    t_slowest = max_over_ranks(0.5 + rank)   # rank 1 pretends to be slower
    if rank == 0:
        full = np.concatenate([g[2] for g in sorted(gathered, key=lambda g: g[0])])
        np.save(os.path.join(out_dir, "gathered.npy"), full)
        with open(os.path.join(out_dir, "tmax.txt"), "w") as f:
            f.write(repr(t_slowest))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_gloo(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    import oracle
    import synth
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    got = np.load(tmp_path / "gathered.npy")
    ref = oracle.correlate(synth.tiny()["x"])
    np.testing.assert_array_equal(got, ref)
    tmax = float(open(tmp_path / "tmax.txt").read())
    assert tmax == 1.5
    assert job_throughput([3, 5], tmax) == pytest.approx(8 / 1.5)
