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


def _bench_worker(rank, world, port, out_dir):
    import json

    import torch.distributed as dist

    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    res = {}
    for split in ("none", "channels"):
        lo, hi = bench.rank_channels(split, 480, world, rank)
        ops = bench.ops_of(256, 1024, hi - lo)
        # rank 1 pretends to be slower: 12 ms against 10 ms for the 4 steps
        value, ms_step, ops_job = bench.job_throughput(ops, 10.0 + 2.0 * rank, 4)
        res[split] = {"lo": lo, "hi": hi, "value": value, "ms_step": ms_step, "ops_job": ops_job}
    with open(os.path.join(out_dir, f"bench{rank}.json"), "w") as f:
        json.dump(res, f)
    dist.barrier()
    dist.destroy_process_group()


def test_bench_rank_logic_two_ranks_gloo(tmp_path):
    """bench.py's rank logic on two gloo ranks: with --split channels the
    ranks own 240 channels each and the job's ops are those of the one
    480-channel workload; without a split every rank runs all 480 and the
    job counts both. Either way the time is the slowest rank's."""
    pytest.importorskip("torch")
    import json

    import torch.multiprocessing as mp

    import bench
    port = _free_port()
    mp.start_processes(_bench_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    r = [json.load(open(tmp_path / f"bench{k}.json")) for k in range(2)]
    full = bench.ops_of(256, 1024, 480)
    assert (r[0]["channels"]["lo"], r[0]["channels"]["hi"]) == (0, 240)
    assert (r[1]["channels"]["lo"], r[1]["channels"]["hi"]) == (240, 480)
    assert (r[1]["none"]["lo"], r[1]["none"]["hi"]) == (0, 480)
    for k in range(2):
        assert r[k]["channels"]["ops_job"] == pytest.approx(full)
        assert r[k]["none"]["ops_job"] == pytest.approx(2 * full)
        for split in ("none", "channels"):
            assert r[k][split]["ms_step"] == pytest.approx(3.0)      # 12 ms / 4 steps
            want = r[k][split]["ops_job"] * 4 / 12e-3 / 1e12
            assert r[k][split]["value"] == pytest.approx(want)
    assert bench.parse(["--split", "channels"]).split == "channels"
    assert bench.parse([]).split == "none"


def _np_reorder(x, S, C, T, I, dtype, a, b):
    """Test stand-in for corr_reorder on CPU tensors (the oracle's permutation)."""
    import torch

    import oracle
    return torch.from_numpy(oracle.reorder(x.numpy(), a, b))


def _corner_worker(rank, world, port, out_dir, dtype):
    import torch
    import torch.distributed as dist

    import oracle
    from paper_1702_00844_gb300.shard import channel_range, corner_turn

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    S, C, T, I = 6, 5, 7, 2
    rng = np.random.default_rng(11)
    if dtype == "cf32":
        full = (rng.standard_normal((I, C, S, T, 2)) + 1j * rng.standard_normal((I, C, S, T, 2))).astype(np.complex64)
    else:
        full = rng.integers(-127, 128, size=(I, C, S, T, 2, 2)).astype(np.int8)
    sct = oracle.reorder(full, "cst", "sct")              # every receiver's stream
    Sr = S // world
    mine = torch.from_numpy(np.ascontiguousarray(sct[:, rank * Sr:(rank + 1) * Sr]))
    got = corner_turn(mine, S, C, T, I, dtype, reorder_fn=_np_reorder)
    lo, hi = channel_range(C, world, rank)
    np.testing.assert_array_equal(got.numpy(), full[:, lo:hi])
    # correlating after the turn gives this rank's channels of the whole array
    ref = oracle.correlate(full.reshape((I * C,) + full.shape[2:]), dtype)
    mine_vis = oracle.correlate(got.numpy().reshape((I * (hi - lo),) + full.shape[2:]), dtype)
    ref = ref.reshape((I, C) + ref.shape[1:])[:, lo:hi].reshape(mine_vis.shape)
    np.testing.assert_array_equal(mine_vis, ref)
    with open(os.path.join(out_dir, f"ok{rank}"), "w") as f:
        f.write("ok")
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("dtype", ["cf32", "ci8"])
def test_corner_turn_two_ranks_gloo(tmp_path, dtype):
    """Section 7's corner turn over two gloo ranks: each rank starts with all
    channels of half the stations and ends with its channels of all stations,
    equal to the oracle's layout of the whole array; its correlation equals
    the single-process correlation of those channels."""
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_corner_worker, args=(2, port, str(tmp_path), dtype), nprocs=2, join=True,
                       start_method="spawn")
    assert (tmp_path / "ok0").exists() and (tmp_path / "ok1").exists()
