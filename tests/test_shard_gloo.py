"""Host logic of the multi-rank partitioning on CPU with gloo, world size 2.

The GPU computation itself is covered by tests/test_gpu_shard.py (two processes
driving the CUDA library); here no GPU is needed:
  * the slices cover the range exactly and are balanced;
  * point sharding: each rank's slice of histograms (from the FP64 oracle,
    standing in for the library here) is gathered into the single-process
    table, identical on every rank;
  * event sharding's exchange: the integer all-reduce of uint64 digit columns
    is the exact wrap-around sum, identical on every rank, and the global
    bounds are the maxima over the ranks' slices.
"""
import os
import socket

import numpy as np
import pytest

from paper_1311_7579_gb300 import shard


def test_split_range_covers_exactly():
    for n in (0, 1, 63, 64, 65, 1000, 12345):
        for ws in (1, 2, 3, 8):
            for q in (1, 64):
                got = [shard.split_range(n, ws, r, q) for r in range(ws)]
                pos = 0
                for b, c in got:
                    assert b == pos and c >= 0
                    assert b % q == 0 or c == 0 or b == n
                    pos += c
                assert pos == n
                sizes = [c for _, c in got]
                pad = -(-n // q) * q - n  # the last slice is short by the padding
                assert max(sizes) - min(sizes) <= q + pad


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _digits(rank):
    rng = np.random.default_rng(100 + rank)
    return rng.integers(0, 2 ** 64, size=(2, 3, 5, 4), dtype=np.uint64)


def _worker(rank, ws, port, mode, out_dir):
    import torch.distributed as dist

    import oracle
    from paper_1311_7579_gb300 import shard, synth
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=ws)
    if mode == "points":
        import torch
        s = synth.table1_sample(6000, seed=71)
        pts = synth.scan_points(7, seed=72)
        b, c = shard.shard_points(len(pts), ws, rank)
        local = torch.from_numpy(oracle.histogram(s, pts[b:b + c], 0.0, 5.0, 40))[None]
        full = shard.gather_point_histograms(local, len(pts)).numpy()
        np.save(os.path.join(out_dir, "r%d.npy" % rank), full)
    else:
        total = shard.sum_digits(_digits(rank))
        s = synth.table1_sample(6000, seed=73)
        b, c = shard.shard_events(s["n"], ws, rank)
        w, e = shard.global_bounds(shard.slice_sample(s, b, c))
        np.save(os.path.join(out_dir, "r%d.npy" % rank), total)
        np.save(os.path.join(out_dir, "b%d.npy" % rank), np.array([w, e]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("mode", ["points", "events"])
def test_two_rank_sharding_host_logic(tmp_path, mode):
    pytest.importorskip("torch")
    import torch.multiprocessing as mp

    import oracle
    from paper_1311_7579_gb300 import synth
    oracle.build()
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, mode, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    r0 = np.load(tmp_path / "r0.npy")
    r1 = np.load(tmp_path / "r1.npy")
    assert np.array_equal(r0, r1)  # identical on every rank
    if mode == "points":
        s = synth.table1_sample(6000, seed=71)
        pts = synth.scan_points(7, seed=72)
        assert np.array_equal(r0, oracle.histogram(s, pts, 0.0, 5.0, 40)[None])
    else:
        with np.errstate(over="ignore"):
            ref = _digits(0) + _digits(1)  # uint64 wrap-around
        assert r0.dtype == np.uint64 and np.array_equal(r0, ref)
        s = synth.table1_sample(6000, seed=73)
        bounds = np.load(tmp_path / "b0.npy")
        assert np.array_equal(bounds, np.load(tmp_path / "b1.npy"))
        assert bounds[0] == float(np.max(np.abs(s["w_mc"]))) and bounds[1] == float(np.max(s["e_true"]))
