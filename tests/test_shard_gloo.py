"""Multi-rank partitioning on CPU with gloo, world size 2: point sharding and
event sharding (with the fixed-order sum of partial histograms) reproduce the
single-process result.  Each rank's histograms come from the FP64 oracle, which
stands in for the GPU computation here."""
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


def _worker(rank, ws, port, mode, out_dir):
    import torch
    import torch.distributed as dist

    import oracle
    from paper_1311_7579_gb300 import shard, synth
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=ws)
    s = synth.table1_sample(6000, seed=71)
    pts = synth.scan_points(7, seed=72)
    if mode == "points":
        b, c = shard.shard_points(len(pts), ws, rank)
        local = torch.from_numpy(oracle.histogram(s, pts[b:b + c], 0.0, 5.0, 40))[None]
        full = shard.gather_point_histograms(local, len(pts))
    else:
        b, c = shard.shard_events(s["n"], ws, rank)
        sub = {k: (v[b:b + c] if isinstance(v, np.ndarray) else v) for k, v in s.items()}
        sub["n"] = c
        local = torch.from_numpy(oracle.histogram(sub, pts, 0.0, 5.0, 40))[None]
        full = shard.sum_event_histograms(local)
    np.save(os.path.join(out_dir, "r%d.npy" % rank), full.numpy())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("mode", ["points", "events"])
def test_two_rank_sharding_matches_single_process(tmp_path, mode):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    import oracle
    from paper_1311_7579_gb300 import synth
    oracle.build()
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, mode, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    s = synth.table1_sample(6000, seed=71)
    pts = synth.scan_points(7, seed=72)
    ref = oracle.histogram(s, pts, 0.0, 5.0, 40)[None]
    r0 = np.load(tmp_path / "r0.npy")
    r1 = np.load(tmp_path / "r1.npy")
    assert np.array_equal(r0, r1)  # identical on every rank
    if mode == "points":
        assert np.array_equal(r0, ref)
    else:
        assert np.allclose(r0, ref, rtol=1e-12, atol=0)
