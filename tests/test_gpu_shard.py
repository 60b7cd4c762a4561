"""Sharded histograms through the CUDA library: two processes on the one GPU,
each a rank with its own context, exchanging over gloo on the host (no NCCL,
no multicast; the ranks' kernels never wait on one another).

  * by points: each rank computes its slice of the point table; the gathered
    table equals one osc_histogram call over all points, bit for bit;
  * by events: each rank holds a slice of every sample's events, bounded with
    the whole sample's bounds; the digit columns are summed exactly and
    converted once, and the bins equal one osc_histogram call over all events,
    bit for bit, for FP32-bulk and FP64.
"""
import os
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

NB, LO, HI = 50, 0.0, 12.0


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _inputs():
    from paper_1311_7579_gb300 import synth
    samples = [synth.all_channel_sample(40_003, seed=91, L_km=810.0, rho=2.8, e_hi=12.0),
               synth.all_channel_sample(25_017, seed=93, L_km=295.0, rho=2.6, e_hi=6.0)]
    pts = synth.scan_points(5, seed=92)
    return samples, pts


def _worker(rank, ws, port, mode, out_dir):
    import torch.distributed as dist

    from paper_1311_7579_gb300 import api, shard
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=ws)
    samples, pts = _inputs()
    with api.Context(0) as c:
        ids = []
        for s in samples:
            if mode == "points":
                ids.append(api.osc_load_sample(c.ptr, s))
            else:
                b, n = shard.shard_events(s["n"], ws, rank)
                sub = shard.slice_sample(s, b, n)
                sid = api.osc_load_sample(c.ptr, sub)
                api.osc_sample_set_bounds(c.ptr, sid, *shard.global_bounds(sub))
                ids.append(sid)
        api.osc_set_params(c.ptr, pts)
        for prec in ("fp32", "fp64"):
            if mode == "points":
                h = shard.point_sharded_histogram(api, c.ptr, ids, len(pts), prec, LO, HI, NB)
            else:
                h = shard.event_sharded_histogram(api, c.ptr, ids, 0, len(pts), prec, LO, HI, NB)
            np.save(os.path.join(out_dir, "%s_r%d.npy" % (prec, rank)), h)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("mode", ["points", "events"])
def test_two_ranks_on_one_gpu_match_one_call_bitwise(tmp_path, mode):
    pytest.importorskip("torch")
    import torch.multiprocessing as mp

    from paper_1311_7579_gb300 import api
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, mode, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    samples, pts = _inputs()
    with api.Context(0) as c:
        ids = [api.osc_load_sample(c.ptr, s) for s in samples]
        api.osc_set_params(c.ptr, pts)
        for prec in ("fp32", "fp64"):
            ref = api.osc_histogram(c.ptr, ids, 0, len(pts), prec, LO, HI, NB)
            assert ref.sum() > 0
            for r in range(2):
                got = np.load(tmp_path / ("%s_r%d.npy" % (prec, r)))
                assert got.shape == ref.shape
                assert np.array_equal(got, ref), (mode, prec, r, float(np.max(np.abs(got - ref))))


def test_digits_round_trip_in_one_process():
    """osc_histogram_digits followed by osc_histogram_from_digits equals
    osc_histogram bit for bit (host and device buffers), and summing the digits
    of two halves of a sample (bounded with the whole sample's bounds) equals
    the whole sample's bins."""
    torch = pytest.importorskip("torch")
    from paper_1311_7579_gb300 import api, shard
    samples, pts = _inputs()
    s = samples[0]
    with api.Context(0) as c:
        sid = api.osc_load_sample(c.ptr, s)
        api.osc_set_params(c.ptr, pts)
        ref = api.osc_histogram(c.ptr, [sid], 0, len(pts), "fp32", LO, HI, NB)
        dg = api.osc_histogram_digits(c.ptr, [sid], 0, len(pts), "fp32", LO, HI, NB)
        assert dg.shape == (1, len(pts), NB, 4)
        assert np.array_equal(api.osc_histogram_from_digits(c.ptr, [sid], 0, len(pts), NB, dg), ref)
        ddev = torch.zeros((1, len(pts), NB, 4), dtype=torch.int64, device="cuda")
        api.osc_histogram_digits(c.ptr, [sid], 0, len(pts), "fp32", LO, HI, NB, out=ddev)
        odev = torch.zeros((1, len(pts), NB), dtype=torch.float64, device="cuda")
        api.osc_histogram_from_digits(c.ptr, [sid], 0, len(pts), NB, ddev, out=odev)
        torch.cuda.synchronize()
        assert np.array_equal(odev.cpu().numpy(), ref)
        w = float(np.max(np.abs(s["w_mc"])))
        e = float(np.max(s["e_true"]))
        half = (s["n"] // 128) * 64
        parts = []
        for b, n in ((0, half), (half, s["n"] - half)):
            pid = api.osc_load_sample(c.ptr, shard.slice_sample(s, b, n))
            with pytest.raises(api.OscError):
                api.osc_sample_set_bounds(c.ptr, pid, 0.5 * w, e)  # below the slice's own largest weight
            api.osc_sample_set_bounds(c.ptr, pid, w, e)
            parts.append((pid, api.osc_histogram_digits(c.ptr, [pid], 0, len(pts), "fp32", LO, HI, NB)))
        with np.errstate(over="ignore"):
            total = parts[0][1] + parts[1][1]
        assert np.array_equal(api.osc_histogram_from_digits(c.ptr, [parts[0][0]], 0, len(pts), NB, total), ref)
