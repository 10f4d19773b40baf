"""Multi-rank host logic of bench.py on CPU: two gloo ranks (the GPU runs use one NCCL rank per GPU).

The path shards over independent samples (replicas, weak scaling): each rank draws its own seed, the
job time is the maximum over ranks, and the job throughput counts the units of all ranks.  Under
torchrun only rank 0 prints; the reference arm does its work on rank 0 alone.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    seed = bench.rank_seed(rank)
    ms = 100.0 + 50.0 * rank          # rank 1 is the slow one
    ms_max = bench.max_over_ranks(ms, dist, "cpu")
    value = bench.job_throughput(1000.0, world, ms_max)
    seeds = [None] * world
    dist.all_gather_object(seeds, seed)
    out[rank] = (ms_max, value, seeds)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        ms_max, value, seeds = res[rank]
        assert ms_max == 150.0
        assert abs(value - 2000.0 / 0.150) < 1e-6
        assert len(set(seeds)) == world


def test_reference_arm_only_on_rank_zero(capsys):
    import bench
    import argparse
    args = argparse.Namespace(workload="rf_4x2^25", warmup=0, steps=1, gpus=2)
    bench.run_reference(args, rank=1, world=2)
    assert capsys.readouterr().out == ""


def test_cpu_sample_fits_every_workload():
    """The CPU baseline's light-cone window (w sites, n steps: w + 2 n sites of the chain) fits every
    preset, the 2^16-site random-bond chains included, with the same 2^27 site-updates per thread."""
    import bench
    for name in ["rf_4x2^25", "rf_16x2^20", "rb_1024x2^16", "uneven_256", "rbg_linear_4x2^25", "none_16x2^20"]:
        wl = bench.workload(name, 0)
        L = wl["cpu"]["L"]
        w, n = bench.cpu_sample_shape(L)
        assert w >= 1 and n >= 1 and w + 2 * n <= L, name
        assert w * n == 1 << 27, name
    wl = bench.workload("rb_1024x2^16", 0)
    r = bench.oracle_sample(wl, 1024, 16)
    assert r["value"] > 0 and r["kind"] == "oracle"
