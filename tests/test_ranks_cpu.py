"""Host logic of the multi-rank benchmark on CPU (gloo, two ranks): every
rank simulates its own seeded replica, the reported time is the slowest
rank's, and the whole-job rate counts every rank's gates over that time.
There is no data exchange between replicas."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [120.0, 250.0][rank]                 # rank 1 is the slower one
        ms = bench.max_over_ranks(local_ms, world, "cpu")
        seeds = [None] * world
        dist.all_gather_object(seeds, bench.replica_seed(rank))
        out[rank] = (ms, bench.job_rate(world, 420, 3, ms), tuple(seeds))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(worker, args=(world, free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        ms, rate, seeds = res[rank]
        assert ms == 250.0
        assert rate == pytest.approx(2 * 420 * 3 / 0.25)
        assert len(set(seeds)) == world                 # independent replicas


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(17.5, 1, "cpu") == 17.5
    assert bench.job_rate(1, 420, 5, 1000.0) == 2100.0


def test_serving_mix_is_seeded_and_shaped():
    """The serving workload's request stream: the same seed gives the same
    circuits; the class mix is about 40 / 30 / 30 (QFT / Grover / grid); n,
    the bounds and the read-out qubits stay in range."""
    a = bench.serving_requests(400, 10, 14, 77)
    b = bench.serving_requests(400, 10, 14, 77)
    assert [(r["n"], r["cls"], r["x"], r["eps"], r["readout"], len(r["gates"])) for r in a] == \
           [(r["n"], r["cls"], r["x"], r["eps"], r["readout"], len(r["gates"])) for r in b]
    counts = {k: sum(r["cls"] == k for r in a) for k in ("qft", "grover", "grid")}
    assert abs(counts["qft"] / 400 - 0.4) < 0.08
    assert abs(counts["grover"] / 400 - 0.3) < 0.08
    assert abs(counts["grid"] / 400 - 0.3) < 0.08
    for r in a:
        assert 10 <= r["n"] <= 14 and r["eps"] in (1e-3, 1e-4)
        assert 1 <= len(r["readout"]) <= 3 and len(set(r["readout"])) == len(r["readout"])
        assert all(0 <= q < r["n"] for q in r["readout"])
        assert 0 <= r["x"] < (1 << r["n"])
        assert all(max(g.targets) < r["n"] for g in r["gates"])
