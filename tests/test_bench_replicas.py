"""The N > 1 path of bench.py on the CPU (two gloo ranks): the path does
not shard, so N GPUs run N independent replicas; the job's time is the
slowest rank's, its throughput the work of all ranks over that time, each
rank solves its own seeded problem, and the reference arm prints from rank 0
only."""
import importlib.util
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench = _bench()
        local = [3.0, 5.0][rank]                     # rank 1 is the slow replica
        t = bench.max_over_ranks(local, world, "cpu")
        out[rank] = (t, bench.job_tflops(2e12, world, t))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank_main, args=(2, _free_port(), out), nprocs=2, start_method="spawn", join=True)
        res = dict(out)
    for rank in (0, 1):
        t, tf = res[rank]
        assert t == 5.0
        assert tf == pytest.approx(2 * 2e12 / 5.0 / 1e12)


def test_single_rank_keeps_its_own_time():
    bench = _bench()
    assert bench.max_over_ranks(1.25, 1, "cpu") == 1.25
    assert bench.job_tflops(1e12, 1, 0.5) == pytest.approx(2.0)


def test_replicas_solve_different_problems():
    bench = _bench()
    w = bench.WORKLOADS["synthetic-4096"]
    a = bench.make_inputs(w, "cpu", rank=0)
    b = bench.make_inputs(w, "cpu", rank=1)
    assert all(x.shape == y.shape for x, y in zip(a, b))
    assert not torch.equal(a[3], b[3]) and not torch.equal(a[1], b[1])
    again = bench.make_inputs(w, "cpu", rank=1)
    assert all(torch.equal(x, y) for x, y in zip(b, again))   # seeded


def test_reference_arm_prints_from_rank_zero_only(capsys, monkeypatch):
    bench = _bench()
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    bench.main(["--impl", "reference", "--steps", "1", "--warmup", "0"])
    assert capsys.readouterr().out == ""
