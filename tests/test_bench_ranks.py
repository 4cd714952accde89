"""The benchmark's multi-rank host logic on CPU with the gloo backend
(world size 2): the slowest rank's time and the sum of launches reach every
rank, the whole-job value counts every rank's work, and under torchrun the
reference arm runs on rank 0 only."""
import importlib.util
import json
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = load_bench()
        t, launches = b.reduce_over_ranks(1.5 + rank, 100 + rank, world, torch.device("cpu"))
        q.put((rank, t, launches, b.whole_job_value(world, 2, 1e12, t)))
    finally:
        dist.destroy_process_group()


def test_reduce_over_ranks_gloo_world2():
    world, port = 2, free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    got = sorted(q.get(timeout=10) for _ in range(world))
    for rank, t, launches, value in got:
        assert t == 2.5                         # the slower rank's time
        assert launches == 201                  # both ranks' launches
        assert value == pytest.approx(2 * 2 * 1e12 / 2.5 / 1e12)


def test_single_rank_is_identity():
    b = load_bench()
    assert b.reduce_over_ranks(3.0, 7, 1, None) == (3.0, 7)
    assert b.whole_job_value(1, 4, 2e12, 2.0) == pytest.approx(4.0)


def test_reference_arm_runs_on_rank0_only(monkeypatch, capsys):
    b = load_bench()
    monkeypatch.setattr("sys.argv", ["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
                                     "--warmup", "0", "--ref-sample-n", "64"])
    a = b.parse()
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    b.run_reference(a)
    assert capsys.readouterr().out == ""        # rank 1: no work, no line
    monkeypatch.setenv("RANK", "0")
    b.run_reference(a)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["cpu_baseline"]["kind"] == "oracle" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0
