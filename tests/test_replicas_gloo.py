"""The N > 1 path of bench.py on CPU: two gloo ranks (127.0.0.1) run the
replica reduction (max of the per-rank times, job throughput over all
ranks) that the GPU run uses over NCCL, and the reference arm's rank
filter (only rank 0 works and prints)."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out):
    import torch
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier()
        t_max = bench.reduce_max(times[rank], "cpu")
        value = bench.job_throughput(2, 100, world, t_max)
        out[rank] = (t_max, value)
        bench.barrier()
    finally:
        torch.distributed.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_count_all_units():
    world, port = 2, _free_port()
    times = [0.25, 0.40]
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank_main, args=(r, world, port, times, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
        res = dict(out)
    for r in range(world):
        t_max, value = res[r]
        assert t_max == 0.40
        assert value == pytest.approx(2 * 100 * world / 0.40)


def test_reduction_without_a_process_group_is_the_local_value():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(1.5, "cpu") == 1.5
    assert bench.job_throughput(7, 10, 1, 2.0) == 35.0


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_reference_arm_prints_one_line_on_rank_zero():
    env = dict(os.environ, WORLD_SIZE="2", RANK="0", LOCAL_RANK="0", MASTER_ADDR="127.0.0.1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--workload", "tiny400", "--steps", "3", "--warmup", "3"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["cpu_baseline"]["kind"] == "oracle"
    # the workload part of the config matches what the GPU arm reports
    sys.path.insert(0, ROOT)
    import bench
    from synth import make_system
    s = make_system("tiny400")
    for key, val in bench.workload_config(s, "tiny400").items():
        assert d["config"][key] == val, key
