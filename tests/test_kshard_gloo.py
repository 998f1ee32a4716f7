"""The N > 1 path of bench.py on CPU.

The k-points of a workload are independent (no potential feedback), so the
benchmark gives each rank a subset of them and sums the per-rank records
once at the end.  Here two gloo ranks (127.0.0.1) run that path with the
FP64 oracle standing in for the GPU step: each rank propagates its own
k-points, the records are reduced with the same function the GPU run uses
over NCCL, and the result must equal the oracle run on all k-points.  The
timing reduction (max of the per-rank times) and the reference arm's rank
filter are covered as well."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _ragged_cfg():
    from synth import tiny_config
    return tiny_config(name="ragged", n_g=0, n_atoms=3, lmax=2, n_lo_per_atom=3, n_s=3, n_aux=20,
                       n_k=4, kgrid=(2, 2, 1), n_b_range=(130, 181), seed=17, lattice="mos2",
                       edir=(1.0, 0.0, 0.0))


def _spawn(target, world, *args):
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=target, args=(r, world, port, out) + args) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(300)
        assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
        return dict(out)


def _init(rank, world, port):
    import torch
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)


def _timing_main(rank, world, port, out, times):
    import torch
    _init(rank, world, port)
    try:
        bench.barrier()
        t_max = bench.reduce_max(times[rank], "cpu")
        out[rank] = (t_max, bench.job_throughput(2, 100, world, t_max),
                     bench.reduce_sum(3 * (rank + 1), "cpu"))
        bench.barrier()
    finally:
        torch.distributed.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_count_all_units():
    times = [0.25, 0.40]
    res = _spawn(_timing_main, 2, times)
    for r in range(2):
        t_max, value, states = res[r]
        assert t_max == 0.40
        assert value == pytest.approx(2 * 100 * 2 / 0.40)
        assert states == 9.0


def _shard_main(rank, world, port, out, n_steps):
    import torch
    from oracle import Oracle
    from synth import basis_sizes, make_system, pulse_samples
    _init(rank, world, port)
    try:
        cfg = _ragged_cfg()
        n_g, n_lo = basis_sizes(cfg)
        mine = bench.shard_kpoints([g + n_lo for g in n_g], world)[rank]
        s = make_system(cfg, k_subset=mine)
        a = pulse_samples(cfg, n_steps=n_steps, a0=5.0)
        r = Oracle(s).run(a, s["dt"])
        rec = {"t": r["t"], "j": r["J"], "j_full": r["J_full"], "dmu": r["dmu"], "energy": r["E"],
               "n_exc": r["n_exc"], "norm_dev": r["norm_dev"], "resid": r["resid"]}
        red = bench.reduce_records(rec, "cpu")
        out[rank] = (mine, {k: np.asarray(v).tolist() for k, v in red.items()})
    finally:
        torch.distributed.destroy_process_group()


def test_k_point_shards_sum_to_the_whole_crystal_record():
    """Two ranks, each propagating its shard of a ragged 4-k system with the
    oracle, reduce to the oracle's record of all four k-points."""
    from oracle import Oracle
    from synth import make_system, pulse_samples
    n_steps = 6
    res = _spawn(_shard_main, 2, n_steps)
    owned = sorted(k for r in range(2) for k in res[r][0])
    assert owned == [0, 1, 2, 3] and all(len(res[r][0]) == 2 for r in range(2))
    cfg = _ragged_cfg()
    s = make_system(cfg)
    full = Oracle(s).run(pulse_samples(cfg, n_steps=n_steps, a0=5.0), s["dt"])
    for r in range(2):
        red = {k: np.asarray(v) for k, v in res[r][1].items()}
        for key, ref in (("j", full["J"]), ("j_full", full["J_full"]), ("dmu", full["dmu"]),
                         ("energy", full["E"])):
            scale = max(float(np.max(np.abs(ref))), 1e-300)
            assert np.max(np.abs(red[key] - ref)) / scale < 1e-12, key
        # N_exc = N_e - (kept charge): a small difference of numbers of order N_e
        n_e = float(np.sum(s["wk"]) * np.sum(s["occ"]))
        assert np.max(np.abs(red["n_exc"] - full["n_exc"])) < 1e-14 * n_e
        assert np.allclose(red["norm_dev"], full["norm_dev"], rtol=0, atol=1e-15)
        assert np.allclose(red["resid"], full["resid"], rtol=0, atol=1e-15)
    assert np.max(np.abs(full["dmu"])) > 1e-6  # the pulse drives a dipole well above round-off


def test_shards_cover_every_k_point_once_and_balance_the_load():
    from synth import CONFIGS, basis_sizes
    n_g, n_lo = basis_sizes(CONFIGS["mos2_16k"])
    nb = [g + n_lo for g in n_g]
    for world in (1, 2, 4, 8, 16):
        sh = bench.shard_kpoints(nb, world)
        assert sorted(k for s in sh for k in s) == list(range(16))
        loads = [sum(nb[k] ** 2 for k in s) for s in sh]
        # longest-first to the least-loaded rank: no rank above the mean by more than one k-point
        assert max(loads) <= sum(loads) / world + max(n ** 2 for n in nb)
    assert bench.shard_kpoints([5, 7, 6], 5)[3:] == [[], []]


def test_reduction_without_a_process_group_is_the_local_value():
    assert bench.reduce_max(1.5, "cpu") == 1.5
    assert bench.reduce_sum(2.5, "cpu") == 2.5
    rec = {"j": np.ones((2, 3))}
    assert bench.reduce_records(rec, "cpu") is rec
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
    for key, val in bench.workload_config("tiny400").items():
        assert d["config"][key] == val, key
