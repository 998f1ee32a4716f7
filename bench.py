#!/usr/bin/env python
"""Throughput of the RT-TDDFT auxiliary-subspace step on GB300.

One "step" is one time step of the whole hot path for every k-point of the
workload: HH(t) build, propagation, expansion, operator pass from the
submatrices, projection and reductions.  The metric is state*steps/s
(propagated Kohn-Sham states times time steps per second).

ours (default): the CUDA library through its C ABI.  `value` is device time
(CUDA events on the context's stream, summed over the K timed steps) with
the inputs resident in HBM and L2 flushed (a 256 MiB write) before every
step; `e2e` is the same metric through the public API from host buffers
(pinned sample upload and record read-back inside every timed step).
reference: the FP64 CPU oracle on the host cores, on a bounded number of
steps of the same workload.

Multi-GPU (torchrun): every rank runs an independent replica of the
workload (the k-points of these systems need no exchange); `value` is the
sum over ranks divided by the slowest rank's time.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# precision forms timed beside the headline one ("+fft": FFT route of the interstitial sum)
FORMS = ("fp64", "fp32", "bf16x3", "fp16x3", "fp64+fft", "fp32+fft", "fp64+fft+hartree", "fp32+fft+hartree")
METRIC = "state*steps/sec per GB300, plain FP64 vs split-precision/batched at stated error"
UNIT = "state*steps/s"
FP64_PEAK_TFLOPS = 1.25   # GB300 FP64 (nominal; the profiling recipe's table)
SM_COUNT, SM_MAX_MHZ, FP32_LANES = 152, 2070.0, 128

# dram bytes (read + write) per launch from ncu captures, keyed by kernel slot,
# form and workload; valid only while the kernel source hashes match.
TRAFFIC = {
    # profiles/k_cheb_coop_h2_6000_ncu.md: dram__bytes_read.sum + dram__bytes_write.sum
    ("chebyshev_series", "fp32+fft", "h2_6000", "03e32d7d4661fadf"): 675840.0,
}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def _bf16_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        if "bf16_tflops" in d:
            return float(d["bf16_tflops"]), "measured"
    return 1900.0, "fallback"


def _src_hash():
    h = hashlib.sha256()
    for f in ("k_linalg.cu", "k_step.cu", "k_tc.cu", "k_fft.cu", "common.cuh", "rtd.h"):
        with open(os.path.join(ROOT, "paper_2403_04351_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.lines = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for n, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def algorithmic_work(name, sysd, prec, nterms=1):
    """(flops, bytes) of one launch of a step kernel, from the shapes alone
    (the submatrix form, not the dense H the method avoids)."""
    ns, naux = int(sysd["n_s"]), int(sysd["n_aux"])
    ma = int(np.sum(sysd["n_a"]))
    nlo = int(np.sum(sysd["n_lo"]))
    cb = 8 if prec == "fp32" else 16  # bytes of a stored complex
    fl, by = 0.0, 0.0
    for ng in np.asarray(sysd["n_g"], dtype=np.float64):
        nb = ng + nlo
        if name == "toeplitz_and_backprojection":
            fl += 8 * ns * (ng * ng + 2 * ng * ma)
            by += ma * ng * cb + ng * ns * 16 * 2
        elif name == "backprojection":
            fl += 8 * ns * 2 * ng * ma
            by += ma * ng * cb + ng * ns * 16 * 2
        elif name == "tc_interstitial_and_forward":
            # split-BF16: three bf16 products per complex multiply-add
            fl += 3 * 8 * ns * (ng * ng + ng * ma)
            by += ma * ng * 8 + ng * ns * 8
        elif name == "gemm_expand":
            fl += 8 * nb * naux * ns
            by += nb * naux * cb + nb * ns * 16
        elif name == "gemm_forward":
            fl += 8 * ma * ng * ns
            by += ma * ng * cb
        elif name == "gemm_project":
            fl += 8 * nb * naux * ns
            by += nb * naux * cb + nb * ns * 16
        elif name in ("chebyshev_term", "chebyshev_series"):
            terms = 1 if name == "chebyshev_term" else max(1, nterms - 1)
            fl += terms * 8 * naux * naux * ns
            by += terms * naux * naux * 16
        elif name == "fft_interstitial":
            pass  # counted once over all k below
        elif name == "local_mt":
            m = (ma + nlo)
            fl += 8 * 5 * ns * m * m / max(1, int(sysd["n_atoms"]))
            by += 5 * m * m * 16 / max(1, int(sysd["n_atoms"]))
    if name == "fft_interstitial":
        fl, by = fft_work(sysd)
    return fl, by


def _smooth(n):
    m = n
    while True:
        r = m
        for p in (2, 3, 5):
            while r % p == 0:
                r //= p
        if r == 1:
            return m
        m += 1


def fft_work(sysd):
    """(flops, bytes) of the pruned FFT convolution of all k-points and
    states: 5 L log2 L flops per 1-D transform of L points (the usual count),
    6 per grid point for the product with v(r); bytes: the grid buffers read
    and written once per pass (they stay in L2 at these sizes)."""
    import math
    ns = int(sysd["n_s"])
    F = [_smooth(int(v)) for v in sysd["vt_dim"]]
    f1 = lambda L: 5.0 * L * math.log2(L)
    fl = by = 0.0
    for gi in sysd["g_int"]:
        gi = np.asarray(gi)
        nline = len({(int(a), int(b)) for a, b in gi[:, :2]})
        nplane = len(set(int(a) for a in gi[:, 0]))
        per = (2 * nline * f1(F[2]) + 2 * nplane * F[2] * f1(F[1]) + F[1] * F[2] * (2 * f1(F[0]) + 6 * F[0]))
        pts = 2 * nline * F[2] + 4 * nplane * F[1] * F[2] + 2 * F[0] * F[1] * F[2]
        fl += ns * per
        by += ns * pts * 2 * 16
    return fl, by


def reduce_max(x, device):
    """Max over all ranks of a per-rank float (the slowest replica sets the
    time); the value itself when no process group is running."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if torch.distributed.is_available() and torch.distributed.is_initialized() \
            and torch.distributed.get_world_size() > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def barrier():
    import torch
    if torch.distributed.is_available() and torch.distributed.is_initialized() \
            and torch.distributed.get_world_size() > 1:
        torch.distributed.barrier()


def job_throughput(states_per_rank, steps, world, t_max):
    """Whole-job state*steps/s: every replica advances its own copy of the
    workload, so the units of all ranks count, over the slowest rank's time."""
    return states_per_rank * steps * world / t_max


def roofline_of(name, tr, s, prec, nterms):
    """Roofline entry of one traced kernel slot: algorithmic work per launch
    over its mean event-timed duration, against the peak of its bound."""
    dur = tr[name][0] / tr[name][1] * 1e-3  # seconds per launch
    form = prec
    prec = prec.partition("+")[0]
    fl, by = algorithmic_work(name, s, prec, nterms)
    hbm, src = _peaks()
    if name in ("gemm_expand", "gemm_project", "gemm_forward") and prec != "fp64":
        ach = by / dur / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                "frac": ach / hbm, "peak_source": src}
    elif name == "tc_interstitial_and_forward":
        peak, src = _bf16_peak()
        ach = fl / dur / 1e12
        roof = {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "peak_source": src + " (cuBLAS bf16 burst)"}
    else:
        if prec == "fp64" or name in ("chebyshev_term", "chebyshev_series"):
            peak = FP64_PEAK_TFLOPS
            src = "recipe FP64 nominal"
        else:
            peak = SM_COUNT * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12
            src = "152 SM x 128 FP32 lanes x 2 x 2070 MHz"
        ach = fl / dur / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "peak_source": src}
    roof["kernel"] = name
    roof["ms_per_launch"] = dur * 1e3
    roof["traffic"] = TRAFFIC.get((name, form, s["name"], _src_hash()))
    return roof


def run_ours(args, rank, world, local_rank):
    import torch
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    from paper_2403_04351_gb300 import Context, build
    from synth import make_system, pulse_samples
    build()
    s = make_system(args.workload)
    cfg = s["cfg"]
    K, W = args.steps, args.warmup
    a_all = pulse_samples(s, n_steps=max(cfg.n_steps, K + W + 64))
    a0 = float(cfg.a0)
    # a dedicated stream: the library, the L2 flush and the events all run on it
    # (torch's default stream has handle 0, which the library would replace)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    assert stream.cuda_stream != 0
    # L2 flush by READING 256 MiB (twice the L2): the evicted lines are clean,
    # so the timed step does not pay for writing back the flush buffer
    flush_buf = torch.ones(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    class _Flush:
        def zero_(self):
            torch.sum(flush_buf)
    flush = _Flush()
    n_states = int(s["n_s"]) * int(s["n_k"])

    def timed_form(form, nsteps, nwarm):
        # a form is a precision form, with "+fft" for the FFT route of the interstitial sum
        # and "+hartree" for the density feedback (the per-step potential from the density)
        parts = form.split("+")
        ctx = Context(s, precision=parts[0], graph_steps=1, a_max=a0, max_record=nsteps + nwarm + 8,
                      stream=stream.cuda_stream, interstitial="fft" if "fft" in parts else "toeplitz",
                      hartree="hartree" in parts)
        assert ctx.stream_handle() == stream.cuda_stream
        d_a = torch.from_numpy(a_all[:nsteps + nwarm]).to(dev)
        for i in range(nwarm):
            flush.zero_()
            ctx.step(d_a[i:i + 1])
        torch.cuda.synchronize(dev)
        ctx.observables(clear=True)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(nsteps)]
        barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for i in range(nsteps):
            flush.zero_()
            ev[i][0].record(stream)
            ctx.step(d_a[nwarm + i:nwarm + i + 1])
            ev[i][1].record(stream)
        torch.cuda.synchronize(dev)
        wall = time.perf_counter() - t0
        barrier()
        dev_s = sum(e0.elapsed_time(e1) for e0, e1 in ev) * 1e-3
        obs = ctx.observables(clear=True)
        return ctx, dev_s, wall, obs

    with ClockSampler(local_rank) as clk:
        ctx, dev_s, wall, obs = timed_form(args.precision, K, W)
    clocks = clk.summary()
    dev_max = reduce_max(dev_s, dev)
    value = job_throughput(n_states, K, world, dev_max)

    # per-kernel trace (CUDA events after every launch, L2 flushed before each step)
    tr = {}
    for i in range(args.trace_steps):
        flush.zero_()
        for name, ms in ctx.trace(a_all[W + K + i:W + K + i + 1]):
            t = tr.setdefault(name, [0.0, 0])
            t[0] += ms
            t[1] += 1
    ctx.observables(clear=True)
    # e2e: host samples (pinned) in, the step's record out, every step
    pinned = torch.from_numpy(a_all[:K + W]).pin_memory()
    e2e_s = 0.0
    for i in range(W + K):
        flush.zero_()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        ctx.step(pinned[i:i + 1].numpy())
        rec = ctx.observables(clear=True)
        if i >= W:
            e2e_s += time.perf_counter() - t0
    e2e_value = job_throughput(n_states, K, world, reduce_max(e2e_s, dev))
    info = ctx.info()
    ctx.close()

    # the plain FP64 GPU step, for the ratio the target is stated against
    # the other precision forms over the same samples (same warm-up), for the
    # throughput of each and its error per observable against the plain FP64 form
    forms = {args.precision: {"value": value, "ms_per_step": dev_max / K * 1e3, "steps": K}}
    form_obs = {args.precision: obs}
    if args.fp64_steps > 0:
        for prec in FORMS:
            if prec == args.precision:
                continue
            c2, d2, _, o2 = timed_form(prec, args.fp64_steps, W)
            c2.close()
            forms[prec] = {"value": n_states * args.fp64_steps / d2, "ms_per_step": d2 / args.fp64_steps * 1e3,
                           "steps": args.fp64_steps}
            form_obs[prec] = o2
    if "fp64" in form_obs:
        for prec, o in form_obs.items():
            # the density feedback is another model: its forms compare with its FP64 form
            ref = form_obs.get("fp64+fft+hartree") if "hartree" in prec else form_obs["fp64"]
            if ref is None:
                continue
            n = min(len(o["t"]), len(ref["t"]))
            if n == 0:
                continue

            def relerr(key):
                a_, b_ = np.asarray(o[key][:n]), np.asarray(ref[key][:n])
                return float(np.max(np.abs(a_ - b_)) / max(float(np.max(np.abs(b_))), 1e-300))
            forms[prec]["error_vs_fp64"] = {"dmu": relerr("dmu"), "j": relerr("j"), "energy": relerr("energy"),
                                            "j_full": relerr("j_full"),
                                            "norm_dev_max": float(np.max(o["norm_dev"][:n])), "steps": n}
    fp64 = forms.get("fp64") if args.precision != "fp64" else None

    # roofline of the dominant kernel slot (and of the tensor-core kernel, if any)
    dom = max(tr.items(), key=lambda kv: kv[1][0])[0] if tr else None
    roof = roofline_of(dom, tr, s, args.precision, info["cheb_terms"]) if dom else None
    roof_tc = None
    if "tc_interstitial_and_forward" in tr and dom != "tc_interstitial_and_forward":
        roof_tc = roofline_of("tc_interstitial_and_forward", tr, s, args.precision, info["cheb_terms"])
    roof_fft = None
    if "fft_interstitial" in tr and dom != "fft_interstitial":
        roof_fft = roofline_of("fft_interstitial", tr, s, args.precision, info["cheb_terms"])
    share = {n: round(v[0] / sum(x[0] for x in tr.values()), 4) for n, v in tr.items()}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": dev_max / K * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"fp64": "f64", "fp32": "f32+f64", "bf16x3": "bf16x3+f32+f64",
                  "fp16x3": "fp16x3+f32+f64"}[args.precision.partition("+")[0]],
        "data": "synthetic (seeded generator shaped like the paper's H2 cell)",
        "config": {**workload_config(s, args.workload), "precision_form": args.precision.partition("+")[0],
                   "interstitial": "fft" if args.precision.endswith("+fft") else "toeplitz (direct sum)",
                   "propagator": "chebyshev (exact exponential to FP64 round-off)",
                   "l2": "flushed (256 MiB read) before every timed step",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "tensor_core_plan": info.get("tc") if args.precision in ("bf16x3", "fp16x3") else None},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 3 * 8,
                "d2h_bytes_per_step": 16 * 8},
        "gpu_launches": int(info["kernel_launches_per_step"]) * K,
        "clocks": clocks,
        "roofline": roof,
        "roofline_tc": roof_tc,
        "roofline_fft": roof_fft,
        "kernel_share": share,
        "fp64": fp64,
        "forms": forms,
        "wall_s": wall,
        "observables_last": {"dmu": obs["dmu"][-1].tolist() if len(obs["t"]) else None,
                             "norm_dev_max": float(np.max(obs["norm_dev"])) if len(obs["t"]) else None},
    }
    if rank == 0 and world == 1 and args.cpu_seconds > 0:
        line["cpu_baseline"] = cpu_baseline(s, a_all, args.cpu_seconds)
    return line


def cpu_baseline(s, a_all, budget_s):
    """The oracle, as it stands, on the host cores: set-up excluded, then as
    many steps as fit in about `budget_s` seconds."""
    from oracle import Oracle
    cores = os.cpu_count()
    orc = Oracle(s)
    t0 = time.perf_counter()
    n = 0
    thetas = None
    while True:
        r = orc.run(a_all[n:n + 1], s["dt"], thetas=thetas)
        thetas = r["theta"]
        n += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": int(s["n_s"]) * int(s["n_k"]) * n / dt, "unit": UNIT, "cores": cores,
            "kind": "oracle",
            "sample": "%d steps of %s after set-up (set-up excluded), numpy/OpenBLAS threads = %d"
                      % (n, s["name"], cores)}


def workload_config(s, workload):
    """The workload part of the config, shared by both arms."""
    return {"workload": workload, "n_k": int(s["n_k"]), "n_basis": int(s["n_g"][0]) + int(np.sum(s["n_lo"])),
            "n_states": int(s["n_s"]), "n_aux": int(s["n_aux"]), "dt": float(s["dt"])}


def run_reference(args):
    from oracle import Oracle
    from synth import make_system, pulse_samples
    s = make_system(args.workload)
    a = pulse_samples(s, n_steps=max(s["cfg"].n_steps, args.steps + args.warmup + 1))
    orc = Oracle(s)
    thetas = None
    for i in range(args.warmup):
        thetas = orc.run(a[i:i + 1], s["dt"], thetas=thetas)["theta"]
    nsteps = args.steps if args.ref_steps <= 0 else min(args.steps, args.ref_steps)
    t0 = time.perf_counter()
    r = orc.run(a[args.warmup:args.warmup + nsteps], s["dt"], thetas=thetas)
    dt = time.perf_counter() - t0
    v = int(s["n_s"]) * int(s["n_k"]) * nsteps / dt
    cores = os.cpu_count()
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 1,
            "steps": nsteps, "warmup": args.warmup, "ms_per_step": dt / nsteps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded generator shaped like the paper's H2 cell)",
            "config": {**workload_config(s, args.workload), "precision_form": "fp64 oracle (numpy/scipy, host cores)"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d steps of %s (set-up excluded)" % (nsteps, s["name"])},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "dmu_last": r["dmu"][-1].tolist()}


def main():
    p = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--precision", choices=list(FORMS), default="fp32+fft",
                   help="precision form; '+fft' selects the FFT route of the interstitial sum")
    p.add_argument("--workload", default="h2_6000")
    p.add_argument("--fp64-steps", type=int, default=50, help="steps timed for each other precision form")
    p.add_argument("--trace-steps", type=int, default=5)
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    p.add_argument("--ref-steps", type=int, default=40)
    args = p.parse_args()
    if args.warmup < 3:
        p.error("--warmup must be >= 3")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS"):
                os.environ.setdefault(v, str(os.cpu_count()))
            print(json.dumps(run_reference(args)), flush=True)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    line = run_ours(args, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
