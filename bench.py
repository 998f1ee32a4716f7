#!/usr/bin/env python
"""Throughput of the RT-TDDFT auxiliary-subspace step on GB300.

One "step" is one time step of the whole hot path for every k-point of the
workload: HH(t) build, propagation, expansion, operator pass from the
submatrices, projection and reductions.  The metric is state*steps/s
(propagated Kohn-Sham states times time steps per second).

Default workload: the batched heterostructure mos2_16k (22 atoms, 16
k-points of N_basis 7000-10000, 60 states, N_aux 300), headline form
split-BF16 on the tensor cores with the FP64 subspace.  The plain FP64 form,
the FP32, FFT-route and split-FP16 forms, and the forms with a prescribed
potential change (where the full-basis contractions feed the subspace
Hamiltonian and so the dipole) are timed beside it, each with its error per
observable against the FP64 form; h2_6000 and co_12000 are timed as extra
entries.

ours (default): the CUDA library through its C ABI.  `value` is device time
(CUDA events on the context's stream, summed over the K timed steps) with
the inputs resident in HBM and L2 flushed (a 256 MiB read) before every
step; `e2e` is the same metric through the public API from host buffers
(pinned sample upload and record read-back inside every timed step).
reference: the FP64 CPU oracle on the host cores, on a bounded sample of
the same workload (one k-point of it for the multi-k workload, its time
scaled to all k-points by the oracle's per-k cost, which grows as
N_basis^2).

Multi-GPU (torchrun): the k-points are independent (no potential feedback),
so rank r owns a subset of them (longest-first assignment by N_basis^2);
the records are summed over ranks once at the end, and `value` is the states
of all ranks times the steps over the slowest rank's time (the total work is
fixed: strong scaling).
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
    # dram__bytes_read.sum + dram__bytes_write.sum per launch, keyed by the kernel
    # sources they were taken on.  mos2_16k: an ncu capture of the DRAM counters on two
    # of its k-points (--k-subset 0,1), scaled to all 16: the series by the
    # k-points (8x, every k-point has the same N_aux), the interstitial and matching-
    # row products by sum_k N_G (6.833x; their streams are the matching coefficients
    # and the packed C_G, both proportional to N_G).
    ("chebyshev_series", "bf16x3", "mos2_16k", "7a742d39b168f133"): 27926528.0,
    ("tc_interstitial_and_forward", "bf16x3", "mos2_16k", "7a742d39b168f133"): 4533407514.0,
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
    cb = 16 if prec == "fp64" else 8  # bytes of a stored complex (FP32, or a bf16/fp16 hi/lo pair)
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
    """Max over all ranks of a per-rank float (the slowest rank sets the
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
    """Whole-job state*steps/s when every rank advances the same number of
    states: the units of all ranks count, over the slowest rank's time."""
    return states_per_rank * steps * world / t_max


def shard_kpoints(n_basis, world):
    """k-points of each rank: longest first (by N_basis^2, the per-k cost of
    the interstitial sum) to the least-loaded rank; ties to the lower rank.
    Every k-point goes to exactly one rank; each list is sorted."""
    load = [0.0] * world
    own = [[] for _ in range(world)]
    order = sorted(range(len(n_basis)), key=lambda k: (-float(n_basis[k]) ** 2, k))
    for k in order:
        r = min(range(world), key=lambda i: (load[i], i))
        own[r].append(k)
        load[r] += float(n_basis[k]) ** 2
    return [sorted(o) for o in own]


RECORD_SUM = ("j", "j_full", "dmu", "energy", "n_exc")
RECORD_MAX = ("norm_dev", "resid")


def reduce_records(obs, device):
    """Whole-crystal record from the per-rank records of disjoint k-point
    sets: J, J_full, dmu, E and N_exc are sums over k with the k weights
    (J(t0) subtracts linearly), so they add over ranks; the norm and
    residual deviations are maxima."""
    import torch
    if not (torch.distributed.is_available() and torch.distributed.is_initialized()
            and torch.distributed.get_world_size() > 1):
        return obs
    out = dict(obs)
    for key in RECORD_SUM + RECORD_MAX:
        if key not in obs:
            continue
        t = torch.from_numpy(np.ascontiguousarray(obs[key], dtype=np.float64)).to(device)
        op = torch.distributed.ReduceOp.SUM if key in RECORD_SUM else torch.distributed.ReduceOp.MAX
        torch.distributed.all_reduce(t, op=op)
        out[key] = t.cpu().numpy()
    return out


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


# ------------------------------------------------------------- workloads

DEFAULT_WORKLOAD = "mos2_16k"
DEFAULT_FORM = "bf16x3"
# forms timed beside the headline one; "+dv": a prescribed potential change
# dV(t) = sin(0.1 t) dV_1 rebuilt into the subspace Hamiltonian every step
COMPARE_FORMS = {
    "mos2_16k": ("fp64", "fp64+fft", "fp32", "fp32+fft", "bf16x3+fft", "fp16x3",
                 "fp64+fft+dv", "fp32+fft+dv", "bf16x3+dv", "bf16x3+fft+dv", "fp16x3+fft+dv"),
}
EXTRA_FORMS = ("fp64", "fp32+fft", "bf16x3", "bf16x3+fft", "fp64+fft+dv", "fp32+fft+dv", "bf16x3+dv",
               "bf16x3+fft+dv")
# the basis-size point of the paper's CO table where the two interstitial
# routes differ most: the direct sum (MM) against the FFT route, FP64 and FP32
EXTRA_FORMS_BY = {"co_25727": ("fp64", "fp64+fft", "fp32", "fp32+fft", "bf16x3", "bf16x3+fft")}
FORM_STEPS = {"mos2_16k": 4, "co_12000": 20, "h2_6000": 50, "co_25727": 10}


def parse_form(form):
    """(precision, interstitial route, density feedback, potential change)."""
    parts = form.split("+")
    if parts[0] not in ("fp64", "fp32", "bf16x3", "fp16x3") or any(
            p not in ("fft", "hartree", "dv") for p in parts[1:]):
        raise ValueError("unknown form %r" % form)
    return parts[0], ("fft" if "fft" in parts else "toeplitz"), "hartree" in parts, "dv" in parts


def reference_form(form):
    """The FP64 form a form's error is measured against (the density
    feedback and the potential change are other models)."""
    _, _, hartree, dv = parse_form(form)
    if hartree:
        return "fp64+fft+hartree"
    if dv:
        return "fp64+fft+dv"
    return "fp64"


def workload_samples(cfg, n):
    """Pulse samples A(t_k) and potential-change scales s_k of a workload,
    starting at the pulse's peak (t = T/2, T = n_steps dt), so that a short
    run already carries a dipole well above round-off."""
    from synth import dv_scale_samples, pulse_samples
    period = cfg.n_steps * cfg.dt
    a = pulse_samples(cfg, n_steps=n, t_start=0.5 * period, period=period)
    sc = dv_scale_samples(n, cfg.dt, t_start=0.5 * period)
    return a, sc


def workload_config(workload):
    """The workload part of the config, shared by both arms."""
    from synth import CONFIGS, basis_sizes
    cfg = CONFIGS[workload]
    n_g, n_lo = basis_sizes(cfg)
    nb = [g + n_lo for g in n_g]
    return {"workload": workload, "n_k": int(cfg.n_k),
            "n_basis": int(nb[0]) if len(set(nb)) == 1 else [int(min(nb)), int(max(nb))],
            "n_basis_sum": int(sum(nb)), "n_atoms": int(cfg.n_atoms), "lmax": int(cfg.lmax),
            "n_states": int(cfg.n_s), "n_aux": int(cfg.n_aux), "dt": float(cfg.dt)}


def oracle_sample_k(workload):
    """The k-point the oracle is timed on and the factor that scales its
    time to the whole workload: the k whose N_basis^2 is nearest the mean
    (the oracle's per-k step cost grows as N_basis^2: dense H(t) and its
    products with C), factor = sum_k N_basis(k)^2 / N_basis(sample)^2."""
    from synth import CONFIGS, basis_sizes
    cfg = CONFIGS[workload]
    n_g, n_lo = basis_sizes(cfg)
    nb2 = np.array([(g + n_lo) ** 2 for g in n_g], dtype=np.float64)
    if len(nb2) == 1:
        return 0, 1.0
    k = int(np.argmin(np.abs(nb2 - nb2.mean())))
    return k, float(nb2.sum() / nb2[k])


def oracle_rate(workload, a, warm, nsteps=None, budget_s=None):
    """The oracle, as it stands, on the host cores: set-up excluded, `warm`
    untimed steps, then `nsteps` timed steps (or as many as fit in
    `budget_s` seconds) of one k-point of the workload; returns the
    workload's state*steps/s scaled to all its k-points and a description."""
    from oracle import Oracle
    from synth import CONFIGS, make_system
    cfg = CONFIGS[workload]
    k, scale = oracle_sample_k(workload)
    s = make_system(workload, k_subset=[k] if cfg.n_k > 1 else None)
    orc = Oracle(s)
    thetas = None
    for i in range(warm):
        thetas = orc.run(a[i:i + 1], s["dt"], thetas=thetas)["theta"]
    t0 = time.perf_counter()
    n = 0
    while True:
        r = orc.run(a[warm + n:warm + n + 1], s["dt"], thetas=thetas)
        thetas = r["theta"]
        n += 1
        el = time.perf_counter() - t0
        if (nsteps is not None and n >= nsteps) or (budget_s is not None and el > budget_s) \
                or warm + n >= len(a):
            break
    t_sample = time.perf_counter() - t0
    t_all = t_sample * scale
    v = int(cfg.n_s) * int(cfg.n_k) * n / t_all
    cores = os.cpu_count()
    if cfg.n_k > 1:
        desc = ("%d steps of k-point %d (N_basis %d) of %s after set-up (set-up excluded), its time scaled "
                "by sum_k N_basis^2 / N_basis(%d)^2 = %.3f to all %d k-points (extrapolated: the oracle's "
                "per-k cost grows as N_basis^2); numpy/OpenBLAS threads = %d"
                % (n, k, int(s["n_g"][0]) + int(np.sum(s["n_lo"])), workload, k, scale, cfg.n_k, cores))
    else:
        desc = "%d steps of %s after set-up (set-up excluded), numpy/OpenBLAS threads = %d" % (n, workload, cores)
    return {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc,
            "steps": n, "s_per_step_sample": t_sample / n, "extrapolation_factor": scale,
            "dmu_last": r["dmu"][-1].tolist()}


def data_label(workload):
    if workload.startswith("mos2"):
        return ("synthetic (seeded generator shaped like the paper's pyridine@MoS2 interface: "
                "3x3 MoS2 supercell, 22 atoms, 4x4x1 k-grid)")
    if workload.startswith("co"):
        return "synthetic (seeded generator shaped like the paper's CO cell)"
    return "synthetic (seeded generator shaped like the paper's H2 cell)"


# ------------------------------------------------------------- our arm

class _Timer:
    """Runs forms of one system on one stream with CUDA events; L2 flushed by
    READING 256 MiB (twice the L2) before every step: the evicted lines are
    clean, so the timed step does not pay for writing back the flush buffer."""

    def __init__(self, dev, stream):
        import torch
        self.torch = torch
        self.dev = dev
        self.stream = stream
        self.flush_buf = torch.ones(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def flush(self):
        self.torch.sum(self.flush_buf)

    def context(self, s, form, max_record, a_max):
        from paper_2403_04351_gb300 import Context
        from synth import make_dv
        prec, route, hartree, dv = parse_form(form)
        ctx = Context(s, precision=prec, graph_steps=1, a_max=a_max, s_max=1.0 if dv else 0.0,
                      max_record=max_record, stream=self.stream.cuda_stream, interstitial=route,
                      hartree=hartree)
        assert ctx.stream_handle() == self.stream.cuda_stream
        if dv:
            ctx.set_dv(make_dv(s))
        return ctx

    def run(self, s, form, a_all, sc_all, nsteps, nwarm, keep=False):
        torch = self.torch
        dev, stream = self.dev, self.stream
        dv = parse_form(form)[3]
        ctx = self.context(s, form, nsteps + nwarm + 8, float(s["cfg"].a0))
        d_a = torch.from_numpy(a_all[:nsteps + nwarm]).to(dev)
        d_s = torch.from_numpy(sc_all[:nsteps + nwarm]).to(dev) if dv else None

        def one(i):
            ctx.step(d_a[i:i + 1], None if d_s is None else d_s[i:i + 1])
        for i in range(nwarm):
            self.flush()
            one(i)
        torch.cuda.synchronize(dev)
        ctx.observables(clear=True)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(nsteps)]
        barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        torch.cuda.nvtx.range_push("timed_steps")  # lets a profiler select these launches
        for i in range(nsteps):
            self.flush()
            ev[i][0].record(stream)
            one(nwarm + i)
            ev[i][1].record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize(dev)
        wall = time.perf_counter() - t0
        barrier()
        dev_s = sum(e0.elapsed_time(e1) for e0, e1 in ev) * 1e-3
        obs = ctx.observables(clear=True)
        if not keep:
            ctx.close()
            ctx = None
        return ctx, dev_s, wall, obs


def form_errors(form_obs):
    """Error of every form against its FP64 reference form, per observable:
    max over the common steps of |x - x_ref| / max |x_ref|."""
    out = {}
    for form, o in form_obs.items():
        ref = form_obs.get(reference_form(form))
        if ref is None or form == reference_form(form):
            continue
        n = min(len(o["t"]), len(ref["t"]))
        if n == 0:
            continue

        def relerr(key):
            a_, b_ = np.asarray(o[key][:n]), np.asarray(ref[key][:n])
            return float(np.max(np.abs(a_ - b_)) / max(float(np.max(np.abs(b_))), 1e-300))
        out[form] = {"vs": reference_form(form), "dmu": relerr("dmu"), "j": relerr("j"),
                     "energy": relerr("energy"), "j_full": relerr("j_full"),
                     "norm_dev_max": float(np.max(o["norm_dev"][:n])), "steps": n}
    return out


def time_forms(timer, s, forms, a_all, sc_all, nsteps, nwarm, have=None):
    """Time each form over the same samples; returns ({form: entry}, {form: record})."""
    n_states = int(s["n_s"]) * int(s["n_k"])
    entries, recs = {}, {}
    if have:
        for f, (e, o) in have.items():
            entries[f], recs[f] = e, o
    for form in forms:
        if form in entries:
            continue
        t0 = time.perf_counter()
        _, d2, _, o2 = timer.run(s, form, a_all, sc_all, nsteps, nwarm)
        log("%s %s: %.2f ms/step, %.1f s with set-up" % (s["name"], form, d2 / nsteps * 1e3,
                                                        time.perf_counter() - t0))
        entries[form] = {"value": n_states * nsteps / d2, "ms_per_step": d2 / nsteps * 1e3, "steps": nsteps}
        recs[form] = o2
    errs = form_errors(recs)
    for form, e in errs.items():
        entries[form]["error_vs_fp64"] = e
    for form, e in entries.items():
        ref = entries.get(reference_form(form))
        if ref is not None and form != reference_form(form):
            e["speedup_vs_fp64"] = e["value"] / ref["value"]
    return entries, recs


def shard_refusal(form, world, k_subset):
    """Why a form cannot run on a subset of the k-points, or None: the density
    feedback sums the density over every k-point each step, so a k-point shard
    or subset would feed back a partial density."""
    if parse_form(form)[2] and (world > 1 or k_subset):
        return ("%s: the density feedback couples the k-points through the density and is "
                "not sharded (run it on one GPU, all k-points)" % form)
    return None


def run_ours(args, rank, world, local_rank):
    import torch
    from synth import CONFIGS, make_system
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    from paper_2403_04351_gb300 import build
    build()
    cfg = CONFIGS[args.workload]
    mine = None
    if world > 1:
        n_g, n_lo = __import__("synth").basis_sizes(cfg)
        mine = shard_kpoints([g + n_lo for g in n_g], world)[rank]
    if args.k_subset:
        # a smaller case of the same workload (profiling): these k-points only
        sub = [int(x) for x in args.k_subset.split(",")]
        mine = sub if mine is None else [k for k in mine if k in sub]
    s = make_system(args.workload, k_subset=mine)
    K, W = args.steps, args.warmup
    a_all, sc_all = workload_samples(cfg, K + W + args.trace_steps + 64)
    # a dedicated stream: the library, the L2 flush and the events all run on it
    # (torch's default stream has handle 0, which the library would replace)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    assert stream.cuda_stream != 0
    timer = _Timer(dev, stream)
    n_states = int(s["n_s"]) * int(s["n_k"])
    form = args.precision
    dv_head = parse_form(form)[3]

    t_start = time.perf_counter()
    with ClockSampler(local_rank) as clk:
        ctx, dev_s, wall, obs = timer.run(s, form, a_all, sc_all, K, W, keep=True)
    log("%s %s headline: %.2f ms/step, %.1f s with set-up" % (s["name"], form, dev_s / K * 1e3,
                                                            time.perf_counter() - t_start))
    clocks = clk.summary()
    dev_max = reduce_max(dev_s, dev)
    states_all = reduce_sum(n_states, dev)
    value = states_all * K / dev_max
    obs_all = reduce_records(obs, dev)

    # per-kernel trace (CUDA events after every launch, L2 flushed before each step)
    tr = {}
    for i in range(args.trace_steps):
        timer.flush()
        j = W + K + i
        for name, ms in ctx.trace(a_all[j:j + 1], sc_all[j:j + 1] if dv_head else None):
            t = tr.setdefault(name, [0.0, 0])
            t[0] += ms
            t[1] += 1
    ctx.observables(clear=True)
    # e2e: host samples (pinned) in, the step's record out, every step
    pinned = torch.from_numpy(a_all[:K + W]).pin_memory()
    pinned_s = torch.from_numpy(sc_all[:K + W]).pin_memory()
    e2e_s = 0.0
    for i in range(W + K):
        timer.flush()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        ctx.step(pinned[i:i + 1].numpy(), pinned_s[i:i + 1].numpy() if dv_head else None)
        ctx.observables(clear=True)
        if i >= W:
            e2e_s += time.perf_counter() - t0
    e2e_value = states_all * K / reduce_max(e2e_s, dev)
    info = ctx.info()
    ctx.close()
    del ctx

    forms = {form: {"value": value, "ms_per_step": dev_max / K * 1e3, "steps": K}}
    workloads = {}
    if world == 1 and args.form_steps != 0:
        nf = args.form_steps if args.form_steps > 0 else FORM_STEPS.get(args.workload, 20)
        # the headline form again over the same samples as the others, for its error
        cmp_forms = COMPARE_FORMS.get(args.workload, FORMS)
        fe, _ = time_forms(timer, s, (form,) + tuple(f for f in cmp_forms if f != form), a_all, sc_all, nf, 3)
        for f, e in fe.items():
            if f == form:
                e = dict(e, steps_of_error_run=nf)
                forms[f].update({k: v for k, v in e.items() if k in ("error_vs_fp64", "speedup_vs_fp64")})
                forms[f]["short_run"] = {"value": e["value"], "steps": nf}
            else:
                forms[f] = e
        if "fp64" in forms and form != "fp64":
            forms[form]["speedup_vs_fp64"] = value / forms["fp64"]["value"]
        del s
        for w in [x for x in args.extra_workloads.split(",") if x and x != args.workload]:
            s2 = make_system(w)
            a2, sc2 = workload_samples(CONFIGS[w], 256)
            fe2, _ = time_forms(timer, s2, EXTRA_FORMS_BY.get(w, EXTRA_FORMS), a2, sc2, FORM_STEPS.get(w, 20), 3)
            workloads[w] = {"config": workload_config(w), "forms": fe2}
            del s2
    fp64 = forms.get("fp64") if form != "fp64" else None

    # roofline of the dominant kernel slot (and of the tensor-core kernel, if any)
    s_meta = make_system(args.workload, k_subset=mine, with_amat=False)
    dom = max(tr.items(), key=lambda kv: kv[1][0])[0] if tr else None
    roof = roofline_of(dom, tr, s_meta, form, info["cheb_terms"]) if dom else None
    roof_tc = None
    if "tc_interstitial_and_forward" in tr and dom != "tc_interstitial_and_forward":
        roof_tc = roofline_of("tc_interstitial_and_forward", tr, s_meta, form, info["cheb_terms"])
    roof_fft = None
    if "fft_interstitial" in tr and dom != "fft_interstitial":
        roof_fft = roofline_of("fft_interstitial", tr, s_meta, form, info["cheb_terms"])
    total = sum(x[0] for x in tr.values())
    share = {n: round(v[0] / total, 4) for n, v in tr.items()} if total > 0 else {}

    prec, route, hartree, _ = parse_form(form)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": dev_max / K * 1e3, "higher_is_better": True,
        "scaling": "strong" if world > 1 else "weak",
        "vs_baseline": None,
        "dtype": {"fp64": "f64", "fp32": "f32+f64", "bf16x3": "bf16x3+f32+f64",
                  "fp16x3": "fp16x3+f32+f64"}[prec],
        "data": data_label(args.workload),
        "config": {**workload_config(args.workload),
                   "l2": "flushed (256 MiB read) before every timed step",
                   "parallelism": ("k-point shards over %d ranks" % world) if world > 1 else "single GPU"},
        "form": {"name": form, "precision": prec,
                 "interstitial": "fft" if route == "fft" else "toeplitz (direct sum)",
                 "potential_change": "prescribed, sin(0.1 t) dV_1" if dv_head else
                 ("interstitial Hartree feedback" if hartree else "none"),
                 "propagator": "chebyshev (exact exponential to FP64 round-off)",
                 "subspace": "FP64 (HH, propagator, theta, J, dmu)",
                 "pulse": "samples from the pulse's peak on (t = T/2 of A0 sin^2(pi t/T) sin(w t))",
                 "tensor_core_plan": info.get("tc") if prec in ("bf16x3", "fp16x3") else None,
                 "k_points_this_rank": mine},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": (4 if dv_head else 3) * 8,
                "d2h_bytes_per_step": 16 * 8},
        "gpu_launches": int(info["kernel_launches_per_step"]) * K,
        "clocks": clocks,
        "roofline": roof,
        "roofline_tc": roof_tc,
        "roofline_fft": roof_fft,
        "kernel_share": share,
        "fp64": fp64,
        "forms": forms,
        "workloads": workloads,
        "wall_s": wall,
        "observables_last": {"dmu": obs_all["dmu"][-1].tolist() if len(obs_all["t"]) else None,
                             "norm_dev_max": float(np.max(obs_all["norm_dev"])) if len(obs_all["t"]) else None},
    }
    if rank == 0 and world == 1 and args.cpu_seconds > 0:
        t0 = time.perf_counter()
        cb = oracle_rate(args.workload, a_all, 1, budget_s=args.cpu_seconds)
        log("oracle sample: %.1f s with set-up" % (time.perf_counter() - t0))
        line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
    return line


def log(msg):
    """Progress on stderr (the JSON line alone goes to stdout)."""
    sys.stderr.write("[bench] %s\n" % msg)
    sys.stderr.flush()


def reduce_sum(x, device):
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if torch.distributed.is_available() and torch.distributed.is_initialized() \
            and torch.distributed.get_world_size() > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.SUM)
    return float(t.item())


def run_reference(args):
    from synth import CONFIGS
    cfg = CONFIGS[args.workload]
    a, _ = workload_samples(cfg, args.steps + args.warmup + 1)
    nsteps = args.steps if args.ref_steps <= 0 else min(args.steps, args.ref_steps)
    cb = oracle_rate(args.workload, a, args.warmup, nsteps=nsteps)
    v = cb["value"]
    ms = int(cfg.n_s) * int(cfg.n_k) / v * 1e3
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 1,
            "steps": cb["steps"], "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": data_label(args.workload),
            "config": {**workload_config(args.workload), "l2": "not applicable (host oracle)",
                       "parallelism": "host cores"},
            "form": {"name": "fp64 oracle (numpy/scipy, explicit H, S, P; exact exponential by eigh)"},
            "cpu_baseline": {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "dmu_last": cb["dmu_last"]}


def main():
    p = argparse.ArgumentParser(description=__doc__.split("\n")[1])
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--precision", default=DEFAULT_FORM,
                   help="headline form: fp64|fp32|bf16x3|fp16x3, then +fft (FFT route of the interstitial "
                        "sum), +hartree (density feedback) or +dv (prescribed potential change)")
    p.add_argument("--workload", default=DEFAULT_WORKLOAD)
    p.add_argument("--form-steps", type=int, default=-1,
                   help="steps timed for each other form (-1: per workload; 0: none)")
    p.add_argument("--extra-workloads", default="h2_6000,co_12000,co_25727")
    p.add_argument("--trace-steps", type=int, default=3)
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    p.add_argument("--ref-steps", type=int, default=20)
    p.add_argument("--k-subset", default="",
                   help="comma-separated k-points of the workload to run (a smaller case for profiling)")
    args = p.parse_args()
    if args.warmup < 3:
        p.error("--warmup must be >= 3")
    parse_form(args.precision)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    why = shard_refusal(args.precision, world, args.k_subset)
    if why:
        p.error(why)
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
