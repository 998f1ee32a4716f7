"""Writes tests/golden/mos2_16k_oracle.npz: the FP64 oracle on the full-size
batched heterostructure workload mos2_16k (16 k-points, N_basis 7000-10000,
22 atoms, N_s 60, N_aux 300), for the full-size parity test of the GPU path.

Only `oracle` and `synth` are called.  The k-points are independent (no
potential feedback), and every per-step record of the method is a sum over
k with the k weights (J(t0) subtracts linearly), so the oracle runs one
k-point at a time (each drawn bit-identically to the full draw) and the
records are summed.  Stored:

* the whole-crystal record over 3 steps of a strong pulse (a whole sin^2
  pulse of amplitude 5 over the 3 steps): t, J, J_full, dmu, E, the largest
  |C^H S C - I| and N_exc;
* for k-point 0 and the largest-N_basis k-point: theta after the 3 steps
  (N_aux x N_s), the rows ROWS of C (seeded), and the rows ROWS of H(A) X and
  S X for a seeded N_basis x 8 block X at A = A_APPLY (the operator of
  Appendix A at the explicit matrices), with (|H| |X|) and (|S| |X|) at
  those rows as the scale of reduced-precision error bounds.

Run:  python tests/golden/make_mos2_16k_golden.py   (about half an hour on
8 cores; the dense H, S, P of one k-point take about 8 GB).
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import Oracle  # noqa: E402
from oracle.rttddft_oracle import hamiltonian  # noqa: E402
from synth import CONFIGS, basis_sizes, make_system, pulse_samples  # noqa: E402

WORKLOAD = "mos2_16k"
N_STEPS = 3
A0 = 5.0
A_APPLY = np.array([0.3, -0.2, 0.1])
N_X = 8
N_ROWS_C = 128
N_ROWS_HX = 256
OUT = os.path.join(HERE, "mos2_16k_oracle.npz")


def sample_rows(nb, n, seed):
    """Seeded distinct row indices, plus the first and last plane-wave and LO rows."""
    rng = np.random.default_rng(seed)
    rows = set(rng.choice(nb, size=n - 4, replace=False).tolist())
    rows.update([0, nb - 1])
    return np.array(sorted(rows), dtype=np.int64)


def seeded_block(nb, k):
    rng = np.random.default_rng(1000 + k)
    return np.asfortranarray((rng.standard_normal((nb, N_X)) + 1j * rng.standard_normal((nb, N_X))) / np.sqrt(2))


def main():
    cfg = CONFIGS[WORKLOAD]
    n_g, n_lo = basis_sizes(cfg)
    nb_all = [g + n_lo for g in n_g]
    k_big = int(np.argmax(nb_all))
    keep_k = [0, k_big]
    a = pulse_samples(cfg, n_steps=N_STEPS, a0=A0)
    tot = None
    out = {"a_samples": a, "a_apply": A_APPLY, "keep_k": np.array(keep_k), "n_basis": np.array(nb_all)}
    for k in range(cfg.n_k):
        t0 = time.time()
        s = make_system(WORKLOAD, k_subset=[k])
        orc = Oracle(s)
        r = orc.run(a, s["dt"])
        rec = {"t": r["t"], "J": r["J"], "J_full": r["J_full"], "dmu": r["dmu"], "E": r["E"],
               "n_exc": r["n_exc"], "norm_dev": r["norm_dev"]}
        if tot is None:
            tot = {key: np.array(v, dtype=np.float64) for key, v in rec.items()}
        else:
            for key in ("J", "J_full", "dmu", "E", "n_exc"):
                tot[key] += rec[key]
            tot["norm_dev"] = np.maximum(tot["norm_dev"], rec["norm_dev"])
        if k in keep_k:
            nb = nb_all[k]
            ops = orc.kp[0]["ops"]
            c = r["C"][0]
            rows_c = sample_rows(nb, N_ROWS_C, 10 + k)
            rows_h = sample_rows(nb, N_ROWS_HX, 20 + k)
            x = seeded_block(nb, k)
            h = hamiltonian(ops, A_APPLY, float(s["c_light"]))
            hx = h @ x
            sx = ops["S"] @ x
            # entrywise scales of the products, (|H| |X|) and (|S| |X|) at the rows,
            # for error bounds of reduced-precision forms
            mag_h = np.abs(h[rows_h, :]) @ np.abs(x)
            mag_s = np.abs(ops["S"][rows_h, :]) @ np.abs(x)
            del h
            out.update({
                "theta_k%d" % k: r["theta"][0],
                "rows_c_k%d" % k: rows_c, "c_rows_k%d" % k: c[rows_c, :],
                "rows_hx_k%d" % k: rows_h, "hx_rows_k%d" % k: hx[rows_h, :], "sx_rows_k%d" % k: sx[rows_h, :],
                "hx_norm_k%d" % k: np.array([float(np.max(np.abs(hx)))]),
                "mag_h_k%d" % k: mag_h, "mag_s_k%d" % k: mag_s,
            })
        del orc, r
        print("k %2d  N_basis %5d  %.1f s" % (k, nb_all[k], time.time() - t0), flush=True)
    for key, v in tot.items():
        out["rec_" + key] = v
    np.savez_compressed(OUT, **out)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
