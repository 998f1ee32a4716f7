"""The FFT route of the interstitial sum (Sec. 3: matrix products against
FFTs) against the FP64 oracle, through the C ABI.

The route computes sum_G' V~_{G-G'} C_G' as a circular convolution on a grid
of F_i >= vt_dim[i] points per axis, which equals the direct sum exactly;
only the rounding differs.  Error model: a radix-r FFT of n points has a
relative error of about eps log2(n) in the 2-norm, so the FP64 route stays
near 1e-15 of the operator's scale and is checked with the FP64 form's
tolerances (1e-12 of the largest entry, dipole 1e-8, J and E 1e-10); the
FP32 route (eps 6e-8, three transforms of log2(n) ~ 6 stages per axis) is
checked entrywise against 1e-5 (|H||x|), like the FP32 form.
"""
import numpy as np
import pytest

from oracle import Oracle, explicit_dv, explicit_operators, hamiltonian
from paper_2403_04351_gb300 import Context, RttddftError, build
from synth import dv_scale_samples, make_dv, make_system, pulse_samples, tiny_config
from systems import free_electron_system

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    build()


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(float(np.max(np.abs(b))), 1e-300))


def ragged_cfg():
    return tiny_config(name="ragged", n_g=0, n_atoms=3, lmax=2, n_lo_per_atom=3, n_s=3, n_aux=20,
                       n_k=4, kgrid=(2, 2, 1), n_b_range=(130, 181), seed=17, lattice="mos2",
                       edir=(1.0, 0.0, 0.0))


def chain_cfg(n_g=600):
    """A long thin cell (6 x 6 x 120 bohr^3): the table box needs more than 128
    grid points along z (161 at 600 plane waves, 162 on the FFT grid)."""
    return tiny_config(name="chain", n_g=n_g, n_atoms=2, lmax=2, n_lo_per_atom=2, n_s=3, n_aux=24,
                       lattice="chain", seed=23)


def smooth(n):
    m = n
    while True:
        r = m
        for p in (2, 3, 5):
            while r % p == 0:
                r //= p
        if r == 1:
            return m
        m += 1


def system_for(case):
    dv = None
    if case in ("tiny400", "dv"):
        s = make_system("tiny400")
        dv = make_dv(s) if case == "dv" else None
    elif case == "ragged":
        s = make_system(ragged_cfg())
    elif case == "free":
        s = free_electron_system(n_g=50, n_s=2, n_aux=6)
    elif case == "chain":
        s = make_system(chain_cfg())
    else:  # many states, several column chunks of the operator
        s = make_system(tiny_config(n_g=300, n_atoms=2, lmax=2, n_lo_per_atom=2, n_s=40, n_aux=64, seed=5))
    return s, dv


@pytest.mark.parametrize("launches", ["5", "3"])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16x3", "fp16x3"])
@pytest.mark.parametrize("case", ["tiny400", "ragged", "free", "dv", "wide", "chain"])
def test_operator_by_fft_equals_explicit(case, prec, launches, monkeypatch):
    """Both launch sets (five line passes; plane-fused three) on every case.
    The split forms take the interstitial sum by FP32 FFTs and the
    matching-coefficient products on the tensor cores: their bound is the
    split one, 1e-4 (|H||x|)."""
    rng = np.random.default_rng(4)
    s, dv = system_for(case)
    monkeypatch.setenv("RTTDDFT_FFT_LAUNCHES", launches)
    ctx = Context(s, precision=prec, interstitial="fft")
    info = ctx.info()
    assert info["interstitial"] == 1
    assert info["fft_fused"] == (1 if launches == "3" else 0)
    assert info["fft_grid"] == tuple(smooth(int(v)) for v in s["vt_dim"])
    if dv is not None:
        ctx.set_dv(dv)
    a_vec = np.array([0.3, -0.7, 1.1]) * 20.0
    sdv = 0.8 if dv is not None else 0.0
    for k in range(int(s["n_k"])):
        ops = explicit_operators(s, k)
        nb = ops["nb"]
        ncols = 2 * int(s["n_s"]) + 1
        x = rng.standard_normal((nb, ncols)) + 1j * rng.standard_normal((nb, ncols))
        hx, sx = ctx.apply(k, x, a_vec, sdv)
        h = hamiltonian(ops, a_vec, s["c_light"], explicit_dv(s, k, dv) if dv else None, sdv)
        ref_h, ref_s = h @ x, ops["S"] @ x
        if prec == "fp64":
            assert rel(hx, ref_h) < 1e-12, (k, rel(hx, ref_h))
            assert rel(sx, ref_s) < 1e-12
        else:
            tol = 1e-5 if prec == "fp32" else 1e-4
            assert np.max(np.abs(hx - ref_h) / (np.abs(h) @ np.abs(x))) < tol
            assert np.max(np.abs(sx - ref_s) / (np.abs(ops["S"]) @ np.abs(x))) < tol
    ctx.close()


def test_fft_and_direct_sum_agree_to_rounding():
    """The two routes of the same FP64 operator: equal to a few ulps of the
    operator's scale (they share everything but the interstitial sum)."""
    s = make_system("tiny400")
    rng = np.random.default_rng(8)
    nb = int(s["n_g"][0]) + int(np.sum(s["n_lo"]))
    x = rng.standard_normal((nb, 3)) + 1j * rng.standard_normal((nb, 3))
    a_vec = np.array([0.1, 0.2, -0.4])
    c1 = Context(s, interstitial="toeplitz")
    c2 = Context(s, interstitial="fft")
    h1, s1 = c1.apply(0, x, a_vec, 0.0)
    h2, s2 = c2.apply(0, x, a_vec, 0.0)
    assert rel(h2, h1) < 1e-13
    assert rel(s2, s1) < 1e-14
    c1.close()
    c2.close()


@pytest.mark.parametrize("n_g", [600, 3000])
def test_long_axis_fft_equals_direct_sum(n_g):
    """Axes beyond 128 grid points (fewer lines per block of a pass): the FFT
    route equals the FP64 direct sum to rounding at z extents of 162 and 270
    points."""
    s = make_system(chain_cfg(n_g))
    rng = np.random.default_rng(9)
    nb = int(s["n_g"][0]) + int(np.sum(s["n_lo"]))
    x = rng.standard_normal((nb, 5)) + 1j * rng.standard_normal((nb, 5))
    a_vec = np.array([0.2, -0.1, 0.5])
    c1 = Context(s, interstitial="toeplitz")
    c2 = Context(s, interstitial="fft")
    assert c2.info()["fft_grid"][2] == smooth(int(s["vt_dim"][2])) > 128
    h1, s1 = c1.apply(0, x, a_vec, 0.0)
    h2, s2 = c2.apply(0, x, a_vec, 0.0)
    assert rel(h2, h1) < 1e-13
    assert rel(s2, s1) < 1e-14
    c1.close()
    c2.close()


def test_long_axis_hartree_feedback_matches_oracle():
    """The density passes (full-grid transforms of every axis) on the long
    cell against the oracle's direct density and Hartree matrix."""
    s = make_system(chain_cfg())
    a = pulse_samples(s, n_steps=15, a0=20.0)
    r = Oracle(s).run(a, s["dt"], hartree=True)
    ctx = Context(s, interstitial="fft", hartree=True, graph_steps=5)
    ctx.step(a)
    obs = ctx.observables()
    assert rel(obs["dmu"], r["dmu"]) < 1e-8
    assert rel(obs["energy"], r["E"]) < 1e-10
    ctx.close()


@pytest.mark.parametrize("launches", ["5", "3"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_step_by_fft_matches_oracle_over_200_steps(prec, launches, monkeypatch):
    monkeypatch.setenv("RTTDDFT_FFT_LAUNCHES", launches)
    s = make_system("tiny400")
    a = pulse_samples(s, a0=5.0)
    r = Oracle(s).run(a, s["dt"])
    ctx = Context(s, precision=prec, interstitial="fft", graph_steps=10)
    ctx.step(a)
    obs = ctx.observables()
    assert rel(obs["dmu"], r["dmu"]) < 1e-8
    assert rel(obs["j"], r["J"]) < 1e-10
    if prec == "fp64":
        assert rel(obs["energy"], r["E"]) < 1e-10
        assert rel(obs["j_full"], r["J_full"]) < 1e-10
        assert np.max(obs["norm_dev"]) < 1e-10
        assert np.max(obs["resid"]) < 1e-10
    else:
        assert rel(obs["energy"], r["E"]) < 1e-5
        assert rel(obs["j_full"], r["J_full"]) < 1e-4
        assert np.max(obs["norm_dev"]) < 1e-5
    ctx.close()


def test_ragged_multi_k_step_by_fft():
    s = make_system(ragged_cfg())
    a = pulse_samples(s, n_steps=40, a0=5.0)
    r = Oracle(s).run(a, s["dt"])
    ctx = Context(s, interstitial="fft", graph_steps=10)
    ctx.step(a)
    obs = ctx.observables()
    assert rel(obs["dmu"], r["dmu"]) < 1e-8
    assert rel(obs["energy"], r["E"]) < 1e-10
    assert np.max(obs["norm_dev"]) < 1e-10
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16x3", "fp16x3"])
def test_potential_change_rebuilt_by_fft(prec):
    """dVV = L^H (s dh) L + CC_G^H (s dV~ * CC_G) with the interstitial part by
    FFT over the N_aux columns, every step.  In FP64 the dipole keeps 1e-8; in
    the reduced-precision forms the rebuilt dVV carries FP32 rounding into the
    FP64 subspace Hamiltonian (bound 1e-6, the split forms' target)."""
    s = make_system("tiny400")
    dv = make_dv(s)
    a = pulse_samples(s, n_steps=30, a0=10.0)
    sc = dv_scale_samples(30, s["dt"])
    r = Oracle(s, dv=dv).run(a, s["dt"], dv_scale=sc)
    ctx = Context(s, precision=prec, interstitial="fft")
    ctx.set_dv(dv)
    ctx.step(a, sc)
    obs = ctx.observables()
    if prec == "fp64":
        assert rel(obs["dmu"], r["dmu"]) < 1e-8
        assert rel(obs["energy"], r["E"]) < 1e-10
    else:
        assert rel(obs["dmu"], r["dmu"]) < 1e-6
        assert rel(obs["energy"], r["E"]) < (1e-5 if prec == "fp32" else 1e-4)
    ctx.close()


def test_h2_6000_by_fft_sampled():
    """The benchmark workload over 20 steps through the FFT route in both
    forms, in the benchmark's launch configuration (graphs of 10 steps)."""
    s = make_system("h2_6000")
    a = pulse_samples(s)[:20]
    r = Oracle(s).run(a, s["dt"])
    for prec in ("fp64", "fp32"):
        ctx = Context(s, precision=prec, interstitial="fft", graph_steps=10)
        assert ctx.info()["fft_grid"] == (45, 45, 45)
        print(prec, "fft launches", 3 if ctx.info()["fft_fused"] else 5)
        ctx.step(a)
        obs = ctx.observables()
        assert rel(obs["dmu"], r["dmu"]) < 1e-8
        assert rel(obs["j"], r["J"]) < 1e-10
        assert rel(obs["energy"], r["E"]) < (1e-10 if prec == "fp64" else 1e-5)
        ctx.close()



@pytest.mark.parametrize("prec", ["bf16x3", "fp16x3"])
def test_split_forms_by_fft_over_200_steps(prec):
    """The split forms with the FFT route: the dipole and the current of
    record from the FP64 subspace (1e-8, 1e-10), the full-basis observables
    within the split bounds."""
    s = make_system("tiny400")
    a = pulse_samples(s, a0=5.0)
    r = Oracle(s).run(a, s["dt"])
    ctx = Context(s, precision=prec, interstitial="fft", graph_steps=10)
    ctx.step(a)
    obs = ctx.observables()
    assert rel(obs["dmu"], r["dmu"]) < 1e-8
    assert rel(obs["j"], r["J"]) < 1e-10
    assert rel(obs["energy"], r["E"]) < 1e-4
    assert rel(obs["j_full"], r["J_full"]) < 1e-3
    assert np.max(obs["norm_dev"]) < 1e-4
    ctx.close()
