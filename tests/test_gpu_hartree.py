"""The per-step potential from the evolving density (the interstitial Hartree
potential of the density's change, fed back into HH and the operator of the
next step) against the oracle's explicit run, through the C ABI.

The GPU takes the density from pruned inverse FFTs of the plane-wave rows,
the Poisson equation on the table box and the FFT route of the rebuild; the
oracle sums the autocorrelation of the coefficients directly and forms the
Hartree matrix explicitly.  Same quantity, different rounding: the FP64 form
keeps its tolerances (dipole 1e-8, E 1e-10, norm 1e-10); in the FP32 form
the density, the potential and its projection carry FP32 rounding into the
FP64 subspace Hamiltonian (dipole 1e-6, E 1e-5).  The muffin-tin part
(hartree_mt_u != 0) takes the atoms' density matrices from L theta in FP64
in every form; its blocks go through the same rebuild as a prescribed change.
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_2403_04351_gb300 import Context, RttddftError, build
from synth import make_system, pulse_samples, tiny_config

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    build()


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(float(np.max(np.abs(b))), 1e-300))


@pytest.fixture(scope="module")
def tiny():
    return make_system("tiny400")


@pytest.fixture(scope="module")
def ref(tiny):
    a = pulse_samples(tiny, n_steps=30, a0=20.0)
    return a, Oracle(tiny).run(a, tiny["dt"], hartree=True)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16x3"])
def test_hartree_feedback_matches_oracle(tiny, ref, prec):
    a, r = ref
    ctx = Context(tiny, precision=prec, interstitial="fft", hartree=True, graph_steps=10)
    ctx.step(a)
    obs = ctx.observables()
    if prec == "fp64":
        assert rel(obs["dmu"], r["dmu"]) < 1e-8
        assert rel(obs["energy"], r["E"]) < 1e-10
        assert np.max(obs["norm_dev"]) < 1e-10
        assert np.max(np.abs(obs["n_exc"] - r["n_exc"])) < 1e-10
    else:
        # split-BF16: the interstitial sum by the FP32 FFT route, the matching-
        # coefficient products on the tensor cores; the density and its potential
        # are FP64 in every form
        assert rel(obs["dmu"], r["dmu"]) < 1e-6
        assert rel(obs["energy"], r["E"]) < (1e-5 if prec == "fp32" else 1e-4)
        assert np.max(obs["norm_dev"]) < (1e-5 if prec == "fp32" else 1e-4)
    ctx.close()


def test_hartree_feedback_changes_the_dipole(tiny, ref):
    a, r = ref
    ctx = Context(tiny, interstitial="fft", graph_steps=10)
    ctx.step(a)
    plain = ctx.observables()
    ctx.close()
    assert rel(plain["dmu"], r["dmu"]) > 1e-6


def test_hartree_feedback_is_inert_without_field(tiny):
    ctx = Context(tiny, interstitial="fft", hartree=True)
    ctx.step(np.zeros((10, 3)))
    obs = ctx.observables()
    assert np.max(np.abs(obs["dmu"])) < 1e-12
    assert np.max(np.abs(obs["n_exc"])) < 1e-12
    ctx.close()


def test_hartree_feedback_ragged_multi_k():
    cfg = tiny_config(name="ragged", n_g=0, n_atoms=3, lmax=2, n_lo_per_atom=3, n_s=3, n_aux=20,
                      n_k=4, kgrid=(2, 2, 1), n_b_range=(130, 181), seed=17, lattice="mos2",
                      edir=(1.0, 0.0, 0.0))
    s = make_system(cfg)
    a = pulse_samples(s, n_steps=20, a0=20.0)
    r = Oracle(s).run(a, s["dt"], hartree=True)
    ctx = Context(s, interstitial="fft", hartree=True, graph_steps=5)
    ctx.step(a)
    obs = ctx.observables()
    assert rel(obs["dmu"], r["dmu"]) < 1e-8
    assert rel(obs["energy"], r["E"]) < 1e-10
    ctx.close()


@pytest.fixture(scope="module")
def ref_mt(tiny):
    a = pulse_samples(tiny, n_steps=30, a0=20.0)
    return a, Oracle(tiny).run(a, tiny["dt"], hartree=True, mt_u=0.5)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_muffin_tin_feedback_matches_oracle(tiny, ref_mt, prec):
    """The muffin-tin blocks dh_a = U (n_a - n_a(0)) of the atoms' density
    matrices (Appendix A, Eq. v_MT) added to the interstitial Hartree change."""
    a, r = ref_mt
    ctx = Context(tiny, precision=prec, interstitial="fft", hartree=True, hartree_mt_u=0.5, graph_steps=10)
    ctx.step(a)
    obs = ctx.observables()
    if prec == "fp64":
        assert rel(obs["dmu"], r["dmu"]) < 1e-8
        assert rel(obs["energy"], r["E"]) < 1e-10
        assert np.max(obs["norm_dev"]) < 1e-10
        assert np.max(np.abs(obs["n_exc"] - r["n_exc"])) < 1e-10
    else:
        assert rel(obs["dmu"], r["dmu"]) < 1e-6
        assert rel(obs["energy"], r["E"]) < 1e-5
    ctx.close()


def test_muffin_tin_feedback_changes_the_dipole(tiny, ref, ref_mt):
    """U != 0 moves the dipole away from the interstitial-only feedback by far
    more than the parity tolerance, so the test above checks the MT part."""
    _, r = ref
    _, r_mt = ref_mt
    assert rel(r_mt["dmu"], r["dmu"]) > 1e-5
    a, _ = ref_mt
    ctx = Context(tiny, interstitial="fft", hartree=True, hartree_mt_u=0.0, graph_steps=10)
    ctx.step(a)
    obs = ctx.observables()
    assert rel(obs["dmu"], r_mt["dmu"]) > 1e-5
    ctx.close()


def test_muffin_tin_feedback_ragged_multi_k():
    cfg = tiny_config(name="ragged_mt", n_g=0, n_atoms=3, lmax=2, n_lo_per_atom=3, n_s=3, n_aux=20,
                      n_k=4, kgrid=(2, 2, 1), n_b_range=(130, 181), seed=19, lattice="mos2",
                      edir=(1.0, 0.0, 0.0))
    s = make_system(cfg)
    a = pulse_samples(s, n_steps=20, a0=20.0)
    r = Oracle(s).run(a, s["dt"], hartree=True, mt_u=-0.7)
    ctx = Context(s, interstitial="fft", hartree=True, hartree_mt_u=-0.7, graph_steps=5)
    ctx.step(a)
    obs = ctx.observables()
    assert rel(obs["dmu"], r["dmu"]) < 1e-8
    assert rel(obs["energy"], r["E"]) < 1e-10
    ctx.close()


def test_muffin_tin_feedback_is_inert_without_field(tiny):
    ctx = Context(tiny, interstitial="fft", hartree=True, hartree_mt_u=0.5)
    ctx.step(np.zeros((10, 3)))
    obs = ctx.observables()
    assert np.max(np.abs(obs["dmu"])) < 1e-12
    assert np.max(np.abs(obs["n_exc"])) < 1e-12
    ctx.close()


def test_hartree_bound_is_enforced_and_other_calls_refused(tiny):
    a = pulse_samples(tiny, n_steps=10, a0=20.0)
    ctx = Context(tiny, interstitial="fft", hartree=True, hartree_bound=1e-12)
    with pytest.raises(RttddftError) as e:
        ctx.step(a)
        ctx.observables()
    assert e.value.code == -1
    ctx.close()
    from synth import make_dv
    ctx = Context(tiny, interstitial="fft", hartree=True)
    with pytest.raises(RttddftError) as e:
        ctx.set_dv(make_dv(tiny))
    assert e.value.code == -1
    with pytest.raises(RttddftError) as e:
        ctx.adjoint(a, np.array([0.0, 0.0, 1.0]))
    assert e.value.code == -9
    ctx.close()
