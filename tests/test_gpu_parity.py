"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (FP64 form): the operator from submatrices equals the explicit
H X and S X to 1e-12 of the largest entry (sums of a few hundred FP64
products); the dipole matches to 1e-8 relative (the target of the FP64
form), currents and energies to 1e-10, theta and C to 1e-9 (eigenvector
sensitivity of the Ritz basis times FP64 round-off over the run).
"""
import numpy as np
import pytest

from oracle import Oracle, explicit_dv, explicit_operators, hamiltonian
from paper_2403_04351_gb300 import Context, RttddftError, build
from synth import make_dv, make_system, pulse_samples, tiny_config, dv_scale_samples
from systems import free_electron_system, plane_wave_basis

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build()


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(float(np.max(np.abs(b))), 1e-300))


@pytest.fixture(scope="module")
def tiny():
    return make_system("tiny400")


@pytest.fixture(scope="module")
def tiny_oracle(tiny):
    return Oracle(tiny)


def ragged_cfg():
    return tiny_config(name="ragged", n_g=0, n_atoms=3, lmax=2, n_lo_per_atom=3, n_s=3, n_aux=20,
                       n_k=4, kgrid=(2, 2, 1), n_b_range=(130, 181), seed=17, lattice="mos2",
                       edir=(1.0, 0.0, 0.0))


# ------------------------------------------------------------------ operator

@pytest.mark.parametrize("case", ["tiny400", "ragged", "free", "dv"])
def test_operator_from_submatrices_equals_explicit(case, tiny):
    rng = np.random.default_rng(1)
    dv = None
    if case == "tiny400":
        s = tiny
    elif case == "ragged":
        s = make_system(ragged_cfg())
    elif case == "free":
        s = free_electron_system(n_g=50, n_s=2, n_aux=6)
    else:
        s = tiny
        dv = make_dv(s)
    ctx = Context(s)
    if dv is not None:
        ctx.set_dv(dv)
    a_vec = np.array([0.3, -0.7, 1.1]) * 20.0
    sdv = 0.8 if dv is not None else 0.0
    for k in range(int(s["n_k"])):
        ops = explicit_operators(s, k)
        nb = ops["nb"]
        ncols = 2 * int(s["n_s"]) + 1  # exercises column chunks and a ragged last chunk
        x = rng.standard_normal((nb, ncols)) + 1j * rng.standard_normal((nb, ncols))
        hx, sx = ctx.apply(k, x, a_vec, sdv)
        h = hamiltonian(ops, a_vec, s["c_light"], explicit_dv(s, k, dv) if dv else None, sdv)
        ref_h = h @ x
        ref_s = ops["S"] @ x
        assert rel(hx, ref_h) < 1e-12
        assert rel(sx, ref_s) < 1e-12
    ctx.close()


# ------------------------------------------------------------------ set-up

def test_auxiliary_basis_matches_oracle_ritz_vectors(tiny, tiny_oracle):
    ctx = Context(tiny)
    cc, ev, pp = ctx.get_aux(0)
    kp = tiny_oracle.kp[0]
    assert rel(ev, kp["eps"]) < 1e-12
    assert rel(cc, kp["caux"]) < 1e-9
    assert rel(pp, kp["psub"]) < 1e-9
    ctx.close()


def test_given_basis_is_checked_for_orthonormality(tiny, tiny_oracle):
    kp = tiny_oracle.kp[0]
    ctx = Context(tiny, aux_mode="given", caux=[kp["caux"]], eps=[kp["eps"]])
    cc, ev, _ = ctx.get_aux(0)
    assert np.array_equal(ev, kp["eps"])
    ctx.close()
    with pytest.raises(RttddftError) as e:
        Context(tiny, aux_mode="given", caux=[1.01 * kp["caux"]], eps=[kp["eps"]])
    assert e.value.code == -4


# ------------------------------------------------------------------ steps

def compare_run(obs, r, dmu_tol=1e-8, j_tol=1e-10, e_tol=1e-10):
    assert len(obs["t"]) == len(r["t"])
    assert rel(obs["t"], r["t"]) < 1e-14
    assert rel(obs["j"], r["J"]) < j_tol
    assert rel(obs["j_full"], r["J_full"]) < j_tol
    assert rel(obs["dmu"], r["dmu"]) < dmu_tol
    assert rel(obs["energy"], r["E"]) < e_tol
    assert np.max(obs["norm_dev"]) < 1e-10
    assert np.max(obs["resid"]) < 1e-10
    # excited electrons from the FP64 state: absolute, N_e times a few 1e-12
    assert np.max(np.abs(obs["n_exc"] - r["n_exc"])) < 1e-10


def test_excited_electrons_stay_zero_without_field(tiny):
    ctx = Context(tiny, graph_steps=10)
    ctx.step(np.zeros((40, 3)))
    obs = ctx.observables()
    assert np.max(np.abs(obs["n_exc"])) < 1e-12
    ctx.close()


def test_chebyshev_step_matches_oracle_over_200_steps(tiny, tiny_oracle):
    a = pulse_samples(tiny, a0=5.0)
    r = tiny_oracle.run(a, tiny["dt"])
    ctx = Context(tiny, graph_steps=10)
    ctx.step(a)
    obs = ctx.observables()
    compare_run(obs, r)
    th, c = ctx.get_state(0, with_c=True)
    assert rel(th, r["theta"][0]) < 1e-9
    assert rel(c, r["C"][0]) < 1e-9
    assert ctx.info()["steps_done"] == 200
    ctx.close()


@pytest.mark.parametrize("prop", ["eig", "cn"])
def test_eig_and_crank_nicolson_propagators(tiny, tiny_oracle, prop):
    a = pulse_samples(tiny, n_steps=40, a0=20.0)
    r = tiny_oracle.run(a, tiny["dt"], propagator="exact" if prop == "eig" else "cn")
    ctx = Context(tiny, propagator=prop)
    ctx.step(a)
    obs = ctx.observables()
    compare_run(obs, r)
    if prop == "eig":
        assert rel(obs["dt_cr"], r["dtcr"]) < 1e-10
    ctx.close()


def test_multi_k_ragged_batch_matches_oracle():
    s = make_system(ragged_cfg())
    assert len(set(s["n_g"].tolist())) == 4
    a = pulse_samples(s, n_steps=30, dt=0.2, a0=30.0)
    r = Oracle(s).run(a, 0.2)
    ctx = Context(s, dt=0.2, graph_steps=7)
    ctx.step(a[:13])
    ctx.step(a[13:])
    obs = ctx.observables()
    compare_run(obs, r)
    ctx.close()


def test_reprojection_mode(tiny, tiny_oracle):
    a = pulse_samples(tiny, n_steps=50, a0=10.0)
    r = tiny_oracle.run(a, tiny["dt"], reproject=True)
    ctx = Context(tiny, reproject=True)
    ctx.step(a)
    compare_run(ctx.observables(), r)
    ctx.close()


def test_potential_change_rebuilt_every_step(tiny):
    dv = make_dv(tiny)
    orc = Oracle(tiny, dv=dv)
    a = pulse_samples(tiny, n_steps=30, a0=10.0)
    sc = dv_scale_samples(30, tiny["dt"])
    r = orc.run(a, tiny["dt"], dv_scale=sc)
    ctx = Context(tiny)
    ctx.set_dv(dv)
    ctx.step(a, sc)
    compare_run(ctx.observables(), r)
    ctx.close()


def test_fp32_form_error_per_observable(tiny, tiny_oracle):
    a = pulse_samples(tiny, a0=5.0)
    r = tiny_oracle.run(a, tiny["dt"])
    ctx = Context(tiny, precision="fp32", graph_steps=10)
    ctx.step(a)
    obs = ctx.observables()
    # the state of record (theta) and the current J stay FP64
    assert rel(obs["dmu"], r["dmu"]) < 1e-8
    assert rel(obs["j"], r["J"]) < 1e-10
    assert np.max(np.abs(obs["n_exc"] - r["n_exc"])) < 1e-10
    # observables of the FP32 full-basis pass
    assert rel(obs["energy"], r["E"]) < 1e-5
    assert rel(obs["j_full"], r["J_full"]) < 1e-4
    assert np.max(obs["norm_dev"]) < 1e-5
    ctx.close()


def test_graph_replay_is_bitwise_equal_to_direct_launches(tiny):
    a = pulse_samples(tiny, n_steps=30, a0=5.0)
    outs = []
    for g in (0, 1, 10):
        ctx = Context(tiny, graph_steps=g)
        ctx.step(a)
        outs.append(ctx.observables())
        ctx.close()
    for o in outs[1:]:
        for key in outs[0]:
            assert np.array_equal(o[key], outs[0][key]), key


# ------------------------------------------------------------------ edge cases

@pytest.mark.parametrize("n_s,n_aux", [(1, 7), (5, 5), (3, 13)])
def test_small_and_square_subspaces(n_s, n_aux):
    s = make_system(tiny_config(n_g=50, n_atoms=2, lmax=1, n_lo_per_atom=2, n_s=n_s,
                                n_aux=n_aux, seed=23))
    a = pulse_samples(s, n_steps=25, dt=0.2, a0=40.0)
    r = Oracle(s).run(a, 0.2)
    ctx = Context(s, dt=0.2)
    ctx.step(a)
    compare_run(ctx.observables(), r)
    ctx.close()


def test_complete_subspace_and_free_electrons():
    s = make_system(tiny_config(n_g=24, n_atoms=2, lmax=1, n_lo_per_atom=2, n_s=3, seed=21))
    a = pulse_samples(s, n_steps=6, dt=0.3, a0=20.0, omega=0.5, edir=(0.2, 0.5, 0.8))
    r = Oracle(s).run(a, 0.3)
    ctx = Context(s, dt=0.3)
    ctx.step(a)
    compare_run(ctx.observables(), r)
    ctx.close()
    fe = free_electron_system(n_s=3)
    cc, eps, idx = plane_wave_basis(fe, 8)
    a = pulse_samples(fe, n_steps=40, dt=0.2, a0=3.0, omega=0.4, edir=(0.3, -0.2, 0.9))
    ctx = Context(fe, dt=0.2, aux_mode="given", caux=[cc], eps=[eps])
    ctx.step(a)
    obs = ctx.observables()
    g = fe["gk"][0][idx[:3]]
    j = -(1.0 / fe["omega"]) * (fe["occ"] @ g)[None, :] - (fe["occ"].sum() / fe["omega"]) * a / fe["c_light"]
    assert rel(obs["j"], j) < 1e-12 and rel(obs["j_full"], j) < 1e-12
    ctx.close()


def test_initial_state_given_and_record_overflow(tiny, tiny_oracle):
    rng = np.random.default_rng(4)
    kp = tiny_oracle.kp[0]
    mix = np.linalg.qr(rng.standard_normal((32, 8)) + 1j * rng.standard_normal((32, 8)))[0]
    c0 = kp["caux"] @ mix
    a = pulse_samples(tiny, n_steps=20, a0=5.0)
    r = Oracle(tiny, c0=[c0]).run(a, tiny["dt"])
    ctx = Context(tiny, c0=[c0], max_record=25)
    ctx.step(a)
    compare_run(ctx.observables(clear=False), r)
    with pytest.raises(RttddftError) as e:
        ctx.step(a)
    assert e.value.code == -1
    ctx.observables(clear=True)
    ctx.step(a[:5])
    assert len(ctx.observables()["t"]) == 5
    ctx.close()


# ------------------------------------------------------------------ full size

def test_h2_6000_bench_configuration_sampled():
    """The benchmark's workload and launch configuration (graph of 10 steps),
    compared with the oracle over the first 20 steps in both forms."""
    s = make_system("h2_6000")
    n = 20
    a = pulse_samples(s)[:n]
    orc = Oracle(s)
    r = orc.run(a, s["dt"])
    for prec in ("fp64", "fp32"):
        ctx = Context(s, precision=prec, graph_steps=10)
        ctx.step(a)
        obs = ctx.observables()
        assert rel(obs["dmu"], r["dmu"]) < 1e-8
        assert rel(obs["j"], r["J"]) < 1e-10
        if prec == "fp64":
            compare_run(obs, r)
        else:
            assert rel(obs["energy"], r["E"]) < 1e-5
        ctx.close()


def test_tiled_series_with_ragged_row_tiles_and_k_points(monkeypatch):
    """The row-tile form of the Chebyshev series (forced): 61 rows (a ragged
    last tile of 5), 33 states (a ragged column set), four k-points of ragged
    N_basis; FP64 form, compared with the oracle over 20 steps."""
    monkeypatch.setenv("RTTDDFT_CHEB_TILE", "1")
    cfg = tiny_config(name="tile", n_g=0, n_atoms=2, lmax=1, n_lo_per_atom=2, n_s=33, n_aux=61,
                      n_k=4, kgrid=(2, 2, 1), n_b_range=(120, 150), seed=23, lattice="mos2",
                      edir=(1.0, 0.0, 0.0))
    s = make_system(cfg)
    a = pulse_samples(s, n_steps=20, a0=10.0)
    r = Oracle(s).run(a, s["dt"])
    ctx = Context(s, graph_steps=10)
    ctx.step(a)
    compare_run(ctx.observables(), r)
    ctx.close()


def test_potential_change_pattern_replaced_between_steps():
    """A potential change whose pattern changes during the run: ten steps
    with dV_1, then rttddft_set_dv with another pattern dV_2 and ten more
    steps.  The rebuild takes the pattern current at each step (nothing
    projected is cached), so theta after the twenty steps equals the
    oracle's run of the two halves with their own patterns (1e-9)."""
    s = make_system("tiny400")
    dv1, dv2 = make_dv(s), make_dv(s, seed_offset=7)
    a = pulse_samples(s, n_steps=20, a0=5.0)
    sc = dv_scale_samples(20, s["dt"])
    r1 = Oracle(s, dv=dv1).run(a[:10], s["dt"], dv_scale=sc[:10])
    r2 = Oracle(s, dv=dv2).run(a[10:], s["dt"], dv_scale=sc[10:], thetas=r1["theta"])
    ctx = Context(s)
    ctx.set_dv(dv1)
    ctx.step(a[:10], sc[:10])
    ctx.set_dv(dv2)
    ctx.step(a[10:], sc[10:])
    th = ctx.get_state(0)
    assert rel(th, r2["theta"][0]) < 1e-9
    # and the second pattern mattered: keeping dV_1 for all twenty steps ends elsewhere
    r_same = Oracle(s, dv=dv1).run(a, s["dt"], dv_scale=sc)
    assert rel(r_same["theta"][0], r2["theta"][0]) > 1e-6
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_direct_sum_with_the_table_gathered_through_l2(prec, monkeypatch):
    """When the table window of a row tile does not fit in shared memory (G
    sets whose 128-row tiles span several planes of the table, e.g. the
    N_basis 25727 cell) the direct sum gathers V~ through L1/L2 into the
    interstitial buffer; forced here on the small system: the operator equals
    the explicit H X (1e-12 FP64, 1e-5 (|H||x|) FP32), with and without the
    potential change, and a 30-step run keeps the oracle's dipole (1e-8)."""
    monkeypatch.setenv("RTTDDFT_TOEP_GATHER", "1")
    rng = np.random.default_rng(12)
    a_vec = np.array([0.4, -0.9, 1.3])
    for s in (make_system("tiny400"), make_system(ragged_cfg())):
        dv = make_dv(s)
        ctx = Context(s, precision=prec)
        ctx.set_dv(dv)
        for k in range(int(s["n_k"])):
            ops = explicit_operators(s, k)
            nb = ops["nb"]
            x = rng.standard_normal((nb, 5)) + 1j * rng.standard_normal((nb, 5))
            for sdv in (0.0, 0.7):
                hx, sx = ctx.apply(k, x, a_vec, sdv)
                h = hamiltonian(ops, a_vec, s["c_light"], explicit_dv(s, k, dv), sdv)
                if prec == "fp64":
                    assert rel(hx, h @ x) < 1e-12, k
                    assert rel(sx, ops["S"] @ x) < 1e-12, k
                else:
                    assert np.max(np.abs(hx - h @ x) / (np.abs(h) @ np.abs(x))) < 1e-5, k
        ctx.close()
    s = make_system("tiny400")
    a = pulse_samples(s, n_steps=30, a0=5.0)
    r = Oracle(s).run(a, s["dt"])
    ctx = Context(s, precision=prec, graph_steps=10)
    ctx.step(a)
    obs = ctx.observables()
    assert rel(obs["dmu"], r["dmu"]) < 1e-8
    assert rel(obs["energy"], r["E"]) < (1e-10 if prec == "fp64" else 1e-5)
    ctx.close()
