"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Every test here is CPU-only.  None of them re-types the oracle's formulas:
they check closed forms, an independent algorithm (FFT convolution, Pade
expm), invariants of the exact dynamics, or numbers printed in the paper.
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import (Oracle, critical_timestep, explicit_dv, explicit_operators,
                    full_basis_propagator, hamiltonian, interstitial_potential,
                    overall_speedup, polarizability, propagate_cn, propagate_exact, ritz_basis,
                    interstitial_density, hartree_table, mt_density)
from synth import make_dv, make_system, pulse_samples, tiny_config
from systems import free_electron_system, permutation_mt_system, plane_wave_basis

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def tiny():
    return make_system("tiny400")


@pytest.fixture(scope="module")
def tiny_oracle(tiny):
    return Oracle(tiny)


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


# ----------------------------------------------------------------- operators

def test_operators_hermitian_and_overlap_positive(tiny):
    ops = explicit_operators(tiny, 0)
    for m in [ops["S"], ops["H0"], *ops["P"]]:
        assert np.max(np.abs(m - m.conj().T)) < 1e-14 * max(1.0, np.max(np.abs(m)))
    assert np.min(np.linalg.eigvalsh(ops["S"])) > 0.1


def test_interstitial_sum_equals_fft_convolution(tiny):
    """Eq. v_interstitial: sum_G' V~_{G-G'} y_G' is a convolution; evaluate it
    by zero-padded FFTs (the paper's second route, Sec. 2) and compare."""
    g = tiny["g_int"][0].astype(np.int64)
    vt = tiny["vtab"]
    ext = (np.asarray(tiny["vt_dim"]) - 1) // 2
    rng = np.random.default_rng(0)
    y = rng.standard_normal(len(g)) + 1j * rng.standard_normal(len(g))
    lo = g.min(axis=0)
    span = g.max(axis=0) - lo
    n = [int(2 ** math.ceil(math.log2(3 * s + 2 * e + 2))) for s, e in zip(span, ext)]
    yg = np.zeros(n, dtype=np.complex128)
    yg[tuple((g - lo).T)] = y
    vg = np.zeros(n, dtype=np.complex128)
    r = [np.arange(-e, e + 1) % m for e, m in zip(ext, n)]
    vg[np.ix_(*r)] = vt
    conv = np.fft.ifftn(np.fft.fftn(vg) * np.fft.fftn(yg))
    direct = interstitial_potential(tiny["g_int"][0], tiny["vt_dim"], vt) @ y
    assert _rel(conv[tuple((g - lo).T)], direct) < 1e-12


def test_muffin_tin_blocks_land_on_matched_plane_waves():
    """With A_alpha[p, pi(p)] = d_p, (A^H h A)[pi(p), pi(q)] = conj(d_p) h_pq d_q
    and the LO coupling is conj(d_p) h[p, N_A + j] (Eq. v_MT, Appendix A)."""
    s, perm, d = permutation_mt_system()
    ops = explicit_operators(s, 0)
    ng = int(s["n_g"][0])
    na = int(s["n_a"][0])
    nlo = int(s["n_lo"][0])
    for atom in range(2):
        rows = np.arange(atom * na, (atom + 1) * na)
        pg = perm[rows]
        dd = d[rows]
        lo = ng + atom * nlo + np.arange(nlo)
        h = s["h"][atom]
        got = ops["H0"][np.ix_(pg, pg)]
        assert np.allclose(got, np.conj(dd)[:, None] * h[:na, :na] * dd[None, :], atol=1e-14)
        got = ops["H0"][np.ix_(pg, lo)]
        assert np.allclose(got, np.conj(dd)[:, None] * h[:na, na:], atol=1e-14)
        got = ops["H0"][np.ix_(lo, lo)]
        assert np.allclose(got, h[na:, na:], atol=1e-14)
        o = s["o"][atom]
        got = ops["S"][np.ix_(pg, pg)] - np.eye(na)
        assert np.allclose(got, np.conj(dd)[:, None] * o[:na, :na] * dd[None, :], atol=1e-14)
        for l in range(3):
            got = ops["P"][l][np.ix_(lo, pg)]
            assert np.allclose(got, s["p"][atom][l][na:, :na] * dd[None, :], atol=1e-14)


def test_free_electron_hamiltonian_is_shifted_kinetic_energy():
    """Velocity gauge with no potential: H(A) = |G+k+A/c|^2/2 exactly."""
    s = free_electron_system()
    ops = explicit_operators(s, 0)
    a = np.array([0.7, -1.3, 2.1])
    h = hamiltonian(ops, a, s["c_light"])
    expect = 0.5 * np.sum((s["gk"][0] + a / s["c_light"]) ** 2, axis=1)
    assert np.max(np.abs(h - np.diag(expect))) < 1e-14


def test_free_electron_current_energy_and_dipole_closed_form():
    """Plane waves stay eigenstates under a uniform A(t):
    J = -(1/Omega) sum_j f_j (G_j + k + A/c), E = sum_j f_j |G_j+k+A/c|^2/2,
    and dmu is the trapezoid integral of Omega*(J - J(0))."""
    s = free_electron_system(n_s=3)
    cc, eps, idx = plane_wave_basis(s, 8)
    orc = Oracle(s, aux_mode="given", caux=[cc], eps=[eps])
    a = pulse_samples(s, n_steps=40, dt=0.2, a0=3.0, omega=0.4, edir=(0.3, -0.2, 0.9))
    r = orc.run(a, 0.2)
    gocc = s["gk"][0][idx[:3]]
    f = s["occ"]
    c = s["c_light"]
    om = s["omega"]
    j_exp = -(1.0 / om) * (f @ gocc)[None, :] - (1.0 / om) * f.sum() * a / c
    assert _rel(r["J"], j_exp) < 1e-12
    assert _rel(r["J_full"], j_exp) < 1e-12
    e_exp = np.array([f @ (0.5 * np.sum((gocc + ak / c) ** 2, axis=1)) for ak in a])
    assert _rel(r["E"], e_exp) < 1e-12
    jind = -(1.0 / om) * f.sum() * a / c
    dmu = np.cumsum(om * 0.2 * 0.5 * (np.vstack([np.zeros(3), jind[:-1]]) + jind), axis=0)
    assert _rel(r["dmu"], dmu) < 1e-12


# ------------------------------------------------------------ Ritz subspace

def test_ritz_basis_orthonormal_diagonal_and_bounded_by_exact(tiny):
    ops = explicit_operators(tiny, 0)
    cc, eps = ritz_basis(ops, tiny["caux"][0])
    assert np.max(np.abs(cc.conj().T @ ops["S"] @ cc - np.eye(len(eps)))) < 1e-12
    assert np.max(np.abs(cc.conj().T @ ops["H0"] @ cc - np.diag(eps))) < 1e-12
    assert np.all(np.diff(eps) > 0)
    exact = sla.eigvalsh(ops["H0"], ops["S"])[:len(eps)]
    assert np.all(eps >= exact - 1e-12)          # Courant-Fischer bound
    sums = cc.sum(axis=0)
    assert np.max(np.abs(sums.imag)) < 1e-12 and np.all(sums.real > 0)


def test_complete_subspace_equals_full_basis_propagation():
    """N_aux = N_basis: the subspace step is the exact solution of
    S dC/dt = -i H C (Eq. evolution_wf_coeff) with H held per step."""
    s = make_system(tiny_config(n_g=24, n_atoms=2, lmax=1, n_lo_per_atom=2, n_s=3,
                                seed=21))
    orc = Oracle(s)
    ops = explicit_operators(s, 0)
    a = pulse_samples(s, n_steps=6, dt=0.3, a0=20.0, omega=0.5, edir=(0.2, 0.5, 0.8))
    r = orc.run(a, 0.3)
    c = orc.kp[0]["caux"] @ orc.kp[0]["theta0"]
    for k in range(6):
        c = full_basis_propagator(ops, a[k], s["c_light"], 0.3) @ c
    assert _rel(r["C"][0], c) < 1e-11


def test_excited_electrons_match_full_basis_projection():
    """N_exc = N_e - sum_j f_j sum_{i < N_s} |<phi_i(0)| S |psi_j(t)>|^2 from an
    independent route: brute-force full-basis propagation and the occupied
    generalized eigenvectors of (H0, S) from LAPACK, in a complete subspace;
    zero when no field acts."""
    s = make_system(tiny_config(n_g=24, n_atoms=2, lmax=1, n_lo_per_atom=2, n_s=3,
                                seed=21))
    orc = Oracle(s)
    ops = explicit_operators(s, 0)
    still = orc.run(np.zeros((8, 3)), 0.3)
    assert np.max(np.abs(still["n_exc"])) < 1e-13
    a = pulse_samples(s, n_steps=6, dt=0.3, a0=20.0, omega=0.5, edir=(0.2, 0.5, 0.8))
    r = orc.run(a, 0.3)
    h0 = hamiltonian(ops, np.zeros(3), s["c_light"])
    w, phi = sla.eigh(h0, ops["S"])
    occ = np.asarray(s["occ"])
    ns = int(s["n_s"])
    c = orc.kp[0]["caux"] @ orc.kp[0]["theta0"]
    assert r["n_exc"].min() > 0.0
    for k in range(6):
        c = full_basis_propagator(ops, a[k], s["c_light"], 0.3) @ c
        ov = phi[:, :ns].conj().T @ ops["S"] @ c
        brute = float(np.sum(occ)) - float(np.sum(occ[None, :] * np.abs(ov) ** 2))
        assert abs(r["n_exc"][k] - brute) < 1e-11


def test_excited_electrons_are_second_order_in_a_weak_field(tiny_oracle, tiny):
    n1 = tiny_oracle.run(pulse_samples(tiny, n_steps=100, a0=5e-3), 0.1)["n_exc"][-1]
    n2 = tiny_oracle.run(pulse_samples(tiny, n_steps=100, a0=1e-2), 0.1)["n_exc"][-1]
    assert n1 > 0.0
    assert abs(n2 / n1 - 4.0) < 1e-3


# -------------------------------------------------------------- propagators

def test_exact_propagator_matches_pade_expm_and_two_level_closed_form():
    rng = np.random.default_rng(3)
    n = 32
    x = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    h = 0.5 * (x + x.conj().T)
    y = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    sm = np.eye(n) + 0.05 * (y @ y.conj().T) / n
    th = rng.standard_normal((n, 4)) + 1j * rng.standard_normal((n, 4))
    out, _ = propagate_exact(h, np.eye(n), th, 0.37)
    assert _rel(out, sla.expm(-0.37j * h) @ th) < 1e-12
    out, _ = propagate_exact(h, sm, th, 0.37)
    assert _rel(out, sla.expm(-0.37j * np.linalg.solve(sm, h)) @ th) < 1e-11
    # two-level system: exp(-iHt) = e^{-i m t}(cos(w t) - i sin(w t)/w (H - m))
    a_, d_, b_ = 0.3, -0.8, 0.25 + 0.4j
    h2 = np.array([[a_, b_], [np.conj(b_), d_]])
    m = 0.5 * (a_ + d_)
    w = math.sqrt((0.5 * (a_ - d_)) ** 2 + abs(b_) ** 2)
    t = 1.7
    u = np.exp(-1j * m * t) * (math.cos(w * t) * np.eye(2)
                               - 1j * math.sin(w * t) / w * (h2 - m * np.eye(2)))
    out, lam = propagate_exact(h2, np.eye(2), np.eye(2), t)
    assert np.max(np.abs(out - u)) < 1e-14
    assert abs(critical_timestep(lam) - 0.2 / (2 * w)) < 1e-14


def test_crank_nicolson_is_second_order(tiny_oracle, tiny):
    a = np.tile(np.array([[0.0, 0.0, 20.0]]), (1, 1))
    errs = []
    for dt in (0.2, 0.1, 0.05):
        n = int(round(4.0 / dt))
        aa = np.repeat(a, n, axis=0)
        ex = tiny_oracle.run(aa, dt, propagator="exact")["theta"][0]
        cn = tiny_oracle.run(aa, dt, propagator="cn")["theta"][0]
        errs.append(np.max(np.abs(cn - ex)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.8 < r1 < 4.2 and 3.8 < r2 < 4.2


# ---------------------------------------------------------------- dynamics

def test_field_free_ground_state_only_gains_phase(tiny_oracle, tiny):
    n, dt = 50, 0.1
    r = tiny_oracle.run(np.zeros((n, 3)), dt)
    eps = tiny_oracle.kp[0]["eps"]
    t = n * dt
    expect = np.zeros_like(r["theta"][0])
    ns = tiny["n_s"]
    expect[np.arange(ns), np.arange(ns)] = np.exp(-1j * eps[:ns] * t)
    assert np.max(np.abs(r["theta"][0] - expect)) < 1e-12
    assert np.max(np.abs(r["dmu"])) < 1e-13
    assert np.max(np.abs(r["J"] - tiny_oracle.j_gs)) < 1e-15


def test_norm_conserved_and_projection_consistent(tiny_oracle, tiny):
    a = pulse_samples(tiny, a0=5.0)
    r = tiny_oracle.run(a, tiny["dt"])
    assert r["norm_dev"].max() < 1e-10
    assert r["resid"].max() < 1e-12
    assert _rel(r["J"], r["J_full"]) < 1e-11


def test_energy_conserved_for_static_field(tiny_oracle):
    a = np.repeat(np.array([[3.0, -2.0, 5.0]]), 100, axis=0)
    r = tiny_oracle.run(a, 0.1)
    assert np.max(np.abs(r["E"] - r["E"][0])) < 1e-10 * abs(r["E"][0])


def test_discrete_work_theorem_links_energy_and_current(tiny_oracle, tiny):
    """For piecewise-constant A the exact step conserves <H(A_k)>, so
    E(t_{k+1}) - E(t_k) = -(Omega/c) (A_k - A_{k-1}).J(t_k)
                          + N_e |A_k - A_{k-1}|^2 / (2 c^2)
    (velocity gauge: dH/dA = (P + (A/c) S)/c, J = -(1/Omega) sum f <P + A/c>)."""
    a = pulse_samples(tiny, n_steps=60, dt=0.1, a0=40.0, omega=0.8,
                      edir=(0.5, 0.3, 0.8))
    r = tiny_oracle.run(a, 0.1)
    c = tiny["c_light"]
    om = tiny["omega"]
    ne = float(np.sum(tiny["occ"]))
    e_prev = tiny_oracle.energy([tiny_oracle.kp[0]["theta0"]], np.zeros(3))
    j_prev = tiny_oracle.j_gs
    a_prev = np.zeros(3)
    for k in range(len(a)):
        da = a[k] - a_prev
        pred = e_prev - (om / c) * da @ j_prev + ne * (da @ da) / (2 * c * c)
        assert abs(r["E"][k] - pred) < 1e-12 * max(1.0, abs(pred))
        e_prev, j_prev, a_prev = r["E"][k], r["J_full"][k], a[k]


def test_time_reversal_returns_to_start(tiny_oracle, tiny):
    a = pulse_samples(tiny, n_steps=80, dt=0.1, a0=30.0)
    fwd = tiny_oracle.run(a, 0.1)
    back = tiny_oracle.run(a[::-1], -0.1, thetas=fwd["theta"])
    assert np.max(np.abs(back["theta"][0] - tiny_oracle.kp[0]["theta0"])) < 1e-12


def test_dipole_is_linear_in_weak_field(tiny_oracle, tiny):
    r1 = tiny_oracle.run(pulse_samples(tiny, n_steps=100, a0=1e-4), 0.1)["dmu"][-1]
    r2 = tiny_oracle.run(pulse_samples(tiny, n_steps=100, a0=2e-4), 0.1)["dmu"][-1]
    assert np.max(np.abs(r2 - 2 * r1)) < 1e-4 * np.max(np.abs(r2))


def test_multi_k_totals_are_weighted_sums():
    cfg = tiny_config(n_g=30, n_atoms=2, lmax=1, n_lo_per_atom=2, n_s=2, n_aux=12,
                      n_k=4, kgrid=(2, 2, 1), n_b_range=(30, 40), seed=9)
    s = make_system(cfg)
    a = pulse_samples(s, n_steps=10, dt=0.2, a0=10.0)
    full = Oracle(s).run(a, 0.2)
    parts = [Oracle(make_system(cfg, k_subset=[k])) for k in range(4)]
    for p in parts:
        p.wk = np.array([0.25])
        p.j_gs = p._current_full([p.kp[0]["caux"] @ p.kp[0]["theta0"]], np.zeros(3))
    runs = [p.run(a, 0.2) for p in parts]
    assert _rel(full["J"], sum(r["J"] for r in runs)) < 1e-12
    assert _rel(full["E"], sum(r["E"] for r in runs)) < 1e-12
    assert _rel(full["dmu"], sum(r["dmu"] for r in runs)) < 1e-12


# ------------------------------------------------------------ potential change

def test_potential_change_four_block_form_matches_explicit(tiny):
    """Eq. v_MT: CC^H dV CC = R^H dV_LL R + R^H dV_Ll CC_l + CC_l^H dV_lL R
    + CC_l^H dV_ll CC_l (R = A CC_L), plus Eq. v_interstitial."""
    dv = make_dv(tiny)
    ops = explicit_operators(tiny, 0)
    cc, _ = ritz_basis(ops, tiny["caux"][0])
    dense = cc.conj().T @ explicit_dv(tiny, 0, dv) @ cc
    ng = int(tiny["n_g"][0])
    na = int(tiny["n_a"][0])
    nlo = int(tiny["n_lo"][0])
    cl = cc[:ng]
    four = cl.conj().T @ interstitial_potential(tiny["g_int"][0], tiny["vt_dim"],
                                                dv["dvtab"]) @ cl
    for a in range(2):
        r = tiny["amat"][0][a * na:(a + 1) * na] @ cl
        cle = cc[ng + a * nlo: ng + (a + 1) * nlo]
        d = dv["dh"][a]
        four += r.conj().T @ d[:na, :na] @ r + r.conj().T @ d[:na, na:] @ cle \
            + cle.conj().T @ d[na:, :na] @ r + cle.conj().T @ d[na:, na:] @ cle
    assert _rel(four, dense) < 1e-12


def test_potential_change_enters_as_hermitian_perturbation(tiny):
    dv = make_dv(tiny)
    m = explicit_dv(tiny, 0, dv)
    assert np.max(np.abs(m - m.conj().T)) < 1e-15
    orc = Oracle(tiny, dv=dv)
    scale = np.full(40, 0.7)
    r = orc.run(np.zeros((40, 3)), 0.1, dv_scale=scale)
    assert r["norm_dev"].max() < 1e-10
    assert np.max(np.abs(r["E"] - r["E"][0])) < 1e-10 * abs(r["E"][0])


# ---------------------------------------------------------------- gradient

def test_tangent_gradient_matches_central_differences():
    s = make_system(tiny_config(n_g=40, n_atoms=2, lmax=1, n_lo_per_atom=2, n_s=2,
                                n_aux=10, seed=13))
    orc = Oracle(s)
    n, dt = 25, 0.2
    a = pulse_samples(s, n_steps=n, dt=dt, a0=30.0, omega=0.6, edir=(0.2, 0.4, 0.9))
    g = np.array([0.3, -0.5, 0.8])
    seeds = [(0, 2), (7, 0), (12, 1), (24, 2)]
    grad = orc.dipole_gradient(a, dt, g, seeds)
    h = 1e-4
    for (k, l), gv in zip(seeds, grad):
        ap = a.copy()
        am = a.copy()
        ap[k, l] += h
        am[k, l] -= h
        fd = (g @ orc.run(ap, dt)["dmu"][-1] - g @ orc.run(am, dt)["dmu"][-1]) / (2 * h)
        assert abs(gv - fd) < 1e-7 * max(abs(fd), 1e-3)


# --------------------------------------------------------- paper's printed table

def test_overall_speedups_of_table_h2():
    """Table tab:H2: the printed overall speed-ups follow from the printed
    times per step and dt_cr by the time needed to cover 1 a.u."""
    rows = np.loadtxt(os.path.join(HERE, "golden", "paper_table_h2.txt"))
    # the printed inputs are rounded to their last digit: propagate half a unit
    ref_tol = 0.05 / 139.0 + 0.00005 / 0.0012
    for n_empty, t_mm, t_fft, dtcr, s_mm, s_fft in rows:
        for t, s in ((t_mm, s_mm), (t_fft, s_fft)):
            tol = ref_tol + 0.05 / t + 0.005 / dtcr
            got = overall_speedup(t, dtcr, 139.0, 0.0012)
            assert abs(got - s) <= tol * s + 0.5
            # the inverse reading (time x step length) is far off
            assert abs(139.0 * 0.0012 / (t * dtcr) - s) > 0.5 * s


# --------------------------------------------------------------- spectrum

def test_damped_transform_of_a_cosine_is_a_geometric_series():
    """F(w) = dt sum_n cos(w0 t_n) e^{(i w - eta) t_n} in closed form:
    (dt/2) sum_pm e^{z t0} (1 - e^{z N dt}) / (1 - e^{z dt}), z = i(w pm w0) - eta."""
    t0, dt, n, w0, eta = 0.2, 0.05, 3000, 0.7, 0.01
    t = t0 + dt * np.arange(n)
    f = np.stack([np.cos(w0 * t), 2.0 * np.cos(w0 * t), np.zeros(n)], axis=1)
    e = np.ones((n, 3))
    w = np.array([0.3, 0.69, 1.4])
    _, jw, _ = polarizability(t0, dt, f, e, w, 1.0, eta=eta)
    expect = np.zeros(w.size, dtype=complex)
    for sgn in (1.0, -1.0):
        z = 1j * (w + sgn * w0) - eta
        expect += 0.5 * dt * np.exp(z * t0) * (1 - np.exp(z * n * dt)) / (1 - np.exp(z * dt))
    assert np.max(np.abs(jw[:, 0] - expect)) < 1e-12 * np.max(np.abs(expect))
    assert np.max(np.abs(jw[:, 1] - 2 * expect)) < 1e-12 * np.max(np.abs(expect))
    assert np.all(jw[:, 2] == 0)


def test_polarizability_of_a_proportional_response():
    """J_l(t) = kappa_l E_l(t) gives alpha_ll = i Omega kappa_l / w and
    alpha_{l l'} = (i Omega / w) kappa_l E_l(w) / E_l'(w); a zero field
    component leaves its column at 0."""
    rng = np.random.default_rng(2)
    n = 500
    e = rng.standard_normal((n, 3))
    e[:, 2] = 0.0
    kappa = np.array([0.3, -1.2, 0.5])
    j = e * kappa[None, :]
    w = np.array([0.1, 0.5, 2.0])
    om = 123.0
    al, jw, ew = polarizability(0.0, 0.1, j, e, w, om, eta=0.02)
    for l in range(2):
        assert np.max(np.abs(al[:, l, l] - 1j * om * kappa[l] / w)) < 1e-12 * om / w.min()
    assert np.max(np.abs(al[:, 0, 1] - 1j * om / w * kappa[0] * ew[:, 0] / ew[:, 1])) < 1e-9
    assert np.all(al[:, :, 2] == 0)


# ------------------------------------------------------- Hartree feedback

def test_interstitial_density_equals_fft_of_the_squared_orbitals(tiny, tiny_oracle):
    """n_g from the explicit autocorrelation of the plane-wave coefficients
    equals |psi(r)|^2 summed on a real-space grid and taken back to G space by
    numpy's FFT (grid wider than the table box, so nothing aliases)."""
    rng = np.random.default_rng(4)
    ng = int(tiny["n_g"][0])
    nb = ng + int(np.sum(tiny["n_lo"]))
    c = rng.standard_normal((nb, 3)) + 1j * rng.standard_normal((nb, 3))
    occ = np.array([2.0, 1.0, 0.5])
    n = interstitial_density(tiny, [c], occ, np.array([1.0]), tiny["omega"])
    dim = np.asarray(tiny["vt_dim"])
    e = (dim - 1) // 2
    F = dim + 3
    gi = np.asarray(tiny["g_int"][0])
    dens = np.zeros(tuple(F))
    for j in range(3):
        grid = np.zeros(tuple(F), dtype=np.complex128)
        grid[gi[:, 0] % F[0], gi[:, 1] % F[1], gi[:, 2] % F[2]] = c[:ng, j]
        psi = np.fft.ifftn(grid) * np.prod(F)       # sum_G C_G e^{+2 pi i G.r/F}
        dens += occ[j] * np.abs(psi) ** 2
    ng_fft = np.fft.fftn(dens) / np.prod(F) / tiny["omega"]
    r = [np.arange(-x, x + 1) for x in e]
    d1, d2, d3 = np.meshgrid(r[0], r[1], r[2], indexing="ij")
    ref = ng_fft[d1 % F[0], d2 % F[1], d3 % F[2]]
    assert _rel(n, ref) < 1e-12
    # the density is real: n_{-g} = conj(n_g)
    assert np.max(np.abs(n - np.conj(n[::-1, ::-1, ::-1]))) < 1e-15 * np.max(np.abs(n))


def test_hartree_potential_has_positive_energy_and_zero_mean(tiny):
    rng = np.random.default_rng(6)
    dim = tuple(int(x) for x in tiny["vt_dim"])
    z = rng.standard_normal(dim) + 1j * rng.standard_normal(dim)
    dn = 0.5 * (z + np.conj(z[::-1, ::-1, ::-1]))  # a real density change
    dv = hartree_table(tiny, dn, np.zeros(dim))
    e = [(x - 1) // 2 for x in dim]
    assert dv[e[0], e[1], e[2]] == 0.0
    # E_H = (Omega/2) sum_g dV_g conj(dn_g) = (Omega/2) sum_g 4 pi |dn_g|^2/|g|^2 > 0
    eh = 0.5 * tiny["omega"] * np.sum(dv * np.conj(dn))
    assert abs(eh.imag) < 1e-12 * abs(eh.real) and eh.real > 0
    # the potential of a real density is real in space: dV_{-g} = conj(dV_g)
    assert np.max(np.abs(dv - np.conj(dv[::-1, ::-1, ::-1]))) < 1e-15 * np.max(np.abs(dv))


def test_hartree_feedback_is_inert_without_field_and_keeps_the_norm(tiny_oracle, tiny):
    still = tiny_oracle.run(np.zeros((12, 3)), 0.1, hartree=True)
    plain = tiny_oracle.run(np.zeros((12, 3)), 0.1)
    assert np.max(np.abs(still["theta"][0] - plain["theta"][0])) < 1e-13
    a = pulse_samples(tiny, n_steps=20, a0=20.0)
    r = tiny_oracle.run(a, tiny["dt"], hartree=True)
    assert r["norm_dev"].max() < 1e-10
    assert r["resid"].max() < 1e-12
    r0 = tiny_oracle.run(a, tiny["dt"])
    assert np.max(np.abs(r["dmu"] - r0["dmu"])) > 1e-6 * np.max(np.abs(r0["dmu"]))


def test_hartree_potential_of_a_single_plane_wave_density():
    """A density change cos(g0 . r) (n_{+-g0} = 1/2) has the Hartree potential
    (4 pi / |g0|^2) cos(g0 . r): with |g0| from the real-space cell (b = 2 pi
    A^-T) of a hexagonal cell, where rows and columns of the reciprocal matrix
    differ, independently of the system's stored reciprocal vectors."""
    tiny = make_system(tiny_config(name="hex", n_g=30, n_atoms=1, lmax=1, n_lo_per_atom=1, n_s=1, n_aux=4,
                                   seed=2, lattice="mos2"))
    dim = tuple(int(x) for x in tiny["vt_dim"])
    e = np.array([(x - 1) // 2 for x in dim])
    b = 2 * math.pi * np.linalg.inv(np.asarray(tiny["lattice"])).T  # rows b_i
    assert abs(b[0] @ b[1]) > 1e-3  # a non-orthogonal pair
    for g0 in ([1, 0, 0], [1, 1, 0], [1, -1, 1]):
        g0 = np.array(g0)
        assert np.all(np.abs(g0) <= e)  # inside the table box
        dn = np.zeros(dim, dtype=np.complex128)
        dn[tuple(e + g0)] = 0.5
        dn[tuple(e - g0)] = 0.5
        dv = hartree_table(tiny, dn, np.zeros(dim))
        gc = g0 @ b
        expect = 4 * math.pi / float(gc @ gc) * 0.5
        assert abs(dv[tuple(e + g0)] - expect) < 1e-14 * expect
        assert abs(dv[tuple(e - g0)] - expect) < 1e-14 * expect
        mask = np.ones(dim, dtype=bool)
        mask[tuple(e + g0)] = mask[tuple(e - g0)] = False
        assert np.max(np.abs(dv[mask])) == 0.0


# ------------------------------------------------ muffin-tin density feedback

def test_muffin_tin_density_of_phased_unit_rows():
    """With A_alpha[p, pi(p)] = d_p every matching channel p of an atom reads
    one plane-wave coefficient, v_p = d_p c_pi(p), and the local-orbital
    channels read the LO rows: n_a[p, q] = sum_j f_j v_p conj(v_q), written
    here entry by entry from the coefficients (no embedding matrix)."""
    s, perm, d = permutation_mt_system()
    ng = int(s["n_g"][0])
    na = int(s["n_a"][0])
    nlo = int(s["n_lo"][0])
    nb = ng + 2 * nlo
    rng = np.random.default_rng(21)
    c = rng.standard_normal((nb, 3)) + 1j * rng.standard_normal((nb, 3))
    occ = np.array([2.0, 1.5, 0.25])
    n = mt_density(s, [c], occ, np.array([0.5]))
    for atom in range(2):
        m = na + nlo
        ref = np.zeros((m, m), dtype=np.complex128)
        for p in range(m):
            for q in range(m):
                for j in range(3):
                    vp = d[atom * na + p] * c[perm[atom * na + p], j] if p < na else c[ng + atom * nlo + p - na, j]
                    vq = d[atom * na + q] * c[perm[atom * na + q], j] if q < na else c[ng + atom * nlo + q - na, j]
                    ref[p, q] += 0.5 * occ[j] * vp * np.conj(vq)
        assert _rel(n[atom], ref) < 1e-14
        assert np.max(np.abs(n[atom] - n[atom].conj().T)) < 1e-15 * np.max(np.abs(ref))


def test_muffin_tin_feedback_inert_without_field_effective_with_one(tiny_oracle, tiny):
    """The ground state keeps its muffin-tin density (only phases change), so
    the contact feedback does nothing without a field; with a pulse it changes
    the dipole, and the run keeps the norm."""
    still = tiny_oracle.run(np.zeros((10, 3)), 0.1, hartree=True, mt_u=0.5)
    plain = tiny_oracle.run(np.zeros((10, 3)), 0.1)
    assert np.max(np.abs(still["theta"][0] - plain["theta"][0])) < 1e-13
    a = pulse_samples(tiny, n_steps=20, a0=20.0)
    r_mt = tiny_oracle.run(a, tiny["dt"], hartree=True, mt_u=0.5)
    r_i = tiny_oracle.run(a, tiny["dt"], hartree=True)
    assert r_mt["norm_dev"].max() < 1e-10
    assert np.max(np.abs(r_mt["dmu"] - r_i["dmu"])) > 1e-6 * np.max(np.abs(r_i["dmu"]))


def test_muffin_tin_potential_lands_on_matched_plane_waves():
    """The feedback's potential matrix for a state with a muffin-tin density
    change: its blocks sit on the matched plane waves exactly as Eq. v_MT
    places h (conj(d_p) dh_pq d_q on (pi(p), pi(q))), with dh = U (n - n0)."""
    from oracle.rttddft_oracle import Oracle
    s, perm, d = permutation_mt_system()
    ng = int(s["n_g"][0])
    na = int(s["n_a"][0])
    nlo = int(s["n_lo"][0])
    orc = Oracle(s)
    th0 = [kp["theta0"] for kp in orc.kp]
    rng = np.random.default_rng(5)
    th1 = [t + 0.1 * (rng.standard_normal(t.shape) + 1j * rng.standard_normal(t.shape)) for t in th0]
    cs0 = [kp["caux"] @ t for kp, t in zip(orc.kp, th0)]
    cs1 = [kp["caux"] @ t for kp, t in zip(orc.kp, th1)]
    n0 = interstitial_density(s, cs0, orc.occ, orc.wk, orc.omega)
    mt0 = mt_density(s, cs0, orc.occ, orc.wk)
    mt1 = mt_density(s, cs1, orc.occ, orc.wk)
    u = 0.7
    vh, _ = orc.hartree_matrices(th1, n0, mt0, u)
    vi, _ = orc.hartree_matrices(th1, n0)
    vmt = vh[0] - vi[0]
    for atom in range(2):
        rows = np.arange(atom * na, (atom + 1) * na)
        pg, dd = perm[rows], d[rows]
        lo = ng + atom * nlo + np.arange(nlo)
        dh = u * (mt1[atom] - mt0[atom])
        assert np.allclose(vmt[np.ix_(pg, pg)], np.conj(dd)[:, None] * dh[:na, :na] * dd[None, :], atol=1e-14)
        assert np.allclose(vmt[np.ix_(pg, lo)], np.conj(dd)[:, None] * dh[:na, na:], atol=1e-14)
        assert np.allclose(vmt[np.ix_(lo, lo)], dh[na:, na:], atol=1e-14)
