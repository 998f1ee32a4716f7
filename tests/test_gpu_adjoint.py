"""Adjoint of the step (reverse mode through the Chebyshev polynomial) against
the oracle's tangent-linear gradient (Daleckii-Krein divided differences of
the exact exponential) and against central differences of the CUDA path."""
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


def small_system():
    return make_system(tiny_config(n_g=40, n_atoms=2, lmax=1, n_lo_per_atom=2, n_s=2, n_aux=10,
                                   seed=13))


def test_adjoint_equals_oracle_tangent_gradient_for_every_sample():
    s = small_system()
    n, dt = 25, 0.2
    a = pulse_samples(s, n_steps=n, dt=dt, a0=30.0, omega=0.6, edir=(0.2, 0.4, 0.9))
    g = np.array([0.3, -0.5, 0.8])
    ctx = Context(s, dt=dt)
    grad, dmu = ctx.adjoint(a, g, ckpt_every=7)
    orc = Oracle(s)
    seeds = [(k, l) for k in range(n) for l in range(3)]
    ref = orc.dipole_gradient(a, dt, g, seeds).reshape(n, 3)
    assert np.max(np.abs(grad - ref)) < 1e-9 * np.max(np.abs(ref))
    r = orc.run(a, dt)
    assert np.max(np.abs(dmu - r["dmu"][-1])) < 1e-9 * np.max(np.abs(r["dmu"][-1]))
    ctx.close()


def test_adjoint_matches_central_differences_and_leaves_state():
    s = small_system()
    n, dt, h = 20, 0.2, 1e-6
    a = pulse_samples(s, n_steps=n, dt=dt, a0=30.0, omega=0.6, edir=(0.0, 0.0, 1.0))
    g = np.array([0.0, 0.0, 1.0])
    ctx = Context(s, dt=dt)
    ctx.step(a[:5])
    ctx.observables(clear=True)
    th0 = ctx.get_state(0)
    info0 = ctx.info()
    grad, _ = ctx.adjoint(a[5:], g, ckpt_every=4)
    assert np.array_equal(ctx.get_state(0), th0)
    assert ctx.info()["steps_done"] == info0["steps_done"]
    ctx.close()

    def dmu_end(aa):
        c = Context(s, dt=dt)
        c.step(aa)
        d = c.observables()["dmu"]
        c.close()
        return g @ (d[-1] - d[4])

    rng = np.random.default_rng(2)
    for kk in rng.choice(n - 5, size=4, replace=False):
        ap, am = a.copy(), a.copy()
        ap[5 + kk, 2] += h
        am[5 + kk, 2] -= h
        fd = (dmu_end(ap) - dmu_end(am)) / (2 * h)
        assert abs(grad[kk, 2] - fd) < 1e-6 * max(abs(fd), 1e-3 * np.max(np.abs(grad)))


def test_adjoint_requires_the_chebyshev_propagator():
    s = small_system()
    ctx = Context(s, propagator="eig")
    with pytest.raises(RttddftError) as e:
        ctx.adjoint(pulse_samples(s, n_steps=3), np.array([0, 0, 1.0]))
    assert e.value.code == -9
    ctx.close()


def test_adjoint_workload_h2_6000_400_steps_sampled():
    """The adjoint workload: the H2-like system over 400 steps, FP64,
    theta checkpointed every 50 steps; 10 random samples against central
    differences (h = 1e-6) of the CUDA path and against the oracle's
    tangent-linear gradient."""
    s = make_system("h2_6000_adj")
    n = 400
    a = pulse_samples(s, n_steps=n)
    g = np.array([0.0, 0.0, 1.0])
    ctx = Context(s, max_record=n + 8)
    grad, dmu = ctx.adjoint(a, g, ckpt_every=50)
    ctx.close()
    rng = np.random.default_rng(5)
    picks = sorted(rng.choice(n, size=10, replace=False).tolist())
    h = 1e-6

    def dmu_end(aa):
        c = Context(s, max_record=n + 8)
        c.step(aa)
        d = c.observables()["dmu"][-1]
        c.close()
        return g @ d

    # Central differences are limited by round-off here: dmu(T) sums 400 values of
    # J_ind = J - J(t0), a small difference of nearly equal currents, so dmu carries
    # an absolute error of ~1e-14 and the h = 1e-6 quotient ~1e-14/1e-6 = 1e-8,
    # about 2e-6 of the gradient.  h = 1e-6 is checked at 3e-6, h = 1e-5 at 1e-6.
    # Every one of the 10 samples at both step sizes.
    scale = np.max(np.abs(grad[:, 2]))
    for kk in picks:
        for hh, tol in ((h, 3e-6), (1e-5, 1e-6)):
            ap, am = a.copy(), a.copy()
            ap[kk, 2] += hh
            am[kk, 2] -= hh
            fd = (dmu_end(ap) - dmu_end(am)) / (2 * hh)
            assert abs(grad[kk, 2] - fd) < tol * max(abs(fd), 1e-2 * scale), (kk, hh, grad[kk, 2], fd)
    ref = Oracle(s).dipole_gradient(a, s["dt"], g, [(kk, 2) for kk in picks])
    assert np.max(np.abs(grad[picks, 2] - ref)) < 1e-9 * max(np.max(np.abs(ref)), 1e-12)


def test_autograd_function_gives_the_adjoint_gradient():
    """dipole_increment (a torch.autograd.Function over rttddft_adjoint): its
    value is the oracle's dipole after the run, and loss.backward() with
    loss = g . dmu gives the adjoint's gradient for direction g."""
    import torch
    from paper_2403_04351_gb300 import dipole_increment
    s = small_system()
    n, dt = 25, 0.2
    a = pulse_samples(s, n_steps=n, dt=dt, a0=30.0, omega=0.6, edir=(0.2, 0.4, 0.9))
    g = np.array([0.3, -0.5, 0.8])
    ctx = Context(s, dt=dt)
    at = torch.tensor(a, dtype=torch.float64, requires_grad=True)
    dmu = dipole_increment(at, ctx, ckpt_every=7)
    r = Oracle(s).run(a, dt)
    assert np.max(np.abs(dmu.detach().numpy() - r["dmu"][-1])) < 1e-9 * np.max(np.abs(r["dmu"][-1]))
    loss = (dmu * torch.tensor(g, dtype=torch.float64)).sum()
    loss.backward()
    grad, _ = ctx.adjoint(a, g, ckpt_every=7)
    assert np.max(np.abs(at.grad.numpy() - grad)) <= 1e-13 * np.max(np.abs(grad))
    ctx.close()
