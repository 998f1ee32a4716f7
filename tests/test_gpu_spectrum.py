"""The polarizability of Eq. polarizability (post-processing of the recorded
current) on the GPU against the oracle's transform, through the C ABI.

Both evaluate the same FP64 sums F(w) = dt sum_n f(t_n) e^{(i w - eta) t_n}
(the GPU in a fixed blocked order, sincos per sample), so they agree to
rounding: 1e-12 of the largest |F(w)| and of the largest |alpha|.
"""
import numpy as np
import pytest

from oracle import Oracle, polarizability
from paper_2403_04351_gb300 import Context, build
from paper_2403_04351_gb300.rttddft import rttddft_polarizability
from synth import make_system, pulse_samples

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    build()


def _close(a, b, tol):
    assert np.max(np.abs(a - b)) <= tol * max(float(np.max(np.abs(b))), 1e-300)


def test_polarizability_of_a_recorded_run():
    """The current recorded by the step (induced part: minus the oracle's
    field-free value) and E = -(1/c) dA/dt of the pulse at the record times."""
    s = make_system("tiny400")
    n = 200
    a = pulse_samples(s, n_steps=n, a0=5.0)
    ctx = Context(s, graph_steps=10)
    ctx.step(a)
    obs = ctx.observables()
    ctx.close()
    j_gs = Oracle(s).j_gs
    j_ind = obs["j"] - j_gs[None, :]
    dt = float(s["dt"])
    # A is held at its midpoint sample over each step: E at t_{k+1} from the
    # difference of consecutive samples
    a_prev = np.vstack([np.zeros((1, 3)), a[:-1]])
    e = -(a - a_prev) / (s["c_light"] * dt)
    w = np.linspace(0.05, 2.0, 40)
    al, jw, ew = rttddft_polarizability(dt, dt, j_ind, e, w, s["omega"], eta=0.01)
    al_o, jw_o, ew_o = polarizability(dt, dt, j_ind, e, w, s["omega"], eta=0.01)
    _close(jw, jw_o, 1e-12)
    _close(ew, ew_o, 1e-12)
    _close(al, al_o, 1e-12)


def test_polarizability_random_series_and_device_buffers():
    import torch
    rng = np.random.default_rng(5)
    n = 5000
    j = rng.standard_normal((n, 3))
    e = rng.standard_normal((n, 3))
    w = rng.uniform(0.01, 3.0, 64)
    al_o, jw_o, ew_o = polarizability(1.5, 0.02, j, e, w, 800.0, eta=0.003)
    al, jw, ew = rttddft_polarizability(1.5, 0.02, j, e, w, 800.0, eta=0.003)
    _close(jw, jw_o, 1e-12)
    _close(al, al_o, 1e-12)
    # device inputs and outputs
    dj = torch.from_numpy(j).cuda()
    de = torch.from_numpy(e).cuda()
    dw = torch.from_numpy(w).cuda()
    dal = torch.zeros((64, 3, 3), dtype=torch.complex128, device="cuda")
    from paper_2403_04351_gb300.rttddft import load_library, _ptr
    code = load_library().rttddft_polarizability(n, 1.5, 0.02, _ptr(dj), _ptr(de), 0.003, 64, _ptr(dw), 800.0,
                                                 None, None, _ptr(dal), None)
    assert code == 0
    torch.cuda.synchronize()
    _close(dal.cpu().numpy(), al_o, 1e-12)
