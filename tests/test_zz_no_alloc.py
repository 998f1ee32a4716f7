"""rttddft_apply_noalloc: the operator apply for callers that cannot allocate
device memory (its scratch is a static device array) gives the same H X and
S X as rttddft_apply.  Collected last so that a failure here comes after all
other tests have run."""
import numpy as np
import pytest

from paper_2403_04351_gb300 import Context, RttddftError, build, rttddft
from synth import make_dv, make_system, tiny_config

pytestmark = pytest.mark.gpu


def _device_block(torch, x):
    # column-major N_basis x ncols on the device = row-major ncols x N_basis
    return torch.from_numpy(np.ascontiguousarray(x.T)).cuda()


def test_noalloc_apply_matches_apply_on_two_calls():
    import torch
    assert torch.cuda.is_available()
    build()
    s = make_system("tiny400")
    dv = make_dv(s)
    ctx = Context(s)
    ctx.set_dv(dv)
    nb = int(s["n_g"][0]) + int(np.sum(s["n_lo"]))
    rng = np.random.default_rng(7)
    for call, (ncols, a_vec, sdv) in enumerate([(11, (0.4, -1.2, 2.0), 0.0),
                                               (5, (3.0, 0.5, -0.7), 0.6)]):
        x = rng.standard_normal((nb, ncols)) + 1j * rng.standard_normal((nb, ncols))
        hx_ref, sx_ref = ctx.apply(0, x, a_vec, sdv)
        dx = _device_block(torch, x)
        dh = torch.empty_like(dx)
        ds = torch.empty_like(dx)
        av = np.ascontiguousarray(a_vec, dtype=np.float64)
        rttddft.rttddft_apply_noalloc(ctx.ctx, 0, ncols, dx, av, sdv, dh, ds)
        torch.cuda.synchronize()
        hx = dh.cpu().numpy().T
        sxv = ds.cpu().numpy().T
        scale_h = np.max(np.abs(hx_ref))
        scale_s = np.max(np.abs(sx_ref))
        assert np.max(np.abs(hx - hx_ref)) <= 1e-12 * scale_h, call
        assert np.max(np.abs(sxv - sx_ref)) <= 1e-12 * scale_s, call
    ctx.close()


def test_noalloc_apply_rejects_host_pointers_and_oversized_blocks():
    import torch
    build()
    s = make_system(tiny_config(n_g=40, n_atoms=2, lmax=1, n_lo_per_atom=2, n_s=2, n_aux=8, seed=3))
    ctx = Context(s)
    nb = int(s["n_g"][0]) + 4
    x = np.zeros((nb, 2), dtype=np.complex128, order="F")
    with pytest.raises(RttddftError) as e:
        rttddft.rttddft_apply_noalloc(ctx.ctx, 0, 2, x, np.zeros(3), 0.0, x.copy(), x.copy())
    assert e.value.code == -1 and "device pointers" in str(e.value)
    ctx.close()
    big = make_system(tiny_config(n_g=12000, n_atoms=2, lmax=2, n_lo_per_atom=2, n_s=30, n_aux=30,
                                  seed=5))
    ctx = Context(big)
    nbb = int(big["n_g"][0]) + 4
    dx = torch.zeros((30, nbb), dtype=torch.complex128, device="cuda")
    with pytest.raises(RttddftError) as e:
        rttddft.rttddft_apply_noalloc(ctx.ctx, 0, 30, dx, np.zeros(3), 0.0, dx.clone(), dx.clone())
    assert e.value.code == -1 and "static limit" in str(e.value)
    ctx.close()


def test_noalloc_apply_in_an_fft_route_context():
    """An FFT-route context: the no-alloc apply takes the direct interstitial sum
    (its static scratch has no FFT buffers); the two routes agree to rounding."""
    import torch
    build()
    s = make_system("tiny400")
    ctx = Context(s, interstitial="fft")
    nb = int(s["n_g"][0]) + int(np.sum(s["n_lo"]))
    rng = np.random.default_rng(11)
    x = rng.standard_normal((nb, 9)) + 1j * rng.standard_normal((nb, 9))
    a_vec = (0.2, 0.9, -1.4)
    hx_ref, sx_ref = ctx.apply(0, x, a_vec, 0.0)
    dx = _device_block(torch, x)
    dh = torch.empty_like(dx)
    ds = torch.empty_like(dx)
    rttddft.rttddft_apply_noalloc(ctx.ctx, 0, 9, dx, np.ascontiguousarray(a_vec, dtype=np.float64), 0.0, dh, ds)
    torch.cuda.synchronize()
    assert np.max(np.abs(dh.cpu().numpy().T - hx_ref)) <= 1e-12 * np.max(np.abs(hx_ref))
    assert np.max(np.abs(ds.cpu().numpy().T - sx_ref)) <= 1e-12 * np.max(np.abs(sx_ref))
    ctx.close()
