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


@pytest.mark.parametrize("form", ["fp32", "bf16x3"])
def test_noalloc_apply_in_reduced_precision_contexts(form):
    """FP32 and split-BF16 contexts with the potential change on, at k-point 1
    of a ragged 2-k system: the no-alloc apply runs the FP32 contraction form
    (its static scratch holds no tensor-core operands) and is held to the
    oracle's explicit H X and S X at the FP32 bound, 1e-5 (|H||x|); in the
    FP32 context it also matches rttddft_apply of the same context."""
    import torch
    from oracle import explicit_dv, explicit_operators, hamiltonian
    build()
    cfg = tiny_config(name="ragged2", n_g=0, n_atoms=3, lmax=2, n_lo_per_atom=3, n_s=3, n_aux=20,
                      n_k=2, kgrid=(2, 1, 1), n_b_range=(130, 181), seed=19, lattice="mos2")
    s = make_system(cfg)
    assert s["n_g"][0] != s["n_g"][1]
    dv = make_dv(s)
    ctx = Context(s, precision=form)
    ctx.set_dv(dv)
    rng = np.random.default_rng(13)
    a_vec, sdv = (0.6, -1.1, 0.3), 0.7
    for k in (1, 0):
        ops = explicit_operators(s, k)
        nb = ops["nb"]
        x = rng.standard_normal((nb, 5)) + 1j * rng.standard_normal((nb, 5))
        dx = _device_block(torch, x)
        dh = torch.empty_like(dx)
        ds = torch.empty_like(dx)
        rttddft.rttddft_apply_noalloc(ctx.ctx, k, 5, dx, np.ascontiguousarray(a_vec, dtype=np.float64), sdv, dh, ds)
        torch.cuda.synchronize()
        hx = dh.cpu().numpy().T
        sxv = ds.cpu().numpy().T
        h = hamiltonian(ops, a_vec, s["c_light"], explicit_dv(s, k, dv), sdv)
        assert np.max(np.abs(hx - h @ x) / (np.abs(h) @ np.abs(x))) < 1e-5, (form, k)
        assert np.max(np.abs(sxv - ops["S"] @ x) / (np.abs(ops["S"]) @ np.abs(x))) < 1e-5, (form, k)
        if form == "fp32":
            hx_ref, sx_ref = ctx.apply(k, x, a_vec, sdv)
            assert np.max(np.abs(hx - hx_ref)) <= 1e-6 * np.max(np.abs(hx_ref)), k
            assert np.max(np.abs(sxv - sx_ref)) <= 1e-6 * np.max(np.abs(sx_ref)), k
    ctx.close()


def test_noalloc_apply_rejects_the_co_12000_workload():
    """co_12000 (N_basis 12000, N_states 7) needs more than the 16 MiB static
    scratch (the interstitial partials of the direct sum dominate): ERR_ARG
    with the need in the message, nothing launched."""
    import torch
    build()
    s = make_system("co_12000")
    ctx = Context(s)
    nb = int(s["n_g"][0]) + int(np.sum(s["n_lo"]))
    dx = torch.zeros((7, nb), dtype=torch.complex128, device="cuda")
    with pytest.raises(RttddftError) as e:
        rttddft.rttddft_apply_noalloc(ctx.ctx, 0, 7, dx, np.zeros(3), 0.0, dx.clone(), dx.clone())
    assert e.value.code == -1 and "static limit" in str(e.value)
    ctx.close()
