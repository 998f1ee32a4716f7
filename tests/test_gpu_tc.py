"""The split-BF16 complex GEMM on the tensor cores (tcgen05, TMA-fed), called
through rttddft_zgemm_bf16x3, against FP64 products computed on the host.

Two kinds of check:
  - integer-valued operands that bf16 holds exactly (so lo = 0 and every FP32
    partial sum is exact): the result must be bit-exact, which pins the
    operand layout, the complex-as-real mapping, conjugation, the K slices,
    the tile edges and the epilogue;
  - random operands: the element error must stay within the split bound
    (3 * 2^-16 + 2 K_slice * 2^-24) * sum_k |a_ik| |x_kj| (the dropped lo.lo
    term, the rounding of lo, and FP32 accumulation), and be far below plain
    bf16 (2^-8).
"""
import numpy as np
import pytest

from paper_2403_04351_gb300 import RttddftError, build
from paper_2403_04351_gb300 import rttddft as R

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    build()


def _dev(mat_colmajor):
    """Device copy of a complex column-major matrix given as a numpy (rows, cols) array."""
    import torch
    return torch.from_numpy(np.asfortranarray(mat_colmajor).T.copy()).to("cuda")


def _host(t, rows):
    return t.cpu().numpy().T[:rows]


def _run(trans, m, n, k, a, x, c0=None, beta_add=0):
    import torch
    da, dx = _dev(a), _dev(x)
    dc = _dev(c0 if c0 is not None else np.zeros((m, n), complex))
    R.rttddft_zgemm_bf16x3(trans, m, n, k, da, a.shape[0], dx, k, dc, m, beta_add)
    torch.cuda.synchronize()
    return _host(dc, m)


def _ints(rng, shape, lim=3):
    return rng.integers(-lim, lim + 1, shape) + 1j * rng.integers(-lim, lim + 1, shape)


SHAPES = [  # (trans, m, n, k)
    (0, 300, 2, 200),     # expansion-like: N_b x N_aux times N_aux x N_s
    (1, 200, 2, 6000),    # projection-like: CC^H (N_aux x N_b) times N_b x N_s
    (0, 128, 8, 32),      # one M tile, K inside one K block
    (0, 129, 17, 65),     # ragged M, N and K
    (1, 1, 1, 1),
    (0, 257, 130, 300),   # two N tiles (2N = 260 real columns)
    (1, 162, 60, 1000),   # matching-coefficient-like with N_s = 60
]


@pytest.mark.parametrize("trans,m,n,k", SHAPES)
def test_exact_on_bf16_representable_integers(trans, m, n, k):
    rng = np.random.default_rng(m * 7 + n * 3 + k)
    a = _ints(rng, (k, m) if trans else (m, k))
    x = _ints(rng, (k, n))
    ref = (a.conj().T if trans else a) @ x
    got = _run(trans, m, n, k, a, x)
    assert np.array_equal(got, ref), np.max(np.abs(got - ref))


@pytest.mark.parametrize("trans,m,n,k", SHAPES)
def test_random_operands_within_split_bound(trans, m, n, k):
    rng = np.random.default_rng(1000 + m + n + k)
    a = rng.standard_normal((k, m) if trans else (m, k)) + 1j * rng.standard_normal((k, m) if trans else (m, k))
    a *= np.exp(rng.uniform(-3, 3, a.shape))  # a spread of magnitudes
    x = rng.standard_normal((k, n)) + 1j * rng.standard_normal((k, n))
    op = a.conj().T if trans else a
    ref = op @ x
    mag = np.abs(op) @ np.abs(x)
    got = _run(trans, m, n, k, a, x)
    err = np.abs(got - ref)
    kslice = 3 * ((2 * k + 63) // 64) * 64  # the K one FP32 accumulator can see at most
    bound = 2.0 * (3 * 2.0 ** -16 + 2 * kslice * 2.0 ** -24) * mag
    assert np.all(err <= bound), np.max(err / bound)
    assert np.max(err / mag) < 2.0 ** -12


def test_beta_add_accumulates():
    rng = np.random.default_rng(4)
    m, n, k = 190, 3, 77
    a, x, c0 = _ints(rng, (m, k)), _ints(rng, (k, n)), _ints(rng, (m, n), 50)
    got = _run(0, m, n, k, a, x, c0=c0, beta_add=1)
    assert np.array_equal(got, c0 + a @ x)


def test_degenerate_sizes_and_bad_arguments():
    import torch
    c = _dev(np.full((4, 2), 5 + 1j))
    R.rttddft_zgemm_bf16x3(0, 4, 2, 0, c, 4, c, 1, c, 4, 1)  # k = 0, += nothing
    assert np.all(_host(c, 4) == 5 + 1j)
    R.rttddft_zgemm_bf16x3(0, 4, 2, 0, c, 4, c, 1, c, 4, 0)  # k = 0, C = 0
    assert np.all(_host(c, 4) == 0)
    R.rttddft_zgemm_bf16x3(0, 0, 2, 3, c, 1, c, 3, c, 1, 0)  # m = 0
    with pytest.raises(RttddftError) as e:
        R.rttddft_zgemm_bf16x3(0, 4, 2, 3, c, 3, c, 3, c, 4, 0)  # lda < m
    assert e.value.code == -1
    h = np.zeros(8, complex)
    with pytest.raises(RttddftError) as e:
        R.rttddft_zgemm_bf16x3(0, 4, 2, 1, h, 4, c, 1, c, 4, 0)  # host pointer
    assert e.value.code == -1
    torch.cuda.synchronize()
