"""The seeded input generator (no method arithmetic): reproducible draws, a
k-point subset drawn bit-identically to the same k-points of the full set
(the full-size GPU test compares a batched run's k-point 0 with a run of that
k-point alone), and the structural properties the method assumes."""
import numpy as np

from synth import make_system, tiny_config


def _cfg():
    return tiny_config(name="sub", n_g=0, n_atoms=2, lmax=1, n_lo_per_atom=2, n_s=2, n_aux=10,
                       n_k=4, kgrid=(2, 2, 1), n_b_range=(60, 80), seed=31, lattice="mos2",
                       edir=(1.0, 0.0, 0.0))


def test_draws_are_reproducible():
    a, b = make_system(_cfg()), make_system(_cfg())
    for key in ("vtab", "n_g"):
        assert np.array_equal(a[key], b[key])
    for k in range(4):
        assert np.array_equal(a["caux"][k], b["caux"][k])
        assert np.array_equal(a["amat"][k], b["amat"][k])


def test_k_subset_is_bit_identical_to_the_full_draw():
    full = make_system(_cfg())
    for k in (0, 2):
        sub = make_system(_cfg(), k_subset=[k])
        assert np.array_equal(sub["vt_dim"], full["vt_dim"])
        assert np.array_equal(sub["vtab"], full["vtab"])
        assert np.array_equal(sub["g_int"][0], full["g_int"][k])
        assert np.array_equal(sub["gk"][0], full["gk"][k])
        assert np.array_equal(sub["amat"][0], full["amat"][k])
        assert np.array_equal(sub["caux"][0], full["caux"][k])
        for a in range(2):
            assert np.array_equal(sub["h"][a], full["h"][a])


def test_table_is_hermitian_and_covers_the_differences():
    s = make_system(_cfg())
    v = s["vtab"]
    assert np.max(np.abs(v - np.conj(v[::-1, ::-1, ::-1]))) == 0.0
    e = (np.asarray(s["vt_dim"]) - 1) // 2
    for gi in s["g_int"]:
        assert np.all(gi.max(axis=0) - gi.min(axis=0) <= e)
        # lexicographic order of the G list
        keys = [tuple(x) for x in gi]
        assert keys == sorted(keys)
