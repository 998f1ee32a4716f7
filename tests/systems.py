"""Hand-built special-case systems for the tests (no method arithmetic)."""
import numpy as np

from synth import make_system, tiny_config


def free_electron_system(n_g=30, n_s=3, n_aux=None, seed=5):
    """Plane waves only: no atoms, no local orbitals, zero potential table.
    Its Hamiltonian is diagonal: H(A) = |G+k+A/c|^2 / 2."""
    s = make_system(tiny_config(n_g=n_g, n_s=n_s, n_aux=n_aux or n_g, seed=seed))
    ng = int(s["n_g"][0])
    s.update(n_atoms=0, n_a=np.zeros(0, np.int32), n_lo=np.zeros(0, np.int32),
             h=[], o=[], p=[], amat=[np.zeros((0, ng), dtype=np.complex128, order="F")])
    s["vtab"] = np.zeros_like(s["vtab"])
    s["caux"] = [np.asfortranarray(s["caux"][0][:ng, :])]
    return s


def plane_wave_basis(s, n_aux):
    """Unit vectors on the n_aux plane waves of lowest |G+k|^2 and their energies."""
    gk = s["gk"][0]
    e = 0.5 * np.sum(gk * gk, axis=1)
    order = np.argsort(e, kind="stable")[:n_aux]
    cc = np.zeros((len(e), n_aux), dtype=np.complex128, order="F")
    cc[order, np.arange(n_aux)] = 1.0
    return cc, e[order], order


def permutation_mt_system(seed=7):
    """A small system whose matching coefficients are phased unit rows:
    A_alpha[p, pi(p)] = d_p, zero elsewhere, so each muffin-tin block lands on
    known plane-wave positions."""
    s = make_system(tiny_config(n_g=40, n_atoms=2, lmax=1, n_lo_per_atom=2, n_s=2,
                                n_aux=10, seed=seed))
    ng = int(s["n_g"][0])
    rng = np.random.default_rng(seed)
    n_rows = int(np.sum(s["n_a"]))
    perm = rng.permutation(ng)[:n_rows]
    d = np.exp(2j * np.pi * rng.random(n_rows))
    a = np.zeros((n_rows, ng), dtype=np.complex128, order="F")
    a[np.arange(n_rows), perm] = d
    s["amat"] = [a]
    s["vtab"] = np.zeros_like(s["vtab"])
    s["gk"] = [np.zeros_like(s["gk"][0])]
    return s, perm, d
