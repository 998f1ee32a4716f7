"""Seeded synthetic systems shaped like the paper's molecules and interface.

The paper's workloads (H2 and CO in vacuum boxes, pyridine@MoS2 with a 3x3x1
k-grid; Sec. 3) need exciting ground states, species files and the NOMAD
archive, none of which are available.  This module draws stand-ins with the
same structure:

* LAPW+LO basis per k-point (Eq. expansion_LAPW_lo): N_G plane waves G+k
  followed by the local orbitals, grouped by atom.
* per atom alpha: matching coefficients A_alpha (N_A x N_G, k-dependent) and
  Hermitian muffin-tin blocks h_alpha, o_alpha (overlap, positive definite)
  and p_alpha (three momentum components) of order N_A + n_lo (Eq. v_MT,
  Appendix A); N_A = 2 (lmax+1)^2 counts (u, u') for every (l, m).
* interstitial potential table V~_{G-G'} indexed by the integer difference
  vector (Eq. v_interstitial, Appendix A), Hermitian: V~_{-g} = conj(V~_g).
* a block of N_aux trial vectors per k whose span is the auxiliary subspace
  (Eq. auxiliary_basis); the step's set-up turns it into S-orthonormal Ritz
  vectors.
* pulse samples A(t) = A0 sin^2(pi t / T) sin(omega t) e at step midpoints.

Every array is drawn from numpy PCG64 streams keyed by (seed, role, k, atom),
so any subset of k-points can be regenerated identically.  Complex matrices
are returned as complex128 numpy arrays in column-major (Fortran) order, the
layout the C ABI takes.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

BOHR_PER_ANGSTROM = 1.0 / 0.529177210903
C_LIGHT = 137.035999084  # atomic units (CODATA 2018)

# role tags for independent random streams
_T_VTAB, _T_AMAT, _T_H, _T_O, _T_P, _T_CAUX, _T_NB, _T_DH, _T_DV = range(1, 10)


def _rng(*key):
    return np.random.Generator(np.random.PCG64(list(int(x) for x in key)))


def _cnormal(rng, shape):
    """Complex normal with E|z|^2 = 1."""
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    return (re + 1j * im) * (1.0 / math.sqrt(2.0))


def _haar_unitary(rng, n):
    z = _cnormal(rng, (n, n))
    q, r = np.linalg.qr(z)
    d = np.diag(r)
    ph = d / np.where(np.abs(d) > 0, np.abs(d), 1.0)
    return q * ph[None, :]


def _hermitian_with_spectrum(rng, n, lo, hi):
    q = _haar_unitary(rng, n)
    lam = rng.uniform(lo, hi, size=n)
    m = (q * lam[None, :]) @ q.conj().T
    m = 0.5 * (m + m.conj().T)
    return np.asfortranarray(m)


@dataclass(frozen=True)
class Config:
    name: str
    seed: int
    n_atoms: int
    lmax: int
    n_lo_per_atom: int
    n_s: int
    n_aux: int
    dt: float
    n_steps: int
    lattice: str               # "h2box", "mos2" or "chain"
    n_k: int = 1
    n_g: int = 0               # plane waves (single k) ...
    n_b_range: tuple = (0, 0)  # ... or per-k basis size drawn uniformly
    kgrid: tuple = (1, 1, 1)
    edir: tuple = (0.0, 0.0, 1.0)
    a0: float = 0.05
    omega: float = 0.3

    @property
    def n_a(self):
        return 2 * (self.lmax + 1) ** 2


CONFIGS = {
    # tiny system: 1 k, 2 atoms, lmax 4, 360 PW + 40 LO, 8 states, N_aux 32
    "tiny400": Config("tiny400", 1, 2, 4, 20, 8, 32, 0.1, 200, "h2box", n_g=360),
    # H2-like large cell: 5900 PW + 100 LO, 2 states, N_aux 200
    "h2_6000": Config("h2_6000", 2, 2, 8, 50, 2, 200, 0.2, 2000, "h2box", n_g=5900),
    # CO-like cell: 11800 PW + 200 LO, 7 states, N_aux 400
    "co_12000": Config("co_12000", 3, 2, 8, 100, 7, 400, 0.2, 1000, "h2box", n_g=11800),
    # CO-like cell at the largest basis of the paper's basis-size table (N_basis 25727,
    # where the FFT route of the interstitial sum pays most): 25527 PW + 200 LO
    "co_25727": Config("co_25727", 6, 2, 8, 100, 7, 400, 0.2, 1000, "h2box", n_g=25527),
    # heterostructure: 22 atoms, 16 k-points, N_basis in [7000, 10000]
    "mos2_16k": Config("mos2_16k", 4, 22, 8, 5, 60, 300, 0.2, 500, "mos2", n_k=16,
                       n_b_range=(7000, 10000), kgrid=(4, 4, 1), edir=(1.0, 0.0, 0.0)),
    # adjoint workload: the H2-like system over 400 steps
    "h2_6000_adj": Config("h2_6000_adj", 2, 2, 8, 50, 2, 200, 0.2, 400, "h2box", n_g=5900),
}


def tiny_config(name="micro", n_g=40, n_atoms=2, lmax=1, n_lo_per_atom=2, n_s=3,
                n_aux=None, n_k=1, seed=11, dt=0.1, n_steps=20, kgrid=(1, 1, 1),
                n_b_range=(0, 0), a0=0.05, omega=0.3, lattice="h2box",
                edir=(0.0, 0.0, 1.0)):
    """A small configuration for brute-force checks (N_aux defaults to N_basis)."""
    if n_aux is None:
        n_aux = n_g + n_atoms * n_lo_per_atom
    return Config(name, seed, n_atoms, lmax, n_lo_per_atom, n_s, n_aux, dt, n_steps,
                  lattice, n_k=n_k, n_g=n_g, n_b_range=n_b_range, kgrid=kgrid,
                  edir=edir, a0=a0, omega=omega)


def _lattice(kind):
    if kind == "h2box":  # 21.401 x 20 x 20 bohr^3 box (Sec. 3.1)
        return np.diag([21.401, 20.0, 20.0])
    if kind == "mos2":   # 3a x 3a hexagonal supercell, a = 3.16 A, L = 14.71 A (Sec. 3.3)
        a = 3.16 * BOHR_PER_ANGSTROM
        c = 14.71 * BOHR_PER_ANGSTROM
        return np.array([[3 * a, 0.0, 0.0],
                         [1.5 * a, 1.5 * a * math.sqrt(3.0), 0.0],
                         [0.0, 0.0, c]])
    if kind == "chain":  # a long thin box (6 x 6 x 120 bohr^3): many plane waves along z
        return np.diag([6.0, 6.0, 120.0])
    raise ValueError(kind)


def _kpoints(kgrid):
    pts = []
    for i in range(kgrid[0]):
        for j in range(kgrid[1]):
            for l in range(kgrid[2]):
                pts.append((i / kgrid[0], j / kgrid[1], l / kgrid[2]))
    return np.array(pts, dtype=np.float64)


def basis_sizes(cfg):
    """Per-k plane-wave counts and the LO count of a configuration."""
    n_lo = cfg.n_atoms * cfg.n_lo_per_atom
    if cfg.n_b_range[1] > 0:
        rng = _rng(cfg.seed, _T_NB)
        nb = rng.integers(cfg.n_b_range[0], cfg.n_b_range[1] + 1, size=cfg.n_k)
        return [int(x) - n_lo for x in nb], n_lo
    return [cfg.n_g] * cfg.n_k, n_lo


def _gset(recip, kcart, n_g):
    """The n_g integer triples with the shortest |G+k|, listed in
    lexicographic (n1, n2, n3) order; ties at the cut are broken
    lexicographically."""
    vol_recip = abs(np.linalg.det(recip))
    gmax = (3.0 * n_g * vol_recip / (4.0 * math.pi)) ** (1.0 / 3.0)
    lat = 2.0 * math.pi * np.linalg.inv(recip).T  # rows: real-space vectors
    nmax = [int(math.ceil(1.3 * gmax * np.linalg.norm(lat[i]) / (2 * math.pi))) + 2
            for i in range(3)]
    r = [np.arange(-m, m + 1) for m in nmax]
    n1, n2, n3 = np.meshgrid(r[0], r[1], r[2], indexing="ij")
    ints = np.stack([n1.ravel(), n2.ravel(), n3.ravel()], axis=1)
    cart = ints @ recip + kcart[None, :]
    len2 = np.einsum("ij,ij->i", cart, cart)
    order = np.lexsort((ints[:, 2], ints[:, 1], ints[:, 0], len2))
    sel = ints[order[:n_g]]
    if n_g >= len(ints) or np.max(np.abs(sel), axis=0).tolist() >= list(nmax):
        raise RuntimeError("G-vector search box too small")
    lex = np.lexsort((sel[:, 2], sel[:, 1], sel[:, 0]))
    sel = np.ascontiguousarray(sel[lex]).astype(np.int32)
    gk = sel.astype(np.float64) @ recip + kcart[None, :]
    return sel, np.ascontiguousarray(gk)


def make_system(cfg, k_subset=None, with_amat=True):
    """Draw the synthetic system for configuration `cfg` (a Config or a name).

    Returns a dict of numpy arrays (see module docstring).  `k_subset`
    restricts the k-points that are materialised (the others keep their
    random streams, so a subset is bit-identical to the full draw).
    """
    if isinstance(cfg, str):
        cfg = CONFIGS[cfg]
    lattice = _lattice(cfg.lattice)
    omega = abs(np.linalg.det(lattice))
    recip = 2.0 * math.pi * np.linalg.inv(lattice).T
    kfrac_all = _kpoints(cfg.kgrid)
    if len(kfrac_all) != cfg.n_k:
        raise ValueError("k-grid does not match n_k")
    n_g_all, n_lo_tot = basis_sizes(cfg)
    ks = list(range(cfg.n_k)) if k_subset is None else list(k_subset)
    n_a = cfg.n_a
    n_lo = [cfg.n_lo_per_atom] * cfg.n_atoms

    g_int, gk = [], []
    for k in ks:
        kc = kfrac_all[k] @ recip
        gi, gc = _gset(recip, kc, n_g_all[k])
        g_int.append(gi)
        gk.append(gc)

    # interstitial potential table over the integer difference box
    ext = np.zeros(3, dtype=np.int64)
    for gi in g_int:
        ext = np.maximum(ext, gi.max(axis=0) - gi.min(axis=0))
    # the box must not depend on the k subset: use all k-points' extents
    if k_subset is not None:
        ext = np.zeros(3, dtype=np.int64)
        for k in range(cfg.n_k):
            gi, _ = _gset(recip, kfrac_all[k] @ recip, n_g_all[k])
            ext = np.maximum(ext, gi.max(axis=0) - gi.min(axis=0))
    vt_dim = (2 * ext + 1).astype(np.int32)
    vtab = _make_vtab(_rng(cfg.seed, _T_VTAB), recip, ext, amp=0.1, width=4.0)

    # per-atom muffin-tin blocks (k-independent)
    h, o, p = [], [], []
    for a in range(cfg.n_atoms):
        m = n_a + n_lo[a]
        h.append(_hermitian_with_spectrum(_rng(cfg.seed, _T_H, a), m, -1.0, 1.0))
        o.append(_hermitian_with_spectrum(_rng(cfg.seed, _T_O, a), m, 0.5, 2.0))
        pr = _rng(cfg.seed, _T_P, a)
        p.append(np.stack([_hermitian_with_spectrum(pr, m, -0.5, 0.5) for _ in range(3)]))

    # matching coefficients, stacked over atoms: (n_atoms*N_A) x N_G per k
    amat = []
    if with_amat:
        for i, k in enumerate(ks):
            ng = n_g_all[k]
            env = np.exp(-np.einsum("ij,ij->i", gk[i], gk[i]) / 20.0) / math.sqrt(ng)
            blocks = []
            for a in range(cfg.n_atoms):
                z = _cnormal(_rng(cfg.seed, _T_AMAT, k, a), (n_a, ng))
                blocks.append(z * env[None, :])
            amat.append(np.asfortranarray(np.concatenate(blocks, axis=0)))

    # trial vectors spanning the auxiliary subspace
    caux = []
    for i, k in enumerate(ks):
        ng = n_g_all[k]
        nb = ng + n_lo_tot
        g2 = np.einsum("ij,ij->i", gk[i], gk[i])
        sigma2 = 0.25 * float(np.max(g2))
        z = _cnormal(_rng(cfg.seed, _T_CAUX, k), (nb, cfg.n_aux))
        z[:ng] *= np.exp(-g2 / (2.0 * sigma2))[:, None]
        z[ng:] *= 0.3
        caux.append(np.asfortranarray(z))

    return dict(
        name=cfg.name, cfg=cfg, omega=float(omega), c_light=C_LIGHT,
        lattice=lattice, recip=recip,
        n_k=len(ks), k_index=np.array(ks, dtype=np.int32),
        kfrac=kfrac_all[ks], wk=np.full(len(ks), 1.0 / cfg.n_k),
        n_atoms=cfg.n_atoms, n_a=np.full(cfg.n_atoms, n_a, dtype=np.int32),
        n_lo=np.array(n_lo, dtype=np.int32),
        n_s=cfg.n_s, n_aux=cfg.n_aux, occ=np.full(cfg.n_s, 2.0),
        n_g=np.array([n_g_all[k] for k in ks], dtype=np.int32),
        g_int=g_int, gk=gk, amat=amat, h=h, o=o, p=p,
        vt_dim=vt_dim, vtab=vtab, caux=caux,
        dt=cfg.dt, n_steps=cfg.n_steps,
    )


def _make_vtab(rng, recip, ext, amp, width):
    """V~_g = amp * exp(-|g|^2/width) * (z_g + conj(z_{-g}))/2 over the box
    |g_i| <= ext_i; Hermitian in g, real at g = 0."""
    r = [np.arange(-e, e + 1) for e in ext]
    d1, d2, d3 = np.meshgrid(r[0], r[1], r[2], indexing="ij")
    gi = np.stack([d1, d2, d3], axis=-1).astype(np.float64)
    gc = gi @ recip
    env = amp * np.exp(-np.einsum("...i,...i->...", gc, gc) / width)
    z = _cnormal(rng, d1.shape)
    zm = z[::-1, ::-1, ::-1]  # z at -g
    v = env * 0.5 * (z + np.conj(zm))
    return np.ascontiguousarray(v)


def pulse_samples(cfg_or_sys, n_steps=None, dt=None, a0=None, omega=None, edir=None,
                  t_start=0.0, period=None):
    """A(t) = A0 sin^2(pi t/T) sin(omega t) e, sampled at step midpoints
    t_k + dt/2; T defaults to n_steps*dt.  Returns an (n_steps, 3) array."""
    cfg = cfg_or_sys["cfg"] if isinstance(cfg_or_sys, dict) else cfg_or_sys
    if isinstance(cfg, str):
        cfg = CONFIGS[cfg]
    n_steps = cfg.n_steps if n_steps is None else n_steps
    dt = cfg.dt if dt is None else dt
    a0 = cfg.a0 if a0 is None else a0
    omega = cfg.omega if omega is None else omega
    e = np.asarray(cfg.edir if edir is None else edir, dtype=np.float64)
    period = n_steps * dt if period is None else period
    t = t_start + (np.arange(n_steps) + 0.5) * dt
    amp = a0 * np.sin(math.pi * t / period) ** 2 * np.sin(omega * t)
    return np.ascontiguousarray(amp[:, None] * e[None, :])


def make_dv(sys, amp=1e-2, seed_offset=0):
    """A potential-change pattern dV_1: per-atom Hermitian muffin-tin blocks
    dh_alpha (order N_A + n_lo) and an interstitial table dV~ over the same
    difference box as V~ (Hermitian in g)."""
    cfg = sys["cfg"]
    dh = []
    for a in range(sys["n_atoms"]):
        m = int(sys["n_a"][a] + sys["n_lo"][a])
        dh.append(_hermitian_with_spectrum(_rng(cfg.seed + seed_offset, _T_DH, a), m,
                                           -amp, amp))
    ext = (np.asarray(sys["vt_dim"]) - 1) // 2
    dvt = _make_vtab(_rng(cfg.seed + seed_offset, _T_DV), sys["recip"], ext, amp=amp,
                     width=4.0)
    return dict(dh=dh, dvtab=dvt)


def dv_scale_samples(n_steps, dt, freq=0.1, t_start=0.0):
    """Scale s_k = sin(freq t) of the potential-change pattern at step midpoints."""
    t = t_start + (np.arange(n_steps) + 0.5) * dt
    return np.ascontiguousarray(np.sin(freq * t))
