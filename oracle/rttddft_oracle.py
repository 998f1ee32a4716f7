"""FP64 CPU oracle for the velocity-gauge RT-TDDFT step in an auxiliary subspace.

TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's CPU
baseline may import this module.  It shares no code with the CUDA path; the
two meet only in the seeded inputs drawn by `synth`.

The oracle is deliberately plain: it forms the LAPW+LO matrices H, S and P
explicitly (the matrices the method is designed to avoid) and then follows
the method step by step with dense linear algebra from numpy/scipy.

Paper sections and equations followed (arXiv 2403.04351):
* Sec. 2, Eq. (TDKS) and the velocity-gauge Hamiltonian
  H(t) = 1/2 (-i nabla + A/c)^2 + V, which in the basis becomes
  H(t) = H0 + (A/c).P + |A|^2/(2c^2) S + dV(t).
* Eq. expansion_LAPW_lo / expansion_basis: coefficient matrix C_k of order
  N_basis x N_states, rows = [plane waves G+k ; local orbitals].
* Eq. evolution_wf_coeff: S C' = -i H C.
* Eq. auxiliary_basis, approximation_coefficients: C(t) ~= CC(0) theta(t),
  theta = CC^H S C.
* Eq. evolution_of_projection_coeff, definition_auxiliary_hamiltonian:
  theta' = -i HH theta with HH = CC^H H CC.
* Eq. auxiliary_hamiltonian_with_parts: HH = T + (A/c).PP + A^2/(2c^2) SS + VV(t).
* Eq. v_interstitial and Eq. v_MT, Appendix A: the matrix elements of V in
  the basis (interstitial Toeplitz table plus the muffin-tin blocks mapped
  by the matching coefficients).
* Eq. dipole: delta mu(t) = Omega * int_0^t J_ind.
* Eq. critical_timestep: dt_cr = f / (eps_max - eps_min), f = 0.2.

Readings where the paper is silent (each listed in the design notes):
* the muffin-tin overlap/Hamiltonian/momentum blocks o, h, p of each atom
  act through E_alpha = [A_alpha 0; 0 I] exactly as V does in Eq. v_MT; the
  interstitial overlap is the identity on the plane waves;
* the propagator is the exact exponential of the subspace Hamiltonian held
  at the step midpoint (or Crank-Nicolson), with A_k = A(t_k + dt/2);
* J(t) = -(1/Omega) sum_k w_k sum_j f_j Re c_j^H (P + (A/c) S) c_j and
  J_ind = J - J(t0) with J(t0) the field-free ground-state value;
* the dipole integral is the trapezoid rule on the step grid, dmu(t0) = 0;
* the auxiliary basis is the set of Ritz vectors of H0 in the span of the
  given trial vectors (S-orthonormal, H0 diagonal on them), each scaled so
  that the sum of its coefficients is real and positive;
* the per-step potential from the evolving density (Sec. 2: VV(t) is what
  changes from step to step) is modelled by its Hartree part: in the
  interstitial n_g = (1/Omega) sum_k w_k sum_j f_j sum_G C_G conj(C_{G-g})
  over the plane-wave rows, dV_g = 4 pi (n_g(t) - n_g(0)) / |g|^2 (g != 0,
  cartesian g), on the table box; in the spheres, optionally, the density
  matrix n_a = sum_k w_k sum_j f_j (E_a c)(E_a c)^H of each atom's channels
  and the on-site blocks dh_a = U (n_a(t) - n_a(0)) (a contact stand-in for
  the sphere's Hartree response, whose radial functions and Gaunt
  coefficients are not available); the potential of step k comes from C_k.

What pins each function (tests/test_oracle_pins.py; no function is
parity-unpinned):
* interstitial_potential: the FFT convolution of the same sum;
* embedding, explicit_operators: muffin-tin blocks landing on the matched plane
  waves, Hermiticity and positivity, the free-electron closed forms;
* explicit_dv: the four-block form of Eq. v_MT, a Hermitian perturbation;
* hamiltonian: free-electron closed forms, the discrete work theorem;
* ritz_basis, fix_phases: orthonormality, diagonal H0, bounds by the exact
  eigenvalues;
* propagate_exact, critical_timestep: Pade expm, the two-level closed form;
* propagate_cn: second-order convergence;
* full_basis_propagator and Oracle.run: the complete-subspace equivalence,
  the field-free phase, norm and energy conservation, time reversal,
  weak-field linearity, k-point weighting;
* Oracle.excited_electrons: full-basis projection on the LAPACK ground state,
  second order in a weak field;
* Oracle.dipole_gradient: central differences;
* overall_speedup: the speed-ups printed in Table tab:H2;
* polarizability: the closed-form geometric series, a proportional response;
* interstitial_density: |psi(r)|^2 on a grid through numpy's FFT;
* hartree_table: a single plane-wave density in a hexagonal cell, the sign of
  the Hartree energy; Oracle.run(hartree=True): field-free inertness, norm;
* mt_density: the closed form of a system whose matching coefficients are
  phased unit rows (each channel reads one plane-wave coefficient);
  Oracle.run(hartree=True, mt_u): field-free inertness, its effect on the
  dipole, and the muffin-tin potential matrix against its own blocks placed
  on the matched plane waves.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla

F_CRIT = 0.2  # Eq. critical_timestep: f = 0.2


# ---------------------------------------------------------------- operators

def interstitial_potential(g_int, vt_dim, vtab):
    """V_I[G, G'] = V~_{G-G'} (Eq. v_interstitial, Appendix A)."""
    ext = (np.asarray(vt_dim) - 1) // 2
    d = g_int[:, None, :].astype(np.int64) - g_int[None, :, :].astype(np.int64)
    return vtab[d[..., 0] + ext[0], d[..., 1] + ext[1], d[..., 2] + ext[2]]


def embedding(sys, ik, atom):
    """E_alpha = [A_alpha 0 ; 0 I_lo(alpha)] as a dense (N_A+n_lo) x N_basis
    matrix: the block map of Eq. v_MT for one atom."""
    ng = int(sys["n_g"][ik])
    n_lo = np.asarray(sys["n_lo"])
    nb = ng + int(n_lo.sum())
    n_a = int(sys["n_a"][atom])
    row0 = int(np.sum(sys["n_a"][:atom]))
    lo0 = ng + int(n_lo[:atom].sum())
    e = np.zeros((n_a + int(n_lo[atom]), nb), dtype=np.complex128)
    e[:n_a, :ng] = sys["amat"][ik][row0:row0 + n_a, :]
    e[n_a:, lo0:lo0 + int(n_lo[atom])] = np.eye(int(n_lo[atom]))
    return e


def explicit_operators(sys, ik):
    """Dense S, H0 and P_x, P_y, P_z of one k-point (Appendix A):
    S  = [I_G 0; 0 0] + sum_a E_a^H o_a E_a
    H0 = [diag(|G+k|^2/2) + V_I 0; 0 0] + sum_a E_a^H h_a E_a
    P_l = [diag((G+k)_l) 0; 0 0] + sum_a E_a^H p_a,l E_a
    """
    ng = int(sys["n_g"][ik])
    nb = ng + int(np.sum(sys["n_lo"]))
    gk = sys["gk"][ik]
    s = np.zeros((nb, nb), dtype=np.complex128)
    h0 = np.zeros((nb, nb), dtype=np.complex128)
    p = np.zeros((3, nb, nb), dtype=np.complex128)
    s[:ng, :ng] = np.eye(ng)
    h0[:ng, :ng] = np.diag(0.5 * np.sum(gk * gk, axis=1))
    h0[:ng, :ng] += interstitial_potential(sys["g_int"][ik], sys["vt_dim"], sys["vtab"])
    for l in range(3):
        p[l, :ng, :ng] = np.diag(gk[:, l])
    for a in range(int(sys["n_atoms"])):
        e = embedding(sys, ik, a)
        eh = e.conj().T
        s += eh @ sys["o"][a] @ e
        h0 += eh @ sys["h"][a] @ e
        for l in range(3):
            p[l] += eh @ sys["p"][a][l] @ e
    return dict(S=s, H0=h0, P=p, nb=nb, ng=ng)


def explicit_dv(sys, ik, dv):
    """Dense potential change dV_1 of one k-point from its muffin-tin blocks
    dh_a and interstitial table dV~ (Appendix A, Eq. v_MT / v_interstitial)."""
    ng = int(sys["n_g"][ik])
    nb = ng + int(np.sum(sys["n_lo"]))
    m = np.zeros((nb, nb), dtype=np.complex128)
    m[:ng, :ng] = interstitial_potential(sys["g_int"][ik], sys["vt_dim"], dv["dvtab"])
    for a in range(int(sys["n_atoms"])):
        e = embedding(sys, ik, a)
        m += e.conj().T @ dv["dh"][a] @ e
    return m


def interstitial_density(sys, cs, occ, wk, omega):
    """Fourier coefficients n_g of the interstitial density on the table box
    (shape vt_dim, g_i from -e_i to e_i): n_g = (1/Omega) sum_k w_k sum_j f_j
    sum_{G, G - g in the set} C_Gj conj(C_{G-g, j}), from the plane-wave rows
    of the coefficient matrices cs[k] (n_b x n_s); the e^{ik.r} phase of a
    Bloch state drops out of |psi|^2."""
    dim = np.asarray(sys["vt_dim"])
    e = (dim - 1) // 2
    box = np.zeros(tuple(int(x) for x in dim), dtype=np.complex128)
    for ik, c in enumerate(cs):
        gi = np.asarray(sys["g_int"][ik])
        cg = np.asarray(c)[:gi.shape[0], :]
        for g in range(gi.shape[0]):
            d = gi[g][None, :] - gi + e[None, :]
            val = wk[ik] * ((cg[g][None, :] * np.conj(cg)) @ occ)
            np.add.at(box, (d[:, 0], d[:, 1], d[:, 2]), val)
    return box / omega


def mt_density(sys, cs, occ, wk):
    """Muffin-tin density matrices of every atom: n_a = sum_k w_k sum_j f_j
    v_kj v_kj^H with v_kj = E_a c_kj = [A_a c_G ; c_lo(a)], the occupations of
    the atom's matching (u, u') and local-orbital channels, i.e. the
    coefficients of the sphere's density in products of its radial functions
    (Appendix A, the muffin-tin part of Eq. v_MT).  cs[k] is n_b x n_s."""
    out = []
    for a in range(int(sys["n_atoms"])):
        m = int(sys["n_a"][a]) + int(sys["n_lo"][a])
        n = np.zeros((m, m), dtype=np.complex128)
        for ik, c in enumerate(cs):
            v = embedding(sys, ik, a) @ np.asarray(c)
            n += wk[ik] * (v * np.asarray(occ)[None, :]) @ v.conj().T
        out.append(n)
    return out


def hartree_table(sys, n, n0):
    """dV_g = 4 pi (n_g - n0_g) / |g|^2 on the table box, 0 at g = 0 (the
    Poisson equation in G space; g cartesian from the reciprocal vectors)."""
    dim = np.asarray(sys["vt_dim"])
    e = (dim - 1) // 2
    r = [np.arange(-x, x + 1) for x in e]
    d1, d2, d3 = np.meshgrid(r[0], r[1], r[2], indexing="ij")
    gc = np.stack([d1, d2, d3], axis=-1).astype(np.float64) @ np.asarray(sys["recip"])
    g2 = np.einsum("...i,...i->...", gc, gc)
    out = np.zeros_like(n)
    nz = g2 > 0
    out[nz] = 4.0 * math.pi * (n[nz] - n0[nz]) / g2[nz]
    return out


def hamiltonian(ops, a_vec, c_light, dv_mat=None, dv_scale=0.0):
    """H(t) = H0 + (A/c).P + |A|^2/(2c^2) S (+ s dV_1): the velocity-gauge
    Hamiltonian of Sec. 2 in the LAPW+LO basis."""
    a = np.asarray(a_vec, dtype=np.float64)
    h = ops["H0"].copy()
    for l in range(3):
        if a[l] != 0.0:
            h += (a[l] / c_light) * ops["P"][l]
    h += (float(a @ a) / (2.0 * c_light ** 2)) * ops["S"]
    if dv_mat is not None and dv_scale != 0.0:
        h += dv_scale * dv_mat
    return h


# ------------------------------------------------------- auxiliary subspace

def fix_phases(cc):
    """Scale each column so that the sum of its entries is real positive."""
    s = cc.sum(axis=0)
    ph = np.where(np.abs(s) > 0, np.conj(s) / np.abs(s), 1.0)
    return cc * ph[None, :]


def ritz_basis(ops, trial):
    """Ritz vectors of H0 in span(trial), S-orthonormal, ascending Ritz values
    (the auxiliary basis of Eq. auxiliary_basis for the synthetic system)."""
    hr = trial.conj().T @ ops["H0"] @ trial
    mr = trial.conj().T @ ops["S"] @ trial
    hr = 0.5 * (hr + hr.conj().T)
    mr = 0.5 * (mr + mr.conj().T)
    eps, y = sla.eigh(hr, mr)
    cc = fix_phases(trial @ y)
    return cc, eps


def critical_timestep(eigvals, f=F_CRIT):
    """Eq. critical_timestep: dt_cr = f / (eps_max - eps_min)."""
    return f / (float(np.max(eigvals)) - float(np.min(eigvals)))


def overall_speedup(t_step, dt_cr, t_step_ref, dt_cr_ref):
    """Speed-up in propagating 1 a.u. of time against a reference code: the
    ratio of (time per step / step length) (Sec. 3.1, Table tab:H2)."""
    return (t_step_ref / dt_cr_ref) / (t_step / dt_cr)


def propagate_exact(hsub, ssub, theta, dt):
    """theta' = exp(-i SS^{-1} HH dt) theta for SS theta' = -i HH theta
    (Eq. evolution_of_projection_coeff), by the generalized eigenproblem
    HH V = SS V Lambda, V^H SS V = I: theta' = V e^{-i Lambda dt} V^H SS theta."""
    lam, v = sla.eigh(0.5 * (hsub + hsub.conj().T), 0.5 * (ssub + ssub.conj().T))
    return v @ (np.exp(-1j * lam * dt)[:, None] * (v.conj().T @ (ssub @ theta))), lam


def propagate_cn(hsub, ssub, theta, dt):
    """Crank-Nicolson: (SS + i dt/2 HH) theta' = (SS - i dt/2 HH) theta."""
    lhs = ssub + 0.5j * dt * hsub
    rhs = (ssub - 0.5j * dt * hsub) @ theta
    lam = sla.eigvalsh(0.5 * (hsub + hsub.conj().T), 0.5 * (ssub + ssub.conj().T))
    return np.linalg.solve(lhs, rhs), lam


# ------------------------------------------------------------------ the run

class Oracle:
    """The method on one synthetic system, every operator explicit.

    aux_mode "ritz": the auxiliary basis is built from sys["caux"] (trial
    vectors); "given": `caux` and `eps` are used as they are.
    """

    def __init__(self, sys, aux_mode="ritz", caux=None, eps=None, c0=None, dv=None):
        self.sys = sys
        self.c = float(sys["c_light"])
        self.omega = float(sys["omega"])
        self.occ = np.asarray(sys["occ"], dtype=np.float64)
        self.wk = np.asarray(sys["wk"], dtype=np.float64)
        self.n_s = int(sys["n_s"])
        self.n_aux = int(sys["n_aux"]) if aux_mode == "ritz" else int(caux[0].shape[1])
        self.kp = []
        for ik in range(int(sys["n_k"])):
            ops = explicit_operators(sys, ik)
            if aux_mode == "ritz":
                cc, ev = ritz_basis(ops, np.asarray(sys["caux"][ik]))
            else:
                cc, ev = np.asarray(caux[ik]), np.asarray(eps[ik])
            # projected, time-independent parts of Eq. auxiliary_hamiltonian_with_parts
            h0s = cc.conj().T @ ops["H0"] @ cc
            ps = np.stack([cc.conj().T @ ops["P"][l] @ cc for l in range(3)])
            ss = cc.conj().T @ ops["S"] @ cc
            dvm = explicit_dv(sys, ik, dv) if dv is not None else None
            if c0 is None:
                theta0 = np.zeros((self.n_aux, self.n_s), dtype=np.complex128)
                theta0[np.arange(self.n_s), np.arange(self.n_s)] = 1.0
            else:
                theta0 = cc.conj().T @ ops["S"] @ c0[ik]
            self.kp.append(dict(ops=ops, caux=cc, eps=ev, h0sub=h0s, psub=ps, ssub=ss,
                                dv=dvm, theta0=theta0))
        self.j_gs = self._current_full([kp["caux"] @ kp["theta0"] for kp in self.kp],
                                       np.zeros(3))

    # Eq. auxiliary_hamiltonian_with_parts with VV(t) = VV(0) + dVV(t),
    # T + VV(0) = CC^H H0 CC, dVV(t) = CC^H (s dV_1) CC recomputed per step
    def subspace_hamiltonian(self, ik, a_vec, dv_scale=0.0, extra=None):
        kp = self.kp[ik]
        a = np.asarray(a_vec, dtype=np.float64)
        h = kp["h0sub"].copy()
        for l in range(3):
            h += (a[l] / self.c) * kp["psub"][l]
        h += (float(a @ a) / (2.0 * self.c ** 2)) * kp["ssub"]
        if kp["dv"] is not None and dv_scale != 0.0:
            cc = kp["caux"]
            h += cc.conj().T @ (dv_scale * kp["dv"]) @ cc
        if extra is not None:
            cc = kp["caux"]
            h += cc.conj().T @ extra @ cc
        return h

    def hartree_matrices(self, thetas, n0, mt0=None, mt_u=0.0):
        """Dense potential change of every k-point for the state C = CC theta:
        the interstitial Hartree potential of its density against the
        reference n0 and, when mt_u != 0, the muffin-tin blocks
        dh_a = mt_u (n_a - mt0_a) of its muffin-tin density matrices."""
        cs = [kp["caux"] @ t for kp, t in zip(self.kp, thetas)]
        table = hartree_table(self.sys, interstitial_density(self.sys, cs, self.occ, self.wk, self.omega), n0)
        dh = None
        if mt_u != 0.0:
            dh = [mt_u * (na - n0a) for na, n0a in zip(mt_density(self.sys, cs, self.occ, self.wk), mt0)]
        out = []
        for ik, kp in enumerate(self.kp):
            ng = kp["ops"]["ng"]
            m = np.zeros((kp["ops"]["nb"], kp["ops"]["nb"]), dtype=np.complex128)
            m[:ng, :ng] = interstitial_potential(self.sys["g_int"][ik], self.sys["vt_dim"], table)
            if dh is not None:
                for a in range(int(self.sys["n_atoms"])):
                    e = embedding(self.sys, ik, a)
                    m += e.conj().T @ dh[a] @ e
            out.append(m)
        return out, table

    def _current_full(self, cs, a_vec):
        a = np.asarray(a_vec, dtype=np.float64)
        j = np.zeros(3)
        for ik, c in enumerate(cs):
            kp = self.kp[ik]
            sc = kp["ops"]["S"] @ c
            for l in range(3):
                m = kp["ops"]["P"][l] @ c + (a[l] / self.c) * sc
                val = np.real(np.sum(np.conj(c) * m, axis=0))
                j[l] += self.wk[ik] * (-1.0 / self.omega) * float(self.occ @ val)
        return j

    def _current_sub(self, thetas, a_vec):
        a = np.asarray(a_vec, dtype=np.float64)
        j = np.zeros(3)
        for ik, th in enumerate(thetas):
            kp = self.kp[ik]
            st = kp["ssub"] @ th
            for l in range(3):
                m = kp["psub"][l] @ th + (a[l] / self.c) * st
                val = np.real(np.sum(np.conj(th) * m, axis=0))
                j[l] += self.wk[ik] * (-1.0 / self.omega) * float(self.occ @ val)
        return j

    def run(self, a_samples, dt, propagator="exact", reproject=False, dv_scale=None,
            thetas=None, keep_states=False, hartree=False, mt_u=0.0):
        """Propagate len(a_samples) steps.  Returns a dict of per-step records
        (t, J, J_full, dmu, E, norm_dev, resid, dtcr, n_exc), final theta and C.
        hartree: the interstitial Hartree potential of the density of C_k
        (against that of the starting state) acts during step k; with
        mt_u != 0 also the muffin-tin blocks mt_u (n_a(C_k) - n_a(C_0))."""
        a_samples = np.asarray(a_samples, dtype=np.float64)
        n = a_samples.shape[0]
        nk = len(self.kp)
        th = [kp["theta0"].copy() for kp in self.kp] if thetas is None else \
            [t.copy() for t in thetas]
        rec = {key: [] for key in ("t", "J", "J_full", "dmu", "E", "norm_dev", "resid",
                                   "dtcr", "n_exc")}
        states = []
        dmu = np.zeros(3)
        jind_prev = np.zeros(3)
        if hartree:
            cs0 = [kp["caux"] @ t for kp, t in zip(self.kp, th)]
            n0 = interstitial_density(self.sys, cs0, self.occ, self.wk, self.omega)
            mt0 = mt_density(self.sys, cs0, self.occ, self.wk) if mt_u != 0.0 else None
            rec["hartree_l1"] = []
        for k in range(n):
            a = a_samples[k]
            s = 0.0 if dv_scale is None else float(dv_scale[k])
            cs, hcs, e_tot, ndev, res, lam_rng = [], [], 0.0, 0.0, 0.0, []
            vh = [None] * nk
            if hartree:
                vh, table = self.hartree_matrices(th, n0, mt0, mt_u)
                rec["hartree_l1"].append(float(np.sum(np.abs(table))))
            for ik in range(nk):
                kp = self.kp[ik]
                hsub = self.subspace_hamiltonian(ik, a, s, extra=vh[ik])
                if propagator == "exact":
                    th[ik], lam = propagate_exact(hsub, kp["ssub"], th[ik], dt)
                elif propagator == "cn":
                    th[ik], lam = propagate_cn(hsub, kp["ssub"], th[ik], dt)
                else:
                    raise ValueError(propagator)
                lam_rng.append(float(lam[-1] - lam[0]))
                # expand back (Eq. approximation_coefficients)
                c = kp["caux"] @ th[ik]
                # apply H(t) and S with the explicit matrices
                h = hamiltonian(kp["ops"], a, self.c, kp["dv"], s)
                if vh[ik] is not None:
                    h = h + vh[ik]
                hc = h @ c
                sc = kp["ops"]["S"] @ c
                # project (theta = CC^H S C)
                tt = kp["caux"].conj().T @ sc
                res = max(res, float(np.max(np.abs(tt - th[ik]))))
                norm = c.conj().T @ sc
                ndev = max(ndev, float(np.max(np.abs(norm - np.eye(self.n_s)))))
                e_tot += self.wk[ik] * float(self.occ @ np.real(np.sum(np.conj(c) * hc, 0)))
                if reproject:
                    g = tt.conj().T @ tt
                    w, u = np.linalg.eigh(0.5 * (g + g.conj().T))
                    th[ik] = tt @ (u @ np.diag(w ** -0.5) @ u.conj().T)
                cs.append(c)
            j_sub = self._current_sub(th, a)
            j_full = self._current_full(cs, a)
            jind = j_sub - self.j_gs
            dmu = dmu + self.omega * dt * 0.5 * (jind_prev + jind)
            jind_prev = jind
            rec["t"].append((k + 1) * dt)
            rec["J"].append(j_sub)
            rec["J_full"].append(j_full)
            rec["dmu"].append(dmu.copy())
            rec["E"].append(e_tot)
            rec["norm_dev"].append(ndev)
            rec["resid"].append(res)
            rec["dtcr"].append(F_CRIT / max(lam_rng))
            rec["n_exc"].append(self.excited_electrons(th))
            if keep_states:
                states.append([t.copy() for t in th])
        out = {key: np.asarray(v) for key, v in rec.items()}
        out["theta"] = th
        out["C"] = [kp["caux"] @ t for kp, t in zip(self.kp, th)]
        if keep_states:
            out["states"] = states
        return out

    def excited_electrons(self, thetas):
        """N_exc = N_e - sum_k w_k sum_j f_j sum_{i < N_s} |theta_ij|^2: the
        charge outside the N_s lowest auxiliary vectors, i.e. the occupied
        ground state (the quantity the paper plots for CO and pyridine@MoS2
        without a formula; this is the reading used here)."""
        ne = float(np.sum(self.wk) * np.sum(self.occ))
        kept = 0.0
        for ik, th in enumerate(thetas):
            occ_block = th[:self.n_s, :]
            kept += self.wk[ik] * float(np.sum(self.occ[None, :] * np.abs(occ_block) ** 2))
        return ne - kept

    def energy(self, thetas, a_vec, dv_scale=0.0):
        """E = sum_k w_k sum_j f_j Re c_j^H H(A) c_j with c = CC theta."""
        e = 0.0
        for ik, th in enumerate(thetas):
            kp = self.kp[ik]
            c = kp["caux"] @ th
            h = hamiltonian(kp["ops"], a_vec, self.c, kp["dv"], dv_scale)
            e += self.wk[ik] * float(self.occ @ np.real(np.sum(np.conj(c) * (h @ c), 0)))
        return e

    # ------------------------------------------------------------ gradient
    def dipole_gradient(self, a_samples, dt, gdir, seeds, dv_scale=None):
        """d(gdir . dmu(T)) / d A_{k,l} for the (k, l) pairs in `seeds`, by
        forward-mode tangent propagation through the exact-exponential steps.
        The derivative of exp(-i dt HH) along E uses the Daleckii-Krein
        formula V (Gamma o (V^H E V)) V^H with the divided differences
        Gamma_ij = (e^{-i dt l_i} - e^{-i dt l_j}) / (l_i - l_j).
        Requires SS = I (Ritz basis)."""
        a_samples = np.asarray(a_samples, dtype=np.float64)
        g = np.asarray(gdir, dtype=np.float64)
        n = a_samples.shape[0]
        nk = len(self.kp)
        # forward sweep: store theta_k and the eigen-decompositions
        th = [kp["theta0"].copy() for kp in self.kp]
        hist_th = [[t.copy() for t in th]]
        eig = []
        for k in range(n):
            s = 0.0 if dv_scale is None else float(dv_scale[k])
            step = []
            for ik in range(nk):
                hsub = self.subspace_hamiltonian(ik, a_samples[k], s)
                lam, v = np.linalg.eigh(0.5 * (hsub + hsub.conj().T))
                step.append((lam, v))
                th[ik] = v @ (np.exp(-1j * lam * dt)[:, None] * (v.conj().T @ th[ik]))
            eig.append(step)
            hist_th.append([t.copy() for t in th])
        wts = np.ones(n)
        wts[-1] = 0.5
        out = []
        for (k0, l0) in seeds:
            dth = [np.zeros_like(t) for t in th]
            total = 0.0
            for ik in range(nk):
                lam, v = eig[k0][ik]
                e_dir = self.kp[ik]["psub"][l0] / self.c + \
                    (a_samples[k0, l0] / self.c ** 2) * np.eye(self.n_aux)
                d = lam[:, None] - lam[None, :]
                x = 0.5 * dt * d
                sinc = np.where(np.abs(x) > 1e-30, np.sin(x) / np.where(x == 0, 1, x), 1.0)
                gam = -1j * dt * np.exp(-0.5j * dt * (lam[:, None] + lam[None, :])) * sinc
                du = v @ (gam * (v.conj().T @ e_dir @ v)) @ v.conj().T
                dth[ik] = du @ hist_th[k0][ik]
            # direct dependence of J(t_{k0+1}) on A_{k0}
            nel = sum(self.wk[ik] * float(self.occ @ np.real(np.sum(
                np.conj(hist_th[k0 + 1][ik]) * (self.kp[ik]["ssub"] @ hist_th[k0 + 1][ik]),
                0))) for ik in range(nk))
            total += dt * wts[k0] * g[l0] * (-1.0) * nel / self.c
            for m in range(k0 + 1, n + 1):
                if m > k0 + 1:
                    for ik in range(nk):
                        lam, v = eig[m - 1][ik]
                        dth[ik] = v @ (np.exp(-1j * lam * dt)[:, None] * (v.conj().T @ dth[ik]))
                # dJ_l(t_m) = -(1/Omega) sum f 2 Re theta^H (P_l + a/c S) dtheta
                am = a_samples[m - 1]
                for ik in range(nk):
                    kp = self.kp[ik]
                    t_m = hist_th[m][ik]
                    for l in range(3):
                        if g[l] == 0.0:
                            continue
                        mm = kp["psub"][l] @ dth[ik] + (am[l] / self.c) * (kp["ssub"] @ dth[ik])
                        val = 2.0 * np.real(np.sum(np.conj(t_m) * mm, 0))
                        dj = self.wk[ik] * (-1.0 / self.omega) * float(self.occ @ val)
                        total += self.omega * dt * wts[m - 1] * g[l] * dj
            out.append(total)
        return np.asarray(out)


def full_basis_propagator(ops, a_vec, c_light, dt):
    """exp(-i S^{-1} H dt) for the full coefficient ODE (Eq. evolution_wf_coeff),
    evaluated as S^{-1/2} expm(-i dt S^{-1/2} H S^{-1/2}) S^{1/2} with the
    Pade scaling-and-squaring expm."""
    h = hamiltonian(ops, a_vec, c_light)
    s = ops["S"]
    w, u = np.linalg.eigh(0.5 * (s + s.conj().T))
    s_mh = (u * w ** -0.5) @ u.conj().T
    s_h = (u * w ** 0.5) @ u.conj().T
    ht = s_mh @ h @ s_mh
    return s_mh @ sla.expm(-1j * dt * 0.5 * (ht + ht.conj().T)) @ s_h


def polarizability(t0, dt, j_ind, e_field, w, omega_cell, eta=0.0):
    """Eq. polarizability: alpha_{l l'}(w) = (i Omega / w) J_l(w) / E_l'(w), the
    time series taken to the frequency domain by the damped discrete transform
    F(w) = dt sum_n f(t_n) e^{(i w - eta) t_n}, t_n = t0 + n dt (the paper does
    not give its transform; this is the reading used here).  Entries whose
    E_l'(w) is exactly zero are 0.  Returns (alpha [n_w, 3, 3], J(w), E(w))."""
    j_ind = np.asarray(j_ind, dtype=np.float64).reshape(-1, 3)
    e_field = np.asarray(e_field, dtype=np.float64).reshape(-1, 3)
    w = np.asarray(w, dtype=np.float64).ravel()
    t = t0 + dt * np.arange(j_ind.shape[0])
    kern = np.exp((1j * w[:, None] - eta) * t[None, :])  # [n_w, n_t]
    jw = dt * kern @ j_ind
    ew = dt * kern @ e_field
    alpha = np.zeros((w.size, 3, 3), dtype=np.complex128)
    for lp in range(3):
        nz = ew[:, lp] != 0
        alpha[nz, :, lp] = (1j * omega_cell / w[nz, None]) * jw[nz, :] / ew[nz, lp, None]
    return alpha, jw, ew
