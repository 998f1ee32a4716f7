"""ctypes binding of the rttddft C ABI (include/rttddft.h).

Argument marshalling only: every step of the method runs in the CUDA
library.  The functions carry the ABI's names; `Context` wraps them for a
system given as the dict produced by `synth.make_system` (or any dict with
the same keys).  Importing this module does not load the library; the first
call does, and fails loudly if it has not been built.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB_PATH

RTTDDFT_OK = 0
ERRORS = {
    -1: "ERR_ARG", -2: "ERR_NOT_HERMITIAN", -3: "ERR_NOT_PD", -4: "ERR_NOT_ORTHONORMAL",
    -5: "ERR_NONFINITE", -6: "ERR_OOM", -7: "ERR_CUDA", -8: "ERR_TIMEOUT", -9: "ERR_UNSUPPORTED",
}
PROP = {"chebyshev": 0, "eig": 1, "cn": 2}
PREC = {"fp64": 0, "fp32": 1, "bf16x3": 2, "fp16x3": 3}
AUX = {"ritz": 0, "given": 1}
INTERSTITIAL = {"toeplitz": 0, "fft": 1}

EXPORTED = ["rttddft_default_options", "rttddft_setup", "rttddft_step", "rttddft_observables",
            "rttddft_set_dv", "rttddft_apply", "rttddft_get_state", "rttddft_set_state",
            "rttddft_get_aux", "rttddft_get_info", "rttddft_adjoint", "rttddft_trace_steps",
            "rttddft_apply_noalloc", "rttddft_zgemm_bf16x3", "rttddft_polarizability",
            "rttddft_destroy", "rttddft_last_error", "rttddft_version"]

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


class rttddft_system(ctypes.Structure):
    _fields_ = [("n_k", ctypes.c_int), ("n_atoms", ctypes.c_int), ("n_s", ctypes.c_int),
                ("n_aux", ctypes.c_int), ("omega", ctypes.c_double), ("c_light", ctypes.c_double),
                ("occ", _dp), ("wk", _dp), ("n_g", _ip), ("g_int", _ip), ("gk", _dp),
                ("n_a", _ip), ("n_lo", _ip), ("amat", _dp), ("h", _dp), ("o", _dp), ("p", _dp),
                ("vt_dim", ctypes.c_int * 3), ("vtab", _dp), ("caux", _dp), ("eps", _dp),
                ("c0", _dp), ("recip", ctypes.c_double * 9)]


class rttddft_options(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("propagator", ctypes.c_int), ("precision", ctypes.c_int),
                ("reproject", ctypes.c_int), ("aux_mode", ctypes.c_int),
                ("max_record", ctypes.c_int), ("graph_steps", ctypes.c_int),
                ("cheb_tol", ctypes.c_double), ("ortho_tol", ctypes.c_double),
                ("max_sweeps", ctypes.c_int), ("a_max", ctypes.c_double),
                ("s_max", ctypes.c_double), ("interstitial", ctypes.c_int), ("hartree", ctypes.c_int),
                ("hartree_bound", ctypes.c_double), ("hartree_mt_u", ctypes.c_double)]


class rttddft_obs(ctypes.Structure):
    _fields_ = [("capacity", ctypes.c_int), ("count", ctypes.c_int), ("t", _dp), ("j", _dp),
                ("j_full", _dp), ("dmu", _dp), ("energy", _dp), ("norm_dev", _dp),
                ("resid", _dp), ("dt_cr", _dp), ("n_exc", _dp)]


class rttddft_info(ctypes.Structure):
    _fields_ = [("steps_done", ctypes.c_longlong), ("time", ctypes.c_double),
                ("n_basis_max", ctypes.c_int), ("cheb_terms", ctypes.c_int),
                ("dt_cr0", ctypes.c_double), ("kernel_launches_per_step", ctypes.c_int),
                ("precision", ctypes.c_int), ("tc_tile_n", ctypes.c_int), ("tc_stages", ctypes.c_int),
                ("tc_kblocks", ctypes.c_int), ("tc_slices", ctypes.c_int), ("tc_window", ctypes.c_int),
                ("tc_smem", ctypes.c_int), ("tc_candidates", ctypes.c_int),
                ("tc_interstitial_ns", ctypes.c_int), ("tc_matching_ns", ctypes.c_int),
                ("interstitial", ctypes.c_int), ("fft_grid", ctypes.c_int * 3), ("fft_fused", ctypes.c_int),
                ("tc_gen_threads", ctypes.c_int), ("tc_a_tmem", ctypes.c_int),
                ("tc_back_parts", ctypes.c_int)]


class rttddft_trace(ctypes.Structure):
    _fields_ = [("capacity", ctypes.c_int), ("count", ctypes.c_int),
                ("names", ctypes.POINTER(ctypes.c_char_p)), ("ms", _dp)]


class RttddftError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code


_lib = None


def load_library(path=None):
    """Load librttddft.so (built in-tree); raises if it is missing."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError("librttddft.so is not built (%s); run __graft_entry__.build()" % p)
    lib = ctypes.CDLL(p)
    vp = ctypes.c_void_p
    lib.rttddft_default_options.argtypes = [ctypes.POINTER(rttddft_options)]
    lib.rttddft_default_options.restype = None
    lib.rttddft_setup.argtypes = [ctypes.POINTER(rttddft_system), ctypes.POINTER(rttddft_options),
                                  vp, ctypes.POINTER(vp)]
    lib.rttddft_setup.restype = ctypes.c_int
    lib.rttddft_step.argtypes = [vp, ctypes.c_int, vp, vp]
    lib.rttddft_step.restype = ctypes.c_int
    lib.rttddft_observables.argtypes = [vp, ctypes.POINTER(rttddft_obs), ctypes.c_int]
    lib.rttddft_observables.restype = ctypes.c_int
    lib.rttddft_set_dv.argtypes = [vp, vp, vp]
    lib.rttddft_set_dv.restype = ctypes.c_int
    lib.rttddft_apply.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, vp, ctypes.c_double, vp, vp]
    lib.rttddft_apply.restype = ctypes.c_int
    lib.rttddft_apply_noalloc.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, vp, ctypes.c_double,
                                          vp, vp]
    lib.rttddft_apply_noalloc.restype = ctypes.c_int
    lib.rttddft_get_state.argtypes = [vp, ctypes.c_int, vp, vp]
    lib.rttddft_get_state.restype = ctypes.c_int
    lib.rttddft_set_state.argtypes = [vp, ctypes.c_int, vp]
    lib.rttddft_set_state.restype = ctypes.c_int
    lib.rttddft_get_aux.argtypes = [vp, ctypes.c_int, vp, vp, vp]
    lib.rttddft_get_aux.restype = ctypes.c_int
    lib.rttddft_get_info.argtypes = [vp, ctypes.POINTER(rttddft_info)]
    lib.rttddft_get_info.restype = ctypes.c_int
    lib.rttddft_adjoint.argtypes = [vp, ctypes.c_int, vp, vp, vp, ctypes.c_int, vp, vp]
    lib.rttddft_adjoint.restype = ctypes.c_int
    lib.rttddft_trace_steps.argtypes = [vp, ctypes.c_int, vp, vp, ctypes.POINTER(rttddft_trace)]
    lib.rttddft_trace_steps.restype = ctypes.c_int
    lib.rttddft_zgemm_bf16x3.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp,
                                         ctypes.c_int, vp, ctypes.c_int, vp, ctypes.c_int, ctypes.c_int, vp]
    lib.rttddft_zgemm_bf16x3.restype = ctypes.c_int
    d = ctypes.c_double
    lib.rttddft_polarizability.argtypes = [ctypes.c_int, d, d, vp, vp, d, ctypes.c_int, vp, d, vp, vp, vp, vp]
    lib.rttddft_polarizability.restype = ctypes.c_int
    lib.rttddft_destroy.argtypes = [vp]
    lib.rttddft_destroy.restype = None
    lib.rttddft_last_error.argtypes = [vp]
    lib.rttddft_last_error.restype = ctypes.c_char_p
    lib.rttddft_version.argtypes = []
    lib.rttddft_version.restype = ctypes.c_char_p
    if path is None:
        _lib = lib
    return lib


def _ptr(a):
    """Address of a numpy array, a torch tensor, an int address, or None."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _check(ctx, code):
    if code != RTTDDFT_OK:
        msg = load_library().rttddft_last_error(ctx).decode()
        raise RttddftError(code, msg)


# ------------------------------------------------------------------ the ABI

def rttddft_default_options():
    o = rttddft_options()
    load_library().rttddft_default_options(ctypes.byref(o))
    return o


def rttddft_setup(system, options, stream=None):
    ctx = ctypes.c_void_p()
    code = load_library().rttddft_setup(ctypes.byref(system), ctypes.byref(options),
                                        stream, ctypes.byref(ctx))
    _check(None, code)
    return ctx


def rttddft_step(ctx, nsteps, a_samples, dv_scale=None):
    _check(ctx, load_library().rttddft_step(ctx, int(nsteps), _ptr(a_samples), _ptr(dv_scale)))


def rttddft_observables(ctx, obs, clear=1):
    _check(ctx, load_library().rttddft_observables(ctx, ctypes.byref(obs), int(clear)))


def rttddft_set_dv(ctx, dh, dvtab):
    _check(ctx, load_library().rttddft_set_dv(ctx, _ptr(dh), _ptr(dvtab)))


def rttddft_apply(ctx, k, ncols, x, a_vec, dv_scale, hx, sx):
    _check(ctx, load_library().rttddft_apply(ctx, int(k), int(ncols), _ptr(x), _ptr(a_vec),
                                             float(dv_scale), _ptr(hx), _ptr(sx)))


def rttddft_apply_noalloc(ctx, k, ncols, x, a_vec, dv_scale, hx, sx):
    """Operator apply with the library's static scratch (device pointers only)."""
    _check(ctx, load_library().rttddft_apply_noalloc(ctx, int(k), int(ncols), _ptr(x), _ptr(a_vec),
                                                     float(dv_scale), _ptr(hx), _ptr(sx)))


def rttddft_polarizability(t0, dt, j_ind, e_field, w, omega_cell, eta=0.0, stream=None):
    """alpha(w) of Eq. polarizability with J(w) and E(w) (numpy in, numpy out)."""
    j = np.ascontiguousarray(j_ind, dtype=np.float64).reshape(-1, 3)
    e = np.ascontiguousarray(e_field, dtype=np.float64).reshape(-1, 3)
    if j.shape != e.shape:
        raise ValueError("j_ind and e_field need the same [n_t][3] shape")
    wv = np.ascontiguousarray(w, dtype=np.float64).ravel()
    oj = np.zeros((wv.size, 3), dtype=np.complex128)
    oe = np.zeros((wv.size, 3), dtype=np.complex128)
    al = np.zeros((wv.size, 3, 3), dtype=np.complex128)
    lib = load_library()
    code = lib.rttddft_polarizability(int(j.shape[0]), float(t0), float(dt), _ptr(j), _ptr(e), float(eta),
                                      int(wv.size), _ptr(wv), float(omega_cell), _ptr(oj), _ptr(oe), _ptr(al),
                                      _ptr(stream))
    _check(None, code)
    return al, oj, oe


def rttddft_zgemm_bf16x3(trans, m, n, k, a, lda, x, ldx, c, ldc, beta_add=0, stream=None):
    """Split-BF16 complex GEMM on the tensor cores (device pointers)."""
    code = load_library().rttddft_zgemm_bf16x3(int(trans), int(m), int(n), int(k), _ptr(a), int(lda),
                                               _ptr(x), int(ldx), _ptr(c), int(ldc), int(beta_add),
                                               _ptr(stream))
    if code != RTTDDFT_OK:
        raise RttddftError(code, "rttddft_zgemm_bf16x3 failed (%s)" % ERRORS.get(code, code))


def rttddft_get_state(ctx, k, theta, c=None):
    _check(ctx, load_library().rttddft_get_state(ctx, int(k), _ptr(theta), _ptr(c)))


def rttddft_set_state(ctx, k, theta):
    _check(ctx, load_library().rttddft_set_state(ctx, int(k), _ptr(theta)))


def rttddft_get_aux(ctx, k, caux, eps, pp=None):
    _check(ctx, load_library().rttddft_get_aux(ctx, int(k), _ptr(caux), _ptr(eps), _ptr(pp)))


def rttddft_get_info(ctx):
    info = rttddft_info()
    _check(ctx, load_library().rttddft_get_info(ctx, ctypes.byref(info)))
    return info


def rttddft_adjoint(ctx, nsteps, a_samples, dv_scale, gdir, ckpt_every, grad, dmu_out=None):
    _check(ctx, load_library().rttddft_adjoint(ctx, int(nsteps), _ptr(a_samples), _ptr(dv_scale),
                                               _ptr(gdir), int(ckpt_every), _ptr(grad),
                                               _ptr(dmu_out)))


def rttddft_trace_steps(ctx, nsteps, a_samples, dv_scale, trace):
    _check(ctx, load_library().rttddft_trace_steps(ctx, int(nsteps), _ptr(a_samples), _ptr(dv_scale),
                                                   ctypes.byref(trace)))


def rttddft_destroy(ctx):
    load_library().rttddft_destroy(ctx)


def rttddft_last_error(ctx=None):
    return load_library().rttddft_last_error(ctx).decode()


def rttddft_version():
    return load_library().rttddft_version().decode()


# ------------------------------------------------------------------ wrapper

def _cat_f(mats, dtype=np.complex128):
    if not mats:
        return np.zeros(1, dtype=dtype)
    return np.ascontiguousarray(np.concatenate([np.asarray(m, dtype=dtype).ravel(order="F")
                                                for m in mats]))


class Context:
    """One rttddft context for a system dict (see synth.make_system)."""

    def __init__(self, sys, dt=None, propagator="chebyshev", precision="fp64", reproject=False,
                 aux_mode="ritz", caux=None, eps=None, c0=None, max_record=4096, graph_steps=1,
                 cheb_tol=1e-16, stream=None, max_sweeps=30, a_max=0.0, s_max=0.0,
                 interstitial="toeplitz", hartree=False, hartree_bound=None, hartree_mt_u=0.0):
        self.n_k = int(sys["n_k"])
        self.n_s = int(sys["n_s"])
        self.n_aux = int(sys["n_aux"]) if caux is None else int(np.asarray(caux[0]).shape[1])
        self.n_g = np.ascontiguousarray(sys["n_g"], dtype=np.int32)
        n_lo = np.ascontiguousarray(sys["n_lo"], dtype=np.int32)
        self.n_b = self.n_g + int(n_lo.sum())
        self._keep = keep = {}
        keep["occ"] = np.ascontiguousarray(sys["occ"], dtype=np.float64)
        keep["wk"] = np.ascontiguousarray(sys["wk"], dtype=np.float64)
        keep["n_g"] = self.n_g
        keep["g_int"] = np.ascontiguousarray(np.concatenate(sys["g_int"]), dtype=np.int32)
        keep["gk"] = np.ascontiguousarray(np.concatenate(sys["gk"]), dtype=np.float64)
        keep["n_a"] = np.ascontiguousarray(sys["n_a"], dtype=np.int32)
        keep["n_lo"] = n_lo
        keep["amat"] = _cat_f(sys["amat"])
        keep["h"] = _cat_f(sys["h"])
        keep["o"] = _cat_f(sys["o"])
        keep["p"] = _cat_f([pl for pa in sys["p"] for pl in pa])
        keep["vtab"] = np.ascontiguousarray(np.asarray(sys["vtab"], dtype=np.complex128).ravel(order="C"))
        keep["caux"] = _cat_f(sys["caux"] if caux is None else caux)
        keep["eps"] = None if eps is None else np.ascontiguousarray(np.concatenate(eps), dtype=np.float64)
        keep["c0"] = None if c0 is None else _cat_f(c0)
        s = rttddft_system()
        s.n_k, s.n_atoms, s.n_s, s.n_aux = self.n_k, int(sys["n_atoms"]), self.n_s, self.n_aux
        s.omega, s.c_light = float(sys["omega"]), float(sys["c_light"])
        for name in ("occ", "wk", "gk", "amat", "h", "o", "p", "vtab", "caux", "eps", "c0"):
            arr = keep[name]
            setattr(s, name, None if arr is None else arr.ctypes.data_as(_dp))
        for name in ("n_g", "g_int", "n_a", "n_lo"):
            setattr(s, name, keep[name].ctypes.data_as(_ip))
        s.vt_dim[:] = [int(x) for x in sys["vt_dim"]]
        if "recip" in sys:
            s.recip[:] = [float(x) for x in np.asarray(sys["recip"], dtype=np.float64).ravel()]
        o = rttddft_default_options()
        o.dt = float(sys["dt"] if dt is None else dt)
        o.propagator = PROP[propagator]
        o.precision = PREC[precision]
        o.reproject = int(bool(reproject))
        o.aux_mode = AUX[aux_mode]
        o.max_record = int(max_record)
        o.graph_steps = int(graph_steps)
        o.cheb_tol = float(cheb_tol)
        o.max_sweeps = int(max_sweeps)
        o.a_max = float(a_max)
        o.s_max = float(s_max)
        o.interstitial = INTERSTITIAL[interstitial]
        o.hartree = int(bool(hartree))
        if hartree_bound is not None:
            o.hartree_bound = float(hartree_bound)
        o.hartree_mt_u = float(hartree_mt_u)
        self.options = o
        self.max_record = int(max_record)
        self._stream = stream
        self.ctx = rttddft_setup(s, o, stream)

    def stream_handle(self):
        """The cudaStream_t given at set-up (0/None: the library's own stream)."""
        return self._stream or 0

    def step(self, a_samples, dv_scale=None):
        a = a_samples
        if isinstance(a, np.ndarray):
            a = np.ascontiguousarray(a, dtype=np.float64)
        n = int(a.shape[0])
        d = dv_scale
        if isinstance(d, np.ndarray):
            d = np.ascontiguousarray(d, dtype=np.float64)
        rttddft_step(self.ctx, n, a, d)

    def observables(self, clear=True):
        cap = self.max_record
        out = {k: np.zeros(cap) for k in ("t", "energy", "norm_dev", "resid", "dt_cr", "n_exc")}
        for k in ("j", "j_full", "dmu"):
            out[k] = np.zeros((cap, 3))
        obs = rttddft_obs()
        obs.capacity = cap
        for k, v in out.items():
            setattr(obs, k, v.ctypes.data_as(_dp))
        rttddft_observables(self.ctx, obs, int(clear))
        n = obs.count
        return {k: v[:n].copy() for k, v in out.items()}

    def apply(self, k, x, a_vec=(0.0, 0.0, 0.0), dv_scale=0.0):
        if hasattr(x, "data_ptr"):
            hx = x.new_empty(x.shape)
            sx = x.new_empty(x.shape)
            ncols = x.shape[1] if x.dim() == 2 else 1
        else:
            x = np.asfortranarray(x, dtype=np.complex128)
            hx = np.zeros_like(x, order="F")
            sx = np.zeros_like(x, order="F")
            ncols = x.shape[1] if x.ndim == 2 else 1
        av = np.ascontiguousarray(a_vec, dtype=np.float64)
        rttddft_apply(self.ctx, k, ncols, x, av, dv_scale, hx, sx)
        return hx, sx

    def get_state(self, k, with_c=False):
        th = np.zeros((self.n_aux, self.n_s), dtype=np.complex128, order="F")
        c = np.zeros((int(self.n_b[k]), self.n_s), dtype=np.complex128, order="F") if with_c else None
        rttddft_get_state(self.ctx, k, th, c)
        return (th, c) if with_c else th

    def set_state(self, k, theta):
        th = np.asfortranarray(theta, dtype=np.complex128)
        rttddft_set_state(self.ctx, k, th)

    def get_aux(self, k):
        cc = np.zeros((int(self.n_b[k]), self.n_aux), dtype=np.complex128, order="F")
        ev = np.zeros(self.n_aux)
        pp = np.zeros((3, self.n_aux, self.n_aux), dtype=np.complex128)
        ppf = np.zeros(3 * self.n_aux * self.n_aux, dtype=np.complex128)
        rttddft_get_aux(self.ctx, k, cc, ev, ppf)
        for l in range(3):
            pp[l] = ppf[l * self.n_aux ** 2:(l + 1) * self.n_aux ** 2].reshape(
                self.n_aux, self.n_aux, order="F")
        return cc, ev, pp

    def info(self):
        i = rttddft_get_info(self.ctx)
        return dict(steps_done=i.steps_done, time=i.time, n_basis_max=i.n_basis_max,
                    cheb_terms=i.cheb_terms, dt_cr0=i.dt_cr0,
                    kernel_launches_per_step=i.kernel_launches_per_step, precision=i.precision,
                    tc=dict(tile_n=i.tc_tile_n, stages=i.tc_stages, kblocks=i.tc_kblocks,
                            slices=i.tc_slices, window=i.tc_window, smem=i.tc_smem,
                            candidates=i.tc_candidates, interstitial_ns=i.tc_interstitial_ns,
                            matching_ns=i.tc_matching_ns, gen_threads=i.tc_gen_threads,
                            a_tmem=i.tc_a_tmem, back_parts=i.tc_back_parts),
                    interstitial=i.interstitial, fft_grid=tuple(int(x) for x in i.fft_grid),
                    fft_fused=i.fft_fused)

    def set_dv(self, dv):
        self._dh = _cat_f(dv["dh"])
        self._dvt = np.ascontiguousarray(np.asarray(dv["dvtab"], dtype=np.complex128).ravel(order="C"))
        rttddft_set_dv(self.ctx, self._dh, self._dvt)

    def adjoint(self, a_samples, gdir, ckpt_every=50, dv_scale=None):
        a = np.ascontiguousarray(a_samples, dtype=np.float64)
        n = a.shape[0]
        g = np.ascontiguousarray(gdir, dtype=np.float64)
        grad = np.zeros((n, 3))
        dmu = np.zeros(3)
        d = None if dv_scale is None else np.ascontiguousarray(dv_scale, dtype=np.float64)
        rttddft_adjoint(self.ctx, n, a, d, g, int(ckpt_every), grad, dmu)
        return grad, dmu

    def trace(self, a_samples, dv_scale=None):
        """Per-launch device milliseconds of the steps, summed over the samples."""
        a = np.ascontiguousarray(a_samples, dtype=np.float64)
        d = None if dv_scale is None else np.ascontiguousarray(dv_scale, dtype=np.float64)
        cap = 256
        t = rttddft_trace()
        t.capacity = cap
        names = (ctypes.c_char_p * cap)()
        ms = np.zeros(cap)
        t.names = names
        t.ms = ms.ctypes.data_as(_dp)
        rttddft_trace_steps(self.ctx, a.shape[0], a, d, t)
        return [(names[i].decode(), float(ms[i])) for i in range(t.count)]

    def close(self):
        if getattr(self, "ctx", None):
            rttddft_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
