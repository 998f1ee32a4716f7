"""The C-ABI library builds, loads and exports what include/rttddft.h declares,
and set-up rejects malformed inputs on the host (no GPU needed)."""
import ctypes
import os
import re
import shutil

import numpy as np
import pytest

from paper_2403_04351_gb300 import build, rttddft
from synth import make_system, tiny_config

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rttddft.h")


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"RTTDDFT_API\s+[\w\s\*]*?\b(rttddft_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    path = build()
    return rttddft.load_library(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("rttddft_setup", "rttddft_step", "rttddft_observables", "rttddft_destroy",
              "rttddft_last_error", "rttddft_apply", "rttddft_adjoint"):
        assert n in names
    assert sorted(rttddft.EXPORTED) == names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    raw = ctypes.CDLL(rttddft.LIB_PATH)
    for name in ("k_jacobi", "launch_step", "_Z11launch_stepRK8StepArgsRK8StepPlanP11CUstream_stPi"):
        with pytest.raises(AttributeError):
            getattr(raw, name)


def test_version_and_default_options(lib):
    assert "sm_103a" in rttddft.rttddft_version()
    o = rttddft.rttddft_default_options()
    assert o.propagator == 0 and o.precision == 0 and o.aux_mode == 0
    assert o.max_record >= 1 and o.cheb_tol == 1e-16 and o.max_sweeps >= 1


def _expect(code_name, sys, **kw):
    with pytest.raises(rttddft.RttddftError) as e:
        rttddft.Context(sys, **kw)
    assert rttddft.ERRORS[e.value.code] == code_name, str(e.value)


@pytest.fixture(scope="module")
def small():
    return make_system(tiny_config(n_g=40, n_atoms=2, lmax=1, n_lo_per_atom=2, n_s=2, n_aux=8,
                                   seed=3))


def test_setup_rejects_sizes(lib, small):
    s = dict(small)
    s["n_s"] = 9
    _expect("ERR_ARG", s)
    s = dict(small)
    s["n_aux"] = 100
    _expect("ERR_ARG", s)
    _expect("ERR_ARG", small, dt=-0.1)
    _expect("ERR_UNSUPPORTED", dict(small, n_aux=2000))


def test_setup_rejects_non_hermitian_and_non_pd_blocks(lib, small):
    s = dict(small)
    h = [x.copy() for x in small["h"]]
    h[1][0, 1] += 0.3
    s["h"] = h
    _expect("ERR_NOT_HERMITIAN", s)
    s = dict(small)
    o = [x.copy() for x in small["o"]]
    o[0] = o[0] - 3.0 * np.eye(o[0].shape[0])
    s["o"] = o
    _expect("ERR_NOT_PD", s)
    s = dict(small)
    v = small["vtab"].copy()
    v[0, 0, 1] += 0.01j
    s["vtab"] = v
    _expect("ERR_NOT_HERMITIAN", s)


def test_setup_rejects_non_finite_and_small_table(lib, small):
    s = dict(small)
    c = [x.copy() for x in small["caux"]]
    c[0][3, 2] = np.nan
    s["caux"] = c
    _expect("ERR_NONFINITE", s)
    s = dict(small)
    ext = (np.asarray(small["vt_dim"]) - 1) // 2
    s["vtab"] = small["vtab"][1:-1, :, :]
    s["vt_dim"] = np.array([2 * ext[0] - 1, small["vt_dim"][1], small["vt_dim"][2]])
    _expect("ERR_ARG", s)
    assert "vtab box" in rttddft.rttddft_last_error(None)


def test_fft_route_options_are_checked_on_the_host(lib, small):
    """The direct sum is the default interstitial route, and an unknown route
    value is refused before any device work."""
    assert rttddft.rttddft_default_options().interstitial == 0
    o = rttddft.INTERSTITIAL
    try:
        rttddft.INTERSTITIAL = dict(o, bogus=7)
        _expect("ERR_UNSUPPORTED", small, interstitial="bogus")
    finally:
        rttddft.INTERSTITIAL = o


def test_polarizability_arguments_checked_on_the_host(lib):
    j = np.zeros((10, 3))
    w = np.array([0.5, 1.0])
    f = lib.rttddft_polarizability
    P = rttddft._ptr
    assert f(0, 0.0, 0.1, P(j), P(j), 0.0, 2, P(w), 1.0, None, None, None, None) == -1
    assert f(10, 0.0, 0.0, P(j), P(j), 0.0, 2, P(w), 1.0, None, None, None, None) == -1
    assert f(10, 0.0, 0.1, P(j), P(j), -1.0, 2, P(w), 1.0, None, None, None, None) == -1
    wb = np.array([0.5, 0.0])
    assert f(10, 0.0, 0.1, P(j), P(j), 0.0, 2, P(wb), 1.0, None, None, None, None) == -1
    assert f(10, 0.0, 0.1, P(j), P(j), 0.0, 2, P(w), 0.0, None, None, None, None) == -1


def test_hartree_options_checked_on_the_host(lib, small):
    """The density feedback needs the FFT route, the reciprocal vectors, a
    positive bound and a finite muffin-tin coupling; all refused before any
    device work."""
    _expect("ERR_UNSUPPORTED", small, hartree=True)
    _expect("ERR_ARG", small, interstitial="fft", hartree=True, hartree_bound=-1.0)
    s = dict(small)
    del s["recip"]
    _expect("ERR_ARG", s, interstitial="fft", hartree=True)
    _expect("ERR_NONFINITE", small, interstitial="fft", hartree=True, hartree_mt_u=float("nan"))
    assert rttddft.rttddft_default_options().hartree == 0
    assert rttddft.rttddft_default_options().hartree_mt_u == 0.0


def _header_fields(name):
    text = open(HEADER).read()
    end = text.index("} " + name + ";")
    start = text.rfind("typedef struct {", 0, end)
    body = re.sub(r"/\*.*?\*/", "", text[start + len("typedef struct {"):end], flags=re.S)
    return re.findall(r"([A-Za-z_][A-Za-z_0-9]*)\s*(?:\[[^\]]*\])?\s*;", body)


def test_ctypes_structs_follow_the_header():
    """The binding's structures list the header's fields in the header's order
    (the C ABI passes them by pointer, so an order or a missing field would
    shift every later field)."""
    for name in ("rttddft_system", "rttddft_options", "rttddft_obs", "rttddft_info", "rttddft_trace"):
        cls = getattr(rttddft, name)
        assert [f[0] for f in cls._fields_] == _header_fields(name), name
