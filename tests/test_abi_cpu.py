"""C ABI checks that need no GPU: the library loads, exports every symbol the headers
declare, and its host-side plan math (decomposition, cell tables) agrees with the oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import decomposition as odec

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def sigw():
    from paper_2605_27231_gb300 import build, sigw as s
    build.build()
    s.lib()
    return s


def _declared_symbols():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(sigw_\w+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol(sigw):
    lib = ctypes.CDLL(sigw.LIB_PATH)
    names = _declared_symbols()
    assert len(names) >= 15
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_strerror_and_defaults(sigw):
    o = sigw.default_opts()
    assert (o.n_modes, o.n_alpha, o.precision, o.max_batch) == (200, 50, 32, 1)
    assert o.umin == 1e-3 and o.umax == 15.0 and o.upiv == 1.0 and o.sigp == 0.5 and o.Ap == 10.0
    assert sigw.lib().sigw_strerror(0) == b"ok"
    assert sigw.lib().sigw_opts_default(None) == sigw.EINVAL


def test_invalid_arguments_rejected_without_gpu(sigw):
    lib = sigw.lib()
    h = ctypes.c_void_p()
    o = sigw.default_opts()
    for N in (0, 7, 12, 1024):
        assert lib.sigw_plan_create(N, 1.0, ctypes.byref(o), None, ctypes.byref(h)) == sigw.EINVAL
    assert lib.sigw_plan_create(32, -1.0, ctypes.byref(o), None, ctypes.byref(h)) == sigw.EINVAL
    bad = sigw.default_opts(n_alpha=300)
    assert lib.sigw_plan_create(32, 1.0, ctypes.byref(bad), None, ctypes.byref(h)) == sigw.EINVAL
    assert lib.sigw_generate(None, None, None, None, 1, None) == sigw.EINVAL


def test_footprint_scales_with_terms(sigw):
    a = sigw.footprint(64, sigw.default_opts(n_alpha=10))
    b = sigw.footprint(64, sigw.default_opts(n_alpha=50))
    assert b > a > 0
    c = sigw.footprint(64, sigw.default_opts(precision=64))
    assert c > b


def test_decomposition_matches_oracle(sigw):
    """C++ Jacobi decomposition vs numpy eigh: eigenvalues and the basis-independent truncated kernel."""
    dec = odec.build()
    for m, key in ((0, "s"), (1, "c")):
        sigma, phi, edges, sall = sigw.decompose(m, all_sigma=True)
        np.testing.assert_allclose(edges, dec.edges, rtol=0, atol=1e-13)
        np.testing.assert_allclose(sall, dec.sigma_all[key], rtol=1e-11, atol=1e-13 * abs(sall[0]))
        K = (phi.T * sigma) @ phi
        Kref = (dec.phi[key].T * dec.sigma[key]) @ dec.phi[key]
        np.testing.assert_allclose(K, Kref, atol=1e-10 * np.abs(Kref).max())


def test_cell_table_matches_oracle(sigw):
    dec = odec.build()
    msq_max = 3 * 256 ** 2
    msq = np.arange(msq_max + 1)
    for n_c in (1, 5, 64, 256):
        lut = sigw.cell_table(n_c, msq_max)
        ref = odec.cell_of(msq, n_c, dec.edges)
        ref = np.where(ref < 0, 200, ref)
        np.testing.assert_array_equal(lut, ref)


def test_target_box_matches_oracle(sigw):
    """The per-target box rule (host only) against the oracle's own implementation."""
    from oracle import semi_analytic
    for N in (32, 64, 128, 256):
        for sigma in (0.1, 0.5, 1.0):
            for k in np.geomspace(0.05, 8.0, 23):
                L, nc = sigw.target_box(N, k, 1e-2, sigma, 1.3)
                Lo, nco = semi_analytic.target_box(N, k, 1e-2, sigma, 1.3)
                assert nc == nco and abs(L / Lo - 1) < 1e-12
    with pytest.raises(sigw.SigwError):
        sigw.target_box(64, -1.0, 1e-2, 0.5, 1.0)
    with pytest.raises(sigw.SigwError):
        sigw.target_box(64, 1.0, 1e-2, 0.5, 1.0, eps=1.5)


def test_decomposition_error_matches_oracle(sigw):
    """The host decomposition study routine against the oracle's truncation error (independent eigen-solvers;
    the truncated matrix is basis-independent when the cut is not degenerate)."""
    for up, ap in ((1.0, 10.0), (0.8, 0.0)):
        d = odec.build(n_modes=60, n_alpha=20, upiv=up, Ap=ap)
        for m, mk in ((0, "s"), (1, "c")):
            for k in (10, 20, 40):
                f, mx, g = sigw.decomposition_error(m, n_modes=60, n_alpha=k, upiv=up, Ap=ap)
                fo, mxo, go = odec.truncation_error(d, mk, k)
                assert abs(f - fo) < 1e-9 and abs(mx - mxo) < 1e-9 and abs(g - go) < 1e-9


def test_decomposition_sweep_and_optimal_choice(sigw):
    from paper_2605_27231_gb300 import decomp_study
    rows = decomp_study.sweep(0, n_modes=(60,), n_alpha=(10, 20, 30), upiv=(1.0,), Ap=(10.0,))
    errs = [r["frob"] for r in sorted(rows, key=lambda r: r["n_alpha"])]
    assert errs[0] >= errs[1] >= errs[2]
    best = decomp_study.optimal(errs[1] * 1.0001, m=(0,), n_modes=(60,), n_alpha=(10, 20, 30), upiv=(1.0,),
                                Ap=(10.0,))
    assert best["n_alpha"] == 20
    assert decomp_study.optimal(0.0, m=(0,), n_modes=(60,), n_alpha=(10,), upiv=(1.0,), Ap=(10.0,)) is None
