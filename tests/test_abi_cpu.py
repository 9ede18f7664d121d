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
