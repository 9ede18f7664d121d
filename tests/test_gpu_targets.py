"""GPU: the paper's frequency scan with one box per target (Sec. sec_numerical), through the C ABI, against the
oracle's scan and, as physics, against the semi-analytic Gaussian Omega_GW (Eq. eq_semi_anal)."""
import numpy as np
import pytest

from oracle import decomposition as odec
from oracle import semi_analytic, targets

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_27231_gb300 import build, sigw
    build.build()
    sigw.lib()
    return sigw


@pytest.fixture(scope="module")
def dec():
    return odec.build()


@pytest.mark.parametrize("kind,F", [("gauss", 0.0), ("local", 3.0)])
@pytest.mark.parametrize("precision,rtol", [(64, 1e-9), (32, 1e-4)])
def test_target_scan_matches_oracle(lib, dec, kind, F, precision, rtol):
    """Three targets below, at and above the peak, each in its own 32^3 box."""
    N, A, sigma, kstar = 32, 1e-2, 0.5, 1.0
    ks = np.array([0.4, 1.0, 2.5]) * kstar
    ref = targets.target_scan(N, ks, A, sigma, kstar, dec, seed=4, kind=kind, F_NL=F)
    with lib.Plan(N, 1.0, precision=precision) as p:
        got = p.target_scan(ks, A, sigma, kstar, kind=kind, F_NL=F, seed=4)
    np.testing.assert_array_equal(got["n_c"], ref["n_c"])
    np.testing.assert_allclose(got["L"], ref["L"], rtol=1e-14)
    np.testing.assert_allclose(got["omega"], ref["omega"], rtol=rtol)


def test_set_box_requires_a_new_field(lib):
    with lib.Plan(16, 1.0, n_alpha=2) as p:
        p.generate(1e-2, 0.5, 4 * 2 * np.pi)
        p.set_box(2.0)
        with pytest.raises(lib.SigwError) as e:
            p.spectrum([1])
        assert e.value.status == lib.ESTATE
        with pytest.raises(lib.SigwError):
            p.set_box(-1.0)


@pytest.mark.slow
def test_paper_scan_n64_gaussian_vs_semi_analytic(lib, dec):
    """The paper's Gaussian benchmark: 20 targets k/k* in [0.2, 3], N = 64, sigma = 0.5, one box each.
    Seed 1 against the oracle's scan (FP32 bound); the mean of four seeds against Eq. eq_semi_anal within the
    paper's stated accuracy (< ~10 %) wherever the target shell is not an infrared one (n_c >= 3)."""
    N, A, sigma, kstar = 64, 1e-2, 0.5, 1.0
    ks = np.geomspace(0.2, 3.0, 20) * kstar
    vals = []
    with lib.Plan(N, 1.0, precision=32) as p:
        for seed in (1, 2, 3, 4):
            r = p.target_scan(ks, A, sigma, kstar, seed=seed)
            vals.append(r["omega"])
    ref = targets.target_scan(N, ks, A, sigma, kstar, dec, seed=1)
    np.testing.assert_allclose(vals[0], ref["omega"], rtol=1e-4)
    sa = np.array([semi_analytic.omega_gauss(k, A, sigma, kstar) for k in ks])
    ratio = np.mean(vals, 0) / sa
    sel = r["n_c"] >= 3
    assert np.all(np.abs(ratio[sel] - 1) < 0.10), ratio


def _scan_golden(name):
    """A stored oracle scan (tests/golden/make_golden.py, oracle only): rows k L n_c Omega."""
    import os
    return np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", name), comments="#", ndmin=2)


@pytest.mark.parametrize("fname,N,sigma", [("scan64_sigma0.1.txt", 64, 0.1), ("scan64_sigma1.0.txt", 64, 1.0),
                                           ("scan128_sigma0.5.txt", 128, 0.5)])
def test_paper_scan_breadth_matches_oracle(lib, fname, N, sigma):
    """The paper's 20-target Gaussian scan (Sec. sec_numerical) for a narrow and a broad peak at N = 64 and the
    sigma = 0.5 peak at N = 128, seed 1, FP32: the box of every target exactly, Omega within 1e-4 of the oracle in
    every target whose Omega is at least 1e-10 of the scan's largest.  FP32 transforms carry round-off relative to a
    field's overall size, so a bin 1e-12 below the peak (k = 3 k* for the narrow peak, beyond its 2 k* cut-off) is
    held to 1e-3 (measured: 3.3e-4)."""
    rows = _scan_golden(fname)
    with lib.Plan(N, 1.0, precision=32) as p:
        got = p.target_scan(rows[:, 0], 1e-2, sigma, 1.0, seed=1)
    np.testing.assert_array_equal(got["n_c"], rows[:, 2].astype(int))
    np.testing.assert_allclose(got["L"], rows[:, 1], rtol=1e-14)
    ref = rows[:, 3]
    big = ref >= 1e-10 * ref.max()
    np.testing.assert_allclose(got["omega"][big], ref[big], rtol=1e-4)
    np.testing.assert_allclose(got["omega"][~big], ref[~big], rtol=1e-3)


@pytest.mark.slow
@pytest.mark.parametrize("N", [64, 128])
@pytest.mark.parametrize("sigma", [0.1, 0.5, 1.0])
def test_paper_scan_seed_mean_vs_semi_analytic(lib, N, sigma):
    """The paper's accuracy claim (sub ~10 % against Eq. eq_semi_anal, Sec. sec_numerical) for sigma = 0.1, 0.5, 1 at
    N = 64 and 128: the mean of 16 seeds of the GPU scan within 10 % of the semi-analytic Omega at every target whose
    shell is neither an infrared one (n_c >= 5) nor above a third of the Nyquist wave number (n_c <= N/6), and whose
    Omega is at least 1 % of the scan's largest (the cut-off tail of a narrow peak falls by orders of magnitude
    within one shell width).  The lowest shells differ from the continuum by the lattice's own discreteness (the
    exact lattice expectation, without noise, is 0.2-1.3 times the semi-analytic value at n_c = 1, 2 for sigma = 1)."""
    A, kstar = 1e-2, 1.0
    ks = np.geomspace(0.2, 3.0, 20) * kstar
    vals = []
    with lib.Plan(N, 1.0, precision=32) as p:
        for seed in range(1, 17):
            r = p.target_scan(ks, A, sigma, kstar, seed=seed)
            vals.append(r["omega"])
    sa = np.array([semi_analytic.omega_gauss(k, A, sigma, kstar) for k in ks])
    ratio = np.mean(vals, 0) / sa
    sel = (r["n_c"] >= 5) & (r["n_c"] <= N / 6) & (sa >= 1e-2 * sa.max())
    assert sel.sum() >= 5
    worst = np.abs(ratio[sel] - 1).max()
    print("N=%d sigma=%.1f: %d targets, worst |mean/semi-analytic - 1| = %.3f" % (N, sigma, sel.sum(), worst))
    assert worst < 0.10, (ratio[sel], r["n_c"][sel])
