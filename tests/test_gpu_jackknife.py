"""GPU: jackknife error bars of the shell spectra (Sec. sec_envelope_obs) through the C ABI, against the oracle."""
import numpy as np
import pytest

import workloads
from oracle import decomposition as odec
from oracle import jackknife as ojk
from oracle import synth

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


@pytest.mark.parametrize("N,M", [(16, 4), (32, 4), (32, 2)])
@pytest.mark.parametrize("precision", [64, 32])
def test_jackknife_matches_oracle(lib, dec, N, M, precision):
    spec = workloads.Spec(N=N, L=1.0, A=2e-2, sigma=0.5, kstar=(N // 4) * 2 * np.pi, kind="local", F_NL=2.0, seed=21)
    shells = [1, 3, N // 2 - 1]
    Phi, _ = synth.phi_tilde(spec.N, spec.L, spec.A, spec.sigma, spec.kstar, spec.seed, spec.kind, spec.F_NL)
    ref = ojk.jackknife(Phi, spec.L, dec, shells, M=M)
    with lib.Plan(N, spec.L, precision=precision) as p:
        p.generate_spec(spec)
        got = p.spectrum_jackknife(shells, M=M)
        plain = p.spectrum(shells)
    rm, rs = (1e-9, 1e-8) if precision == 64 else (1e-4, 2e-3)
    for k in ("omega", "PA", "PB"):
        np.testing.assert_allclose(got[k][0], ref[k], rtol=rm)
        np.testing.assert_allclose(got["sigma_" + k][0], ref["sigma_" + k], rtol=rs)
        np.testing.assert_allclose(got[k][0], plain[k][0], rtol=1e-12 if precision == 64 else 1e-5)


def test_jackknife_batch_equals_single(lib):
    spec = workloads.scaled(workloads.workload("usr256"), 32)
    shells = [2, 9, 15]
    with lib.Plan(32, spec.L, precision=32, max_batch=2) as p:
        p.generate_spec(spec, seeds=[5, 6])
        both = p.spectrum_jackknife(shells)
    for i, s in enumerate((5, 6)):
        with lib.Plan(32, spec.L, precision=32) as p:
            p.generate_spec(spec, seeds=[s])
            one = p.spectrum_jackknife(shells)
        for k in ("omega", "sigma_omega"):
            assert np.array_equal(both[k][i], one[k][0])


def test_jackknife_rejects_bad_arguments(lib):
    with lib.Plan(16, 1.0, n_alpha=2) as p:
        p.generate(1e-2, 0.5, 4 * 2 * np.pi)
        for kw in ({"shells": [8]}, {"shells": [2], "M": 3}, {"shells": [0]}):
            with pytest.raises(lib.SigwError) as e:
                p.spectrum_jackknife(**kw)
            assert e.value.status == lib.EINVAL
        r = p.spectrum_jackknife([2])  # the plan stays usable
        assert np.isfinite(r["sigma_omega"]).all()
