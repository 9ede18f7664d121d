"""GPU parity: the CUDA path through the C ABI against the CPU FP64 oracle, element by element.

Tolerances: FP64 path rtol 1e-9 per shell (round-off of different summation orders);
FP32 path rtol 1e-4 per shell, the stated bound for FP32 fields/FFTs against the FP64 oracle.
"""
import numpy as np
import pytest

import workloads
from oracle import decomposition as odec
from oracle import sigw as osigw
from oracle import synth

pytestmark = pytest.mark.gpu

RTOL = {64: 1e-9, 32: 1e-4}


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


def _oracle(spec, dec, shells):
    Phi, hits = synth.phi_tilde(spec.N, spec.L, spec.A, spec.sigma, spec.kstar, spec.seed, spec.kind, spec.F_NL,
                                spec.G_NL, spec.usr_floor, spec.alpha_NL, spec.beta_NL)
    return osigw.omega(Phi, spec.L, dec, shells=shells), Phi, hits


def _gpu(lib, spec, shells, precision, **opts):
    with lib.Plan(spec.N, spec.L, precision=precision, **opts) as p:
        hits = p.generate_spec(spec)
        out = p.spectrum(shells)
        phi = p.copy_phi(0)
    return out, phi, hits


# ------------------------------------------------------------------ FFT
@pytest.mark.parametrize("N", [8, 16, 32, 64, 128])
@pytest.mark.parametrize("precision", [32, 64])
def test_fft3d_matches_numpy(lib, N, precision):
    import torch
    rdt = torch.float64 if precision == 64 else torch.float32
    cdt = torch.complex128 if precision == 64 else torch.complex64
    rng = np.random.default_rng(N)
    x = rng.standard_normal((N, N, N))
    with lib.Plan(N, 1.0, precision=precision, n_alpha=2) as p:
        xd = torch.tensor(x, dtype=rdt, device="cuda")
        Xd = torch.empty((N, N, N // 2 + 1), dtype=cdt, device="cuda")
        p.fft3d(-1, xd.data_ptr(), Xd.data_ptr())
        p.synchronize()
        X = Xd.cpu().numpy()
        ref = np.fft.rfftn(x)
        tol = 1e-12 if precision == 64 else 2e-6
        assert np.abs(X - ref).max() <= tol * np.abs(ref).max() * np.sqrt(np.log2(N ** 3))
        yd = torch.empty((N, N, N), dtype=rdt, device="cuda")
        p.fft3d(+1, Xd.data_ptr(), yd.data_ptr())
        p.synchronize()
        y = yd.cpu().numpy() / N ** 3
        assert np.abs(y - x).max() <= tol * 10 * np.abs(x).max()


# ------------------------------------------------------------------ synthesis
@pytest.mark.parametrize("kind,F", [("gauss", 0.0), ("local", 3.0), ("usr", 0.0)])
@pytest.mark.parametrize("precision", [64, 32])
def test_phi_matches_oracle(lib, dec, kind, F, precision):
    spec = workloads.Spec(N=32, L=1.0, A=1e-2, sigma=0.5, kstar=8 * 2 * np.pi, kind=kind, F_NL=F, seed=3)
    Phi, hits = synth.phi_tilde(spec.N, spec.L, spec.A, spec.sigma, spec.kstar, spec.seed, kind, F)
    with lib.Plan(spec.N, spec.L, precision=precision, n_alpha=2) as p:
        ghits = p.generate_spec(spec)
        phi = p.copy_phi(0)
    ref = Phi[:, :, :spec.N // 2 + 1]
    tol = 1e-12 if precision == 64 else 3e-6
    assert np.abs(phi - ref).max() <= tol * np.abs(ref).max()
    if precision == 64:
        assert int(ghits[0]) == hits


# ------------------------------------------------------------------ full spectra, small lattices
@pytest.mark.parametrize("N", [8, 16])
@pytest.mark.parametrize("kind,F", [("gauss", 0.0), ("local", 3.0), ("usr", 0.0)])
@pytest.mark.parametrize("precision", [64, 32])
def test_omega_all_shells_small(lib, dec, N, kind, F, precision):
    spec = workloads.Spec(N=N, L=1.0, A=2e-2, sigma=0.5, kstar=(N // 4) * 2 * np.pi, kind=kind, F_NL=F, seed=11)
    ref, _, _ = _oracle(spec, dec, None)
    got, _, _ = _gpu(lib, spec, None, precision)
    np.testing.assert_array_equal(got["Nk"][0], ref["Nk"])
    np.testing.assert_allclose(got["omega"][0], ref["omega"], rtol=RTOL[precision])
    np.testing.assert_allclose(got["PA"][0], ref["PA"], rtol=RTOL[precision])
    np.testing.assert_allclose(got["PB"][0], ref["PB"], rtol=RTOL[precision])


@pytest.mark.parametrize("N", [16, 32])
@pytest.mark.parametrize("F,G", [(0.0, 1.0), (0.0, 50.0), (3.0, 10.0)])
@pytest.mark.parametrize("precision", [64, 32])
def test_cubic_gnl_all_shells(lib, dec, N, F, G, precision):
    """The cubic term of the local map (Sec. "Local Non-Gaussianities": F_NL = 0 with G_NL in {1, 5, 10, 50}, and a
    mixed F_NL, G_NL case): Phi~ element by element and every shell against the oracle."""
    spec = workloads.Spec(N=N, L=1.0, A=1e-2, sigma=0.5, kstar=(N // 4) * 2 * np.pi, kind="local", F_NL=F, G_NL=G,
                          seed=19)
    ref, Phi, _ = _oracle(spec, dec, None)
    got, phi, _ = _gpu(lib, spec, None, precision)
    refh = Phi[:, :, :N // 2 + 1]
    assert np.abs(phi - refh).max() <= (1e-12 if precision == 64 else 3e-6) * np.abs(refh).max()
    np.testing.assert_array_equal(got["Nk"][0], ref["Nk"])
    np.testing.assert_allclose(got["omega"][0], ref["omega"], rtol=RTOL[precision])
    np.testing.assert_allclose(got["PA"][0], ref["PA"], rtol=RTOL[precision])
    np.testing.assert_allclose(got["PB"][0], ref["PB"], rtol=RTOL[precision])


@pytest.mark.parametrize("N", [16, 32])
@pytest.mark.parametrize("precision", [64, 32])
def test_nonlocal_map_all_shells(lib, dec, N, precision):
    """Eq. eq_nonlocal (alpha_NL = 5, beta_NL = -3 in units of 1/k*^2): Phi~ and every shell against the oracle."""
    spec = workloads.Spec(N=N, L=1.0, A=2e-2, sigma=0.5, kstar=(N // 4) * 2 * np.pi, kind="nonlocal", seed=13,
                          alpha_NL=5.0, beta_NL=-3.0)
    ref, Phi, _ = _oracle(spec, dec, None)
    got, phi, _ = _gpu(lib, spec, None, precision)
    refh = Phi[:, :, :N // 2 + 1]
    assert np.abs(phi - refh).max() <= (1e-12 if precision == 64 else 3e-6) * np.abs(refh).max()
    np.testing.assert_array_equal(got["Nk"][0], ref["Nk"])
    np.testing.assert_allclose(got["omega"][0], ref["omega"], rtol=RTOL[precision])


def test_mixed_batch_with_nonlocal_member(lib, dec):
    """A batch mixing the non-local, local and Gaussian maps gives each member the spectrum it has alone."""
    base = dict(N=16, L=1.0, A=2e-2, sigma=0.5, kstar=4 * 2 * np.pi)
    specs = [workloads.Spec(kind="nonlocal", seed=1, alpha_NL=2.0, beta_NL=1.0, **base),
             workloads.Spec(kind="local", F_NL=2.0, seed=2, **base), workloads.Spec(kind="gauss", seed=3, **base)]
    with lib.Plan(16, 1.0, precision=64, max_batch=3) as p:
        p.generate_batch(specs)
        mixed = p.spectrum()["omega"]
    for i, sp in enumerate(specs):
        ref, _, _ = _oracle(sp, dec, None)
        np.testing.assert_allclose(mixed[i], ref["omega"], rtol=1e-9)


@pytest.mark.parametrize("precision", [64, 32])
def test_omega_gauss32_all_shells(lib, dec, precision):
    """The 32^3 Gaussian workload (log-normal A = 1e-2, sigma = 0.5, k* = 8 k_f), every shell."""
    spec = workloads.workload("gauss32")
    ref, _, _ = _oracle(spec, dec, None)
    got, _, _ = _gpu(lib, spec, None, precision)
    np.testing.assert_array_equal(got["Nk"][0], ref["Nk"])
    np.testing.assert_allclose(got["omega"][0], ref["omega"], rtol=RTOL[precision])


def test_omega_64_local_fp32(lib, dec):
    spec = workloads.scaled(workloads.workload("local128"), 64)
    shells = [1, 2, 7, 8, 9, 16, 31, 32]
    ref, _, _ = _oracle(spec, dec, shells)
    got, _, _ = _gpu(lib, spec, shells, 32)
    np.testing.assert_allclose(got["omega"][0], ref["omega"], rtol=1e-4)


def test_odd_alpha_and_small_batches(lib, dec):
    """An odd number of terms (the last pair has one member) and an alpha batch that does not divide it."""
    spec = workloads.Spec(N=16, L=2.0, A=1e-2, sigma=0.7, kstar=3 * np.pi, kind="local", F_NL=-1.2, seed=5)
    shells = [1, 4, 8]
    d = odec.build(n_alpha=7)
    ref, _, _ = _oracle(spec, d, shells)
    got, _, _ = _gpu(lib, spec, shells, 64, n_alpha=7, alpha_batch=3)
    np.testing.assert_allclose(got["omega"][0], ref["omega"], rtol=1e-9)


def test_batch_equals_single_bitwise(lib):
    """Four seeds in one call give the bits of four single-seed calls."""
    spec = workloads.scaled(workloads.workload("usr256"), 32)
    seeds = [1, 2, 3, 4]
    shells = [2, 4, 9, 16]
    with lib.Plan(spec.N, spec.L, precision=32, max_batch=4) as p:
        p.generate_spec(spec, seeds=seeds)
        batched = p.spectrum(shells)["omega"]
    for i, s in enumerate(seeds):
        with lib.Plan(spec.N, spec.L, precision=32) as p:
            p.generate_spec(spec, seeds=[s])
            single = p.spectrum(shells)["omega"][0]
        assert np.array_equal(batched[i], single)


def test_degenerate_inputs(lib, dec):
    """A = 0 gives an exactly zero field and spectrum; one separable term; shells in any order with repeats give
    the values of the sorted call; an empty shell list is rejected."""
    with lib.Plan(16, 1.0, n_alpha=2, precision=32) as p:
        p.generate(0.0, 0.5, 4 * 2 * np.pi, kind="local", F_NL=3.0)
        r = p.spectrum()
        assert np.all(r["omega"] == 0.0) and np.all(r["PA"] == 0.0)
        import ctypes
        one = (ctypes.c_int * 1)(1)
        assert lib.lib().sigw_spectrum(p._h, one, 0, None, None, None, None) == lib.EINVAL
    spec = workloads.Spec(N=16, L=1.0, A=2e-2, sigma=0.5, kstar=4 * 2 * np.pi, kind="usr", seed=17)
    d1 = odec.build(n_alpha=1)
    ref, _, _ = _oracle(spec, d1, [2, 5, 8])
    with lib.Plan(16, 1.0, precision=64, n_alpha=1) as p:
        p.generate_spec(spec)
        got = p.spectrum([8, 2, 5, 2])["omega"][0]
    np.testing.assert_allclose(got, ref["omega"][[2, 0, 1, 0]], rtol=1e-9)


def test_state_errors(lib):
    with lib.Plan(16, 1.0, n_alpha=2) as p:
        with pytest.raises(lib.SigwError) as e:
            p.spectrum()
        assert e.value.status == lib.ESTATE
        p.generate(1e-2, 0.5, 4 * 2 * np.pi)
        with pytest.raises(lib.SigwError) as e:
            p.spectrum([0])
        assert e.value.status == lib.EINVAL
        with pytest.raises(lib.SigwError) as e:
            p.spectrum([9])
        assert e.value.status == lib.EINVAL


def test_injected_allocation_failure_reports_enomem(lib):
    lib.debug_fail_alloc(3)
    try:
        with pytest.raises(lib.SigwError) as e:
            lib.Plan(16, 1.0, n_alpha=2)
        assert e.value.status == lib.ENOMEM
    finally:
        lib.debug_fail_alloc(0)
    with lib.Plan(16, 1.0, n_alpha=2) as p:  # the library is usable afterwards
        p.generate(1e-2, 0.5, 4 * 2 * np.pi)
        assert np.all(np.isfinite(p.spectrum()["omega"]))


@pytest.mark.parametrize("N", [64, 128])
def test_bulk_copy_wait_timeout_is_reported_and_recoverable(lib, dec, N):
    """The last inverse pass's bounded waits (bulk-copy ring) given a one-cycle limit give up while every copy
    still lands: the call reports SIGW_ETIMEOUT; with the default limit restored the same plan gives the oracle's
    values, on direct launches and on the (re-captured) all-shells graph."""
    spec = workloads.Spec(N=N, L=1.0, A=1e-2, sigma=0.5, kstar=(N // 8) * 2 * np.pi, kind="local", F_NL=2.0, seed=23)
    shells = [3, N // 4]
    ref, _, _ = _oracle(spec, dec, shells)
    with lib.Plan(N, spec.L, precision=32) as p:
        p.generate_spec(spec)
        first = p.spectrum()["omega"][0]  # captures the all-shells graph with the default limit
        for call in (lambda: p.spectrum(shells), lambda: p.spectrum()):
            p.debug_wait_limit(1)
            with pytest.raises(lib.SigwError) as e:
                call()
            assert e.value.status == lib.ETIMEOUT
            p.debug_wait_limit(0)
            np.testing.assert_allclose(p.spectrum(shells)["omega"][0], ref["omega"], rtol=1e-4)
            assert np.array_equal(p.spectrum()["omega"][0], first)


def test_tensor_memory_last_pass_wait_timeout_and_recovery(lib):
    """The last pass with its accumulators in tensor memory (variant bit 8, 256^3): its bounded waits given a
    one-cycle limit report SIGW_ETIMEOUT, after which the same plan gives the bits it gives without the hook, and
    the same values as the register-accumulator form within FP32 round-off."""
    spec = workloads.Spec(N=256, L=1.0, A=1e-2, sigma=0.5, kstar=32 * 2 * np.pi, kind="local", F_NL=2.0, seed=29)
    shells = [5, 77]
    with lib.Plan(256, 1.0, precision=32, n_alpha=6) as p:
        p.generate_spec(spec)
        p.set_tuning(6, 2)
        regs = p.spectrum(shells)["omega"][0]
        p.set_tuning(6, 8)
        clean = p.spectrum(shells)["omega"][0]
        p.debug_wait_limit(1)
        with pytest.raises(lib.SigwError) as e:
            p.spectrum(shells)
        assert e.value.status == lib.ETIMEOUT
        p.debug_wait_limit(0)
        assert np.array_equal(p.spectrum(shells)["omega"][0], clean)
    np.testing.assert_allclose(clean, regs, rtol=2e-6)


def test_usr_strict_mode(lib):
    spec = workloads.Spec(N=16, L=1.0, A=5e-1, sigma=0.5, kstar=4 * 2 * np.pi, kind="usr", seed=2)
    with lib.Plan(16, 1.0, n_alpha=2, strict_domain=1, precision=64) as p:
        with pytest.raises(lib.SigwError) as e:
            p.generate_spec(spec)
        assert e.value.status == lib.EDOMAIN
    _, hits = synth.phi_tilde(spec.N, spec.L, spec.A, spec.sigma, spec.kstar, spec.seed, "usr")
    assert hits > 0


# ------------------------------------------------------------------ full-size workloads, sampled shells
@pytest.mark.slow
def test_local128_sampled_shells_fp32(lib, dec):
    """The 128^3 local f_NL = 5 workload in the bench's launch configuration, sampled shells."""
    spec = workloads.workload("local128")
    shells = [1, 16, 33, 64]
    ref, _, _ = _oracle(spec, dec, shells)
    got, _, _ = _gpu(lib, spec, shells, 32)
    np.testing.assert_allclose(got["omega"][0], ref["omega"], rtol=1e-4)


@pytest.mark.slow
def test_usr256_sampled_shell_fp32(lib, dec):
    """The 256^3 USR-tail workload (A = 5e-3, sigma = 0.3, k* = 32 k_f) at the spectral peak, FP32."""
    spec = workloads.workload("usr256")
    shells = [32]
    ref, _, hits = _oracle(spec, dec, shells)
    got, _, ghits = _gpu(lib, spec, shells, 32)
    np.testing.assert_allclose(got["omega"][0], ref["omega"], rtol=1e-4)
    assert abs(int(ghits[0]) - hits) <= max(2, hits // 100)


def _golden(name):
    """Per-shell oracle values written by tests/golden/make_golden.py (oracle only): rows n_c N_k Omega P_A P_B,
    and the USR floor-hit count of the realisation."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", name)
    hits = None
    for line in open(path):
        if line.startswith("# usr_floor_hits="):
            hits = int(line.split("=")[1])
    return np.loadtxt(path, comments="#", ndmin=2), hits


def _worst(got, ref):
    rel = np.abs(got / ref - 1.0)
    i = int(np.argmax(rel))
    return rel[i], i


@pytest.mark.slow
@pytest.mark.parametrize("name,seed,fname", [("local128", 2, "local128_seed2.txt"), ("usr256", 1, "usr256_seed1.txt"),
                                             ("broad512", 5, "broad512_seed5.txt")])
def test_full_size_fp32_every_stored_shell(lib, name, seed, fname):
    """FP32 Omega, P_A, P_B within 1e-4 relative of the FP64 oracle in every stored shell bin at full size, N_k
    exact.  usr256 runs in the bench's launch configuration (four seeds per launch, autotuned plan, the captured
    all-shells graph); its first seed is compared.  local128 compares all 64 shells, broad512 shells 8 and 32."""
    rows, hits = _golden(fname)
    spec = workloads.workload(name, seed=seed)
    shells = rows[:, 0].astype(int)
    full = len(shells) == spec.N // 2
    if name == "usr256":
        with lib.Plan(spec.N, spec.L, precision=32, max_batch=4) as p:
            ghits = p.generate_spec(spec, seeds=list(workloads.USR256_SEEDS))
            p.autotune()
            out = p.spectrum()
        got = {k: out[k][0] for k in ("omega", "PA", "PB", "Nk")}
        assert abs(int(ghits[0]) - hits) <= max(2, hits // 100)
    else:
        with lib.Plan(spec.N, spec.L, precision=32) as p:
            p.generate_spec(spec)
            out = p.spectrum(None if full else shells)
        got = {k: out[k][0] for k in ("omega", "PA", "PB", "Nk")}
    np.testing.assert_array_equal(got["Nk"], rows[:, 1].astype(np.int64))
    for col, key in ((2, "omega"), (3, "PA"), (4, "PB")):
        w, i = _worst(got[key], rows[:, col])
        print("%s %s: worst relative error %.3g at shell %d" % (name, key, w, shells[i]))
        assert w <= 1e-4, (key, w, int(shells[i]))


@pytest.mark.slow
def test_broad512_small_shells_fp32_fp64(lib, dec):
    """The 512^3 local f_NL = -2 workload (A = 1e-2, sigma = 1, k* = 64 k_f), the largest lattice, on both paths.
    The oracle side is the direct lattice sum over the kernel's support ball (|n1| < u_max n_c), which is
    affordable for the first shells; Phi~ is compared element by element."""
    from oracle import brute
    spec = workloads.workload("broad512")
    shells = [1, 2]
    Phi, hits = synth.phi_tilde(spec.N, spec.L, spec.A, spec.sigma, spec.kstar, spec.seed, spec.kind, spec.F_NL,
                                spec.G_NL, spec.usr_floor)
    ref = brute.omega_brute(Phi, spec.L, dec, shells=shells, ball=True)
    refh = Phi[:, :, :spec.N // 2 + 1]
    for precision, rtol, ptol in ((32, 1e-4, 1e-5), (64, 1e-9, 1e-12)):
        got, phi, _ = _gpu(lib, spec, shells, precision)
        assert np.abs(phi - refh).max() <= ptol * np.abs(refh).max()
        del phi
        np.testing.assert_array_equal(got["Nk"][0], ref["Nk"])
        np.testing.assert_allclose(got["omega"][0], ref["omega"], rtol=rtol)
        np.testing.assert_allclose(got["PA"][0], ref["PA"], rtol=rtol)
    # every radix variant of the FP32 passes at this size (radix 32 strided passes, radix 16 last pass)
    with lib.Plan(spec.N, spec.L, precision=32) as p:
        p.generate_spec(spec)
        for v in (1, 2, 4, 7, 15, 31):
            p.set_tuning(10, v)
            np.testing.assert_allclose(p.spectrum(shells)["omega"][0], ref["omega"], rtol=1e-4)


def test_graph_replay_equals_direct_launches(lib):
    """The all-shells call runs as a captured CUDA graph; it must give the bits of direct launches (explicit
    shell list), on first capture, on replay and after a batch-size change forces a new capture."""
    spec = workloads.scaled(workloads.workload("local128"), 32)
    H = spec.N // 2
    with lib.Plan(spec.N, spec.L, precision=32, max_batch=2) as p:
        p.generate_spec(spec, seeds=[3, 4])
        direct = p.spectrum(np.arange(1, H + 1))["omega"]
        g1 = p.spectrum()["omega"]
        g2 = p.spectrum()["omega"]
        p.generate_spec(spec, seeds=[3])
        g3 = p.spectrum()["omega"]
    assert np.array_equal(direct, g1) and np.array_equal(g1, g2)
    assert np.array_equal(g3[0], direct[0])


@pytest.mark.parametrize("N", [128, 256])
def test_every_variant_matches_oracle(lib, dec, N):
    """Each radix variant (bits 1, 2, 4 and all together; at 256^3 also the last pass with its accumulators in tensor
    memory, bit 8, and the first pass with its tile in tensor memory, bit 16; both also at 128^3) on sampled shells of
    a local-map field, vs the oracle."""
    spec = workloads.scaled(workloads.workload("local128"), N)
    shells = [3, N // 4]
    d10 = odec.build(n_alpha=10)
    ref, _, _ = _oracle(spec, d10, shells)
    with lib.Plan(N, spec.L, precision=32, n_alpha=10) as p:
        p.generate_spec(spec)
        extra = {256: ((10, 8), (4, 15), (10, 16), (8, 26)), 128: ((10, 8), (5, 13), (10, 26))}[N]
        for B, v in ((4, 0), (10, 1), (10, 2), (8, 4), (5, 7)) + extra:
            p.set_tuning(B, v)
            np.testing.assert_allclose(p.spectrum(shells)["omega"][0], ref["omega"], rtol=1e-4)
        with pytest.raises(lib.SigwError):
            p.set_tuning(0, 0)


def test_autotune_keeps_results_and_seeds_later_plans(lib, dec):
    """The autotuner only regroups terms per launch and changes the strided radix: results stay within FP32
    round-off of the untuned plan (and within 1e-4 of the oracle); a later plan starts from the tuned choice."""
    spec = workloads.workload("local128")
    shells = [16, 40]
    with lib.Plan(spec.N, spec.L, precision=32) as p:
        p.generate_spec(spec)
        before = p.spectrum(shells)["omega"][0]
        B, v, ms = p.autotune()
        after = p.spectrum(shells)["omega"][0]
    assert B in (4, 5, 8, 10, 16) and 0 <= v < 32 and ms > 0
    np.testing.assert_allclose(after, before, rtol=2e-5)
    ref, _, _ = _oracle(spec, dec, shells)
    np.testing.assert_allclose(after, ref["omega"], rtol=1e-4)
    with lib.Plan(spec.N, spec.L, precision=32) as q:
        q.generate_spec(spec)
        again = q.spectrum(shells)["omega"][0]
    assert np.array_equal(again, after)
