"""Pins of the CPU FP64 oracle against facts that do not come from the oracle itself.

Each test states what fixes the expected value: a published known-answer vector,
a closed form, a defining integral evaluated by quadrature, an exact identity
(convolution theorem, Parseval, Hermitian symmetry, exact scaling), the direct
O(N^6) sum, the exact Wick expectation, or the paper's semi-analytic result.
"""
import os

import numpy as np
import pytest
from scipy import integrate

from oracle import brute, decomposition, jackknife, kernels, philox, semi_analytic, sigw, synth, wick

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def dec():
    return decomposition.build()


# ---------------------------------------------------------------- Philox / noise
def test_philox_known_answers():
    """Published Philox4x32-10 known-answer vectors (golden fixture with citation)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = philox.philox4x32_10(tuple(v[0:4]), tuple(v[4:6]))
        assert [int(o) for o in out] == v[6:10]


def test_white_noise_moments():
    """Box-Muller output is N(0,1): mean 0, variance 1, kurtosis 3 (closed-form moments)."""
    g = philox.white_noise(64, seed=12345).ravel()
    n = g.size
    assert abs(g.mean()) < 5.0 / np.sqrt(n)
    assert abs(g.var() - 1.0) < 5.0 * np.sqrt(2.0 / n)
    assert abs(np.mean(g ** 4) / g.var() ** 2 - 3.0) < 5.0 * np.sqrt(24.0 / n)
    # different seeds / cells are uncorrelated
    h = philox.white_noise(64, seed=12346).ravel()
    assert abs(np.mean(g * h)) < 5.0 / np.sqrt(n)
    assert abs(np.mean(g[1:] * g[:-1])) < 5.0 / np.sqrt(n)


# ---------------------------------------------------------------- kernels
def _time_integral(m, u, v):
    """I_m(u,v) from its definition, int_0^inf t {sin,cos}(t) f(t,u,v) dt (Sec. sec_lattice),
    by adaptive quadrature on [0, 20] plus QAWF Fourier quadrature on the tail."""
    trig = np.sin if m == "s" else np.cos
    head = integrate.quad(lambda t: t * kernels.f_source(t, u, v) * trig(t), 1e-9, 20.0, limit=500)[0]
    tail = integrate.quad(lambda t: t * kernels.f_source(t, u, v), 20.0, np.inf,
                          weight="sin" if m == "s" else "cos", wvar=1.0, limlst=200, limit=500)[0]
    return head + tail


@pytest.mark.parametrize("u,v", [(1.0, 1.0), (0.8, 1.3), (2.0, 1.5), (3.0, 2.5)])
@pytest.mark.parametrize("m", ["s", "c"])
def test_kernels_match_time_integrals(m, u, v):
    """The closed forms of Eq. eq_kernels equal the defining time integrals (quadrature)."""
    import warnings
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        num = _time_integral(m, u, v)
    assert num == pytest.approx(float(kernels.kernel(m, u, v)), rel=1e-6)


def test_kernel_hand_values():
    """I_s(1,1) = 27 pi / 32 and I_c(1,1) = 27 (4 - ln 3) / 32, worked by hand from Eq. eq_kernels;
    I_s vanishes below the resonance u + v = sqrt3 (the Theta factor)."""
    assert float(kernels.I_s(1.0, 1.0)) == pytest.approx(27 * np.pi / 32, rel=1e-14)
    assert float(kernels.I_c(1.0, 1.0)) == pytest.approx(27 * (4 - np.log(3)) / 32, rel=1e-14)
    assert float(kernels.I_s(0.6, 0.9)) == 0.0
    # symmetric kernels
    assert float(kernels.I_c(0.7, 1.4)) == pytest.approx(float(kernels.I_c(1.4, 0.7)), rel=1e-15)


def test_transfer_function_limits():
    """T(y) follows the series of 3 j1(z)/z, 1 - y^2/30 + y^4/2520, at small y (T -> 1, the stated
    initial condition) and T + y T' equals the numerical derivative (Sec. sec_envelope)."""
    y0 = 0.05
    assert float(kernels.transfer(y0)) == pytest.approx(1 - y0 ** 2 / 30 + y0 ** 4 / 2520, abs=1e-10)
    y = np.array([0.3, 1.7, 5.0, 12.0])
    h = 1e-6
    dT = (kernels.transfer(y + h) - kernels.transfer(y - h)) / (2 * h)
    np.testing.assert_allclose(kernels.transfer_log_derivative_term(y), kernels.transfer(y) + y * dT, rtol=1e-7, atol=1e-9)


# ---------------------------------------------------------------- decomposition
def test_grid_cumulative_is_linear_in_n():
    """Eq. eq_grid_density: n(u_n) = n, i.e. equal integrated density between edges."""
    p = dict(umin=1e-3, upiv=1.0, sigp=0.5, Ap=10.0)
    e = decomposition.grid_edges(200, umax=15.0, **p)
    R = decomposition.cumulative_density(e, **p)
    np.testing.assert_allclose(np.diff(R), R[-1] / 200, rtol=1e-10)
    # the closed-form cumulative is the integral of rho
    rho = lambda u: 1 + 10.0 * np.exp(-(u - 1.0) ** 2 / (2 * 0.25))
    assert integrate.quad(rho, 1e-3, 2.3)[0] == pytest.approx(float(decomposition.cumulative_density(2.3, **p)), rel=1e-12)


def test_grid_uniform_when_no_bump():
    """A_p = 0 gives a uniform grid (stated under Eq. eq_grid_density)."""
    e = decomposition.grid_edges(50, umin=0.5, umax=3.0, upiv=1.0, sigp=0.5, Ap=0.0)
    np.testing.assert_allclose(e, np.linspace(0.5, 3.0, 51), rtol=0, atol=1e-13)


def test_full_rank_reconstruction_and_orthonormality(dec):
    """Eq. eq_diagonalization with all modes reproduces C; phi_a are orthonormal in L2(du)
    because the f_i of Eq. eq_basis are; the reconstructed kernel on cell centres is I on the strip."""
    for m in ("s", "c"):
        Q, s = dec.Q_all[m], dec.sigma_all[m]
        np.testing.assert_allclose((Q * s) @ Q.T, dec.C[m], atol=1e-12 * np.abs(dec.C[m]).max())
        ph = Q / np.sqrt(dec.widths)[:, None]
        gram = ph.T @ (ph * dec.widths[:, None])
        np.testing.assert_allclose(gram, np.eye(len(s)), atol=1e-11)
        Kfull = dec.kernel_matrix(m)
        u = dec.centres
        strip = (np.abs(u[:, None] - u[None, :]) <= 1) & (u[:, None] + u[None, :] >= 1)
        with np.errstate(all="ignore"):
            ref = np.where(strip, kernels.kernel(m, u[:, None], u[None, :]), 0.0)
        np.testing.assert_allclose(Kfull, ref, atol=1e-10 * np.abs(ref).max())


def test_truncation_properties(dec):
    """|sigma| sorted descending, a real gap at the cut (basis-independent truncation),
    and the reconstruction error falls as N_alpha grows (Sec. sec_decomposition)."""
    for m in ("s", "c"):
        s = np.abs(dec.sigma_all[m])
        assert np.all(np.diff(s) <= 0)
        assert s[49] / s[50] - 1 > 1e-8
        C = dec.C[m]
        errs = []
        for na in (10, 30, 50, 100):
            Q = dec.Q_all[m][:, :na]
            errs.append(np.linalg.norm((Q * dec.sigma_all[m][:na]) @ Q.T - C))
        assert errs == sorted(errs, reverse=True)


def test_cell_lookup_matches_definition(dec):
    """cell_of puts u = |n|/n_c in [e_i, e_{i+1}) (checked point by point with sqrt)."""
    rng = np.random.default_rng(0)
    msq = rng.integers(0, 3 * 128 ** 2, size=5000)
    for n_c in (1, 7, 64):
        c = decomposition.cell_of(msq, n_c, dec.edges)
        u = np.sqrt(msq) / n_c
        inside = (u >= dec.edges[0]) & (u < dec.edges[-1])
        assert np.all((c >= 0) == inside)
        ci = c[inside]
        assert np.all(dec.edges[ci] <= u[inside]) and np.all(u[inside] < dec.edges[ci + 1])


# ---------------------------------------------------------------- synthesis / maps
@pytest.mark.parametrize("sigma", [0.1, 0.5, 1.0])
def test_lognormal_normalisation_and_width(sigma):
    """Eq. eq_lognormal is a normalised Gaussian in ln k: its integral over ln k is the amplitude A, its mean
    is ln k* and its variance sigma^2 (quadrature, not the closed form).  The dimensionful spectrum then gives
    the same total variance, <zeta^2> = int d^3k/(2 pi)^3 P(k) = int P k^2 dk / (2 pi^2) = A, which pins the
    2 pi^2 / k^3 of Eq. eq_adimensional_P as well."""
    A, kstar = 3e-3, 7.5
    lo, hi = np.log(kstar) - 12 * sigma, np.log(kstar) + 12 * sigma
    f = lambda lk: synth.delta2_lognormal(np.exp(lk), A, sigma, kstar)
    m0 = integrate.quad(f, lo, hi, epsabs=0, epsrel=1e-13, limit=200)[0]
    m1 = integrate.quad(lambda lk: (lk - np.log(kstar)) * f(lk), lo, hi, epsabs=1e-14 * A, epsrel=1e-10, limit=200)[0]
    m2 = integrate.quad(lambda lk: (lk - np.log(kstar)) ** 2 * f(lk), lo, hi, epsabs=0, epsrel=1e-12, limit=200)[0]
    assert m0 == pytest.approx(A, rel=1e-10)
    assert abs(m1) < 1e-12 * A
    assert m2 / m0 == pytest.approx(sigma ** 2, rel=1e-10)
    var = integrate.quad(lambda lk: synth.p_zeta(np.exp(lk), A, sigma, kstar) * np.exp(3 * lk) / (2 * np.pi ** 2),
                         lo, hi, epsabs=0, epsrel=1e-13, limit=200)[0]
    assert var == pytest.approx(A, rel=1e-10)


def test_synthesis_hermitian_zeroed_and_normalised():
    """zeta_g is real (Hermitian spectrum), DC and Nyquist planes are zero, and the shell-averaged
    |zeta_g~|^2 / (V P_zeta) is 1 within sampling error (<X~X~*> = V P, Sec. sec_envelope_obs)."""
    N, L = 64, 3.0
    kstar = 8 * 2 * np.pi / L
    zt = synth.zeta_g_tilde(N, L, 1e-2, 0.5, kstar, seed=3)
    x, imag = synth.to_real(zt, L)
    assert imag < 1e-12 * np.abs(x).max()
    assert zt[0, 0, 0] == 0 and np.all(zt[N // 2] == 0) and np.all(zt[:, N // 2] == 0) and np.all(zt[:, :, N // 2] == 0)
    n = synth.wavenumbers(N)
    n0, n1, n2 = np.meshgrid(n, n, n, indexing="ij")
    r = np.sqrt(n0 ** 2 + n1 ** 2 + n2 ** 2)
    P = synth.p_zeta(2 * np.pi / L * r, 1e-2, 0.5, kstar)
    ok = (r > 0) & (n0 != N // 2) & (n1 != N // 2) & (n2 != N // 2)
    for nc in (6, 8, 12):
        sh = ok & (np.abs(r - nc) < 0.5)
        ratio = np.mean(np.abs(zt[sh]) ** 2 / (L ** 3 * P[sh]))
        assert abs(ratio - 1) < 5 / np.sqrt(sh.sum() / 2)


def test_parseval_of_conventions():
    """dx^3 sum |x|^2 = (1/V) sum |X~|^2 for the continuum-normalised transform pair."""
    N, L = 16, 2.0
    x = np.random.default_rng(1).standard_normal((N, N, N))
    X = synth.to_fourier(x, L)
    dx = L / N
    assert dx ** 3 * np.sum(x ** 2) == pytest.approx(np.sum(np.abs(X) ** 2) / L ** 3, rel=1e-12)
    y, imag = synth.to_real(X, L)
    np.testing.assert_allclose(y, x, atol=1e-12)


def test_maps_special_cases():
    """Local map with F_NL = G_NL = 0 is the identity; the USR map -1/3 ln(1-3z) is, by its
    Taylor series, z + (3/2) z^2 + 3 z^3 + O(z^4); floor hits are counted."""
    z = np.linspace(-0.01, 0.01, 101)
    y, _ = synth.apply_map(z, "local", 0.0, 0.0)
    np.testing.assert_array_equal(y, z)
    u, hits = synth.apply_map(z, "usr")
    np.testing.assert_allclose(u, z + 1.5 * z ** 2 + 3 * z ** 3, atol=7.0 * 0.01 ** 4)  # next term (81/12) z^4
    assert hits == 0
    _, hits = synth.apply_map(np.array([0.0, 0.34, 0.5]), "usr", usr_floor=1e-6)
    assert hits == 2


# ---------------------------------------------------------------- TT projection
def test_polarisation_tensors_transverse_traceless_orthonormal():
    """e^l k = 0, tr e^l = 0, e^l : e^l' = delta (Sec. sec_sigw), incl. k_hat parallel to e_0,
    and sum_l e^l e^l = Lambda (the TT projector)."""
    rng = np.random.default_rng(2)
    n = rng.integers(-8, 9, size=(500, 3))
    n = n[np.linalg.norm(n, axis=1) > 0]
    n = np.vstack([n, [[3, 0, 0], [-5, 0, 0]]])
    ep, ex = sigw.polarisation_tensors(n)
    kh = n / np.linalg.norm(n, axis=1, keepdims=True)
    for e in (ep, ex):
        assert np.abs(np.einsum("mij,mj->mi", e, kh)).max() < 1e-12
        assert np.abs(np.einsum("mii->m", e)).max() < 1e-12
        np.testing.assert_allclose(np.einsum("mij,mij->m", e, e), 1.0, atol=1e-12)
    assert np.abs(np.einsum("mij,mij->m", ep, ex)).max() < 1e-12
    P = np.eye(3)[None] - kh[:, :, None] * kh[:, None, :]
    Lam = 0.5 * (np.einsum("mil,mjn->mijln", P, P) + np.einsum("min,mjl->mijln", P, P)
                 - np.einsum("mij,mln->mijln", P, P))
    S = np.einsum("mij,mln->mijln", ep, ep) + np.einsum("mij,mln->mijln", ex, ex)
    np.testing.assert_allclose(S, Lam, atol=1e-12)


# ---------------------------------------------------------------- convolution route
@pytest.mark.parametrize("kind,F", [("gauss", 0.0), ("local", 3.0), ("usr", 0.0)])
def test_fft_route_equals_direct_sum_N8(dec, kind, F):
    """Convolution theorem: the FFT route (Eq. eq_final_envelopes) equals the direct lattice sum
    (Eqs. eq_naive_A/B) with the same truncated kernel, in every shell, to round-off."""
    N, L = 8, 1.0
    Phi, _ = synth.phi_tilde(N, L, 2e-2, 0.5, 2 * 2 * np.pi / L, seed=1, kind=kind, F_NL=F)
    a = sigw.omega(Phi, L, dec)
    b = brute.omega_brute(Phi, L, dec)
    np.testing.assert_allclose(a["omega"], b["omega"], rtol=1e-11)
    np.testing.assert_allclose(a["PA"], b["PA"], rtol=1e-11)
    np.testing.assert_allclose(a["PB"], b["PB"], rtol=1e-11)
    np.testing.assert_array_equal(a["Nk"], b["Nk"])


def test_fft_route_equals_direct_sum_N16(dec):
    """As above at N = 16 for the first and last shells (the last touches the Nyquist planes)."""
    N, L = 16, 1.0
    Phi, _ = synth.phi_tilde(N, L, 1e-2, 0.5, 4 * 2 * np.pi / L, seed=7, kind="usr")
    a = sigw.omega(Phi, L, dec, shells=[1, 8])
    b = brute.omega_brute(Phi, L, dec, shells=[1, 8])
    np.testing.assert_allclose(a["omega"], b["omega"], rtol=1e-11)


def test_ball_restricted_direct_sum_equals_full_sum():
    """Summing only over |n1| < u_max n_c drops exact zeros of the kernel: with u_max = 3 the ball is smaller
    than the lattice for n_c <= 2 and covers it beyond; both forms agree in every shell to round-off."""
    d3 = decomposition.build(n_modes=40, n_alpha=12, umax=3.0)
    N, L = 16, 1.0
    Phi, _ = synth.phi_tilde(N, L, 1e-2, 0.5, 3 * 2 * np.pi / L, seed=8, kind="local", F_NL=1.5)
    a = brute.omega_brute(Phi, L, d3, shells=[1, 2, 3, 8])
    b = brute.omega_brute(Phi, L, d3, shells=[1, 2, 3, 8], ball=True)
    np.testing.assert_allclose(b["omega"], a["omega"], rtol=1e-12)
    np.testing.assert_allclose(b["PB"], a["PB"], rtol=1e-12)
    f = sigw.omega(Phi, L, d3, shells=[1, 2])
    np.testing.assert_allclose(b["omega"][:2], f["omega"], rtol=1e-11)


def test_full_rank_fft_route_equals_exact_kernel_sum(dec):
    """Keeping all N_modes eigenpairs, the FFT route equals the direct sum with the plain cell-centre
    kernel I(u_i, u_j) on the strip (no eigendecomposition on that side)."""
    N, L = 8, 1.0
    Phi, _ = synth.phi_tilde(N, L, 1e-2, 0.5, 2 * 2 * np.pi / L, seed=4, kind="local", F_NL=2.0)
    terms = {m: (dec.sigma_all[m], (dec.Q_all[m] / np.sqrt(dec.widths)[:, None]).T) for m in "sc"}
    a = sigw.omega(Phi, L, dec, terms=terms)
    u = dec.centres
    strip = (np.abs(u[:, None] - u[None, :]) <= 1) & (u[:, None] + u[None, :] >= 1)
    with np.errstate(all="ignore"):
        Km = {m: np.where(strip, kernels.kernel(m, u[:, None], u[None, :]), 0.0) for m in "sc"}
    b = brute.omega_brute(Phi, L, dec, kernel_matrices=Km)
    np.testing.assert_allclose(a["omega"], b["omega"], rtol=1e-9)


def test_rank_one_kernel_is_single_convolution(dec):
    """A separable kernel I = g(u) g(v) is one convolution term (Eq. eq_decomposition with one term)."""
    N, L = 8, 1.0
    Phi, _ = synth.phi_tilde(N, L, 1e-2, 0.5, 2 * 2 * np.pi / L, seed=5)
    g = np.exp(-dec.centres)
    terms = {m: (np.array([1.0]), g[None, :]) for m in "sc"}
    a = sigw.omega(Phi, L, dec, terms=terms)
    b = brute.omega_brute(Phi, L, dec, kernel_matrices={m: np.outer(g, g) for m in "sc"})
    np.testing.assert_allclose(a["omega"], b["omega"], rtol=1e-11)


def test_omega_scales_as_amplitude_squared(dec):
    """Gaussian case: Phi~ is linear in sqrt(A) and Omega quartic in Phi~, so Omega(2A) = 4 Omega(A)."""
    N, L = 16, 1.0
    a = sigw.omega(synth.phi_tilde(N, L, 1e-2, 0.5, 4 * 2 * np.pi / L, seed=9)[0], L, dec, shells=[3, 5])
    b = sigw.omega(synth.phi_tilde(N, L, 2e-2, 0.5, 4 * 2 * np.pi / L, seed=9)[0], L, dec, shells=[3, 5])
    np.testing.assert_allclose(b["omega"], 4 * a["omega"], rtol=1e-12)


def test_local_map_mean_shift_is_invisible(dec):
    """Subtracting <zeta_g^2> only moves k = 0, where phi(0) = 0: Omega is unchanged."""
    N, L = 16, 1.0
    zt = synth.zeta_g_tilde(N, L, 1e-2, 0.5, 4 * 2 * np.pi / L, seed=11)
    zg, _ = synth.to_real(zt, L)
    p1 = (2 / 3) * synth.to_fourier(zg + 3.0 * (zg ** 2 - np.mean(zg ** 2)), L)
    p2 = (2 / 3) * synth.to_fourier(zg + 3.0 * zg ** 2, L)
    a = sigw.omega(p1, L, dec, shells=[2, 6])
    b = sigw.omega(p2, L, dec, shells=[2, 6])
    np.testing.assert_allclose(a["omega"], b["omega"], rtol=1e-10)


def test_usr_map_matches_its_taylor_series(dec):
    """At small amplitude the USR map equals the local map with F_NL = 3/2, G_NL = 3 (Taylor series
    of -1/3 ln(1 - 3 z)); Omega agrees to the size of the neglected z^4 term."""
    N, L = 16, 1.0
    args = (N, L, 1e-6, 0.5, 4 * 2 * np.pi / L)
    a = sigw.omega(synth.phi_tilde(*args, seed=13, kind="usr")[0], L, dec, shells=[3, 6])
    b = sigw.omega(synth.phi_tilde(*args, seed=13, kind="local", F_NL=1.5, G_NL=3.0)[0], L, dec, shells=[3, 6])
    c = sigw.omega(synth.phi_tilde(*args, seed=13, kind="gauss")[0], L, dec, shells=[3, 6])
    np.testing.assert_allclose(a["omega"], b["omega"], rtol=1e-6)
    assert np.max(np.abs(a["omega"] / c["omega"] - 1)) > 1e-4  # the quadratic term is visible


def test_stilde_hermitian(dec):
    """S_ij(x) is real, so S~(-k) = S~(k)* (exact symmetry of the forward DFT)."""
    N, L = 8, 1.0
    Phi, _ = synth.phi_tilde(N, L, 1e-2, 0.5, 2 * 2 * np.pi / L, seed=1, kind="usr")
    St = sigw.envelope_fields(Phi, L, dec.edges, dec.sigma["s"], dec.phi["s"], 2)
    i = np.arange(N)
    mi = (-i) % N
    for c in range(6):
        np.testing.assert_allclose(St[c][np.ix_(mi, mi, mi)], np.conj(St[c]), atol=1e-14 * np.abs(St[c]).max())


# ---------------------------------------------------------------- statistics and physics
def test_seed_mean_matches_wick_expectation(dec):
    """Gaussian Phi: the mean of the FFT-route Omega over seeds equals the exact Wick expectation
    within its standard error (ties synthesis normalisation to the estimator)."""
    N, L = 8, 1.0
    kstar = 2 * 2 * np.pi / L
    ex = wick.expected_omega(N, L, 1e-2, 0.8, kstar, dec, [1, 2, 3])
    vals = np.array([sigw.omega(synth.phi_tilde(N, L, 1e-2, 0.8, kstar, seed=s)[0], L, dec, shells=[1, 2, 3])["omega"]
                     for s in range(100, 164)])
    mean, se = vals.mean(0), vals.std(0, ddof=1) / np.sqrt(len(vals))
    assert np.all(np.abs(mean - ex["omega"]) < 4 * se), (mean, ex["omega"], se)


def _semi_analytic_dense(k, A, sigma, kstar, n=3000):
    """Eq. eq_semi_anal by a plain midpoint sum in other variables: x = ln(k(s+q)/2k*), y = ln(k(s-q)/2k*), in
    which the two Delta^2 factors are Gaussians and dq ds = (s^2 - q^2)/2 dx dy; the domain q in [0, 1], s >= 1
    is a mask on the grid (half weight on the q = 0 diagonal).  The kernel T of Eq. eq_semi_anal is written out
    vectorised here; this pins the quadrature, not T (T is tied to the kernels I_s, I_c by the Wick-sum test)."""
    lim = 9.0 * sigma
    h = 2.0 * lim / n
    x = -lim + h * (np.arange(n) + 0.5)
    X, Y = np.meshgrid(x, x, indexing="ij")
    c = 2.0 * kstar / k
    up, um = c * np.exp(X), c * np.exp(Y)
    s, q = (up + um) / 2.0, (up - um) / 2.0
    ok = (q >= 0.0) & (q <= 1.0) & (s >= 1.0)
    g = A / np.sqrt(2.0 * np.pi * sigma ** 2)
    w = (g * np.exp(-X ** 2 / (2 * sigma ** 2)) * g * np.exp(-Y ** 2 / (2 * sigma ** 2)))[ok]
    w *= np.where(np.eye(n, dtype=bool), 0.5, 1.0)[ok]
    qq, ss = q[ok], s[ok]
    lg = np.log(np.abs((3.0 - qq ** 2) / (3.0 - ss ** 2)))
    T = 12.0 * (qq ** 2 + ss ** 2 - 6) ** 4 * (qq ** 2 - 1) ** 2 * (ss ** 2 - 1) ** 2 / (ss ** 2 - qq ** 2) ** 8 * (
        (lg + 2.0 * (ss ** 2 - qq ** 2) / (qq ** 2 + ss ** 2 - 6)) ** 2 + np.pi ** 2 * (ss > np.sqrt(3.0)))
    return float(np.sum(w * T * (ss ** 2 - qq ** 2) / 2.0) * h * h)


@pytest.mark.parametrize("sigma", [0.5, 1.0])
@pytest.mark.parametrize("k", [0.5, 1.0, 2.0])
def test_semi_analytic_quadrature_converges(sigma, k):
    """The adaptive quadrature of Eq. eq_semi_anal equals a plain midpoint sum of the same integral in other
    variables (the two momenta's logarithms) to within that sum's own discretisation error (< 1 %).  A broad
    peak (sigma = 1) is where a quadrature over a linear s axis loses the narrow peak of its integrand."""
    a = semi_analytic.omega_gauss(k, 1e-2, sigma, 1.0)
    b = _semi_analytic_dense(k, 1e-2, sigma, 1.0)
    assert abs(a / b - 1) < 1e-2


@pytest.mark.parametrize("k", [0.5, 1.5])
def test_semi_analytic_narrow_peak_limit(k):
    """As sigma -> 0, Delta^2 -> A delta(ln k/k*) and Eq. eq_semi_anal collapses onto q = 0, s0 = 2 k*/k: with
    dq ds = (s^2 - q^2)/2 dx dy and half of the peak's mass on the q >= 0 side, Omega -> A^2 s0^2 T(0, s0) / 4.
    (k = 0.5 and 1.5 keep s0 away from sqrt3 and sqrt6, where T varies too fast for the limit at sigma = 0.002.)"""
    s0 = 2.0 / k
    limit = 1e-4 * s0 ** 2 * semi_analytic.T_kernel(0.0, s0) / 4.0
    assert semi_analytic.omega_gauss(k, 1e-2, 0.002, 1.0) == pytest.approx(limit, rel=5e-4)


@pytest.mark.slow
def test_wick_expectation_matches_semi_analytic(dec):
    """The exact lattice expectation for Gaussian zeta agrees with Eq. eq_semi_anal at the paper's
    stated accuracy (< ~10 %, Sec. sec_numerical / Sec. sec_conclusions), here at N = 32, k = k*."""
    N, n_c, A, sig = 32, 6, 1e-2, 0.5
    kstar = 1.0
    L = n_c * 2 * np.pi / kstar
    w = wick.expected_omega(N, L, A, sig, kstar, dec, [n_c])["omega"][0]
    s = semi_analytic.omega_gauss(kstar, A, sig, kstar)
    assert abs(w / s - 1) < 0.10


# ---------------------------------------------------------------- per-target box (Sec. sec_numerical)
@pytest.mark.parametrize("sigma", [0.1, 0.5, 1.0])
def test_k_bar_is_the_quantile_of_the_integrated_spectrum(sigma):
    """k_bar encloses 1 - eps of int Delta^2 dln k: checked by quadrature, not through erfinv."""
    A, kstar, eps = 1e-2, 2.0, 0.1
    kb = semi_analytic.k_bar(sigma, kstar, eps)
    f = lambda lk: synth.delta2_lognormal(np.exp(lk), A, sigma, kstar)
    lo, hi = np.log(kstar) - 12 * sigma, np.log(kstar) + 12 * sigma
    part = integrate.quad(f, lo, np.log(kb), epsabs=0, epsrel=1e-12)[0]
    tot = integrate.quad(f, lo, hi, epsabs=0, epsrel=1e-12)[0]
    assert abs(part / tot - (1 - eps)) < 1e-9


def test_target_box_puts_k_on_a_shell_near_the_rule():
    """k = n_c k_f exactly; the box differs from pi N / k_max only by the rounding of n_c."""
    A, sigma, kstar = 1e-2, 0.5, 1.0
    for N in (32, 64, 128):
        for k in np.geomspace(0.05, 5.0, 37):
            L, n_c = semi_analytic.target_box(N, k, A, sigma, kstar)
            assert abs(n_c * 2 * np.pi / L - k) < 1e-12 * k
            L0 = semi_analytic.box_size(N, k, A, sigma, kstar)
            x = k * L0 / (2 * np.pi)  # the unrounded shell index
            if 1 <= round(x) <= N // 2:
                assert abs(n_c - x) <= 0.5 + 1e-12 and abs(L / L0 - 1) <= 0.5 / x + 1e-12
            if k >= semi_analytic.k_bar(sigma, kstar):
                assert abs(L0 - np.pi * N / (3 * k)) < 1e-12 * L0


# ---------------------------------------------------------------- non-local map (Eq. eq_nonlocal)
def test_nonlocal_map_on_a_plane_wave():
    """For zeta_g = a cos(k.x): lap(zeta_g^2) = -2 k^2 a^2 cos(2 k.x) and zeta_g lap(zeta_g) = -k^2 a^2 cos^2(k.x)
    (closed forms), so the map is known exactly."""
    N, L, a, kstar, al, be = 16, 2.0, 0.3, 5.0, 1.7, -0.6
    kf = 2 * np.pi / L
    kv = kf * np.array([1.0, 2.0, 3.0])
    x = np.arange(N) * L / N
    X0, X1, X2 = np.meshgrid(x, x, x, indexing="ij")
    ph = kv[0] * X0 + kv[1] * X1 + kv[2] * X2
    k2 = kv @ kv
    zg = a * np.cos(ph)
    want = zg + al / kstar ** 2 * (-2 * k2 * a * a * np.cos(2 * ph)) + be / kstar ** 2 * (-k2 * a * a * np.cos(ph) ** 2)
    got = synth.nonlocal_map(zg, L, al, be, kstar)
    np.testing.assert_allclose(got, want, atol=1e-12)


def test_nonlocal_map_with_zero_coefficients_is_the_identity():
    a = synth.phi_tilde(16, 1.0, 1e-2, 0.5, 4 * 2 * np.pi, 3, "nonlocal", alpha_NL=0.0, beta_NL=0.0)[0]
    b = synth.phi_tilde(16, 1.0, 1e-2, 0.5, 4 * 2 * np.pi, 3, "local", F_NL=0.0)[0]
    assert np.array_equal(a, b)


# ---------------------------------------------------------------- decomposition study
def test_truncation_error_is_the_eigenvalue_tail():
    """For a symmetric matrix the Frobenius error of the rank-k eigen truncation is the root of the tail sum of
    squared eigenvalues over the total (Eckart-Young); the oracle's matrix-based error must equal it."""
    d = decomposition.build(n_modes=80, n_alpha=20)
    for m in ("s", "c"):
        w = d.sigma_all[m]
        for k in (5, 20, 50):
            f, mx, gap = decomposition.truncation_error(d, m, k)
            assert abs(f - np.sqrt(np.sum(w[k:] ** 2) / np.sum(w ** 2))) < 1e-12
            assert 0 < mx <= 1 and 0 < gap <= 1
        errs = [decomposition.truncation_error(d, m, k)[0] for k in range(1, 80)]
        assert np.all(np.diff(errs) <= 1e-15)


# ---------------------------------------------------------------- jackknife (Sec. sec_envelope_obs)
def test_jackknife_replica_mean_is_the_shell_estimator(dec):
    """The mean of the leave-one-out replicas equals the k-space shell average (Parseval links the real-space
    energies to sum_k |X_k|^2), in every offered shell."""
    N, L = 16, 1.0
    Phi, _ = synth.phi_tilde(N, L, 2e-2, 0.5, 4 * 2 * np.pi / L, seed=21, kind="local", F_NL=2.0)
    j = jackknife.jackknife(Phi, L, dec, shells=[1, 3, 7], M=4)
    o = sigw.omega(Phi, L, dec, shells=[1, 3, 7])
    for k in ("PA", "PB", "omega"):
        np.testing.assert_allclose(j[k], o[k], rtol=1e-12)
    assert np.all(j["sigma_omega"] > 0) and np.all(j["sigma_omega"] < j["omega"])


def test_jackknife_variance_is_the_squared_standard_error():
    """For replicas of a mean, the jackknife variance equals the squared standard error of the per-sub-volume
    estimates P_i = M^3 E_i / (V N_k) (a classical identity, independent of the replica formula)."""
    rng = np.random.default_rng(3)
    N, M = 16, 4
    X = rng.standard_normal((N, N, N)) + 1j * rng.standard_normal((N, N, N))
    E = jackknife.subvolume_energies(X, M)
    n3 = M ** 3
    assert abs(E.sum() - np.sum(np.abs(X) ** 2)) < 1e-9 * E.sum()  # Parseval
    rep = (E.sum() - E) / (1 - 1 / n3)
    per = n3 * E
    assert abs(jackknife.jackknife_sigma(rep) - per.std(ddof=1) / np.sqrt(n3)) < 1e-10 * per.mean()


def test_jackknife_single_mode_has_no_spread():
    """One Fourier mode has a uniform real-space energy density: every replica is equal, sigma = 0."""
    N, M = 16, 4
    X = np.zeros((N, N, N), dtype=np.complex128)
    X[3, 5, 2] = 2.0 - 1.0j
    E = jackknife.subvolume_energies(X, M)
    np.testing.assert_allclose(E, E.mean(), rtol=1e-12)
    assert jackknife.jackknife_sigma((E.sum() - E)) < 1e-12 * E.sum()
