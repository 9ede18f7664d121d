"""Curvature field synthesis and non-Gaussian maps (oracle side).

Conventions (Sec. sec_envelope_obs, the P_X definition read on a periodic box
of side L with N^3 cells, dx = L/N, V = L^3, k = (2 pi / L) n):
  X~(k) = dx^3 sum_x X(x) e^{-i k.x},   X(x) = (1/V) sum_k X~(k) e^{i k.x},
  <X~(k) X~*(k')> = V delta_kk' P_X(k)  (the continuum (2pi)^3 delta -> V delta).
Lattice wave numbers n_j in (-N/2, N/2] (index N/2 is +N/2).

Steps:
  1. g(x) = Philox white noise (``philox.white_noise``).
  2. zeta_g~(k) = sqrt(P_zeta(k) dx^3) DFT[g](k), P_zeta = 2 pi^2 Delta^2(k) / k^3,
     Delta^2 the log-normal peak of Eq. eq_lognormal; the k = 0 mode and every
     plane with some n_j = N/2 are set to zero.
  3. zeta(x) = map(zeta_g(x)) in real space:
       local  : zeta_g + F_NL (zeta_g^2 - <zeta_g^2>) + G_NL zeta_g^3   (Sec. "Local
                Non-Gaussianities"; <.> the box mean, F_NL = 3/5 f_NL)
       usr    : -(1/3) ln(max(1 - 3 zeta_g, floor))   (the USR-tail map; not in the
                paper, a workload choice; cells with 1 - 3 zeta_g < floor are counted)
       gauss  : identity (no FFT round trip).
  4. Phi~ = (2/3) zeta~  (Phi = 3(1+w)/(5+3w) zeta at w = 1/3, Sec. sec_sigw).

Test infrastructure only (see the package docstring).
"""
import numpy as np
import scipy.fft as sfft

from . import philox


def wavenumbers(N):
    """Integer lattice wave numbers n in (-N/2, N/2] along one axis (index N/2 -> +N/2)."""
    n = np.arange(N)
    return np.where(n <= N // 2, n, n - N)


def delta2_lognormal(k, A, sigma, kstar):
    """Eq. eq_lognormal: Delta^2(k) = A / sqrt(2 pi sigma^2) exp(-ln^2(k/k*) / (2 sigma^2))."""
    k = np.asarray(k, dtype=np.float64)
    with np.errstate(divide="ignore"):
        lk = np.log(k / kstar)
    return A / np.sqrt(2.0 * np.pi * sigma ** 2) * np.exp(-lk * lk / (2.0 * sigma ** 2))


def p_zeta(k, A, sigma, kstar):
    """Dimensionful P(k) = 2 pi^2 Delta^2(k) / k^3 (Eq. eq_adimensional_P)."""
    k = np.asarray(k, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        return 2.0 * np.pi ** 2 * delta2_lognormal(k, A, sigma, kstar) / k ** 3


def zeta_g_tilde(N, L, A, sigma, kstar, seed):
    """Step 2: full-lattice complex zeta_g~ (N^3, FP64), continuum normalisation."""
    dx = L / N
    g = philox.white_noise(N, seed)
    G = sfft.fftn(g, workers=-1)
    n = wavenumbers(N)
    n0, n1, n2 = np.meshgrid(n, n, n, indexing="ij")
    kmag = (2.0 * np.pi / L) * np.sqrt(n0 ** 2 + n1 ** 2 + n2 ** 2)
    P = p_zeta(kmag, A, sigma, kstar)
    P[0, 0, 0] = 0.0
    amp = np.sqrt(P * dx ** 3)
    nyq = (n0 == N // 2) | (n1 == N // 2) | (n2 == N // 2)
    amp[nyq] = 0.0
    return amp * G


def to_real(Xt, L):
    """X(x) = (1/V) sum_k X~ e^{ikx}; the imaginary part must vanish (Hermitian input)."""
    N = Xt.shape[0]
    dx = L / N
    x = sfft.ifftn(Xt, workers=-1) / dx ** 3
    return x.real, np.abs(x.imag).max()


def to_fourier(x, L):
    N = x.shape[0]
    dx = L / N
    return dx ** 3 * sfft.fftn(x, workers=-1)


def apply_map(zg, kind, F_NL=0.0, G_NL=0.0, usr_floor=1e-6):
    """Step 3.  Returns (zeta, n_floor_hits)."""
    if kind == "gauss":
        return zg.copy(), 0
    if kind == "local":
        return zg + F_NL * (zg * zg - np.mean(zg * zg)) + G_NL * zg ** 3, 0
    if kind == "usr":
        arg = 1.0 - 3.0 * zg
        hits = int(np.count_nonzero(arg < usr_floor))
        return -np.log(np.maximum(arg, usr_floor)) / 3.0, hits
    raise ValueError(kind)


def laplacian(xt, L):
    """Spectral Laplacian of a full-lattice spectrum: -k^2 X~ with k = k_f |n| (n_j = +-N/2 give the same k^2)."""
    N = xt.shape[0]
    n = wavenumbers(N)
    n0, n1, n2 = np.meshgrid(n, n, n, indexing="ij")
    return -((2.0 * np.pi / L) ** 2) * (n0 ** 2 + n1 ** 2 + n2 ** 2) * xt


def nonlocal_map(zg, L, alpha_NL, beta_NL, kstar):
    """Eq. eq_nonlocal: zeta = zeta_g + alpha_NL / k*^2 lap(zeta_g^2) + beta_NL / k*^2 zeta_g lap(zeta_g)."""
    lap_zg2, _ = to_real(laplacian(to_fourier(zg * zg, L), L), L)
    lap_zg, _ = to_real(laplacian(to_fourier(zg, L), L), L)
    return zg + alpha_NL / kstar ** 2 * lap_zg2 + beta_NL / kstar ** 2 * zg * lap_zg


def phi_tilde(N, L, A, sigma, kstar, seed, kind="gauss", F_NL=0.0, G_NL=0.0, usr_floor=1e-6, alpha_NL=0.0,
              beta_NL=0.0):
    """Steps 1-4: full-lattice Phi~ (N^3 complex, FP64) and the USR floor-hit count."""
    zgt = zeta_g_tilde(N, L, A, sigma, kstar, seed)
    if kind == "gauss":
        return (2.0 / 3.0) * zgt, 0
    zg, _ = to_real(zgt, L)
    if kind == "nonlocal":
        return (2.0 / 3.0) * to_fourier(nonlocal_map(zg, L, alpha_NL, beta_NL, kstar), L), 0
    z, hits = apply_map(zg, kind, F_NL, G_NL, usr_floor)
    return (2.0 / 3.0) * to_fourier(z, L), hits
