"""Semi-analytic Gaussian Omega_GW in radiation domination (oracle side).

Eq. eq_semi_anal (Sec. sec_envelope_obs), with the kernel T(q, s) the paper
quotes from Witkowski:
  Omega(k) = int_0^1 dq int_1^inf ds T(q,s) Delta^2(k (s+q)/2) Delta^2(k (s-q)/2)
  T(q,s)   = 12 (q^2+s^2-6)^4 (q^2-1)^2 (s^2-1)^2 / (s^2-q^2)^8
             * [ (ln|(3-q^2)/(3-s^2)| + 2(s^2-q^2)/(q^2+s^2-6))^2 + pi^2 Theta(s - sqrt3) ]
evaluated by adaptive quadrature in FP64 over q and t = ln s, the t range split at
the integrable log singularity s = sqrt3 and at the peak s = 2 k*/k, and cut where
the integrand's Delta^2 factors fall below 1e-30 of their peak.

Also the paper's box-size rule (Sec. sec_numerical): L = pi N / k_max,
k_max = 3 max(k, k_bar), with k_bar the (1 - eps) quantile of int Delta^2 dln k.

Test infrastructure only (see the package docstring).
"""
import numpy as np
from scipy import integrate

from .synth import delta2_lognormal

SQRT3 = np.sqrt(3.0)


def T_kernel(q, s):
    q2, s2 = q * q, s * s
    a = q2 + s2 - 6.0
    lg = np.log(np.abs((3.0 - q2) / (3.0 - s2)))
    br = (lg + 2.0 * (s2 - q2) / a) ** 2 + (np.pi ** 2 if s > SQRT3 else 0.0)
    return 12.0 * a ** 4 * (q2 - 1.0) ** 2 * (s2 - 1.0) ** 2 / (s2 - q2) ** 8 * br


def omega_gauss(k, A, sigma, kstar):
    """Eq. eq_semi_anal for the log-normal Delta^2 of Eq. eq_lognormal.

    The s integral runs over t = ln s: the Delta^2 factors put the integrand's weight near s = 2 k*/k, a
    feature of relative width ~sigma that, on a linear s axis, would sit in an interval up to ~1e5 long for a
    broad peak (sigma = 1), where adaptive quadrature does not resolve it.  Breakpoints at s = sqrt3 (the
    integrable log singularity) and at the peak s = 2 k*/k."""
    # support of Delta^2(k (s+q)/2): |ln(k (s+q)/(2 k*))| < sigma sqrt(2 ln 1e30)
    width = sigma * np.sqrt(2.0 * np.log(1e30))
    tmax = np.log(2.0 * kstar * np.exp(width) / k + 1.0)
    tpk = np.log(2.0 * kstar / k)
    pts = sorted({0.0, np.log(SQRT3), tmax} | ({tpk} if 0.0 < tpk < tmax else set()))

    def inner(q):
        def f(t):
            s = np.exp(t)
            return s * T_kernel(q, s) * delta2_lognormal(k * (s + q) / 2.0, A, sigma, kstar) \
                * delta2_lognormal(k * (s - q) / 2.0, A, sigma, kstar)
        tot = 0.0
        for a, b in zip(pts[:-1], pts[1:]):
            tot += integrate.quad(f, a, b, limit=800, epsabs=0.0, epsrel=1e-11)[0]
        return tot

    return integrate.quad(inner, 0.0, 1.0, limit=400, epsabs=0.0, epsrel=1e-10)[0]


def k_bar(sigma, kstar, eps=0.1):
    """(1 - eps) quantile of int Delta^2 dln k for the log-normal: a Gaussian CDF in ln k."""
    from scipy.special import erfinv
    return kstar * np.exp(sigma * np.sqrt(2.0) * erfinv(2.0 * (1.0 - eps) - 1.0))


def target_box(N, k, A, sigma, kstar, eps=0.1):
    """The paper's box for target k, placed on the lattice: n_c = round(k L / 2 pi) in [1, N/2] from the
    rule's L, then L = 2 pi n_c / k so that k_c = k.  Returns (L, n_c)."""
    L0 = box_size(N, k, A, sigma, kstar, eps)
    n_c = int(min(N // 2, max(1, np.floor(k * L0 / (2.0 * np.pi) + 0.5))))
    return 2.0 * np.pi * n_c / k, n_c


def box_size(N, k, A, sigma, kstar, eps=0.1):
    """Paper's rule: L = pi N / k_max, k_max = 3 max(k, k_bar)."""
    # int_0^kbar Delta^2 dln k / int_0^inf = 1 - eps  -> for the log-normal, a Gaussian CDF in ln k
    from scipy.special import erfinv
    kbar = kstar * np.exp(sigma * np.sqrt(2.0) * erfinv(2.0 * (1.0 - eps) - 1.0))
    kmax = 3.0 * max(k, kbar)
    return np.pi * N / kmax
