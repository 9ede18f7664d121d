"""Separable decomposition of I_s, I_c (oracle side), Sec. sec_decomposition.

Steps, in the paper's order:
  1. grid density rho(u) = 1 + A_p exp(-(u-u_p)^2 / (2 sigma_p^2))   (Eq. eq_grid_density)
     and its normalised cumulative n(u); the grid is u(n) for n = 0..N_modes.
     Reading: these N_modes+1 values are the cell EDGES; cell i has centre
     u_i = (e_{i-1}+e_i)/2 and width L_i = e_i - e_{i-1}.
  2. piecewise-constant orthonormal basis f_i = 1_i / sqrt(L_i)      (Eq. eq_basis)
  3. C_ij ~= sqrt(L_i L_j) I(u_i, u_j)                                (Eq. eq_C_matrix_discrete)
     restricted to the triangle strip |u_i - u_j| <= 1 <= u_i + u_j (the paper's
     "|u +- v| < 1" is read as the triangle condition for u + v = k_hat).
  4. C = sum_a sigma_a q^a q^a^T, keep the N_alpha largest |sigma|    (Eq. eq_diagonalization)
  5. phi_a(u) = sum_i q^a_i f_i(u) = q^a_{i(u)} / sqrt(L_{i(u)}), zero outside [u_min, u_max).

Defaults (the paper's meta-parameters, Fig. fig_eigenvalues caption and
Sec. sec_numerical): u_min = 1e-3, u_max = 15, N_modes = 200, u_p = 1,
sigma_p = 0.5, A_p = 10, N_alpha = 50.

Test infrastructure only (see the package docstring).
"""
from dataclasses import dataclass, field

import numpy as np
from scipy.special import erf

from . import kernels

DEFAULTS = dict(n_modes=200, n_alpha=50, umin=1e-3, umax=15.0, upiv=1.0, sigp=0.5, Ap=10.0)


def cumulative_density(u, umin, upiv, sigp, Ap):
    """R(u) = int_{u_min}^u rho(u') du' for Eq. eq_grid_density, in closed form."""
    s2 = np.sqrt(2.0) * sigp
    return (u - umin) + Ap * sigp * np.sqrt(np.pi / 2.0) * (
        erf((u - upiv) / s2) - erf((umin - upiv) / s2))


def grid_edges(n_modes, umin, umax, upiv, sigp, Ap):
    """Edges e_n = u(n), n = 0..n_modes: n(u) = n_modes R(u)/R(u_max) inverted by bisection."""
    Rmax = cumulative_density(umax, umin, upiv, sigp, Ap)
    edges = np.empty(n_modes + 1)
    edges[0], edges[-1] = umin, umax
    for n in range(1, n_modes):
        target = n * Rmax / n_modes
        lo, hi = umin, umax
        for _ in range(200):  # R is strictly increasing (rho >= 1)
            mid = 0.5 * (lo + hi)
            if cumulative_density(mid, umin, upiv, sigp, Ap) < target:
                lo = mid
            else:
                hi = mid
            if hi - lo <= 1e-15 * max(1.0, abs(mid)):
                break
        edges[n] = 0.5 * (lo + hi)
    return edges


def c_matrix(m, centres, widths):
    """C_ij = sqrt(L_i L_j) I_m(u_i, u_j) on the triangle strip, else 0 (Eq. eq_C_matrix_discrete)."""
    ui = centres[:, None]
    uj = centres[None, :]
    strip = (np.abs(ui - uj) <= 1.0) & (ui + uj >= 1.0)
    with np.errstate(divide="ignore", invalid="ignore"):
        val = kernels.kernel(m, ui, uj)
    C = np.where(strip, np.sqrt(widths[:, None] * widths[None, :]) * val, 0.0)
    return C


@dataclass
class Decomposition:
    """Truncated separable form I_m(u,v) ~= sum_a sigma_a phi_a(u) phi_a(v) for m in (s, c)."""
    edges: np.ndarray
    centres: np.ndarray
    widths: np.ndarray
    sigma: dict = field(default_factory=dict)   # m -> (n_alpha,)
    phi: dict = field(default_factory=dict)     # m -> (n_alpha, n_modes), value of phi_a on cell i
    C: dict = field(default_factory=dict)       # m -> full C matrix
    sigma_all: dict = field(default_factory=dict)
    Q_all: dict = field(default_factory=dict)

    def kernel_matrix(self, m, n_alpha=None):
        """K_ij = sum_{a < n_alpha} sigma_a phi_a(cell i) phi_a(cell j): the truncated kernel on cells."""
        s = self.sigma_all[m] if n_alpha is None else self.sigma_all[m][:n_alpha]
        Q = self.Q_all[m][:, :len(s)]
        ph = Q / np.sqrt(self.widths)[:, None]
        return (ph * s[None, :]) @ ph.T


def build(n_modes=200, n_alpha=50, umin=1e-3, umax=15.0, upiv=1.0, sigp=0.5, Ap=10.0):
    """Steps 1-5 above for both kernels."""
    edges = grid_edges(n_modes, umin, umax, upiv, sigp, Ap)
    centres = 0.5 * (edges[:-1] + edges[1:])
    widths = edges[1:] - edges[:-1]
    dec = Decomposition(edges=edges, centres=centres, widths=widths)
    for m in ("s", "c"):
        C = c_matrix(m, centres, widths)
        w, Q = np.linalg.eigh(C)
        order = np.lexsort((np.arange(len(w)), -np.abs(w)))  # |sigma| descending, ties by index
        w, Q = w[order], Q[:, order]
        dec.C[m] = C
        dec.sigma_all[m] = w
        dec.Q_all[m] = Q
        dec.sigma[m] = w[:n_alpha].copy()
        dec.phi[m] = (Q[:, :n_alpha] / np.sqrt(widths)[:, None]).T.copy()
    return dec


def truncation_error(dec, m, n_alpha):
    """Rank-n_alpha truncation of C (Eq. eq_C_matrix_discrete) against C itself: (Frobenius relative error,
    max-entry error relative to max |C|, |sigma_k| / |sigma_{k-1}| at the cut)."""
    C = dec.C[m]
    s, Q = dec.sigma_all[m][:n_alpha], dec.Q_all[m][:, :n_alpha]
    D = C - (Q * s[None, :]) @ Q.T
    w = dec.sigma_all[m]
    gap = abs(w[n_alpha]) / abs(w[n_alpha - 1]) if n_alpha < len(w) and w[n_alpha - 1] != 0 else 0.0
    return np.linalg.norm(D) / np.linalg.norm(C), np.abs(D).max() / np.abs(C).max(), gap


def cell_of(msq, n_c, edges):
    """Cell index of lattice points with integer |n|^2 = msq for target shell n_c.

    u = |n| / n_c lies in cell i (0-based) when e_i <= u < e_{i+1}; written on
    squares so that integer |n|^2 is compared with (e_i n_c)^2 in FP64.
    Returns -1 outside [u_min, u_max).
    """
    msq = np.asarray(msq, dtype=np.float64)
    thr = (edges * n_c) ** 2
    k = np.searchsorted(thr, msq, side="right")  # number of edges with thr <= msq
    cell = k - 1
    cell[(k == 0) | (k == len(edges))] = -1
    return cell
