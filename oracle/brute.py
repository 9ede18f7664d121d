"""Direct O(N^6) lattice evaluation of the envelopes (oracle side, small N only).

Eqs. eq_naive_A / eq_naive_B of Sec. sec_lattice on the periodic lattice, with
the integrals read as lattice sums (int d^3q/(2pi)^3 -> (1/V) sum_q,
(2pi)^3 delta -> V delta) and the kernel replaced by the same truncated
separable form the FFT route uses, I~(u,v) = sum_a sigma_a phi_a(u) phi_a(v):

  A_l(k) = +(4 / (k_c^2 V)) e^l_ij(k_hat) sum_{q1} q1_i q2_j I~_s(|q1|/k_c, |q2|/k_c) Phi~(q1) Phi~(q2)
  B_l(k) = -(4 / (k_c^2 V)) e^l_ij(k_hat) sum_{q1} q1_i q2_j I~_c(...)         ...
  with q2 = wrap(k - q1), and q_j := 0 where n_j = N/2 (the derivative reading).

No FFT is used: this is the sum the convolution theorem rewrites, so it pins
the FFT route to round-off.

Test infrastructure only (see the package docstring).
"""
import numpy as np

from .decomposition import cell_of
from .sigw import polarisation_tensors, shell_modes
from .synth import wavenumbers


def omega_brute(Phi, L, dec, shells=None, kernel_matrices=None):
    """Omega_GW, P_A, P_B, N_k per shell by the direct sum.

    kernel_matrices : optional {m: K} with K_ij the kernel value on cells (i, j);
    defaults to dec.kernel_matrix(m, n_alpha) (the truncated separable kernel).
    """
    N = Phi.shape[0]
    if shells is None:
        shells = range(1, N // 2 + 1)
    kf = 2.0 * np.pi / L
    V = L ** 3
    n = wavenumbers(N)
    n0, n1, n2 = [a.ravel() for a in np.meshgrid(n, n, n, indexing="ij")]
    msq = n0 ** 2 + n1 ** 2 + n2 ** 2
    nD = np.stack([np.where(a == N // 2, 0, a) for a in (n0, n1, n2)], axis=1).astype(np.float64)
    Pf = Phi.ravel()
    i0, i1, i2 = [a.ravel() for a in np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")]
    n_alpha = len(dec.sigma["s"])
    K = {}
    for m in ("s", "c"):
        Km = kernel_matrices[m] if kernel_matrices is not None else dec.kernel_matrix(m, n_alpha)
        Kp = np.zeros((Km.shape[0] + 1, Km.shape[1] + 1))
        Kp[:-1, :-1] = Km  # last row/column: the "outside the grid" cell, kernel 0
        K[m] = Kp
    out = {"n_c": [], "omega": [], "PA": [], "PB": [], "Nk": []}
    for n_c in shells:
        kc = n_c * kf
        cells = cell_of(msq, n_c, dec.edges)
        cells = np.where(cells < 0, K["s"].shape[0] - 1, cells)
        idx, nvec = shell_modes(N, n_c)
        ep, ex = polarisation_tensors(nvec)
        P = {"s": 0.0, "c": 0.0}
        for mode in range(len(nvec)):
            k0, k1, k2 = idx[0][mode], idx[1][mode], idx[2][mode]
            j0, j1, j2 = (k0 - i0) % N, (k1 - i1) % N, (k2 - i2) % N
            q2 = (j0 * N + j1) * N + j2
            base = Pf * Pf[q2]
            for m, sign in (("s", +1.0), ("c", -1.0)):
                w = K[m][cells, cells[q2]] * base
                M = np.einsum("q,qi,qj->ij", w, nD, nD[q2])
                fac = sign * 4.0 * kf ** 2 / (kc ** 2 * V)
                Ap = fac * np.sum(ep[mode] * M)
                Ax = fac * np.sum(ex[mode] * M)
                P[m] += abs(Ap) ** 2 + abs(Ax) ** 2
        Nk = len(nvec)
        out["n_c"].append(n_c)
        out["PA"].append(P["s"] / (V * Nk))
        out["PB"].append(P["c"] / (V * Nk))
        out["Nk"].append(Nk)
        out["omega"].append(kc ** 3 / (48.0 * np.pi ** 2) * (P["s"] + P["c"]) / (V * Nk))
    return {k: np.array(v) for k, v in out.items()}
