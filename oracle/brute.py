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


def omega_brute(Phi, L, dec, shells=None, kernel_matrices=None, ball=False):
    """Omega_GW, P_A, P_B, N_k per shell by the direct sum.

    kernel_matrices : optional {m: K} with K_ij the kernel value on cells (i, j);
    defaults to dec.kernel_matrix(m, n_alpha) (the truncated separable kernel).
    ball : sum only over the q1 with |n1| < u_max n_c.  The kernel vanishes once
    |q1| / k_c leaves the u-grid (phi_a = 0 outside [u_min, u_max)), so the terms
    dropped are exact zeros; this makes small shells of large lattices affordable.
    """
    N = Phi.shape[0]
    if shells is None:
        shells = range(1, N // 2 + 1)
    kf = 2.0 * np.pi / L
    V = L ** 3
    n = wavenumbers(N)
    Pf = Phi.ravel()
    n_alpha = len(dec.sigma["s"])
    K = {}
    for m in ("s", "c"):
        Km = kernel_matrices[m] if kernel_matrices is not None else dec.kernel_matrix(m, n_alpha)
        Kp = np.zeros((Km.shape[0] + 1, Km.shape[1] + 1))
        Kp[:-1, :-1] = Km  # last row/column: the "outside the grid" cell, kernel 0
        K[m] = Kp
    outside = K["s"].shape[0] - 1

    def cells_at(n0, n1, n2, n_c):
        c = cell_of(n0 * n0 + n1 * n1 + n2 * n2, n_c, dec.edges)
        return np.where(c < 0, outside, c)

    def deriv(n0, n1, n2):  # q_j / k_f with the Nyquist reading
        return np.stack([np.where(a == N // 2, 0, a) for a in (n0, n1, n2)], axis=1).astype(np.float64)

    out = {"n_c": [], "omega": [], "PA": [], "PB": [], "Nk": []}
    for n_c in shells:
        kc = n_c * kf
        if ball:  # lattice wave numbers n1 (each axis in (-N/2, N/2]) with |n1| < u_max n_c
            R = int(np.ceil(dec.edges[-1] * n_c))
            r = n[(n >= -R) & (n <= R)]
            a0, a1, a2 = [x.ravel() for x in np.meshgrid(r, r, r, indexing="ij")]
            keep = a0 * a0 + a1 * a1 + a2 * a2 < (dec.edges[-1] * n_c) ** 2
            a0, a1, a2 = a0[keep], a1[keep], a2[keep]
        else:
            a0, a1, a2 = [x.ravel() for x in np.meshgrid(n, n, n, indexing="ij")]
        i0, i1, i2 = a0 % N, a1 % N, a2 % N  # array indices of q1
        q1 = (i0 * N + i1) * N + i2
        c1 = cells_at(a0, a1, a2, n_c)
        d1 = deriv(a0, a1, a2)
        idx, nvec = shell_modes(N, n_c)
        ep, ex = polarisation_tensors(nvec)
        P = {"s": 0.0, "c": 0.0}
        for mode in range(len(nvec)):
            k0, k1, k2 = idx[0][mode], idx[1][mode], idx[2][mode]
            j0, j1, j2 = (k0 - i0) % N, (k1 - i1) % N, (k2 - i2) % N
            q2 = (j0 * N + j1) * N + j2
            b0, b1, b2 = n[j0], n[j1], n[j2]
            c2 = cells_at(b0, b1, b2, n_c)
            d2 = deriv(b0, b1, b2)
            base = Pf[q1] * Pf[q2]
            for m, sign in (("s", +1.0), ("c", -1.0)):
                w = K[m][c1, c2] * base
                M = np.einsum("q,qi,qj->ij", w, d1, d2)
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
