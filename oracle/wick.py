"""Exact Gaussian expectation of the lattice Omega estimator (oracle side).

For Gaussian Phi~ with <Phi~(q) Phi~*(q')> = V P_Phi(q) delta_qq' (P_Phi = (4/9) P_zeta,
zero on the k = 0 mode and the Nyquist planes, as synthesised), Wick's theorem
applied to the direct sum of Eq. eq_naive_A gives, for k != 0,

  <|A_l(k)|^2> = 2 (4 / k_c^2)^2 sum_{q1} |F_sym(q1, q2)|^2 P_Phi(q1) P_Phi(q2),
  F(q1, q2)    = e^l_ij(k_hat) q1_i q2_j I~_s(|q1|/k_c, |q2|/k_c),   F_sym = (F(q1,q2) + F(q2,q1)) / 2,

with q2 = wrap(k - q1) and the derivative reading q_j := 0 at n_j = N/2; the
same with I~_c for B.  The expected Omega(k_c) then follows from the shell
average of Sec. sec_envelope_obs.  This is deterministic (no noise draw) and
ties the synthesis normalisation, the kernels and the Omega constants together.

Test infrastructure only (see the package docstring).
"""
import numpy as np

from .decomposition import cell_of
from .sigw import polarisation_tensors, shell_modes
from .synth import p_zeta, wavenumbers


def expected_omega(N, L, A, sigma, kstar, dec, shells, kernel_matrices=None):
    kf = 2.0 * np.pi / L
    V = L ** 3
    n = wavenumbers(N)
    n0, n1, n2 = [a.ravel() for a in np.meshgrid(n, n, n, indexing="ij")]
    msq = n0 ** 2 + n1 ** 2 + n2 ** 2
    nD = np.stack([np.where(a == N // 2, 0, a) for a in (n0, n1, n2)], axis=1).astype(np.float64)
    nyq = (n0 == N // 2) | (n1 == N // 2) | (n2 == N // 2)
    PPhi = (4.0 / 9.0) * p_zeta(kf * np.sqrt(msq.astype(np.float64)), A, sigma, kstar)
    PPhi[(msq == 0) | nyq] = 0.0
    i0, i1, i2 = [a.ravel() for a in np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")]
    n_alpha = len(dec.sigma["s"])
    K = {}
    for m in ("s", "c"):
        Km = kernel_matrices[m] if kernel_matrices is not None else dec.kernel_matrix(m, n_alpha)
        Kp = np.zeros((Km.shape[0] + 1, Km.shape[1] + 1))
        Kp[:-1, :-1] = Km
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
            q2 = (((k0 - i0) % N) * N + (k1 - i1) % N) * N + (k2 - i2) % N
            pp = PPhi * PPhi[q2]
            live = pp > 0.0
            a1, a2 = nD[live], nD[q2[live]]
            for m in ("s", "c"):
                Kv = K[m][cells[live], cells[q2[live]]]
                for e in (ep[mode], ex[mode]):
                    F12 = np.einsum("ij,qi,qj->q", e, a1, a2) * Kv
                    F21 = np.einsum("ij,qi,qj->q", e, a2, a1) * Kv
                    Fs = 0.5 * (F12 + F21) * kf ** 2
                    P[m] += 2.0 * (4.0 / kc ** 2) ** 2 * np.sum(Fs * Fs * pp[live])
        Nk = len(nvec)
        out["n_c"].append(n_c)
        out["PA"].append(P["s"] / (V * Nk))
        out["PB"].append(P["c"] / (V * Nk))
        out["Nk"].append(Nk)
        out["omega"].append(kc ** 3 / (48.0 * np.pi ** 2) * (P["s"] + P["c"]) / (V * Nk))
    return {k: np.array(v) for k, v in out.items()}
