"""Jackknife error bars of the shell power spectra (Sec. sec_envelope_obs), oracle side.

For a target shell and each field X in {A_+, A_x, B_+, B_x}: keep X_k on the shell modes (zero elsewhere),
transform to real space, split the box into M^3 equal sub-volumes, and form M^3 leave-one-out estimates
  P^(i)_X = (E_X - E_X,i) / ((1 - M^-3) V N_k),
where e_X(x) = N^3 |IDFT[X](x)|^2 is the real-space energy density (sum_x e_X = sum_k |X_k|^2, Parseval),
E_X its total and E_X,i its sum over sub-volume i.  Then
  sigma^2_P = (M^3 - 1) / M^3 sum_i (P^(i) - P_bar)^2,   P_bar = mean_i P^(i),
for P_A = P_A,+ + P_A,x, P_B likewise, and Omega = k_c^3 / (48 pi^2) (P_A + P_B) (the replicas of the sum).

Readings: the polarisation basis is the one of Sec. sec_sigw (oracle.sigw.polarisation_tensors); the
sub-volumes are the M^3 blocks of N/M cells per side (N divisible by M); the Nyquist shell n_c = N/2 is not
offered (its modes have no distinct Hermitian partners).

Test infrastructure only (see the package docstring).
"""
import numpy as np

from .sigw import envelope_fields, project, shell_modes


def subvolume_energies(Xfull, M):
    """Energies of the M^3 sub-volumes of e(x) = N^3 |IDFT[X](x)|^2 for a full-lattice spectrum X."""
    N = Xfull.shape[0]
    e = N ** 3 * np.abs(np.fft.ifftn(Xfull)) ** 2
    s = N // M
    return e.reshape(M, s, M, s, M, s).sum(axis=(1, 3, 5)).ravel()


def jackknife_sigma(replicas):
    """sigma^2 = (n - 1) / n sum_i (P^(i) - mean)^2 over the n replicas."""
    r = np.asarray(replicas, dtype=np.float64)
    n = len(r)
    return np.sqrt((n - 1) / n * np.sum((r - r.mean()) ** 2))


def jackknife(Phi, L, dec, shells, M=4):
    """Per shell: PA, PB, omega (replica means) and their jackknife sigmas; dict of arrays."""
    N = Phi.shape[0]
    if N % M or M < 2:
        raise ValueError("N must be a multiple of M >= 2")
    kf = 2.0 * np.pi / L
    V = L ** 3
    n3 = M ** 3
    keys = ("PA", "PB", "omega", "sigma_PA", "sigma_PB", "sigma_omega")
    out = {k: [] for k in keys}
    for n_c in shells:
        if not 1 <= n_c < N // 2:
            raise ValueError("shell out of range (the Nyquist shell is not offered)")
        kc = n_c * kf
        idx, nvec = shell_modes(N, n_c)
        Nk = len(nvec)
        rep = {}
        for m, sign, name in (("s", -1.0, "PA"), ("c", +1.0, "PB")):
            St = envelope_fields(Phi, L, dec.edges, dec.sigma[m], dec.phi[m], n_c)
            Xp, Xx = project(St, idx, nvec)
            fac = sign * 4.0 / kc ** 2
            E = np.zeros(n3)
            for Xl in (Xp, Xx):
                X = np.zeros((N, N, N), dtype=np.complex128)
                X[idx] = fac * Xl
                E += subvolume_energies(X, M)
            rep[name] = (E.sum() - E) / ((1.0 - 1.0 / n3) * V * Nk)
        rep["omega"] = kc ** 3 / (48.0 * np.pi ** 2) * (rep["PA"] + rep["PB"])
        for name in ("PA", "PB", "omega"):
            out[name].append(rep[name].mean())
            out["sigma_" + name].append(jackknife_sigma(rep[name]))
    return {k: np.array(v) for k, v in out.items()}
