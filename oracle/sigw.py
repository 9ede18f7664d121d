"""Lattice envelopes A, B and Omega_GW by the FFT-convolution route (oracle side).

Follows Sec. sec_lattice and Sec. sec_envelope_obs step by step:

  For a target shell n_c (k_c = n_c k_f, k_f = 2 pi / L) and m in {s, c}:
    V_a(q)     = phi_a^(m)(|q| / k_c) Phi~(q)                               (V_{alpha,q}(k))
    dV_a,j(x)  = (1/V) sum_q i q_j V_a(q) e^{iq.x}                          (gradient fields)
    S_ij(x)    = sum_a sigma_a dV_a,i(x) dV_a,j(x)
    S~_ij(k)   = dx^3 sum_x S_ij(x) e^{-ik.x}
    A_l(k)     = -(4 / k_c^2) e^l_ij(k_hat) S~^(s)_ij(k)                     (Eq. eq_final_envelopes)
    B_l(k)     = +(4 / k_c^2) e^l_ij(k_hat) S~^(c)_ij(k)
  Shell power and spectrum (the P_X estimator and Omega^(RD) of Sec. sec_envelope_obs):
    P_X(k_c)   = sum_{|n| in [n_c - 1/2, n_c + 1/2)} |X_k|^2 / (V N_k)     (full lattice, each mode once)
    Omega(k_c) = k_c^3 / (48 pi^2) sum_l [P_A,l + P_B,l]

Readings where the paper is silent or garbled (shared with the CUDA path):
  * shell width Delta k = k_f (the paper writes pi/L and calls it the fundamental);
    shells n_c = 1..N/2; the scalar k in phi(q/k), 4/k^2 and k^3 is k_c for every
    mode of the shell (only the direction k_hat is per mode).
  * the cell of a lattice point comes from comparing integer |n|^2 with (e_i n_c)^2.
  * derivative factor q_j := 0 where n_j = N/2 (the Nyquist plane); |q| and k_hat
    use n_j = +N/2 there.
  * polarisation basis: u_hat = k_hat x e_0 / |k_hat x e_0| (e_0 the unit vector of
    array axis 0), e_1 in place of e_0 when |k_hat x e_0| < 1e-12; v_hat = k_hat x u_hat
    (Sec. sec_sigw).  Omega does not depend on this choice.

Inverse transforms use ``scipy.fft.irfftn`` on the half spectrum (the fields are
Hermitian, so this equals the full inverse DFT), forward transforms use
``scipy.fft.fftn`` on the full lattice.

Test infrastructure only (see the package docstring).
"""
import numpy as np
import scipy.fft as sfft

from .decomposition import cell_of
from .synth import wavenumbers

PAIRS = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))


def polarisation_tensors(n):
    """e^+ and e^x (each (M,3,3)) for integer direction vectors n (M,3), Sec. sec_sigw."""
    n = np.asarray(n, dtype=np.float64)
    khat = n / np.linalg.norm(n, axis=1, keepdims=True)
    ref = np.zeros_like(khat)
    ref[:, 0] = 1.0
    u = np.cross(khat, ref)
    un = np.linalg.norm(u, axis=1)
    bad = un < 1e-12
    if np.any(bad):
        ref2 = np.zeros((int(bad.sum()), 3))
        ref2[:, 1] = 1.0
        u[bad] = np.cross(khat[bad], ref2)
        un[bad] = np.linalg.norm(u[bad], axis=1)
    u = u / un[:, None]
    v = np.cross(khat, u)
    ep = (u[:, :, None] * u[:, None, :] - v[:, :, None] * v[:, None, :]) / np.sqrt(2.0)
    ex = (u[:, :, None] * v[:, None, :] + v[:, :, None] * u[:, None, :]) / np.sqrt(2.0)
    return ep, ex


def shell_modes(N, n_c):
    """Full-lattice modes with |n| in [n_c - 1/2, n_c + 1/2): (index triples, integer n)."""
    n = wavenumbers(N)
    n0, n1, n2 = np.meshgrid(n, n, n, indexing="ij")
    msq = n0 ** 2 + n1 ** 2 + n2 ** 2
    lo, hi = (n_c - 0.5) ** 2, (n_c + 0.5) ** 2
    idx = np.nonzero((msq >= lo) & (msq < hi))
    nvec = np.stack([n0[idx], n1[idx], n2[idx]], axis=1)
    return idx, nvec


def project(Stilde6, idx, nvec):
    """Sum over polarisations of |e^l_ij S~_ij|^2 at the listed modes -> (M,) per-mode and per-l."""
    ep, ex = polarisation_tensors(nvec)
    S = np.zeros((len(nvec), 3, 3), dtype=np.complex128)
    for c, (i, j) in enumerate(PAIRS):
        val = Stilde6[c][idx]
        S[:, i, j] = val
        S[:, j, i] = val
    Xp = np.einsum("mij,mij->m", ep, S)
    Xx = np.einsum("mij,mij->m", ex, S)
    return Xp, Xx


def envelope_fields(Phi, L, edges, sigma, phi, n_c):
    """S~_ij(k) (6 full-lattice complex arrays) for one target shell and one kernel.

    sigma : (n_alpha,) eigenvalues, phi : (n_alpha, n_modes) values of phi_a on the cells.
    """
    N = Phi.shape[0]
    kf = 2.0 * np.pi / L
    dx = L / N
    n = wavenumbers(N)
    n0, n1, n2 = np.meshgrid(n, n, n, indexing="ij")
    msq = n0 ** 2 + n1 ** 2 + n2 ** 2
    h = N // 2 + 1
    cells = cell_of(msq[:, :, :h], n_c, edges)
    inside = cells >= 0
    cl = np.where(inside, cells, 0)
    qD = []
    for nj in (n0, n1, n2):
        d = np.where(nj == N // 2, 0, nj).astype(np.float64)
        qD.append(kf * d[:, :, :h])
    Ph = Phi[:, :, :h]
    S = np.zeros((6, N, N, N))
    for a in range(len(sigma)):
        Vh = np.where(inside, phi[a][cl], 0.0) * Ph
        G = [sfft.irfftn(1j * qD[j] * Vh, s=(N, N, N), workers=-1) / dx ** 3 for j in range(3)]
        for c, (i, j) in enumerate(PAIRS):
            S[c] += sigma[a] * G[i] * G[j]
    return [dx ** 3 * sfft.fftn(S[c], workers=-1) for c in range(6)]


def omega(Phi, L, dec, shells=None, terms=None):
    """Omega_GW, P_A, P_B (summed over polarisations) and N_k per target shell.

    Phi   : full-lattice complex Phi~ (N^3), continuum normalisation.
    dec   : oracle.decomposition.Decomposition (edges + truncated terms).
    terms : optional {m: (sigma, phi)} overriding dec's truncated terms.
    """
    N = Phi.shape[0]
    if shells is None:
        shells = range(1, N // 2 + 1)
    kf = 2.0 * np.pi / L
    V = L ** 3
    out = {"n_c": [], "omega": [], "PA": [], "PB": [], "Nk": []}
    for n_c in shells:
        kc = n_c * kf
        idx, nvec = shell_modes(N, n_c)
        Nk = len(nvec)
        P = {}
        for m, sign in (("s", -1.0), ("c", +1.0)):
            sig, ph = (terms[m] if terms is not None else (dec.sigma[m], dec.phi[m]))
            St = envelope_fields(Phi, L, dec.edges, sig, ph, n_c)
            Xp, Xx = project(St, idx, nvec)
            fac = sign * 4.0 / kc ** 2
            P[m] = (np.sum(np.abs(fac * Xp) ** 2) + np.sum(np.abs(fac * Xx) ** 2)) / (V * Nk)
        out["n_c"].append(n_c)
        out["PA"].append(P["s"])
        out["PB"].append(P["c"])
        out["Nk"].append(Nk)
        out["omega"].append(kc ** 3 / (48.0 * np.pi ** 2) * (P["s"] + P["c"]))
    return {k: np.array(v) for k, v in out.items()}
