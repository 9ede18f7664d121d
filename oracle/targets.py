"""The paper's frequency scan (Sec. sec_numerical), oracle side: each target wavenumber k gets its own box
(semi_analytic.target_box), its own realisation and Omega_GW in the one shell that holds k.

Test infrastructure only (see the package docstring).
"""
import numpy as np

from . import semi_analytic, sigw, synth


def target_scan(N, ks, A, sigma, kstar, dec, seed=1, kind="gauss", F_NL=0.0, G_NL=0.0, usr_floor=1e-6, eps=0.1):
    """Omega_GW(k) for each k in ks; returns dict omega, L, n_c (arrays)."""
    om, Ls, ncs = [], [], []
    for k in ks:
        L, n_c = semi_analytic.target_box(N, k, A, sigma, kstar, eps)
        Phi, _ = synth.phi_tilde(N, L, A, sigma, kstar, seed, kind, F_NL, G_NL, usr_floor)
        om.append(sigw.omega(Phi, L, dec, shells=[n_c])["omega"][0])
        Ls.append(L)
        ncs.append(n_c)
    return {"omega": np.array(om), "L": np.array(Ls), "n_c": np.array(ncs)}
