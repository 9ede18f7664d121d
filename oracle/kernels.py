"""Analytic radiation-era kernels I_s(u, v), I_c(u, v) (oracle side).

Sec. sec_lattice, Eq. eq_kernels: the asymptotic time integrals
    I_s(u,v) = int_0^inf dt t sin t f(t,u,v),   I_c(u,v) = int_0^inf dt t cos t f(t,u,v)
of the w = 1/3 source kernel f have the closed forms
    I_s = 27 pi (u^2+v^2-3)^2 / (32 u^3 v^3) * Theta(u+v-sqrt3)
    I_c = 27 (u^2+v^2-3) / (32 u^3 v^3) * ( -4uv + (u^2+v^2-3) ln|(3-(u+v)^2)/(3-(u-v)^2)| )
with Theta(0) = 0.  The defining integrals themselves are also given here
(``f_source``, ``transfer``) so the tests can check the closed forms against
direct quadrature.

Test infrastructure only (see the package docstring).
"""
import numpy as np

SQRT3 = np.sqrt(3.0)


def I_s(u, v):
    """Sine kernel, Eq. eq_kernels (Theta(0) = 0)."""
    u = np.asarray(u, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    a = u * u + v * v - 3.0
    theta = (u + v - SQRT3 > 0.0).astype(np.float64)
    return 27.0 * np.pi * a * a / (32.0 * u ** 3 * v ** 3) * theta


def I_c(u, v):
    """Cosine kernel, Eq. eq_kernels."""
    u = np.asarray(u, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    a = u * u + v * v - 3.0
    lg = np.log(np.abs((3.0 - (u + v) ** 2) / (3.0 - (u - v) ** 2)))
    return 27.0 * a / (32.0 * u ** 3 * v ** 3) * (-4.0 * u * v + a * lg)


def kernel(m, u, v):
    """m = 's' (envelope A) or 'c' (envelope B)."""
    if m == "s":
        return I_s(u, v)
    if m == "c":
        return I_c(u, v)
    raise ValueError(m)


def transfer(y):
    """w = 1/3 transfer function T(y) = 3 j1(y/sqrt3) / (y/sqrt3), Sec. sec_envelope."""
    z = np.asarray(y, dtype=np.float64) / SQRT3
    j1 = np.sin(z) / z ** 2 - np.cos(z) / z
    return 3.0 * j1 / z


def transfer_log_derivative_term(y):
    """T(y) + y T'(y) (the combination in the source kernel f), by the closed form
    d/dy [3 j1(z)/z] with z = y / sqrt3."""
    z = np.asarray(y, dtype=np.float64) / SQRT3
    s, c = np.sin(z), np.cos(z)
    # T(z) = 3 (sin z - z cos z) / z^3 ; z dT/dz = 3 (3 z cos z + (z^2 - 3) sin z) / z^3
    T = 3.0 * (s - z * c) / z ** 3
    zT = 3.0 * (3.0 * z * c + (z * z - 3.0) * s) / z ** 3
    return T + zT


def f_source(t, u, v):
    """Source kernel f(t,u,v) = T(ut)T(vt) + 1/2 (T + t dT/dt)_u (T + t dT/dt)_v, Sec. sec_lattice."""
    return (transfer(u * t) * transfer(v * t)
            + 0.5 * transfer_log_derivative_term(u * t) * transfer_log_derivative_term(v * t))
