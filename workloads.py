"""Seeded synthetic workloads shared by the tests, the bench and the oracle checks.

Parameter sets only: lattice size, box, log-normal P_zeta parameters, the
zeta_g -> zeta map and seeds, plus the Poisson arrival stream of the serving
workload.  No step of the SIGW method is computed here, so both the CUDA path
and the CPU oracle can take their inputs from this module without sharing any
of the method's arithmetic.

Workloads (the paper's log-normal Delta^2_zeta of Eq. eq_lognormal and the maps of
Sec. sec_numerical; k* is placed on a lattice mode, k* = n_* (2 pi / L), L = 1):
  gauss32     : 32^3,  Gaussian zeta,           A = 1e-2, sigma = 0.5, n_* = 8,  FP64, seed 1
  local128    : 128^3, local f_NL = 5 (F_NL = 3), A = 1e-2, sigma = 0.5, n_* = 16, seed 2
  usr256      : 256^3, USR tail -1/3 ln(1 - 3 zeta_g), A = 5e-3, sigma = 0.3, n_* = 32, seeds 1..4
  broad512    : 512^3, local f_NL = -2 (F_NL = -1.2), A = 1e-2, sigma = 1.0, n_* = 64, seed 5
  serving     : Poisson arrivals, N in {64, 128, 256}, f_NL ~ U[-5, 20], sigma ~ U[0.1, 1],
                A = 1e-2, map uniform over {gauss, local, usr}, n_* = N / 8, seed = request id
"""
from dataclasses import asdict, dataclass, replace
import math
import random

TWO_PI = 2.0 * math.pi


@dataclass(frozen=True)
class Spec:
    """One spectrum request: lattice, P_zeta, map and seed."""
    N: int
    L: float
    A: float
    sigma: float
    kstar: float          # absolute wave number (1 / length)
    kind: str             # "gauss" | "local" | "usr" | "nonlocal"
    F_NL: float = 0.0     # local map coefficient (F_NL = 3/5 f_NL)
    G_NL: float = 0.0
    usr_floor: float = 1e-6
    seed: int = 1
    alpha_NL: float = 0.0  # non-local map coefficients of Eq. eq_nonlocal (dimensionless; the map divides by k*^2)
    beta_NL: float = 0.0

    def as_dict(self):
        return asdict(self)


def _on_mode(N, nstar, L=1.0):
    return nstar * TWO_PI / L


WORKLOADS = {
    "gauss32": Spec(N=32, L=1.0, A=1e-2, sigma=0.5, kstar=_on_mode(32, 8), kind="gauss", seed=1),
    "local128": Spec(N=128, L=1.0, A=1e-2, sigma=0.5, kstar=_on_mode(128, 16), kind="local", F_NL=0.6 * 5.0, seed=2),
    "usr256": Spec(N=256, L=1.0, A=5e-3, sigma=0.3, kstar=_on_mode(256, 32), kind="usr", seed=1),
    "broad512": Spec(N=512, L=1.0, A=1e-2, sigma=1.0, kstar=_on_mode(512, 64), kind="local", F_NL=0.6 * -2.0, seed=5),
}

USR256_SEEDS = (1, 2, 3, 4)


def workload(name, **over):
    return replace(WORKLOADS[name], **over)


def scaled(spec, N):
    """The same physical setup on another lattice size (n_* scaled with N, L fixed)."""
    nstar = spec.kstar * spec.L / TWO_PI
    return replace(spec, N=N, kstar=(nstar * N / spec.N) * TWO_PI / spec.L)


def serving_stream(n_requests, rate_hz, seed=7, sizes=(64, 128, 256)):
    """Poisson arrivals of spectrum requests: list of (arrival_time_s, Spec)."""
    rng = random.Random(seed)
    t = 0.0
    out = []
    for rid in range(n_requests):
        t += rng.expovariate(rate_hz)
        N = rng.choice(sizes)
        f_nl = rng.uniform(-5.0, 20.0)
        sig = rng.uniform(0.1, 1.0)
        kind = rng.choice(("gauss", "local", "usr"))
        spec = Spec(N=N, L=1.0, A=1e-2, sigma=sig, kstar=(N / 8) * TWO_PI, kind=kind,
                    F_NL=0.6 * f_nl if kind == "local" else 0.0, seed=1000 + rid)
        out.append((t, spec))
    return out
