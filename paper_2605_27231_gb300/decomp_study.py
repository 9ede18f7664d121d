"""Decomposition study: how the grid meta-parameters trade the number of separable terms against the
truncation error of the kernels (Sec. sec_decomposition; the choice is left open in Sec. sec_conclusions).

Every number comes from the library's host routine ``sigw_decomposition_error``; this module only sweeps
its arguments and picks the cheapest grid that meets a target.
"""
import itertools

from . import sigw


def sweep(m, n_modes=(100, 200), n_alpha=(20, 30, 40, 50, 60), upiv=(0.8, 1.0), Ap=(0.0, 10.0), **fixed):
    """Truncation errors of kernel m (0: I_s, 1: I_c) over the grid of parameters; list of dicts."""
    out = []
    for nm, na, up, ap in itertools.product(n_modes, n_alpha, upiv, Ap):
        if na > nm:
            continue
        o = sigw.default_opts(n_modes=nm, n_alpha=na, upiv=up, Ap=ap, **fixed)
        f, mx, g = sigw.decomposition_error(m, o)
        out.append({"m": m, "n_modes": nm, "n_alpha": na, "upiv": up, "Ap": ap, "frob": f, "maxrel": mx, "gap": g})
    return out


def optimal(target, m=(0, 1), **grid):
    """The fewest separable terms (the FFT count scales with them) whose truncation error, in the Frobenius
    norm of the weighted kernel matrix, is at most `target` for every kernel in m; ties go to the smaller grid.
    Returns the winning parameters with both kernels' errors, or None."""
    rows = {}
    for mm in m:
        for r in sweep(mm, **grid):
            key = (r["n_alpha"], r["n_modes"], r["upiv"], r["Ap"])
            rows.setdefault(key, {})[mm] = r["frob"]
    ok = sorted(k for k, v in rows.items() if len(v) == len(m) and max(v.values()) <= target)
    if not ok:
        return None
    na, nm, up, ap = ok[0]
    return {"n_alpha": na, "n_modes": nm, "upiv": up, "Ap": ap, "frob": rows[ok[0]]}
