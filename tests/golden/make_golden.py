"""Write the oracle's per-shell spectra of the full-size workloads to tests/golden/.

The GPU parity tests compare every shell bin of the CUDA path at full size with these files.  They are
written by this script alone, which calls only the CPU FP64 oracle (``oracle/``) and the parameter sets of
``workloads.py``: no value here comes from the CUDA path.

What is computed (the oracle's FFT-convolution route, Sec. sec_lattice and Sec. sec_envelope_obs):
  Omega_GW, P_A, P_B (summed over the two polarisations) and N_k for each target shell n_c of the
  realisation, with the paper's separable decomposition (N_modes = 200, N_alpha = 50, Sec. sec_decomposition).

Files (one line per shell: n_c N_k Omega P_A P_B, 17 significant digits):
  local128_seed2.txt    128^3, local f_NL = 5, every shell 1..64
  usr256_seed1.txt      256^3, USR map, every shell 1..128 (and the USR floor-hit count in the header)
  broad512_seed5.txt    512^3, local f_NL = -2, shells 8 and 32
and the paper's frequency scan (Sec. sec_numerical: 20 targets k/k* log-spaced in [0.2, 3], each in its own box
L = pi N / k_max, one realisation and the one shell holding k; Gaussian log-normal A = 1e-2, k* = 1, seed 1), one
line per target: k L n_c Omega:
  scan64_sigma0.1.txt, scan64_sigma1.0.txt, scan128_sigma0.5.txt

Usage (CPU only; the shells of one workload are spread over worker processes, each of which synthesises the
realisation once):
  python tests/golden/make_golden.py local128 --procs 4
  python tests/golden/make_golden.py usr256 --procs 4
  python tests/golden/make_golden.py broad512 --procs 1
  python tests/golden/make_golden.py scan128_sigma0.5 --procs 4    (and the two scan64 sets)

At 256^3 a worker needs about 3 GB and the whole spectrum takes hours; at 512^3 one worker needs about 35 GB.
"""
import argparse
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

SETS = {  # workload -> (seed, shells (None: every shell))
    "local128": (2, None),
    "usr256": (1, None),
    "broad512": (5, [8, 32]),
}

SCANS = {  # name -> (N, sigma)
    "scan64_sigma0.1": (64, 0.1),
    "scan64_sigma1.0": (64, 1.0),
    "scan128_sigma0.5": (128, 0.5),
}
SCAN_A, SCAN_KSTAR, SCAN_SEED = 1e-2, 1.0, 1

_state = {}


def _init(name, seed):
    import workloads
    from oracle import decomposition, synth
    spec = workloads.workload(name, seed=seed)
    Phi, hits = synth.phi_tilde(spec.N, spec.L, spec.A, spec.sigma, spec.kstar, spec.seed, spec.kind, spec.F_NL,
                                spec.G_NL, spec.usr_floor, spec.alpha_NL, spec.beta_NL)
    _state.update(spec=spec, Phi=Phi, hits=hits, dec=decomposition.build())


def _one(n_c):
    from oracle import sigw
    t0 = time.time()
    r = sigw.omega(_state["Phi"], _state["spec"].L, _state["dec"], shells=[n_c])
    return (n_c, int(r["Nk"][0]), float(r["omega"][0]), float(r["PA"][0]), float(r["PB"][0]), _state["hits"],
            time.time() - t0)


def _init_scan():
    from oracle import decomposition
    _state.update(dec=decomposition.build())


def _one_target(job):
    from oracle import targets
    N, sigma, k = job
    r = targets.target_scan(N, [k], SCAN_A, sigma, SCAN_KSTAR, _state["dec"], seed=SCAN_SEED)
    return k, float(r["L"][0]), int(r["n_c"][0]), float(r["omega"][0])


def scan(name, procs):
    import numpy as np
    N, sigma = SCANS[name]
    ks = np.geomspace(0.2, 3.0, 20) * SCAN_KSTAR
    ctx = mp.get_context("spawn")
    t0 = time.time()
    with ctx.Pool(procs, initializer=_init_scan) as pool:
        rows = sorted(pool.map(_one_target, [(N, sigma, float(k)) for k in ks]))
    out = os.path.join(HERE, name + ".txt")
    with open(out, "w") as f:
        f.write("# Oracle (CPU FP64) frequency scan of Sec. sec_numerical: N=%d, Gaussian log-normal A=%r sigma=%r "
                "kstar=%r, seed %d, eps=0.1, N_modes=200 N_alpha=50\n" % (N, SCAN_A, sigma, SCAN_KSTAR, SCAN_SEED))
        f.write("# written by tests/golden/make_golden.py (calls only oracle/)\n")
        f.write("# k L n_c Omega\n")
        for k, L, n_c, om in rows:
            f.write("%.17g %.17g %d %.17g\n" % (k, L, n_c, om))
    print("wrote", out, "in %.0f s" % (time.time() - t0))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("workload", choices=sorted(SETS) + sorted(SCANS))
    ap.add_argument("--procs", type=int, default=4)
    args = ap.parse_args()
    if args.workload in SCANS:
        return scan(args.workload, args.procs)
    seed, shells = SETS[args.workload]
    import workloads
    spec = workloads.workload(args.workload, seed=seed)
    if shells is None:
        shells = list(range(1, spec.N // 2 + 1))
    # the large shells cost the same as the small ones; interleave so that the workers finish together
    order = shells[::2] + shells[1::2]
    ctx = mp.get_context("spawn")
    rows = []
    t0 = time.time()
    with ctx.Pool(args.procs, initializer=_init, initargs=(args.workload, seed)) as pool:
        for row in pool.imap_unordered(_one, order):
            rows.append(row)
            print("shell %3d  Omega %.6e  (%.0f s, %d/%d done, %.0f s elapsed)" % (row[0], row[2], row[6], len(rows),
                                                                                    len(order), time.time() - t0),
                  flush=True)
    rows.sort()
    out = os.path.join(HERE, "%s_seed%d.txt" % (args.workload, seed))
    with open(out, "w") as f:
        f.write("# Oracle (CPU FP64, FFT-convolution route) per-shell spectrum of the %s workload, seed %d\n"
                % (args.workload, seed))
        f.write("# N=%d L=%r A=%r sigma=%r kstar=%r map=%s F_NL=%r G_NL=%r usr_floor=%r; N_modes=200 N_alpha=50\n"
                % (spec.N, spec.L, spec.A, spec.sigma, spec.kstar, spec.kind, spec.F_NL, spec.G_NL, spec.usr_floor))
        f.write("# usr_floor_hits=%d\n" % rows[0][5])
        f.write("# written by tests/golden/make_golden.py (calls only oracle/); Sec. sec_lattice, "
                "Sec. sec_envelope_obs\n")
        f.write("# n_c N_k Omega P_A P_B\n")
        for n_c, nk, om, pa, pb, _, _ in rows:
            f.write("%d %d %.17g %.17g %.17g\n" % (n_c, nk, om, pa, pb))
    print("wrote", out, "in %.0f s" % (time.time() - t0))


if __name__ == "__main__":
    main()
