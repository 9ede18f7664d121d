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

Usage (CPU only; the shells of one workload are spread over worker processes, each of which synthesises the
realisation once):
  python tests/golden/make_golden.py local128 --procs 4
  python tests/golden/make_golden.py usr256 --procs 4
  python tests/golden/make_golden.py broad512 --procs 1

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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("workload", choices=sorted(SETS))
    ap.add_argument("--procs", type=int, default=4)
    args = ap.parse_args()
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
