"""Benchmark: SIGW spectra/s at 256^3 (FP32 path, FP64 path on the same GPU), one JSON line.

A step is one pass of the whole hot path over one batch of realisations of the
256^3 USR-tail workload (log-normal A = 5e-3, sigma = 0.3, k* = 32 k_f; 4 seeds per
step): Philox synthesis, the USR map, and all 128 target shells of the
FFT-convolution envelopes, TT projection and binning.  One spectrum = Omega_GW in all
N/2 shells for one seed.

  value : spectra/s with the work queued through sigw_generate + sigw_spectrum_async
          (parameters in, results left in HBM); device time from CUDA events on the
          library's stream, max over ranks.
  e2e   : the same through sigw_generate + sigw_spectrum (host seeds in, host Omega out),
          host copies inside the timed region.
Every rank processes its own seeds (no collective on the data path): "scaling": "weak".

--impl reference times the CPU FP64 oracle on a bounded sample of the same workload
(one target shell, a few separable terms) and extrapolates to spectra/s.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

PEAKS_FALLBACK = {"hbm_gbs": 6800.0}

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one ncu capture per kernel kind at 256^3 FP32,
# with the algorithmic bytes of the captured launch (the committed ncu summaries of k_p1, k_p2, k_p3 at 256^3).  These kernels move bytes in
# proportion to the term-realisations of a launch, so the traffic of a bench launch is the algorithmic bytes of
# that launch times the captured ratio.  Valid only while the kernel source is unchanged since the capture.
NCU_TRAFFIC_256 = {
    "p1_inv_axis0_filter": (0.068546e9 + 1.281282e9, 0.0676e9 + 20 * 67.108864e6),
    "p2_inv_axis1": (1.073817e9 + 1.553402e9, 40 * 67.108864e6),
    "p3_inv_axis2_product_fwd_axis2": (2.013373e9 + 0.026424e9, 30 * 67.108864e6 + 6 * 65536 * 2 * 8),
}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return PEAKS_FALLBACK, "fallback"


def _nvtx(torch, name):
    try:
        if name:
            torch.cuda.nvtx.range_push(name)
        else:
            torch.cuda.nvtx.range_pop()
    except Exception:
        pass


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    def __init__(self, index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), "--query-gpu=" + q, "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [l.strip().split(",") for l in self.f.read().splitlines() if l.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for n, v in zip(names, r[5:9]):
                    if "Active" in v and "Not" not in v:
                        reasons.add(n)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2605_27231_gb300 import sigw

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    spec = workloads.workload(args.workload)
    batch = args.batch
    from paper_2605_27231_gb300 import shard
    base = list(workloads.USR256_SEEDS) if args.workload == "usr256" else [spec.seed + i for i in range(batch)]
    seeds = shard.seeds_for_rank((base * batch)[:batch], rank, ws)
    stream = torch.cuda.Stream()
    plan = sigw.Plan(spec.N, spec.L, stream=stream.cuda_stream, precision=args.precision, max_batch=batch,
                     n_alpha=args.n_alpha, alpha_batch=args.alpha_batch)
    n_sh = spec.N // 2
    dev_out = torch.empty(batch * n_sh * 4, dtype=torch.float64, device="cuda")

    def step():
        plan.generate_spec(spec, seeds=seeds)
        plan.spectrum_async(dev_out.data_ptr())

    plan.generate_spec(spec, seeds=seeds)
    tuned = dict(zip(("alpha_batch", "variant_bits", "tune_ms"), plan.autotune()))

    for _ in range(args.warmup):
        step()
    plan.synchronize()

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- device-resident timed region (events on the library's stream) + per-kernel events
    clk = Clocks(local)
    barrier()
    plan.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    _nvtx(torch, "sigw_timed")  # lets a profiler select exactly the timed launches
    for _ in range(args.steps):
        step()
    _nvtx(torch, None)
    e1.record(stream)
    barrier()
    prof = plan.profile_read()
    plan.profile(False)
    clocks = clk.stop()
    ms = e0.elapsed_time(e1)
    t = torch.tensor([ms], dtype=torch.float64, device="cuda")
    if ws > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    value = ws * batch * args.steps / (ms_max / 1e3)

    # ---- end to end through the public API with host buffers
    barrier()
    plan.profile(False)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        plan.generate_spec(spec, seeds=seeds)
        res = plan.spectrum()
    barrier()
    e2e_s = time.perf_counter() - t0
    io = plan.profile_read()
    t = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
    if ws > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    e2e_value = ws * batch * args.steps / float(t.item())
    omega_ok = bool(np.all(np.isfinite(res["omega"])) and np.all(res["omega"] > 0))

    # ---- dominant kernel roofline
    peaks, pk_src = _peaks()
    kinds = [k for k in sigw.KINDS if prof[k]["launches"]]
    dom = max(kinds, key=lambda k: prof[k]["ms"])
    d = prof[dom]
    achieved = d["bytes"] / (d["ms"] / 1e3) / 1e9
    traffic = None
    if dom in NCU_TRAFFIC_256 and spec.N == 256 and args.n_alpha == 50:
        dram, alg = NCU_TRAFFIC_256[dom]
        traffic = d["bytes"] / d["launches"] * dram / alg
    kernels = {k: {"ms_per_step": prof[k]["ms"] / args.steps, "launches_per_step": prof[k]["launches"] / args.steps,
                   "GBps": (prof[k]["bytes"] / (prof[k]["ms"] / 1e3) / 1e9) if prof[k]["ms"] > 0 else None}
               for k in kinds}
    launches = sum(prof[k]["launches"] for k in sigw.KINDS)
    plan.close()

    # ---- FP64 path on the same GPU (sampled shells, extrapolated to a spectrum)
    fp64 = None
    if rank == 0 and args.fp64_shells > 0:
        with sigw.Plan(spec.N, spec.L, stream=stream.cuda_stream, precision=64, max_batch=1) as p64:
            shells = np.unique(np.linspace(1, n_sh, args.fp64_shells).astype(np.int32))
            p64.generate_spec(spec, seeds=seeds[:1])
            p64.spectrum(shells[:1])
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            p64.generate_spec(spec, seeds=seeds[:1])
            b.record(stream)
            b.synchronize()
            gen_ms = a.elapsed_time(b)
            a.record(stream)
            p64.spectrum_async(dev_out.data_ptr(), shells)
            b.record(stream)
            b.synchronize()
            sh_ms = a.elapsed_time(b)
        per_spec_s = (gen_ms + sh_ms * n_sh / len(shells)) / 1e3
        fp64 = {"value": 1.0 / per_spec_s, "unit": "spectra/s", "dtype": "f64",
                "sample": "1 seed, shells %s of 1..%d, extrapolated to all shells" % (shells.tolist(), n_sh),
                "fp32_over_fp64": (value / ws) / (1.0 / per_spec_s)}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample(spec, args.cpu_terms)
    serving = None
    if rank == 0 and args.serve_requests > 0:
        serving = serving_run(args)
    scan = paper_scan() if rank == 0 and not args.no_paper_scan else None
    fftx = fft_crosscheck() if rank == 0 and not args.no_paper_scan else None

    if rank == 0:
        line = {
            "metric": "SIGW spectra/s at 256^3 (FP32 path; FP64 path on the same GPU under fp64_path)",
            "value": value, "unit": "spectra/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == 32 else "f64",
            "data": "synthetic (Philox noise, log-normal P_zeta, USR map)",
            "config": dict(workload_config(args, spec),
                           l2="inputs larger than L2 (%.1f GB device working set per step)" % (sigw.footprint(
                               spec.N, sigw.default_opts(max_batch=batch)) / 1e9), autotuned=tuned),
            "e2e": {"value": e2e_value, "unit": "spectra/s", "h2d_bytes_per_step": io["h2d_bytes"] / args.steps,
                    "d2h_bytes_per_step": io["d2h_bytes"] / args.steps},
            "gpu_launches": launches,
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peaks["hbm_gbs"],
                         "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                         "traffic_note": "bytes per launch, one ncu capture scaled by term-realisations" if traffic
                         else None, "algorithmic_bytes_per_launch": d["bytes"] / d["launches"],
                         "peak_source": pk_src + " (copy)"},
            "kernels": kernels,
            "clocks": clocks,
            "fp64_path": fp64,
            "cpu_baseline": cpu,
            "serving": serving,
            "paper_workload_scan": scan,
            "fft_crosscheck_cufft": fftx,
            "omega_finite_positive": omega_ok,
        }
        print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()


def serving_run(args):
    """Poisson replay of mixed spectrum requests through the continuous-batching server (sigw_submit).

    Service times of one request per size class (alone, plans resident) give the single-slot capacity;
    requests then arrive at args.serve_load times that rate.  Latency = completion - submission."""
    import numpy as np
    from paper_2605_27231_gb300 import sigw
    sizes = (64, 128, 256)
    srv = sigw.Server(args.serve_budget_gb * 1e9, max_slots=args.serve_slots, max_batch=args.serve_batch,
                      precision=32)
    if args.serve_express > 0:
        srv.set_express(args.serve_express, args.serve_express_max_n)
    try:
        service = {}
        for N in sizes:  # warm plans, then time one request alone
            spec = workloads.serving_stream(1, 1.0, seed=1, sizes=(N,))[0][1]
            srv.wait(srv.submit(spec))
            t0 = time.perf_counter()
            srv.wait(srv.submit(spec))
            service[N] = time.perf_counter() - t0
        mean_service = sum(service.values()) / len(service)
        rate = args.serve_load / mean_service
        stream = workloads.serving_stream(args.serve_requests, rate, seed=7, sizes=sizes)
        t_start = time.perf_counter()
        tickets = []
        for t_arr, spec in stream:
            d = t_start + t_arr - time.perf_counter()
            if d > 0:
                time.sleep(d)
            tickets.append((spec.N, srv.submit(spec)))
        lat = {N: [] for N in sizes}
        for N, t in tickets:
            om, l = srv.wait(t, timeout_s=1200)
            lat[N].append(l)
        t_end = time.perf_counter()
        st = srv.stats()
    finally:
        srv.close()
    allv = sorted(l for v in lat.values() for l in v)
    pct = lambda v, q: float(np.percentile(v, q)) if v else None
    return {"requests": len(allv), "arrival_rate_hz": rate, "load": args.serve_load,
            "single_request_service_s": service, "spectra_per_s": len(allv) / (t_end - t_start),
            "p50_latency_s": pct(allv, 50), "p99_latency_s": pct(allv, 99),
            "per_size": {str(N): {"n": len(v), "p50_s": pct(v, 50), "p99_s": pct(v, 99)} for N, v in lat.items()},
            "slots": args.serve_slots, "max_batch": args.serve_batch, "batches": st["batches"],
            "express_slots": args.serve_express, "express_max_n": args.serve_express_max_n,
            "express_batches": st["express_batches"],
            "hbm_peak_gb": st["hbm_peak"] / 1e9, "budget_gb": args.serve_budget_gb,
            "mix": "N uniform over {64,128,256}; f_NL ~ U[-5,20]; sigma ~ U[0.1,1]; map uniform over "
                   "{gauss, local, usr}; Poisson arrivals, seed 7; FP32"}


def fft_crosscheck(N=256, reps=10):
    """The library's 3-D real FFT (sigw_fft3d: rows R2C + two strided passes + unpack) timed beside cuFFT
    (torch.fft.rfftn, a library call) on the same N^3 input, FP32 and FP64, with the largest difference."""
    import torch
    from paper_2605_27231_gb300 import sigw
    out = {}
    for prec, rdt, cdt in ((32, torch.float32, torch.complex64), (64, torch.float64, torch.complex128)):
        st = torch.cuda.Stream()
        with sigw.Plan(N, 1.0, precision=prec, n_alpha=2, stream=st.cuda_stream) as p, torch.cuda.stream(st):
            g = torch.Generator(device="cuda").manual_seed(5)
            x = torch.randn((N, N, N), dtype=rdt, device="cuda", generator=g)
            X = torch.empty((N, N, N // 2 + 1), dtype=cdt, device="cuda")
            res = {}
            for name, fn in (("ours", lambda: p.fft3d(-1, x.data_ptr(), X.data_ptr())),
                             ("cufft", lambda: torch.fft.rfftn(x))):
                for _ in range(3):
                    fn()
                st.synchronize()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(st)
                for _ in range(reps):
                    fn()
                b.record(st)
                b.synchronize()
                res[name] = a.elapsed_time(b) / reps
            p.fft3d(-1, x.data_ptr(), X.data_ptr())
            ref = torch.fft.rfftn(x)
            st.synchronize()
            diff = float((X - ref).abs().max() / ref.abs().max())
        out["fp%d" % prec] = {"ours_ms": res["ours"], "cufft_ms": res["cufft"], "max_abs_diff_over_max": diff}
    out["transform"] = "%d^3 real -> half complex, one realisation" % N
    return out


def paper_scan(steps=3):
    """The paper's own workload (Sec. sec_numerical): 20 target frequencies k/k* in [0.2, 3], each in its own
    box L = pi N / k_max (sigw_target_scan), Gaussian log-normal A = 1e-2, sigma = 0.5, FP32, N = 64 and 128.
    Host wall-clock per 20-frequency scan (each target synthesises its own field and evaluates its shell)."""
    import numpy as np
    from paper_2605_27231_gb300 import sigw
    ks = np.geomspace(0.2, 3.0, 20)
    out = {}
    for N in (64, 128):
        with sigw.Plan(N, 1.0, precision=32) as p:
            p.target_scan(ks, 1e-2, 0.5, 1.0, seed=1)  # warm-up
            t0 = time.perf_counter()
            for s in range(steps):
                p.target_scan(ks, 1e-2, 0.5, 1.0, seed=2 + s)
            out["N%d_s_per_scan" % N] = (time.perf_counter() - t0) / steps
    out["paper"] = "1-2 s for 20 frequencies at N = 64, ~10 s at N = 128, NVIDIA Tesla T4 (PyTorch torch.fft)"
    return out


def oracle_sample(spec, n_terms):
    """The CPU FP64 oracle, as it stands, on a bounded sample of the workload: synthesis of one realisation
    and one target shell (n_c = N/8) of one kernel with n_terms and 2 n_terms separable terms; the per-term
    and fixed costs are extrapolated to all shells, both kernels and 50 terms."""
    import numpy as np
    from oracle import decomposition, sigw as osigw, synth
    dec = decomposition.build()
    t0 = time.perf_counter()
    Phi, _ = synth.phi_tilde(spec.N, spec.L, spec.A, spec.sigma, spec.kstar, spec.seed, spec.kind, spec.F_NL,
                             spec.G_NL, spec.usr_floor)
    t_syn = time.perf_counter() - t0
    n_c = spec.N // 8
    ts = []
    for nt in (n_terms, 2 * n_terms):
        t0 = time.perf_counter()
        osigw.envelope_fields(Phi, spec.L, dec.edges, dec.sigma["s"][:nt], dec.phi["s"][:nt], n_c)
        ts.append(time.perf_counter() - t0)
    per_term = (ts[1] - ts[0]) / n_terms
    fixed = max(ts[0] - n_terms * per_term, 0.0)
    per_spec = t_syn + (spec.N // 2) * 2 * (fixed + 50 * per_term)
    return {"value": 1.0 / per_spec, "unit": "spectra/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": "N=%d: synthesis + shell n_c=%d, kernel I_s, %d and %d terms (%.1f s of CPU); "
                      "extrapolated to %d shells x 2 kernels x 50 terms" % (spec.N, n_c, n_terms, 2 * n_terms,
                                                                            t_syn + sum(ts), spec.N // 2),
            "seconds_per_spectrum": per_spec}


def workload_config(args, spec):
    """The workload keys of the JSON line, shared by both arms."""
    return {"workload": args.workload, "N": spec.N, "L": spec.L, "A": spec.A, "sigma": spec.sigma,
            "kstar_over_kf": round(spec.kstar * spec.L / (2 * 3.141592653589793), 6), "map": spec.kind,
            "seeds_per_step": args.batch, "shells": spec.N // 2, "n_alpha": args.n_alpha, "n_modes": 200,
            "parallelism": "replicas, seeds sharded across ranks"}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    spec = workloads.workload(args.workload)
    vals = []
    t_start = time.perf_counter()
    for i in range(args.warmup + args.steps):
        r = oracle_sample(spec, args.cpu_terms)
        if i >= args.warmup:
            vals.append(r)
    v = statistics.mean(x["value"] for x in vals)
    wall = time.perf_counter() - t_start
    line = {"impl": "reference", "metric": "SIGW spectra/s at 256^3 (FP32 path; FP64 path on the same GPU under fp64_path)",
            "value": v, "unit": "spectra/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * wall / (args.warmup + args.steps), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (Philox noise, log-normal P_zeta, USR map)",
            "config": workload_config(args, spec),
            "cpu_baseline": {"value": v, "unit": "spectra/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": vals[-1]["sample"]},
            "e2e": {"value": v, "unit": "spectra/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="usr256")
    ap.add_argument("--batch", type=int, default=4)
    ap.add_argument("--n-alpha", type=int, default=50, help="separable terms kept (the paper's 50; fewer only to "
                    "shrink a profiling run)")
    ap.add_argument("--fp64-shells", type=int, default=4)
    ap.add_argument("--cpu-terms", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-paper-scan", action="store_true")
    ap.add_argument("--alpha-batch", type=int, default=0,
                    help="separable terms per strided-pass launch (0: chosen by the autotuner)")
    ap.add_argument("--precision", type=int, default=32, choices=[32, 64],
                    help="working precision of the main leg (64 only for profiling the FP64 path)")
    ap.add_argument("--serve-requests", type=int, default=24)
    ap.add_argument("--serve-load", type=float, default=0.8)
    ap.add_argument("--serve-slots", type=int, default=3)
    ap.add_argument("--serve-batch", type=int, default=4)
    ap.add_argument("--serve-express", type=int, default=1, help="express slots for small lattices (0: none)")
    ap.add_argument("--serve-express-max-n", type=int, default=128)
    ap.add_argument("--serve-budget-gb", type=float, default=200.0)
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
