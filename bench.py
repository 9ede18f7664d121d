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
          host copies inside the timed region (a bounded number of steps, stated).
Every rank processes its own seeds (no collective on the data path): "scaling": "weak".

Rank 0 also reports (extra keys of the same line):
  path_fraction : the step against the method's algorithmic bytes (312 field-FFTs per shell, each read + written once)
  fp64_path     : one full FP64 spectrum of the same workload, timed (the metric's second number)
  broad512      : one FP32 512^3 spectrum (per-kernel GB/s, clocks) and the FP64 path on sampled shells
  serving       : the continuous-batching server at 0.5 / 0.8 / 1.0 of its measured capacity on the mixed request
                  stream (FP32), and FP32 against the FP64 plain path on the small-lattice mix
  cpu_baseline, paper_workload_scan, fft_crosscheck_cufft

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
METRIC = "SIGW spectra/s at 256^3 (FP32 path; FP64 path on the same GPU under fp64_path; serving p50/p99 under serving)"

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one ncu capture per kernel kind at 256^3 FP32,
# with the algorithmic bytes of the captured launch (the committed ncu summaries of k_p1_tm, k_p2, k_p3_tm at 256^3).  These move bytes in
# proportion to the term-realisations of a launch, so the traffic of a bench launch is the algorithmic bytes of
# that launch times the captured ratio.  Valid only while the kernel source is unchanged since the capture.
NCU_TRAFFIC_256 = {
    "p1_inv_axis0_filter": (0.06798208e9 + 1.281252e9, 0.0676e9 + 20 * 67.108864e6),  # k_p1_tm (tile in TMEM)
    "p2_inv_axis1": (1.073817e9 + 1.553402e9, 40 * 67.108864e6),
    "p3_inv_axis2_product_fwd_axis2": (2.013404e9 + 0.011483904e9, 30 * 67.108864e6 + 6 * 65536 * 2 * 8),  # k_p3_tm
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
    if args.tuning:  # a fixed choice (terms per launch, variant bits) instead of the autotuner's
        tb, tv = (int(x) for x in args.tuning.split(","))
        plan.set_tuning(tb, tv)
        tuned = {"alpha_batch": tb, "variant_bits": tv, "fixed": True}
    else:
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

    # ---- end to end through the public API with host buffers (a bounded number of steps of the same work)
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    barrier()
    plan.profile(False)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        plan.generate_spec(spec, seeds=seeds)
        res = plan.spectrum()
    barrier()
    e2e_s = time.perf_counter() - t0
    io = plan.profile_read()
    t = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
    if ws > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    e2e_value = ws * batch * e2e_steps / float(t.item())
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

    # ---- FP64 path on the same GPU: one full spectrum (all shells) of the same workload, timed
    fp64 = None
    if rank == 0 and args.fp64_spectrum:
        fp64 = fp64_spectrum(spec, seeds[0], stream, value / ws)
    big = None
    if rank == 0 and args.broad512:
        big = broad512_leg(stream)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample(spec, args.cpu_terms)
    serving = None
    if rank == 0 and args.serve_requests > 0:
        serving = serving_study(args)
    scan = paper_scan() if rank == 0 and not args.no_paper_scan else None
    fftx = fft_crosscheck() if rank == 0 and not args.no_paper_scan else None

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "spectra/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == 32 else "f64",
            "data": "synthetic (Philox noise, log-normal P_zeta, USR map)",
            "config": dict(workload_config(args, spec),
                           l2="inputs larger than L2 (%.1f GB device working set per step)" % (sigw.footprint(
                               spec.N, sigw.default_opts(max_batch=batch)) / 1e9), autotuned=tuned),
            "e2e": {"value": e2e_value, "unit": "spectra/s", "h2d_bytes_per_step": io["h2d_bytes"] / e2e_steps,
                    "d2h_bytes_per_step": io["d2h_bytes"] / e2e_steps, "steps": e2e_steps},
            "gpu_launches": launches,
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peaks["hbm_gbs"],
                         "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                         "traffic_note": "bytes per launch, one ncu capture scaled by term-realisations" if traffic
                         else None, "algorithmic_bytes_per_launch": d["bytes"] / d["launches"],
                         "peak_source": pk_src + " (copy)"},
            "kernels": kernels,
            "clocks": clocks,
            "path_fraction": path_fraction(spec.N, value, peaks["hbm_gbs"]),
            "fp64_path": fp64,
            "broad512": big,
            "cpu_baseline": cpu,
            "serving": serving,
            "paper_workload_scan": scan,
            "fft_crosscheck_cufft": fftx,
            "omega_finite_positive": omega_ok,
        }
        print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()


def _pct(v, q):
    import numpy as np
    return float(np.percentile(v, q)) if len(v) else None


def serving_leg(args, precision, sizes, loads, n_requests):
    """Poisson replays of mixed spectrum requests through one continuous-batching server (sigw_submit).

    The server's plans are made resident first.  Capacity = requests/s the server sustains on the mix: for each
    size class a full batch (max_batch requests) is submitted at once and timed to completion, giving the
    per-request cost c_N; capacity = 1 / mean_N c_N (N uniform over `sizes`).  Each load then replays
    `n_requests` Poisson arrivals (seed 7) at load x capacity; latency = completion - submission."""
    from paper_2605_27231_gb300 import sigw
    srv = sigw.Server(args.serve_budget_gb * 1e9, max_slots=args.serve_slots, max_batch=args.serve_batch,
                      precision=precision)
    if args.serve_express > 0:
        srv.set_express(args.serve_express, args.serve_express_max_n)
    out = {"precision": precision, "sizes": list(sizes), "slots": args.serve_slots, "max_batch": args.serve_batch,
           "express_slots": args.serve_express, "express_max_n": args.serve_express_max_n,
           "budget_gb": args.serve_budget_gb, "loads": []}
    try:
        cost = {}
        for N in sizes:
            specs = [sp for _, sp in workloads.serving_stream(args.serve_batch, 1.0, seed=1, sizes=(N,))]
            for _ in range(2):  # plan made resident, graphs captured for the batch sizes the slots form
                for t in [srv.submit(sp) for sp in specs]:
                    srv.wait(t, timeout_s=3600)
            t0 = time.perf_counter()
            for t in [srv.submit(sp) for sp in specs]:
                srv.wait(t, timeout_s=3600)
            cost[N] = (time.perf_counter() - t0) / len(specs)
        capacity = 1.0 / (sum(cost.values()) / len(cost))
        out["per_request_cost_s"] = {str(N): c for N, c in cost.items()}
        out["capacity_req_per_s"] = capacity
        for load in loads:
            stats0 = srv.stats()
            rate = load * capacity
            stream = workloads.serving_stream(n_requests, rate, seed=7, sizes=sizes)
            t_start = time.perf_counter()
            tickets = []
            for t_arr, sp in stream:
                d = t_start + t_arr - time.perf_counter()
                if d > 0:
                    time.sleep(d)
                tickets.append((sp.N, srv.submit(sp)))
            lat = {N: [] for N in sizes}
            for N, t in tickets:
                _, l = srv.wait(t, timeout_s=3600)
                lat[N].append(l)
            t_end = time.perf_counter()
            st = srv.stats()
            allv = sorted(l for v in lat.values() for l in v)
            out["loads"].append({
                "load": load, "requests": len(allv), "arrival_rate_hz": rate, "spectra_per_s": len(allv) / (t_end - t_start),
                "p50_latency_s": _pct(allv, 50), "p99_latency_s": _pct(allv, 99),
                "per_size": {str(N): {"n": len(v), "p50_s": _pct(v, 50), "p99_s": _pct(v, 99)} for N, v in lat.items()},
                "batches": st["batches"] - stats0["batches"],
                "express_batches": st["express_batches"] - stats0["express_batches"],
                "hbm_peak_gb": st["hbm_peak"] / 1e9})
    finally:
        srv.close()
    return out


def serving_study(args):
    """FP32 serving of the full request mix (N in {64, 128, 256}) at 0.5, 0.8 and 1.0 of measured capacity, and
    FP32 against the FP64 plain path on the small-lattice mix (N in {64, 128}; an FP64 256^3 request takes ~47 s,
    so the full mix does not fit a benchmark run in FP64)."""
    sizes = tuple(int(x) for x in args.serve_sizes.split(","))
    loads = tuple(float(x) for x in args.serve_loads.split(","))
    res = {"mix": "N uniform over the sizes; f_NL ~ U[-5,20]; sigma ~ U[0.1,1]; A = 1e-2; map uniform over "
                  "{gauss, local, usr}; k* = N/8 k_f; seed = request id; Poisson arrivals, seed 7",
           "fp32": serving_leg(args, 32, sizes, loads, args.serve_requests)}
    if args.serve_fp64_requests > 0:
        small = tuple(int(x) for x in args.serve_fp64_sizes.split(","))
        res["fp32_small_mix"] = serving_leg(args, 32, small, (args.serve_fp64_load,), args.serve_requests)
        res["fp64_small_mix"] = serving_leg(args, 64, small, (args.serve_fp64_load,), args.serve_fp64_requests)
    main = [l for l in res["fp32"]["loads"] if abs(l["load"] - 0.8) < 1e-9] or res["fp32"]["loads"]
    res["p50_latency_s"], res["p99_latency_s"] = main[0]["p50_latency_s"], main[0]["p99_latency_s"]
    res["spectra_per_s"] = main[0]["spectra_per_s"]
    res["headline_load"] = main[0]["load"]
    return res


def fp64_spectrum(spec, seed, stream, fp32_per_gpu):
    """The FP64 plain path on the same GPU: one full spectrum (synthesis + all N/2 shells) of one realisation,
    timed with CUDA events on the plan's stream, with the clocks sampled meanwhile."""
    import torch
    from paper_2605_27231_gb300 import sigw
    dev_out = torch.empty(spec.N // 2 * 4, dtype=torch.float64, device="cuda")
    with sigw.Plan(spec.N, spec.L, stream=stream.cuda_stream, precision=64, max_batch=1) as p:
        p.generate_spec(spec, seeds=[seed])
        p.spectrum([1])  # warm
        torch.cuda.synchronize()
        clk = Clocks(torch.cuda.current_device())
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        p.generate_spec(spec, seeds=[seed])
        p.spectrum_async(dev_out.data_ptr())
        b.record(stream)
        b.synchronize()
        clocks = clk.stop()
        s = a.elapsed_time(b) / 1e3
    return {"value": 1.0 / s, "unit": "spectra/s", "dtype": "f64", "seconds_per_spectrum": s,
            "sample": "1 seed, all %d shells, timed (not extrapolated)" % (spec.N // 2),
            "fp32_over_fp64": fp32_per_gpu * s, "clocks": clocks}


def broad512_leg(stream):
    """The 512^3 broad-peak workload (local f_NL = -2, sigma = 1, k* = 64 k_f): one FP32 spectrum (all 256 shells,
    one realisation) timed by CUDA events with per-kernel GB/s; the FP64 path on four sampled shells (labelled as
    sampled: a full FP64 512^3 spectrum takes ~15 minutes)."""
    import numpy as np
    import torch
    from paper_2605_27231_gb300 import sigw
    spec = workloads.workload("broad512")
    n_sh = spec.N // 2
    dev_out = torch.empty(n_sh * 4, dtype=torch.float64, device="cuda")
    peaks, _ = _peaks()
    out = {"workload": "broad512", "N": spec.N, "map": spec.kind, "F_NL": spec.F_NL, "sigma": spec.sigma}
    with sigw.Plan(spec.N, spec.L, stream=stream.cuda_stream, precision=32, max_batch=1) as p:
        p.generate_spec(spec)
        p.spectrum([1])  # warm
        torch.cuda.synchronize()
        clk = Clocks(torch.cuda.current_device())
        p.profile(True)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        p.generate_spec(spec)
        p.spectrum_async(dev_out.data_ptr())
        b.record(stream)
        b.synchronize()
        prof = p.profile_read()
        p.profile(False)
        out["clocks"] = clk.stop()
        s32 = a.elapsed_time(b) / 1e3
        om = dev_out.view(n_sh, 4)[:, 3].cpu().numpy()
    out["fp32"] = {"value": 1.0 / s32, "unit": "spectra/s", "seconds_per_spectrum": s32,
                   "omega_finite_positive": bool(np.all(np.isfinite(om)) and np.all(om > 0)),
                   "kernels": {k: {"ms": prof[k]["ms"], "launches": prof[k]["launches"],
                                   "GBps": prof[k]["bytes"] / (prof[k]["ms"] / 1e3) / 1e9 if prof[k]["ms"] > 0 else None,
                                   "frac_of_peak": (prof[k]["bytes"] / (prof[k]["ms"] / 1e3) / 1e9 / peaks["hbm_gbs"])
                                   if prof[k]["ms"] > 0 else None}
                               for k in sigw.KINDS if prof[k]["launches"]},
                   "path_fraction": path_fraction(spec.N, 1.0 / s32, peaks["hbm_gbs"])}
    shells = np.array([1, 86, 171, 256], dtype=np.int32)
    with sigw.Plan(spec.N, spec.L, stream=stream.cuda_stream, precision=64, max_batch=1) as p:
        a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        a.record(stream)
        p.generate_spec(spec)
        b.record(stream)
        p.spectrum_async(dev_out.data_ptr(), shells)
        c.record(stream)
        c.synchronize()
        gen, sh = a.elapsed_time(b) / 1e3, b.elapsed_time(c) / 1e3
    s64 = gen + sh * n_sh / len(shells)
    out["fp64"] = {"value": 1.0 / s64, "unit": "spectra/s", "seconds_per_spectrum": s64,
                   "sample": "synthesis + shells %s timed, extrapolated to all %d shells (sampled)" % (
                       shells.tolist(), n_sh)}
    out["fp32_over_fp64"] = s64 / s32
    return out


def path_fraction(N, spectra_per_s, peak_gbs):
    """The whole path against the algorithmic byte count of the method: 312 field-FFTs per target shell
    (2 kernels x (3 x 50 inverse + 6 forward)), N/2 shells per spectrum, each field-FFT reading and writing one
    FP32 field once (4 N^3 real + 8 N^2 (N/2 + 1) half-complex bytes)."""
    per_fft = 4.0 * N ** 3 + 8.0 * N * N * (N // 2 + 1)
    per_spec = 312.0 * (N // 2) * per_fft
    achieved = per_spec * spectra_per_s / 1e9
    return {"bytes_per_spectrum": per_spec, "achieved_GBps": achieved, "peak_GBps": peak_gbs,
            "frac": achieved / peak_gbs}


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
    line = {"impl": "reference", "metric": METRIC,
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
    ap.add_argument("--fp64-spectrum", type=int, default=1, help="time one full FP64 spectrum (0: skip)")
    ap.add_argument("--broad512", type=int, default=1, help="run the 512^3 leg (0: skip)")
    ap.add_argument("--e2e-steps", type=int, default=5, help="steps of the end-to-end measurement (at most --steps)")
    ap.add_argument("--cpu-terms", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-paper-scan", action="store_true")
    ap.add_argument("--tuning", default="", help="B,V: terms per launch and variant bits instead of the autotuner")
    ap.add_argument("--alpha-batch", type=int, default=0,
                    help="separable terms per strided-pass launch (0: chosen by the autotuner)")
    ap.add_argument("--precision", type=int, default=32, choices=[32, 64],
                    help="working precision of the main leg (64 only for profiling the FP64 path)")
    ap.add_argument("--serve-requests", type=int, default=200, help="requests per load (0: no serving legs)")
    ap.add_argument("--serve-loads", default="0.5,0.8,1.0", help="loads as fractions of the measured capacity")
    ap.add_argument("--serve-sizes", default="64,128,256")
    ap.add_argument("--serve-fp64-requests", type=int, default=60, help="FP64 serving requests (0: no FP64 leg)")
    ap.add_argument("--serve-fp64-sizes", default="64,128")
    ap.add_argument("--serve-fp64-load", type=float, default=0.8)
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
