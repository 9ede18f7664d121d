"""ctypes binding of libsigw.so (argument marshalling only; every step runs in the library).

Names follow the C ABI in include/sigw.h.  The binding raises ``SigwError`` for
every non-OK status and ``RuntimeError`` when the compiled library is missing:
there is no fallback implementation.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsigw.so")

OK, EINVAL, ENOMEM, ECUDA, EDOMAIN, ETIMEOUT, EBUSY, ENOTREADY, ESTATE = range(9)
MAP_GAUSS, MAP_LOCAL, MAP_USR, MAP_NONLOCAL = 0, 1, 2, 3
MAP_KINDS = {"gauss": MAP_GAUSS, "local": MAP_LOCAL, "usr": MAP_USR, "nonlocal": MAP_NONLOCAL}


class SigwError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("sigw status %d (%s): %s" % (status, _strerror(status), msg))
        self.status = status


class Opts(C.Structure):
    _fields_ = [("n_modes", C.c_int), ("n_alpha", C.c_int), ("umin", C.c_double), ("umax", C.c_double),
                ("upiv", C.c_double), ("sigp", C.c_double), ("Ap", C.c_double), ("precision", C.c_int),
                ("alpha_batch", C.c_int), ("max_batch", C.c_int), ("strict_domain", C.c_int)]


class PZeta(C.Structure):
    _fields_ = [("A", C.c_double), ("sigma", C.c_double), ("kstar", C.c_double)]


class NGMap(C.Structure):
    _fields_ = [("kind", C.c_int), ("F_NL", C.c_double), ("G_NL", C.c_double), ("usr_floor", C.c_double),
                ("alpha_NL", C.c_double), ("beta_NL", C.c_double)]


def _ngmap(kind, F_NL=0.0, G_NL=0.0, usr_floor=1e-6, alpha_NL=0.0, beta_NL=0.0):
    return NGMap(MAP_KINDS[kind] if isinstance(kind, str) else kind, F_NL, G_NL, usr_floor, alpha_NL, beta_NL)


def _spec_map(s):
    return _ngmap(s.kind, s.F_NL, s.G_NL, s.usr_floor, getattr(s, "alpha_NL", 0.0), getattr(s, "beta_NL", 0.0))


NKINDS = 7
KINDS = ("synth", "p1_inv_axis0_filter", "p2_inv_axis1", "p3_inv_axis2_product_fwd_axis2", "f2_fwd_axis1",
         "f3_fwd_axis0_tt_bin", "bin_finalise")


class Profile(C.Structure):
    _fields_ = [("ms", C.c_double * NKINDS), ("bytes", C.c_double * NKINDS), ("launches", C.c_int64 * NKINDS),
                ("h2d_bytes", C.c_double), ("d2h_bytes", C.c_double)]


class ServerStats(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in ("submitted", "completed", "failed", "queued", "batches", "plans_created",
                                          "plans_evicted", "plans_resident")] + \
               [(n, C.c_size_t) for n in ("hbm_in_use", "hbm_peak", "hbm_budget")] + [("express_batches", C.c_uint64)]


_lib = None
_dbl = C.POINTER(C.c_double)
_i64 = C.POINTER(C.c_int64)


def lib():
    """Load libsigw.so (built by paper_2605_27231_gb300.build.build()); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libsigw.so is not built (%s); call __graft_entry__.build() first" % LIB_PATH)
    L = C.CDLL(LIB_PATH)
    P = C.c_void_p
    sig = {
        "sigw_opts_default": (C.c_int, [C.POINTER(Opts)]),
        "sigw_plan_footprint": (C.c_int, [C.c_int, C.POINTER(Opts), C.POINTER(C.c_size_t)]),
        "sigw_plan_create": (C.c_int, [C.c_int, C.c_double, C.POINTER(Opts), P, C.POINTER(P)]),
        "sigw_plan_destroy": (C.c_int, [P]),
        "sigw_plan_last_error": (C.c_char_p, [P]),
        "sigw_plan_kernel_terms": (C.c_int, [P, C.c_int, _dbl, _dbl, _dbl]),
        "sigw_generate": (C.c_int, [P, C.POINTER(PZeta), C.POINTER(NGMap), C.POINTER(C.c_uint64), C.c_int, _i64]),
        "sigw_spectrum": (C.c_int, [P, C.POINTER(C.c_int), C.c_int, _dbl, _dbl, _dbl, _i64]),
        "sigw_spectrum_async": (C.c_int, [P, C.POINTER(C.c_int), C.c_int, P]),
        "sigw_copy_phi": (C.c_int, [P, C.c_int, P]),
        "sigw_fft3d": (C.c_int, [P, C.c_int, P, P]),
        "sigw_synchronize": (C.c_int, [P]),
        "sigw_strerror": (C.c_char_p, [C.c_int]),
        "sigw_decompose": (C.c_int, [C.POINTER(Opts), C.c_int, _dbl, _dbl, _dbl, _dbl]),
        "sigw_cell_table": (C.c_int, [C.POINTER(Opts), C.c_int, C.c_int, C.POINTER(C.c_int16)]),
        "sigw_debug_fail_alloc": (C.c_int, [C.c_int]),
        "sigw_plan_debug_wait_limit": (C.c_int, [P, C.c_longlong]),
        "sigw_plan_profile": (C.c_int, [P, C.c_int]),
        "sigw_plan_autotune": (C.c_int, [P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), _dbl]),
        "sigw_fft3d_noalloc": (C.c_int, [C.c_int, C.c_int, C.c_int, P, P, P]),
        "sigw_generate_batch": (C.c_int, [P, C.POINTER(PZeta), C.POINTER(NGMap), C.POINTER(C.c_uint64), C.c_int, _i64]),
        "sigw_server_create": (C.c_int, [C.c_size_t, C.c_int, C.POINTER(Opts), C.POINTER(P)]),
        "sigw_server_set_express": (C.c_int, [P, C.c_int, C.c_int]),
        "sigw_submit": (C.c_int, [P, C.c_int, C.c_double, C.POINTER(PZeta), C.POINTER(NGMap), C.c_uint64,
                                  C.POINTER(C.c_uint64)]),
        "sigw_poll": (C.c_int, [P, C.c_uint64, _dbl, _dbl]),
        "sigw_wait": (C.c_int, [P, C.c_uint64, C.c_double, _dbl, _dbl]),
        "sigw_server_stats_read": (C.c_int, [P, C.POINTER(ServerStats)]),
        "sigw_server_destroy": (C.c_int, [P]),
        "sigw_plan_profile_read": (C.c_int, [P, C.POINTER(Profile)]),
        "sigw_target_box": (C.c_int, [C.c_int, C.c_double, C.POINTER(PZeta), C.c_double, _dbl, C.POINTER(C.c_int)]),
        "sigw_plan_set_box": (C.c_int, [P, C.c_double]),
        "sigw_plan_set_tuning": (C.c_int, [P, C.c_int, C.c_int]),
        "sigw_decomposition_error": (C.c_int, [C.POINTER(Opts), C.c_int, _dbl, _dbl, _dbl]),
        "sigw_spectrum_jackknife": (C.c_int, [P, C.POINTER(C.c_int), C.c_int, C.c_int, _dbl, _dbl, _dbl, _dbl, _dbl,
                                              _dbl]),
        "sigw_target_scan": (C.c_int, [P, C.POINTER(PZeta), C.POINTER(NGMap), C.c_uint64, _dbl, C.c_int, C.c_double,
                                       _dbl, _dbl, C.POINTER(C.c_int)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _strerror(s):
    try:
        return lib().sigw_strerror(s).decode()
    except Exception:
        return "?"


def _check(status, plan=None, what=""):
    if status != OK:
        msg = what
        if plan is not None:
            msg += ": " + lib().sigw_plan_last_error(plan).decode()
        raise SigwError(status, msg)


def default_opts(**over):
    o = Opts()
    _check(lib().sigw_opts_default(C.byref(o)))
    for k, v in over.items():
        setattr(o, k, v)
    return o


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def decompose(m, opts=None, all_sigma=False):
    """Host-only decomposition: (sigma[n_alpha], phi[n_alpha, n_modes], edges[n_modes+1], sigma_all or None)."""
    o = opts or default_opts()
    sigma = np.zeros(o.n_alpha)
    phi = np.zeros((o.n_alpha, o.n_modes))
    edges = np.zeros(o.n_modes + 1)
    sall = np.zeros(o.n_modes) if all_sigma else None
    _check(lib().sigw_decompose(C.byref(o), m, _ptr(sigma, C.c_double), _ptr(phi, C.c_double),
                                _ptr(edges, C.c_double), _ptr(sall, C.c_double) if all_sigma else None))
    return sigma, phi, edges, sall


def decomposition_error(m, opts=None, **over):
    """sigw_decomposition_error (host only): (frob, maxrel, gap) of the rank-n_alpha truncation of kernel m."""
    o = opts or default_opts(**over)
    f, mx, g = C.c_double(), C.c_double(), C.c_double()
    _check(lib().sigw_decomposition_error(C.byref(o), m, C.byref(f), C.byref(mx), C.byref(g)), None,
           "sigw_decomposition_error")
    return f.value, mx.value, g.value


def cell_table(n_c, msq_max, opts=None):
    o = opts or default_opts()
    lut = np.zeros(msq_max + 1, dtype=np.int16)
    _check(lib().sigw_cell_table(C.byref(o), n_c, msq_max, _ptr(lut, C.c_int16)))
    return lut


def footprint(N, opts=None):
    o = opts or default_opts()
    n = C.c_size_t(0)
    _check(lib().sigw_plan_footprint(N, C.byref(o), C.byref(n)))
    return n.value


def fft3d_noalloc(N, precision, direction, in_ptr, out_ptr, stream=None):
    """sigw_fft3d_noalloc: the 3-D real FFT with no plan and no device allocation (N <= 128 FP32, <= 64 FP64)."""
    _check(lib().sigw_fft3d_noalloc(N, precision, direction, C.c_void_p(in_ptr), C.c_void_p(out_ptr),
                                    C.c_void_p(stream) if stream else None), None, "sigw_fft3d_noalloc")


def target_box(N, k, A, sigma, kstar, eps=0.1):
    """sigw_target_box: the paper's per-target box; returns (L, n_c)."""
    L, nc = C.c_double(), C.c_int()
    pz = PZeta(A, sigma, kstar)
    _check(lib().sigw_target_box(N, k, C.byref(pz), eps, C.byref(L), C.byref(nc)), None, "sigw_target_box")
    return L.value, nc.value


def debug_fail_alloc(n):
    _check(lib().sigw_debug_fail_alloc(n))


class Plan:
    """A lattice (N, L) with its decomposition, tables and device buffers (sigw_plan_create)."""

    def __init__(self, N, L, opts=None, stream=None, **over):
        self.opts = opts or default_opts(**over)
        self.N, self.L = N, L
        h = C.c_void_p()
        st = C.c_void_p(stream) if stream else None
        _check(lib().sigw_plan_create(N, L, C.byref(self.opts), st, C.byref(h)), None, "sigw_plan_create")
        self._h = h
        self.batch = 0

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            lib().sigw_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def dtype(self):
        return np.complex128 if self.opts.precision == 64 else np.complex64

    def kernel_terms(self, m):
        o = self.opts
        sigma, phi, edges = np.zeros(o.n_alpha), np.zeros((o.n_alpha, o.n_modes)), np.zeros(o.n_modes + 1)
        _check(lib().sigw_plan_kernel_terms(self._h, m, _ptr(sigma, C.c_double), _ptr(phi, C.c_double),
                                            _ptr(edges, C.c_double)), self._h, "kernel_terms")
        return sigma, phi, edges

    def generate(self, A, sigma, kstar, kind="gauss", F_NL=0.0, G_NL=0.0, usr_floor=1e-6, seeds=(1,), alpha_NL=0.0,
                 beta_NL=0.0):
        """sigw_generate; returns the USR floor-hit counts per realisation."""
        pz = PZeta(A, sigma, kstar)
        mp = _ngmap(kind, F_NL, G_NL, usr_floor, alpha_NL, beta_NL)
        sd = np.ascontiguousarray(seeds, dtype=np.uint64)
        hits = np.zeros(len(sd), dtype=np.int64)
        _check(lib().sigw_generate(self._h, C.byref(pz), C.byref(mp), _ptr(sd, C.c_uint64), len(sd),
                                   _ptr(hits, C.c_int64)), self._h, "sigw_generate")
        self.batch = len(sd)
        return hits

    def generate_batch(self, specs):
        """sigw_generate_batch: one realisation per workloads.Spec (same N and L), own parameters each."""
        n = len(specs)
        pz = (PZeta * n)(*[PZeta(s.A, s.sigma, s.kstar) for s in specs])
        mp = (NGMap * n)(*[_spec_map(s) for s in specs])
        sd = np.ascontiguousarray([s.seed for s in specs], dtype=np.uint64)
        hits = np.zeros(n, dtype=np.int64)
        _check(lib().sigw_generate_batch(self._h, pz, mp, _ptr(sd, C.c_uint64), n, _ptr(hits, C.c_int64)), self._h,
               "sigw_generate_batch")
        self.batch = n
        return hits

    def generate_spec(self, spec, seeds=None):
        return self.generate(spec.A, spec.sigma, spec.kstar, spec.kind, spec.F_NL, spec.G_NL, spec.usr_floor,
                             seeds=(spec.seed,) if seeds is None else seeds, alpha_NL=getattr(spec, "alpha_NL", 0.0),
                             beta_NL=getattr(spec, "beta_NL", 0.0))

    def spectrum(self, shells=None):
        """sigw_spectrum; dict of [batch, n_shells] arrays: omega, PA, PB, Nk (and n_c)."""
        sh = np.arange(1, self.N // 2 + 1, dtype=np.int32) if shells is None else np.ascontiguousarray(shells, dtype=np.int32)
        ns = len(sh)
        out = {k: np.zeros((self.batch, ns)) for k in ("omega", "PA", "PB")}
        nk = np.zeros((self.batch, ns), dtype=np.int64)
        _check(lib().sigw_spectrum(self._h, _ptr(sh, C.c_int), ns, _ptr(out["omega"], C.c_double),
                                   _ptr(out["PA"], C.c_double), _ptr(out["PB"], C.c_double), _ptr(nk, C.c_int64)),
               self._h, "sigw_spectrum")
        out["Nk"] = nk
        out["n_c"] = sh
        return out

    def spectrum_jackknife(self, shells=None, M=4):
        """sigw_spectrum_jackknife; dict of [batch, n_shells] arrays: omega, sigma_omega, PA, sigma_PA, PB,
        sigma_PB (and n_c).  shells default to 1..N/2-1."""
        sh = np.arange(1, self.N // 2, dtype=np.int32) if shells is None else np.ascontiguousarray(shells, dtype=np.int32)
        ns = len(sh)
        keys = ("omega", "sigma_omega", "PA", "sigma_PA", "PB", "sigma_PB")
        out = {k: np.zeros((self.batch, ns)) for k in keys}
        _check(lib().sigw_spectrum_jackknife(self._h, _ptr(sh, C.c_int), ns, M, *[_ptr(out[k], C.c_double) for k in keys]),
               self._h, "sigw_spectrum_jackknife")
        out["n_c"] = sh
        return out

    def set_box(self, L):
        _check(lib().sigw_plan_set_box(self._h, L), self._h, "sigw_plan_set_box")
        self.L = L

    def target_scan(self, k, A, sigma, kstar, kind="gauss", F_NL=0.0, G_NL=0.0, usr_floor=1e-6, seed=1, eps=0.1):
        """sigw_target_scan: Omega_GW at each target k in its own box; returns dict omega, L, n_c."""
        kk = np.ascontiguousarray(k, dtype=np.float64)
        n = len(kk)
        pz = PZeta(A, sigma, kstar)
        mp = _ngmap(kind, F_NL, G_NL, usr_floor)
        om, Ls, nc = np.zeros(n), np.zeros(n), np.zeros(n, dtype=np.int32)
        _check(lib().sigw_target_scan(self._h, C.byref(pz), C.byref(mp), seed, _ptr(kk, C.c_double), n, eps,
                                      _ptr(om, C.c_double), _ptr(Ls, C.c_double), _ptr(nc, C.c_int)), self._h,
               "sigw_target_scan")
        self.L = float(Ls[-1])
        self.batch = 1
        return {"omega": om, "L": Ls, "n_c": nc}

    def spectrum_async(self, dev_out_ptr, shells=None):
        sh = np.arange(1, self.N // 2 + 1, dtype=np.int32) if shells is None else np.ascontiguousarray(shells, dtype=np.int32)
        _check(lib().sigw_spectrum_async(self._h, _ptr(sh, C.c_int), len(sh), C.c_void_p(dev_out_ptr)), self._h,
               "sigw_spectrum_async")

    def debug_wait_limit(self, cycles):
        """sigw_plan_debug_wait_limit: test hook; 0 restores the default limit of the bulk-copy waits."""
        _check(lib().sigw_plan_debug_wait_limit(self._h, int(cycles)), self._h, "sigw_plan_debug_wait_limit")

    def copy_phi(self, b=0):
        out = np.zeros((self.N, self.N, self.N // 2 + 1), dtype=self.dtype)
        _check(lib().sigw_copy_phi(self._h, b, out.ctypes.data_as(C.c_void_p)), self._h, "sigw_copy_phi")
        return out

    def fft3d(self, direction, in_ptr, out_ptr):
        _check(lib().sigw_fft3d(self._h, direction, C.c_void_p(in_ptr), C.c_void_p(out_ptr)), self._h, "sigw_fft3d")

    def autotune(self, n_c=0):
        """sigw_plan_autotune: returns (terms per launch, radix variant, ms)."""
        b, v, ms = C.c_int(), C.c_int(), C.c_double()
        _check(lib().sigw_plan_autotune(self._h, n_c, C.byref(b), C.byref(v), C.byref(ms)), self._h,
               "sigw_plan_autotune")
        return b.value, v.value, ms.value

    def set_tuning(self, alpha_batch, variant):
        _check(lib().sigw_plan_set_tuning(self._h, alpha_batch, variant), self._h, "sigw_plan_set_tuning")

    def profile(self, enable=True):
        _check(lib().sigw_plan_profile(self._h, 1 if enable else 0), self._h, "sigw_plan_profile")

    def profile_read(self):
        """Counters since the last reset: dict kind -> {ms, bytes, launches}, plus h2d/d2h bytes."""
        pr = Profile()
        _check(lib().sigw_plan_profile_read(self._h, C.byref(pr)), self._h, "sigw_plan_profile_read")
        out = {k: {"ms": pr.ms[i], "bytes": pr.bytes[i], "launches": int(pr.launches[i])} for i, k in enumerate(KINDS)}
        out["h2d_bytes"] = pr.h2d_bytes
        out["d2h_bytes"] = pr.d2h_bytes
        return out

    def synchronize(self):
        _check(lib().sigw_synchronize(self._h), self._h, "sigw_synchronize")


class Server:
    """Continuous-batching spectrum server (sigw_server_create / sigw_submit / sigw_poll / sigw_wait)."""

    def __init__(self, hbm_budget_bytes, max_slots=2, opts=None, **over):
        self.opts = opts or default_opts(**over)
        h = C.c_void_p()
        _check(lib().sigw_server_create(int(hbm_budget_bytes), max_slots, C.byref(self.opts), C.byref(h)), None,
               "sigw_server_create")
        self._h = h
        self._N = {}

    def set_express(self, slots, max_N):
        """sigw_server_set_express: extra slots for requests with N <= max_N."""
        _check(lib().sigw_server_set_express(self._h, slots, max_N), None, "sigw_server_set_express")

    def submit(self, spec):
        t = C.c_uint64()
        _check(lib().sigw_submit(self._h, spec.N, spec.L, C.byref(PZeta(spec.A, spec.sigma, spec.kstar)),
                                 C.byref(_spec_map(spec)),
                                 spec.seed, C.byref(t)), None, "sigw_submit")
        self._N[t.value] = spec.N
        return t.value

    def poll(self, ticket):
        """None while not ready, else (omega, latency_s)."""
        om = np.zeros(self._N.get(ticket, 8) // 2)
        lat = C.c_double()
        st = lib().sigw_poll(self._h, ticket, _ptr(om, C.c_double), C.byref(lat))
        if st == ENOTREADY:
            return None
        self._N.pop(ticket, None)
        _check(st, None, "sigw_poll")
        return om, lat.value

    def wait(self, ticket, timeout_s=600.0):
        om = np.zeros(self._N.get(ticket, 8) // 2)
        lat = C.c_double()
        st = lib().sigw_wait(self._h, ticket, timeout_s, _ptr(om, C.c_double), C.byref(lat))
        if st != ETIMEOUT:
            self._N.pop(ticket, None)
        _check(st, None, "sigw_wait")
        return om, lat.value

    def stats(self):
        s = ServerStats()
        _check(lib().sigw_server_stats_read(self._h, C.byref(s)), None, "sigw_server_stats_read")
        return {n: getattr(s, n) for n, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            lib().sigw_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
