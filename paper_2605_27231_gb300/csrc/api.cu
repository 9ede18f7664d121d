// C ABI of the lattice SIGW library: plan lifetime, device buffers, and the
// orchestration of the synthesis chain and of the per-shell hot loop.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/sigw.h"
#include "ops.h"
#include "plan.h"

namespace {

std::atomic<int> g_fail_alloc{0};

const double kPi = 3.14159265358979323846;

bool is_pow2_in_range(int N) { return N >= 8 && N <= 512 && (N & (N - 1)) == 0; }

sigw::DecompParams params_of(const sigw_opts& o) {
  sigw::DecompParams p;
  p.n_modes = o.n_modes;
  p.n_alpha = o.n_alpha;
  p.umin = o.umin;
  p.umax = o.umax;
  p.upiv = o.upiv;
  p.sigp = o.sigp;
  p.Ap = o.Ap;
  return p;
}

int auto_alpha_batch(const sigw_opts& o) {
  if (o.alpha_batch > 0) return std::min(o.alpha_batch, o.n_alpha);
  return std::min(o.n_alpha, 10);
}

// Largest terms-per-launch the first-pass output buffer holds (the autotuner's largest candidate).
int max_alpha_batch(const sigw_opts& o) {
  if (o.alpha_batch > 0) return std::min(o.alpha_batch, o.n_alpha);
  return std::min(o.n_alpha, 16);
}

// Process-wide autotuning results: (N, precision, realisations, n_alpha) -> (terms per launch, variant).
struct TuneKey {
  int N, prec, batch, n_alpha;
  bool operator<(const TuneKey& o) const {
    return std::tie(N, prec, batch, n_alpha) < std::tie(o.N, o.prec, o.batch, o.n_alpha);
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, std::pair<int, int>> g_tune;

// Sizes (bytes) of every device buffer of a plan.
struct Sizes {
  size_t phi, T, W, synth, F, F2, partial, out, lut, tab, tw, amp, rows_sq;
  int maxblk;
  size_t total() const {
    return phi + T + std::max(W, synth) + F + F2 + partial + out + lut + tab + tw + amp + rows_sq + 4096;
  }
};

Sizes sizes_of(int N, const sigw_opts& o) {
  Sizes s;
  const size_t H = N / 2, NH = H + 1, NN = (size_t)N * N;
  const size_t rel = o.precision == 64 ? 8 : 4, cel = 2 * rel;
  const size_t mb = (size_t)o.max_batch;
  const int B = max_alpha_batch(o);
  sigw::LaunchShape sh = o.precision == 64 ? sigw::OpsRT<double>::shape(N) : sigw::OpsRT<float>::shape(N);
  s.maxblk = sh.maxblk_f3;
  s.phi = mb * NN * NH * cel;
  s.T = 2 * mb * (size_t)B * NN * H * cel;
  s.W = mb * 3 * (size_t)o.n_alpha * NN * H * cel;
  // the jackknife reuses W after each shell: two standard + two packed half spectra + two real fields
  s.W = std::max(s.W, mb * 2 * (NN * NH * cel + NN * H * cel + NN * (size_t)N * rel) + 1024);
  s.synth = mb * (NN * H * cel + NN * NH * cel + 3 * NN * (size_t)N * rel) + 1024;  // + two real fields (non-local map)
  s.F = mb * 6 * NN * NH * cel;
  s.F2 = mb * 6 * NN * NH * cel;
  s.partial = mb * H * 2 * (size_t)s.maxblk * sizeof(double);
  s.out = mb * H * 4 * sizeof(double) + H * (sizeof(int) + sizeof(double));
  const size_t msq = 3 * H * H + 1;
  s.lut = H * msq * sizeof(int16_t);
  s.tab = 2 * ((size_t)o.n_alpha * (o.n_modes + 1) + o.n_alpha) * rel;
  s.tw = (size_t)N * cel;
  s.amp = mb * msq * rel + mb * sizeof(sigw::MapArgs);
  const int rb = o.precision == 64 ? sigw::OpsRT<double>::rows_blocks(N) : sigw::OpsRT<float>::rows_blocks(N);
  s.rows_sq = mb * ((size_t)rb * sizeof(double) + 2 * sizeof(double) + 2 * sizeof(uint64_t));
  return s;
}

bool valid_opts(const sigw_opts& o) {
  return o.n_modes >= 2 && o.n_modes <= 4096 && o.n_alpha >= 1 && o.n_alpha <= o.n_modes && o.umin > 0 &&
         o.umax > o.umin && o.sigp > 0 && o.Ap >= 0 && (o.precision == 32 || o.precision == 64) &&
         o.max_batch >= 1 && o.max_batch <= 64 && o.alpha_batch >= 0;
}

}  // namespace

struct sigw_plan_s {
  int N = 0;
  double L = 0;
  sigw_opts opts{};
  int dev = 0;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  sigw::Decomposition dec;
  Sizes sz{};
  int B = 1;        // terms per first/second-pass launch
  int variant = 0;  // radix variant of the strided inverse passes
  bool tuned_from_table = false;
  size_t msq_max = 0;
  std::vector<double> Nk;  // per shell 1..N/2
  // device buffers
  std::vector<void*> allocs;
  void* d_phi = nullptr;
  void* d_T = nullptr;     // first-pass output (two fields per term of an alpha batch)
  void* d_work = nullptr;  // W during the hot loop, synthesis scratch during sigw_generate / sigw_fft3d
  void* d_F = nullptr;
  void* d_F2 = nullptr;
  double* d_partial = nullptr;
  double* d_out = nullptr;
  int* d_shells = nullptr;
  double* d_Nk = nullptr;
  int16_t* d_lut = nullptr;
  void* d_phitab[2] = {nullptr, nullptr};
  void* d_sigma[2] = {nullptr, nullptr};
  void* d_tw = nullptr;
  void* d_amp = nullptr;            // [max_batch][msq_max + 1] synthesis amplitudes
  sigw::MapArgs* d_maps = nullptr;  // [max_batch] map parameters
  double* d_sq = nullptr;
  double* d_mean = nullptr;
  unsigned long long* d_hits = nullptr;
  uint64_t* d_seeds = nullptr;
  int* d_err = nullptr;  // OR-ed by kernels whose bounded waits gave up
  long long wait_limit = sigw::kDefaultWaitLimit;  // cycles of P3's main-loop waits (sigw_plan_debug_wait_limit)
  int* d_shells_all = nullptr;   // 1..N/2, for the all-shells call (no upload, so it can be captured)
  double* d_Nk_all = nullptr;
  // CUDA graph of the all-shells spectrum loop, per realisation count
  cudaGraphExec_t graph = nullptr;
  int graph_batch = 0;
  bool graphs_ok = true;
  long long graph_launches[SIGW_NKINDS] = {0};
  double graph_bytes[SIGW_NKINDS] = {0};
  int generated = 0;
  std::string err;
  // accounting (see sigw_profile)
  struct Rec {
    int kind;
    cudaEvent_t a, b;
  };
  bool prof_on = false;
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  long long launches[SIGW_NKINDS] = {0};
  double kbytes[SIGW_NKINDS] = {0};
  double h2d = 0, d2h = 0;

  size_t relem() const { return opts.precision == 64 ? 8 : 4; }
  size_t celem() const { return 2 * relem(); }
};

namespace {

sigw_status fail(sigw_plan p, sigw_status s, const std::string& msg) {
  if (p) p->err = msg;
  return s;
}

sigw_status cuda_fail(sigw_plan p, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  (void)cudaGetLastError();
  return fail(p, SIGW_ECUDA, m);
}

#define CKP(plan, call, what)                            \
  do {                                                   \
    cudaError_t _e = (call);                             \
    if (_e != cudaSuccess) return cuda_fail(plan, _e, what); \
  } while (0)

cudaEvent_t get_event(sigw_plan p) {
  if (!p->pool.empty()) {
    cudaEvent_t e = p->pool.back();
    p->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  return e;
}

void prof_reset(sigw_plan p) {
  for (auto& r : p->recs) {
    p->pool.push_back(r.a);
    p->pool.push_back(r.b);
  }
  p->recs.clear();
  for (int k = 0; k < SIGW_NKINDS; ++k) {
    p->launches[k] = 0;
    p->kbytes[k] = 0;
  }
  p->h2d = p->d2h = 0;
}

// Launch one kernel (the callable returns its launch status) with accounting of kind / algorithmic bytes.
template <typename F>
sigw_status run(sigw_plan p, int kind, double bytes, const char* what, F&& f) {
  cudaEvent_t a = nullptr, b = nullptr;
  if (p->prof_on) {
    a = get_event(p);
    if (a) cudaEventRecord(a, p->st);
  }
  cudaError_t e = f();
  if (e != cudaSuccess) return cuda_fail(p, e, what);
  if (p->prof_on && a) {
    b = get_event(p);
    if (b) {
      cudaEventRecord(b, p->st);
      p->recs.push_back({kind, a, b});
    } else {
      p->pool.push_back(a);
    }
  }
  p->launches[kind] += 1;
  p->kbytes[kind] += bytes;
  return SIGW_OK;
}

#define RUN(plan, kind, bytes, what, expr)                                       \
  do {                                                                            \
    sigw_status _s = run(plan, kind, (double)(bytes), what, [&]() { return (expr); }); \
    if (_s != SIGW_OK) return _s;                                                 \
  } while (0)

// After the stream is idle: report (and clear) a bounded wait that gave up inside a kernel.
sigw_status check_err_flag(sigw_plan p) {
  int h = 0;
  cudaError_t e = cudaMemcpy(&h, p->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(p, e, "read error flag");
  if (h) {
    cudaMemset(p->d_err, 0, sizeof(int));
    return fail(p, SIGW_ETIMEOUT, "a bounded wait in the bulk-copy pipeline gave up; results are invalid");
  }
  return SIGW_OK;
}

sigw_status dev_alloc(sigw_plan p, void** ptr, size_t bytes) {
  int c = g_fail_alloc.load();
  if (c > 0) {
    if (g_fail_alloc.fetch_sub(1) == 1) return fail(p, SIGW_ENOMEM, "device allocation failed (injected)");
  }
  cudaError_t e = cudaMalloc(ptr, bytes < 16 ? 16 : bytes);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    *ptr = nullptr;
    return fail(p, e == cudaErrorMemoryAllocation ? SIGW_ENOMEM : SIGW_ECUDA,
                std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
  }
  p->allocs.push_back(*ptr);
  return SIGW_OK;
}

template <typename T>
void to_prec(const std::vector<double>& in, std::vector<unsigned char>& out) {
  out.resize(in.size() * sizeof(T));
  T* o = reinterpret_cast<T*>(out.data());
  for (size_t i = 0; i < in.size(); ++i) o[i] = (T)in[i];
}

void convert(const std::vector<double>& in, int prec, std::vector<unsigned char>& out) {
  if (prec == 64) to_prec<double>(in, out); else to_prec<float>(in, out);
}

// modes of the full lattice n in (-N/2, N/2]^3 per shell: |n|^2 in [n_c^2 - n_c + 1, n_c^2 + n_c]
std::vector<double> count_shell_modes(int N) {
  const int H = N / 2;
  const int msq_max = 3 * H * H;
  std::vector<long long> c2(H * H + 1, 0);
  for (int n = -H + 1; n <= H; ++n) c2[n * n] += 1;
  std::vector<long long> hist(msq_max + 1, 0);
  for (int a = -H + 1; a <= H; ++a)
    for (int b = -H + 1; b <= H; ++b) {
      const int base = a * a + b * b;
      for (int v = 0; v <= H * H; ++v)
        if (c2[v]) hist[base + v] += c2[v];
    }
  std::vector<double> nk(H + 1, 0.0);
  for (int nc = 1; nc <= H; ++nc) {
    long long t = 0;
    for (int m = nc * nc - nc + 1; m <= nc * nc + nc && m <= msq_max; ++m) t += hist[m];
    nk[nc] = (double)t;
  }
  return nk;
}

#define OPS(plan, fn, ...) \
  ((plan)->opts.precision == 64 ? sigw::OpsRT<double>::fn(__VA_ARGS__) : sigw::OpsRT<float>::fn(__VA_ARGS__))

}  // namespace

extern "C" {

sigw_status sigw_opts_default(sigw_opts* o) {
  if (!o) return SIGW_EINVAL;
  o->n_modes = 200;
  o->n_alpha = 50;
  o->umin = 1e-3;
  o->umax = 15.0;
  o->upiv = 1.0;
  o->sigp = 0.5;
  o->Ap = 10.0;
  o->precision = 32;
  o->alpha_batch = 0;
  o->max_batch = 1;
  o->strict_domain = 0;
  return SIGW_OK;
}

const char* sigw_strerror(sigw_status s) {
  switch (s) {
    case SIGW_OK: return "ok";
    case SIGW_EINVAL: return "invalid argument";
    case SIGW_ENOMEM: return "out of memory";
    case SIGW_ECUDA: return "CUDA error";
    case SIGW_EDOMAIN: return "USR map argument below the floor";
    case SIGW_ETIMEOUT: return "timed out";
    case SIGW_EBUSY: return "request does not fit the memory budget";
    case SIGW_ENOTREADY: return "result not ready";
    case SIGW_ESTATE: return "call out of order";
  }
  return "unknown status";
}

sigw_status sigw_debug_fail_alloc(int n) {
  g_fail_alloc.store(n > 0 ? n : 0);
  return SIGW_OK;
}

sigw_status sigw_plan_footprint(int N, const sigw_opts* opts, size_t* bytes) {
  sigw_opts o;
  if (opts) o = *opts; else sigw_opts_default(&o);
  if (!bytes || !is_pow2_in_range(N) || !valid_opts(o)) return SIGW_EINVAL;
  *bytes = sizes_of(N, o).total();
  return SIGW_OK;
}

sigw_status sigw_decompose(const sigw_opts* opts, int m, double* sigma, double* phi, double* edges,
                           double* sigma_all) {
  sigw_opts o;
  if (opts) o = *opts; else sigw_opts_default(&o);
  if (m < 0 || m > 1) return SIGW_EINVAL;
  sigw::Decomposition d;
  std::string e;
  sigw::DecompParams p = params_of(o);
  if (sigma_all) p.n_alpha = p.n_modes;
  if (!sigw::build_decomposition(p, &d, &e)) return SIGW_EINVAL;
  const sigw::KernelTerms& t = d.terms[m];
  if (sigma) std::memcpy(sigma, t.sigma.data(), sizeof(double) * o.n_alpha);
  if (phi) std::memcpy(phi, t.phi.data(), sizeof(double) * (size_t)o.n_alpha * o.n_modes);
  if (edges) std::memcpy(edges, d.edges.data(), sizeof(double) * d.edges.size());
  if (sigma_all) std::memcpy(sigma_all, t.sigma.data(), sizeof(double) * o.n_modes);
  return SIGW_OK;
}

sigw_status sigw_decomposition_error(const sigw_opts* opts, int m, double* frob, double* maxrel, double* gap) {
  sigw_opts o;
  if (opts) o = *opts; else sigw_opts_default(&o);
  if (m < 0 || m > 1 || !valid_opts(o)) return SIGW_EINVAL;
  sigw::DecompParams p = params_of(o);
  const int n = p.n_modes, k = o.n_alpha;
  p.n_alpha = n;  // every eigenpair
  sigw::Decomposition d;
  std::string e;
  if (!sigw::build_decomposition(p, &d, &e)) return SIGW_EINVAL;
  const sigw::KernelTerms& t = d.terms[m];
  // q_a(i) = phi_a(i) sqrt(L_i); the full sum reproduces C, the first k terms give C_k
  std::vector<double> q((size_t)n * n);
  for (int a = 0; a < n; ++a)
    for (int i = 0; i < n; ++i) q[(size_t)a * n + i] = t.phi[(size_t)a * n + i] * std::sqrt(d.widths[i]);
  double num = 0.0, den = 0.0, dmax = 0.0, cmax = 0.0;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double full = 0.0, part = 0.0;
      for (int a = 0; a < n; ++a) {
        const double v = t.sigma[a] * q[(size_t)a * n + i] * q[(size_t)a * n + j];
        full += v;
        if (a < k) part += v;
      }
      num += (full - part) * (full - part);
      den += full * full;
      dmax = std::max(dmax, std::fabs(full - part));
      cmax = std::max(cmax, std::fabs(full));
    }
  if (frob) *frob = den > 0 ? std::sqrt(num / den) : 0.0;
  if (maxrel) *maxrel = cmax > 0 ? dmax / cmax : 0.0;
  if (gap) *gap = (k < n && t.sigma[k - 1] != 0.0) ? std::fabs(t.sigma[k]) / std::fabs(t.sigma[k - 1]) : 0.0;
  return SIGW_OK;
}

sigw_status sigw_cell_table(const sigw_opts* opts, int n_c, int msq_max, int16_t* lut) {
  sigw_opts o;
  if (opts) o = *opts; else sigw_opts_default(&o);
  if (!lut || n_c < 1 || msq_max < 0) return SIGW_EINVAL;
  sigw::Decomposition d;
  std::string e;
  if (!sigw::build_decomposition(params_of(o), &d, &e)) return SIGW_EINVAL;
  sigw::build_cell_lut(d.edges, n_c, msq_max, lut);
  return SIGW_OK;
}

sigw_status sigw_plan_create(int N, double L, const sigw_opts* opts, void* cuda_stream, sigw_plan* out) {
  if (!out) return SIGW_EINVAL;
  *out = nullptr;
  sigw_opts o;
  if (opts) o = *opts; else sigw_opts_default(&o);
  if (!is_pow2_in_range(N) || !(L > 0) || !valid_opts(o)) return SIGW_EINVAL;
  sigw_plan p = new (std::nothrow) sigw_plan_s();
  if (!p) return SIGW_ENOMEM;
  p->N = N;
  p->L = L;
  p->opts = o;
  p->B = auto_alpha_batch(o);
  // Untuned default: the choices measured fastest on GB300 (at 128^3 and 256^3 the first and the radix-16 last pass
  // with their per-thread state in tensor memory; at 512^3 the 512-specific strided passes and the tensor-memory
  // last pass).  sigw_plan_autotune or the table may override it.
  p->variant = o.precision == 32 ? (N == 512 ? 15 : (N >= 128 ? 26 : 0)) : 0;
  std::string e;
  if (!sigw::build_decomposition(params_of(o), &p->dec, &e)) {
    delete p;
    return SIGW_EINVAL;
  }
  auto bail = [&](sigw_status s) {
    sigw_plan_destroy(p);
    return s;
  };
  cudaError_t ce = cudaGetDevice(&p->dev);
  if (ce != cudaSuccess) {
    (void)cudaGetLastError();
    return bail(SIGW_ECUDA);
  }
  if (cuda_stream) {
    p->st = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&p->st, cudaStreamNonBlocking) != cudaSuccess) {
      (void)cudaGetLastError();
      return bail(SIGW_ECUDA);
    }
    p->own_stream = true;
  }
  p->sz = sizes_of(N, o);
  const int H = N / 2;
  p->msq_max = 3 * (size_t)H * H;
  const size_t rel = p->relem(), cel = p->celem();
  const size_t mb = o.max_batch;
  sigw_status s;
#define ALLOC(ptr, bytes)                                   \
  do {                                                      \
    void* _q = nullptr;                                     \
    if ((s = dev_alloc(p, &_q, (bytes))) != SIGW_OK) return bail(s); \
    ptr = reinterpret_cast<decltype(ptr)>(_q);              \
  } while (0)
  ALLOC(p->d_phi, p->sz.phi);
  ALLOC(p->d_T, p->sz.T);
  ALLOC(p->d_work, std::max(p->sz.W, p->sz.synth));
  ALLOC(p->d_F, p->sz.F);
  ALLOC(p->d_F2, p->sz.F2);
  ALLOC(p->d_partial, p->sz.partial);
  ALLOC(p->d_out, mb * H * 4 * sizeof(double));
  ALLOC(p->d_shells, H * sizeof(int));
  ALLOC(p->d_Nk, H * sizeof(double));
  ALLOC(p->d_lut, p->sz.lut);
  for (int m = 0; m < 2; ++m) {
    ALLOC(p->d_phitab[m], (size_t)o.n_alpha * (o.n_modes + 1) * rel);
    ALLOC(p->d_sigma[m], (size_t)o.n_alpha * rel);
  }
  ALLOC(p->d_tw, (size_t)N * cel);
  ALLOC(p->d_amp, mb * (p->msq_max + 1) * rel);
  ALLOC(p->d_maps, mb * sizeof(sigw::MapArgs));
  const int rb = OPS(p, rows_blocks, N);
  ALLOC(p->d_sq, mb * rb * sizeof(double));
  ALLOC(p->d_mean, mb * sizeof(double));
  ALLOC(p->d_hits, mb * sizeof(unsigned long long));
  ALLOC(p->d_seeds, mb * sizeof(uint64_t));
  ALLOC(p->d_err, sizeof(int));
  ALLOC(p->d_shells_all, H * sizeof(int));
  ALLOC(p->d_Nk_all, H * sizeof(double));
#undef ALLOC
  if (cudaMemset(p->d_err, 0, sizeof(int)) != cudaSuccess) return bail(SIGW_ECUDA);
  // tables
  std::vector<unsigned char> buf;
  {
    std::vector<double> tw;
    sigw::build_twiddles(N, tw);
    convert(tw, o.precision, buf);
    if (cudaMemcpy(p->d_tw, buf.data(), buf.size(), cudaMemcpyHostToDevice) != cudaSuccess) return bail(SIGW_ECUDA);
  }
  for (int m = 0; m < 2; ++m) {
    const sigw::KernelTerms& t = p->dec.terms[m];
    std::vector<double> tab((size_t)o.n_alpha * (o.n_modes + 1), 0.0);
    for (int a = 0; a < o.n_alpha; ++a)
      for (int i = 0; i < o.n_modes; ++i) tab[(size_t)a * (o.n_modes + 1) + i] = t.phi[(size_t)a * o.n_modes + i];
    convert(tab, o.precision, buf);
    if (cudaMemcpy(p->d_phitab[m], buf.data(), buf.size(), cudaMemcpyHostToDevice) != cudaSuccess) return bail(SIGW_ECUDA);
    convert(t.sigma, o.precision, buf);
    if (cudaMemcpy(p->d_sigma[m], buf.data(), buf.size(), cudaMemcpyHostToDevice) != cudaSuccess) return bail(SIGW_ECUDA);
  }
  {
    std::vector<int16_t> lut((size_t)H * (p->msq_max + 1));
    for (int nc = 1; nc <= H; ++nc)
      sigw::build_cell_lut(p->dec.edges, nc, (int)p->msq_max, lut.data() + (size_t)(nc - 1) * (p->msq_max + 1));
    if (cudaMemcpy(p->d_lut, lut.data(), lut.size() * sizeof(int16_t), cudaMemcpyHostToDevice) != cudaSuccess)
      return bail(SIGW_ECUDA);
  }
  p->Nk = count_shell_modes(N);
  if (o.alpha_batch == 0) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(TuneKey{N, o.precision, o.max_batch, o.n_alpha});
    if (it != g_tune.end()) {
      p->B = it->second.first;
      p->variant = it->second.second;
      p->tuned_from_table = true;
    }
  }
  {
    std::vector<int> sh(H);
    for (int i = 0; i < H; ++i) sh[i] = i + 1;
    if (cudaMemcpy(p->d_shells_all, sh.data(), sizeof(int) * H, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(p->d_Nk_all, p->Nk.data() + 1, sizeof(double) * H, cudaMemcpyHostToDevice) != cudaSuccess)
      return bail(SIGW_ECUDA);
  }
  *out = p;
  return SIGW_OK;
}

sigw_status sigw_plan_destroy(sigw_plan p) {
  if (!p) return SIGW_OK;
  if (p->st) cudaStreamSynchronize(p->st);
  if (p->graph) cudaGraphExecDestroy(p->graph);
  for (void* q : p->allocs) cudaFree(q);
  prof_reset(p);
  for (cudaEvent_t e : p->pool) cudaEventDestroy(e);
  if (p->own_stream && p->st) cudaStreamDestroy(p->st);
  (void)cudaGetLastError();
  delete p;
  return SIGW_OK;
}

const char* sigw_plan_last_error(sigw_plan p) { return p ? p->err.c_str() : "no plan"; }

sigw_status sigw_plan_kernel_terms(sigw_plan p, int m, double* sigma, double* phi, double* edges) {
  if (!p || m < 0 || m > 1) return SIGW_EINVAL;
  const sigw::KernelTerms& t = p->dec.terms[m];
  if (sigma) std::memcpy(sigma, t.sigma.data(), sizeof(double) * t.sigma.size());
  if (phi) std::memcpy(phi, t.phi.data(), sizeof(double) * t.phi.size());
  if (edges) std::memcpy(edges, p->dec.edges.data(), sizeof(double) * p->dec.edges.size());
  return SIGW_OK;
}

sigw_status sigw_synchronize(sigw_plan p) {
  if (!p) return SIGW_EINVAL;
  CKP(p, cudaSetDevice(p->dev), "cudaSetDevice");
  CKP(p, cudaStreamSynchronize(p->st), "stream synchronize");
  return check_err_flag(p);
}

sigw_status sigw_generate_batch(sigw_plan p, const sigw_pzeta* pz, const sigw_ngmap* maps, const uint64_t* seeds,
                                int batch, int64_t* usr_hits) {
  if (!p) return SIGW_EINVAL;
  if (!pz || !maps || !seeds || batch < 1 || batch > p->opts.max_batch)
    return fail(p, SIGW_EINVAL, "sigw_generate: bad arguments");
  bool all_gauss = true, any_usr = false, any_nonlocal = false;
  for (int b = 0; b < batch; ++b) {
    if (!(pz[b].A >= 0) || !(pz[b].sigma > 0) || !(pz[b].kstar > 0) || maps[b].kind < 0 || maps[b].kind > 3)
      return fail(p, SIGW_EINVAL, "sigw_generate: bad P_zeta or map parameters");
    if (maps[b].kind == SIGW_MAP_NONLOCAL && !(std::isfinite(maps[b].alpha_NL) && std::isfinite(maps[b].beta_NL)))
      return fail(p, SIGW_EINVAL, "sigw_generate: bad non-local map coefficients");
    all_gauss = all_gauss && maps[b].kind == SIGW_MAP_GAUSS;
    any_usr = any_usr || maps[b].kind == SIGW_MAP_USR;
    any_nonlocal = any_nonlocal || maps[b].kind == SIGW_MAP_NONLOCAL;
  }
  CKP(p, cudaSetDevice(p->dev), "cudaSetDevice");
  const int N = p->N, H = N / 2;
  const double L = p->L, dx = L / N, kf = 2.0 * kPi / L;
  const size_t NN = (size_t)N * N;
  const size_t msq1 = p->msq_max + 1;
  // synthesis amplitude sqrt(P_zeta(k) dx^3) per integer |n|^2, P = 2 pi^2 Delta^2 / k^3 (Eq. eq_lognormal)
  std::vector<double> amp(batch * msq1, 0.0);
  std::vector<sigw::MapArgs> margs(batch);
  for (int b = 0; b < batch; ++b) {
    for (size_t msq = 1; msq <= p->msq_max; ++msq) {
      const double k = kf * std::sqrt((double)msq);
      const double lk = std::log(k / pz[b].kstar);
      const double sg = pz[b].sigma;
      const double d2 = pz[b].A / std::sqrt(2.0 * kPi * sg * sg) * std::exp(-lk * lk / (2.0 * sg * sg));
      const double P = 2.0 * kPi * kPi * d2 / (k * k * k);
      amp[b * msq1 + msq] = std::sqrt(P * dx * dx * dx);
    }
    const double ks2 = pz[b].kstar * pz[b].kstar;
    margs[b] = maps[b].kind == SIGW_MAP_NONLOCAL
                   ? sigw::MapArgs{maps[b].kind, maps[b].alpha_NL / ks2, maps[b].beta_NL / ks2, 1e-6}
                   : sigw::MapArgs{maps[b].kind, maps[b].F_NL, maps[b].G_NL,
                                   maps[b].usr_floor > 0 ? maps[b].usr_floor : 1e-6};
  }
  std::vector<unsigned char> buf;
  convert(amp, p->opts.precision, buf);
  CKP(p, cudaMemcpyAsync(p->d_amp, buf.data(), buf.size(), cudaMemcpyHostToDevice, p->st), "upload amp");
  CKP(p, cudaMemcpyAsync(p->d_maps, margs.data(), sizeof(sigw::MapArgs) * batch, cudaMemcpyHostToDevice, p->st),
      "upload maps");
  CKP(p, cudaMemcpyAsync(p->d_seeds, seeds, sizeof(uint64_t) * batch, cudaMemcpyHostToDevice, p->st), "upload seeds");
  p->h2d += buf.size() + sizeof(uint64_t) * batch + sizeof(sigw::MapArgs) * batch;
  const size_t cel = p->celem();
  char* work = (char*)p->d_work;
  void* Y = work;
  void* X = work + (size_t)p->opts.max_batch * NN * H * cel;
  void* R = (char*)X + (size_t)p->opts.max_batch * NN * (H + 1) * cel;
  cudaStream_t st = p->st;
  const double Yb = (double)batch * NN * H * cel, Xb = (double)batch * NN * (H + 1) * cel;
  const double Rb = (double)batch * NN * N * p->relem();
  RUN(p, 0, Yb, "noise + rows R2C", OPS(p, rows_r2c_noise, N, Y, p->d_seeds, batch, p->d_tw, st));
  RUN(p, 0, 2 * Yb, "forward axis 1", OPS(p, pass, N, Y, 1, -1, batch, p->d_tw, st));
  RUN(p, 0, 2 * Yb, "forward axis 0", OPS(p, pass, N, Y, 0, -1, batch, p->d_tw, st));
  if (all_gauss) {
    RUN(p, 0, Yb + Xb, "unpack (Gaussian Phi)",
        OPS(p, unpack, N, Y, p->d_phi, batch, p->d_amp, (long)msq1, 2.0 / 3.0, 0, st));
  } else {  // Gaussian members of a mixed batch go through the identity map
    RUN(p, 0, Yb + Xb, "unpack (zeta_g)", OPS(p, unpack, N, Y, X, batch, p->d_amp, (long)msq1, 1.0, 0, st));
    RUN(p, 0, Yb + Xb, "pack", OPS(p, pack, N, X, Y, batch, st));
    RUN(p, 0, 2 * Yb, "inverse axis 0", OPS(p, pass, N, Y, 0, +1, batch, p->d_tw, st));
    RUN(p, 0, 2 * Yb, "inverse axis 1", OPS(p, pass, N, Y, 1, +1, batch, p->d_tw, st));
    const double scale = 1.0 / ((double)NN * N * dx * dx * dx);
    RUN(p, 0, Yb + Rb, "rows C2R (zeta_g)", OPS(p, rows_c2r, N, Y, R, batch, scale, p->d_sq, p->d_tw, st));
    const int rb = OPS(p, rows_blocks, N);
    RUN(p, 0, (double)batch * rb * 8, "mean zeta_g^2",
        sigw::launch_reduce_mean(p->d_sq, rb, p->d_mean, batch, 1.0 / ((double)NN * N), st));
    void* R2 = nullptr;
    void* R3 = nullptr;
    if (any_nonlocal) {  // Eq. eq_nonlocal: lap(zeta_g) into R2 and lap(zeta_g^2) into R3
      R2 = (char*)R + (size_t)p->opts.max_batch * NN * N * p->relem();
      R3 = (char*)R2 + (size_t)p->opts.max_batch * NN * N * p->relem();
      const double lap = kf * kf;
      RUN(p, 0, Xb + Yb, "pack lap(zeta_g)", OPS(p, pack, N, X, Y, batch, st, lap));
      RUN(p, 0, 2 * Yb, "inverse axis 0", OPS(p, pass, N, Y, 0, +1, batch, p->d_tw, st));
      RUN(p, 0, 2 * Yb, "inverse axis 1", OPS(p, pass, N, Y, 1, +1, batch, p->d_tw, st));
      RUN(p, 0, Yb + Rb, "rows C2R lap(zeta_g)", OPS(p, rows_c2r, N, Y, R2, batch, scale, nullptr, p->d_tw, st));
      RUN(p, 0, Rb + Yb, "zeta_g^2 rows R2C", OPS(p, rows_r2c_square, N, R, Y, batch, p->d_tw, st));
      RUN(p, 0, 2 * Yb, "forward axis 1", OPS(p, pass, N, Y, 1, -1, batch, p->d_tw, st));
      RUN(p, 0, 2 * Yb, "forward axis 0", OPS(p, pass, N, Y, 0, -1, batch, p->d_tw, st));
      RUN(p, 0, Yb + Xb, "unpack (zeta_g^2)", OPS(p, unpack, N, Y, X, batch, nullptr, 0L, dx * dx * dx, 1, st));
      RUN(p, 0, Xb + Yb, "pack lap(zeta_g^2)", OPS(p, pack, N, X, Y, batch, st, lap));
      RUN(p, 0, 2 * Yb, "inverse axis 0", OPS(p, pass, N, Y, 0, +1, batch, p->d_tw, st));
      RUN(p, 0, 2 * Yb, "inverse axis 1", OPS(p, pass, N, Y, 1, +1, batch, p->d_tw, st));
      RUN(p, 0, Yb + Rb, "rows C2R lap(zeta_g^2)", OPS(p, rows_c2r, N, Y, R3, batch, scale, nullptr, p->d_tw, st));
    }
    CKP(p, cudaMemsetAsync(p->d_hits, 0, sizeof(unsigned long long) * batch, st), "memset hits");
    RUN(p, 0, Rb + Yb + (any_nonlocal ? 2 * Rb : 0.0), "map + rows R2C",
        OPS(p, rows_r2c_map, N, R, Y, batch, p->d_maps, p->d_mean, p->d_hits, p->d_tw, st, R2, R3));
    RUN(p, 0, 2 * Yb, "forward axis 1", OPS(p, pass, N, Y, 1, -1, batch, p->d_tw, st));
    RUN(p, 0, 2 * Yb, "forward axis 0", OPS(p, pass, N, Y, 0, -1, batch, p->d_tw, st));
    RUN(p, 0, Yb + Xb, "unpack (Phi)",
        OPS(p, unpack, N, Y, p->d_phi, batch, nullptr, 0L, (2.0 / 3.0) * dx * dx * dx, 1, st));
  }
  std::vector<unsigned long long> hits(batch, 0);
  if (any_usr) {
    CKP(p, cudaMemcpyAsync(hits.data(), p->d_hits, sizeof(unsigned long long) * batch, cudaMemcpyDeviceToHost, st),
        "download hits");
    p->d2h += sizeof(unsigned long long) * batch;
  }
  CKP(p, cudaStreamSynchronize(st), "synthesis");
  p->generated = batch;
  bool any = false;
  for (int b = 0; b < batch; ++b) {
    if (usr_hits) usr_hits[b] = (int64_t)hits[b];
    any = any || hits[b] > 0;
  }
  if (any && p->opts.strict_domain) return fail(p, SIGW_EDOMAIN, "USR floor hits in strict mode");
  return SIGW_OK;
}

sigw_status sigw_generate(sigw_plan p, const sigw_pzeta* pz, const sigw_ngmap* map, const uint64_t* seeds, int batch,
                          int64_t* usr_hits) {
  if (!p) return SIGW_EINVAL;
  if (!pz || !map || batch < 1 || batch > 64) return fail(p, SIGW_EINVAL, "sigw_generate: bad arguments");
  std::vector<sigw_pzeta> pzs(batch, *pz);
  std::vector<sigw_ngmap> ms(batch, *map);
  return sigw_generate_batch(p, pzs.data(), ms.data(), seeds, batch, usr_hits);
}

// Jackknife scratch of one spectrum call (Sec. sec_envelope_obs): M^3 sub-volumes; per (shell, kernel) the TT
// amplitudes go to Xj (standard half spectra, 2 per realisation), are packed into Yj, inverse-transformed into
// the real fields Rj, and reduced per sub-volume x0-plane into part[(si * 2 + m)][2 batch][M^3][N/M].
struct Jackknife {
  int M = 4;
  double* part = nullptr;
  void* Xj = nullptr;
  void* Yj = nullptr;
  void* Rj = nullptr;
};

// Queue the hot loop for the shells sh (device copies in d_sh / d_nk) writing [batch][ns][4] to out.
static sigw_status enqueue_spectrum(sigw_plan p, const std::vector<int>& sh, const int* d_sh, const double* d_nk,
                                    double* out, const Jackknife* jk = nullptr) {
  const int N = p->N, H = N / 2;
  const int ns = (int)sh.size();
  const int batch = p->generated;
  cudaStream_t st = p->st;
  const int n_alpha = p->opts.n_alpha, nm1 = p->opts.n_modes + 1;
  const size_t NN = (size_t)N * N;
  const size_t cel = p->celem();
  void* Ta = p->d_T;
  void* Tb = (char*)p->d_T + (size_t)batch * p->B * NN * H * cel;
  const int var = p->variant;
  const long pbs = (long)ns * 2 * p->sz.maxblk;
  const double fieldb = (double)batch * NN * H * cel;  // one packed complex field per realisation batch
  const double phib = (double)batch * NN * (H + 1) * cel;
  for (int si = 0; si < ns; ++si) {
    const int n_c = sh[si];
    const int16_t* lut = p->d_lut + (size_t)(n_c - 1) * (p->msq_max + 1);
    const int ncp = n_c + 1;
    const int n1lo = std::max(-n_c, -H + 1), nk1 = std::min(n_c, H) - n1lo + 1;
    // columns (n1, n2) of the F3 pass that reach the shell: n1^2 + n2^2 <= n_c^2 + n_c
    long disk = 0;
    for (int n1 = n1lo; n1 < n1lo + nk1; ++n1)
      for (int n2 = 0; n2 <= n_c; ++n2) disk += (n1 * n1 + n2 * n2 <= n_c * n_c + n_c);
    for (int m = 0; m < 2; ++m) {
      for (int a0 = 0; a0 < n_alpha; a0 += p->B) {
        const int nb = std::min(p->B, n_alpha - a0);
        RUN(p, 1, phib + 2.0 * nb * fieldb, "P1",
            OPS(p, p1, N, p->d_phi, Ta, Tb, lut, p->d_phitab[m], nm1, a0, nb, batch, p->d_tw, var, st));
        RUN(p, 2, 5.0 * nb * fieldb, "P2",
            OPS(p, p2, N, Ta, Tb, p->d_work, n_alpha, a0, nb, batch, p->d_tw, var, st));
      }
      RUN(p, 3, 3.0 * n_alpha * fieldb + 6.0 * batch * NN * ncp * cel, "P3",
          OPS(p, p3, N, p->d_work, p->d_sigma[m], n_alpha, p->d_F, n_c, batch, p->d_tw, p->d_err, p->wait_limit,
              var, st));
      RUN(p, 4, 6.0 * batch * ((double)NN * ncp + (double)N * nk1 * ncp) * cel, "F2",
          OPS(p, f2, N, p->d_F, p->d_F2, n_c, batch, p->d_tw, st));
      if (!jk) {
        RUN(p, 5, 6.0 * batch * (double)N * disk * cel, "F3",
            OPS(p, f3, N, p->d_F2, n_c, p->d_partial + ((long)si * 2 + m) * p->sz.maxblk, pbs, batch, p->d_tw, st));
      } else {
        const double xjb = 2.0 * batch * NN * (H + 1) * cel, yjb = 2.0 * batch * NN * H * cel;
        const double rjb = 2.0 * batch * NN * N * p->relem();
        CKP(p, cudaMemsetAsync(jk->Xj, 0, (size_t)xjb, st), "jackknife zero");
        RUN(p, 5, 6.0 * batch * (double)N * disk * cel, "F3 + amplitudes",
            OPS(p, f3, N, p->d_F2, n_c, p->d_partial + ((long)si * 2 + m) * p->sz.maxblk, pbs, batch, p->d_tw, st,
                jk->Xj));
        RUN(p, 0, xjb + yjb, "jackknife pack", OPS(p, pack, N, jk->Xj, jk->Yj, 2 * batch, st));
        RUN(p, 0, 2 * yjb, "jackknife inverse axis 0", OPS(p, pass, N, jk->Yj, 0, +1, 2 * batch, p->d_tw, st));
        RUN(p, 0, 2 * yjb, "jackknife inverse axis 1", OPS(p, pass, N, jk->Yj, 1, +1, 2 * batch, p->d_tw, st));
        RUN(p, 0, yjb + rjb, "jackknife rows C2R",
            OPS(p, rows_c2r, N, jk->Yj, jk->Rj, 2 * batch, 1.0, nullptr, p->d_tw, st));
        const long per = 2L * batch * jk->M * jk->M * jk->M * (N / jk->M);
        RUN(p, 0, rjb, "jackknife sub-volumes",
            OPS(p, subvol, N, jk->M, jk->Rj, 2 * batch, jk->part + ((long)si * 2 + m) * per, st));
      }
    }
  }
  const sigw::LaunchShape shp = OPS(p, shape, N);
  RUN(p, 6, (double)batch * ns * 2 * p->sz.maxblk * 8, "bin finalise",
      sigw::launch_fin(p->d_partial, pbs, p->sz.maxblk, ns, d_sh, d_nk, N, p->L, shp.tc_f3, out, batch, st));
  return SIGW_OK;
}

// Capture the all-shells loop into a CUDA graph for the current realisation count (thread-local capture mode,
// so CUDA calls of other threads are unaffected).  On any failure graphs stay off for this plan.
static bool capture_all_shells(sigw_plan p, const std::vector<int>& sh) {
  if (p->graph) {
    cudaGraphExecDestroy(p->graph);
    p->graph = nullptr;
  }
  long long l0[SIGW_NKINDS];
  double b0[SIGW_NKINDS];
  std::memcpy(l0, p->launches, sizeof(l0));
  std::memcpy(b0, p->kbytes, sizeof(b0));
  if (cudaStreamBeginCapture(p->st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  const sigw_status s = enqueue_spectrum(p, sh, p->d_shells_all, p->d_Nk_all, p->d_out);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(p->st, &g);
  bool ok = (s == SIGW_OK && e == cudaSuccess && g);
  if (ok) ok = cudaGraphInstantiate(&p->graph, g, 0) == cudaSuccess;
  if (g) cudaGraphDestroy(g);
  (void)cudaGetLastError();
  for (int k = 0; k < SIGW_NKINDS; ++k) {  // what one replay launches; not counted until replayed
    p->graph_launches[k] = p->launches[k] - l0[k];
    p->graph_bytes[k] = p->kbytes[k] - b0[k];
    p->launches[k] = l0[k];
    p->kbytes[k] = b0[k];
  }
  if (!ok) {
    if (p->graph) cudaGraphExecDestroy(p->graph);
    p->graph = nullptr;
    return false;
  }
  p->graph_batch = p->generated;
  return true;
}

sigw_status sigw_spectrum_async(sigw_plan p, const int* shells, int n_shells, double* dev_out) {
  if (!p) return SIGW_EINVAL;
  if (!p->generated) return fail(p, SIGW_ESTATE, "sigw_spectrum before sigw_generate");
  const int N = p->N, H = N / 2;
  std::vector<int> sh;
  if (shells) {
    if (n_shells < 1 || n_shells > H) return fail(p, SIGW_EINVAL, "n_shells out of range");
    sh.assign(shells, shells + n_shells);
  } else {
    for (int s = 1; s <= H; ++s) sh.push_back(s);
  }
  for (int s : sh)
    if (s < 1 || s > H) return fail(p, SIGW_EINVAL, "shell index out of range");
  const int ns = (int)sh.size();
  const int batch = p->generated;
  CKP(p, cudaSetDevice(p->dev), "cudaSetDevice");
  cudaStream_t st = p->st;
  double* out = dev_out ? dev_out : p->d_out;
  if (!shells) {
    // all shells: replay a captured graph (per-kernel event timing needs the direct launches)
    if (!p->prof_on && p->graphs_ok) {
      if (!p->graph || p->graph_batch != batch) p->graphs_ok = capture_all_shells(p, sh);
      if (p->graphs_ok) {
        CKP(p, cudaGraphLaunch(p->graph, st), "graph launch");
        for (int k = 0; k < SIGW_NKINDS; ++k) {
          p->launches[k] += p->graph_launches[k];
          p->kbytes[k] += p->graph_bytes[k];
        }
        if (dev_out)
          CKP(p, cudaMemcpyAsync(dev_out, p->d_out, sizeof(double) * 4 * batch * ns, cudaMemcpyDeviceToDevice, st),
              "copy results");
        return SIGW_OK;
      }
    }
    return enqueue_spectrum(p, sh, p->d_shells_all, p->d_Nk_all, out);
  }
  std::vector<double> nk(ns);
  for (int i = 0; i < ns; ++i) nk[i] = p->Nk[sh[i]];
  CKP(p, cudaMemcpyAsync(p->d_shells, sh.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, st), "upload shells");
  CKP(p, cudaMemcpyAsync(p->d_Nk, nk.data(), sizeof(double) * ns, cudaMemcpyHostToDevice, st), "upload Nk");
  p->h2d += sizeof(int) * ns + sizeof(double) * ns;
  return enqueue_spectrum(p, sh, p->d_shells, p->d_Nk, out);
}

sigw_status sigw_spectrum_jackknife(sigw_plan p, const int* shells, int n_shells, int M, double* omega,
                                    double* sigma_omega, double* PA, double* sigma_PA, double* PB, double* sigma_PB) {
  if (!p) return SIGW_EINVAL;
  if (!p->generated) return fail(p, SIGW_ESTATE, "sigw_spectrum_jackknife before sigw_generate");
  const int N = p->N, H = N / 2;
  if (M < 2 || N % M != 0) return fail(p, SIGW_EINVAL, "jackknife: N must be a multiple of M >= 2");
  std::vector<int> sh;
  if (shells) {
    if (n_shells < 1 || n_shells > H) return fail(p, SIGW_EINVAL, "n_shells out of range");
    sh.assign(shells, shells + n_shells);
  } else {
    for (int s = 1; s < H; ++s) sh.push_back(s);
  }
  for (int s : sh)
    if (s < 1 || s >= H) return fail(p, SIGW_EINVAL, "jackknife shells are 1..N/2-1 (no Nyquist shell)");
  const int ns = (int)sh.size(), batch = p->generated;
  CKP(p, cudaSetDevice(p->dev), "cudaSetDevice");
  cudaStream_t st = p->st;
  const size_t NN = (size_t)N * N, cel = p->celem();
  const int M3 = M * M * M, sv = N / M;
  const size_t per = (size_t)2 * batch * M3 * sv;  // partials per (shell, kernel)
  Jackknife jk;
  jk.M = M;
  jk.Xj = p->d_work;
  jk.Yj = (char*)jk.Xj + (size_t)2 * batch * NN * (H + 1) * cel;
  jk.Rj = (char*)jk.Yj + (size_t)2 * batch * NN * H * cel;
  {
    void* q = nullptr;
    sigw_status s = dev_alloc(p, &q, sizeof(double) * per * 2 * ns);
    if (s != SIGW_OK) return s;
    jk.part = (double*)q;
  }
  auto release = [&]() {  // the buffer lives for this call only
    p->allocs.erase(std::remove(p->allocs.begin(), p->allocs.end(), (void*)jk.part), p->allocs.end());
    cudaFree(jk.part);
  };
  std::vector<double> nk(ns);
  for (int i = 0; i < ns; ++i) nk[i] = p->Nk[sh[i]];
  sigw_status s = SIGW_OK;
  if (cudaMemcpyAsync(p->d_shells, sh.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(p->d_Nk, nk.data(), sizeof(double) * ns, cudaMemcpyHostToDevice, st) != cudaSuccess)
    s = cuda_fail(p, cudaGetLastError(), "upload shells");
  p->h2d += sizeof(int) * ns + sizeof(double) * ns;
  if (s == SIGW_OK) s = enqueue_spectrum(p, sh, p->d_shells, p->d_Nk, p->d_out, &jk);
  std::vector<double> part(per * 2 * ns), res((size_t)batch * ns * 4);
  if (s == SIGW_OK &&
      (cudaMemcpyAsync(part.data(), jk.part, sizeof(double) * part.size(), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
       cudaMemcpyAsync(res.data(), p->d_out, sizeof(double) * res.size(), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
       cudaStreamSynchronize(st) != cudaSuccess))
    s = cuda_fail(p, cudaGetLastError(), "jackknife download");
  p->d2h += sizeof(double) * (part.size() + res.size());
  release();
  if (s != SIGW_OK) return s;
  if ((s = check_err_flag(p)) != SIGW_OK) return s;
  // host: E[m][sub] per (realisation, shell), leave-one-out replicas, jackknife variance (FP64, fixed order)
  const double L = p->L, V = L * L * L, dx = L / N;
  for (int b = 0; b < batch; ++b)
    for (int si = 0; si < ns; ++si) {
      const int n_c = sh[si];
      const double C = 4.0 * dx * dx * dx / ((double)n_c * n_c * V * V);
      const double norm = C * C / ((double)NN * N * V * p->Nk[n_c]);
      const double kc = n_c * 2.0 * kPi / L;
      std::vector<double> rep[3];
      double Etot[2] = {0.0, 0.0};
      std::vector<double> E[2] = {std::vector<double>(M3, 0.0), std::vector<double>(M3, 0.0)};
      for (int m = 0; m < 2; ++m)
        for (int f = 0; f < 2; ++f)
          for (int u = 0; u < M3; ++u) {
            const double* q = part.data() + ((size_t)(si * 2 + m) * 2 * batch + (size_t)(b * 2 + f)) * M3 * sv +
                              (size_t)u * sv;
            double t = 0.0;
            for (int x = 0; x < sv; ++x) t += q[x];
            E[m][u] += t;
          }
      for (int m = 0; m < 2; ++m)
        for (int u = 0; u < M3; ++u) Etot[m] += E[m][u];
      for (int u = 0; u < M3; ++u) {
        const double pa = norm * (Etot[0] - E[0][u]) / (1.0 - 1.0 / M3);
        const double pb = norm * (Etot[1] - E[1][u]) / (1.0 - 1.0 / M3);
        rep[0].push_back(pa);
        rep[1].push_back(pb);
        rep[2].push_back(kc * kc * kc / (48.0 * kPi * kPi) * (pa + pb));
      }
      double mean[3], sig[3];
      for (int q = 0; q < 3; ++q) {
        double mu = 0.0;
        for (double v : rep[q]) mu += v;
        mu /= M3;
        double ss = 0.0;
        for (double v : rep[q]) ss += (v - mu) * (v - mu);
        mean[q] = mu;
        sig[q] = std::sqrt((double)(M3 - 1) / M3 * ss);
      }
      const size_t o = (size_t)b * ns + si;
      if (PA) PA[o] = mean[0];
      if (PB) PB[o] = mean[1];
      if (omega) omega[o] = mean[2];
      if (sigma_PA) sigma_PA[o] = sig[0];
      if (sigma_PB) sigma_PB[o] = sig[1];
      if (sigma_omega) sigma_omega[o] = sig[2];
    }
  return SIGW_OK;
}

sigw_status sigw_spectrum(sigw_plan p, const int* shells, int n_shells, double* omega, double* PA, double* PB,
                          int64_t* Nk) {
  if (!p) return SIGW_EINVAL;
  sigw_status s = sigw_spectrum_async(p, shells, n_shells, nullptr);
  if (s != SIGW_OK) return s;
  const int ns = shells ? n_shells : p->N / 2;
  const int batch = p->generated;
  std::vector<double> host((size_t)batch * ns * 4);
  CKP(p, cudaMemcpyAsync(host.data(), p->d_out, host.size() * sizeof(double), cudaMemcpyDeviceToHost, p->st),
      "download results");
  p->d2h += host.size() * sizeof(double);
  CKP(p, cudaStreamSynchronize(p->st), "spectrum");
  {
    sigw_status fs = check_err_flag(p);
    if (fs != SIGW_OK) return fs;
  }
  for (int i = 0; i < batch * ns; ++i) {
    if (PA) PA[i] = host[4 * i + 0];
    if (PB) PB[i] = host[4 * i + 1];
    if (Nk) Nk[i] = (int64_t)host[4 * i + 2];
    if (omega) omega[i] = host[4 * i + 3];
  }
  return SIGW_OK;
}

sigw_status sigw_copy_phi(sigw_plan p, int b, void* host_out) {
  if (!p || !host_out) return SIGW_EINVAL;
  if (b < 0 || b >= p->generated) return fail(p, SIGW_ESTATE, "no generated field for this index");
  const int N = p->N;
  const size_t bytes = (size_t)N * N * (N / 2 + 1) * p->celem();
  CKP(p, cudaSetDevice(p->dev), "cudaSetDevice");
  CKP(p, cudaMemcpyAsync(host_out, (char*)p->d_phi + (size_t)b * bytes, bytes, cudaMemcpyDeviceToHost, p->st),
      "copy Phi");
  CKP(p, cudaStreamSynchronize(p->st), "copy Phi");
  return SIGW_OK;
}

sigw_status sigw_fft3d(sigw_plan p, int direction, const void* in_dev, void* out_dev) {
  if (!p || !in_dev || !out_dev || (direction != -1 && direction != 1)) return SIGW_EINVAL;
  CKP(p, cudaSetDevice(p->dev), "cudaSetDevice");
  const int N = p->N;
  void* Y = p->d_work;
  cudaStream_t st = p->st;
  if (direction < 0) {
    RUN(p, 0, 0, "rows R2C", OPS(p, rows_r2c_real, N, in_dev, Y, 1, p->d_tw, st));
    RUN(p, 0, 0, "forward axis 1", OPS(p, pass, N, Y, 1, -1, 1, p->d_tw, st));
    RUN(p, 0, 0, "forward axis 0", OPS(p, pass, N, Y, 0, -1, 1, p->d_tw, st));
    RUN(p, 0, 0, "unpack", OPS(p, unpack, N, Y, out_dev, 1, nullptr, 0L, 1.0, 1, st));
  } else {
    RUN(p, 0, 0, "pack", OPS(p, pack, N, in_dev, Y, 1, st));
    RUN(p, 0, 0, "inverse axis 0", OPS(p, pass, N, Y, 0, +1, 1, p->d_tw, st));
    RUN(p, 0, 0, "inverse axis 1", OPS(p, pass, N, Y, 1, +1, 1, p->d_tw, st));
    RUN(p, 0, 0, "rows C2R", OPS(p, rows_c2r, N, Y, out_dev, 1, 1.0, nullptr, p->d_tw, st));
  }
  return SIGW_OK;
}

sigw_status sigw_plan_autotune(sigw_plan p, int n_c, int* out_alpha_batch, int* out_variant, double* out_ms) {
  if (!p) return SIGW_EINVAL;
  if (!p->generated) return fail(p, SIGW_ESTATE, "sigw_plan_autotune needs a generated field");
  const int N = p->N, H = N / 2;
  if (n_c == 0) n_c = std::max(1, H / 2);
  if (n_c < 1 || n_c > H) return fail(p, SIGW_EINVAL, "autotune shell out of range");
  CKP(p, cudaSetDevice(p->dev), "cudaSetDevice");
  const int batch = p->generated, n_alpha = p->opts.n_alpha, nm1 = p->opts.n_modes + 1;
  const size_t NN = (size_t)N * N, cel = p->celem();
  const int16_t* lut = p->d_lut + (size_t)(n_c - 1) * (p->msq_max + 1);
  const int bmax = max_alpha_batch(p->opts);
  const int nvar = OPS(p, variants, N);
  cudaStream_t st = p->st;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CKP(p, cudaEventCreate(&e0), "event");
  CKP(p, cudaEventCreate(&e1), "event");
  double best = 1e300;
  int bestB = p->B, bestV = p->variant & 21;
  const int cands[] = {4, 5, 8, 10, 16};
  sigw_status status = SIGW_OK;
  // For each terms-per-launch candidate the two strided passes are timed separately (each with both radix
  // variants, bit 0 for the first pass and bit 2 for the second), so the best pair is found in 2 x nvar runs.
  auto time_pass = [&](int which, int B, int v, float* ms) -> sigw_status {
    void* Ta = p->d_T;
    void* Tb = (char*)p->d_T + (size_t)batch * B * NN * H * cel;
    for (int rep = 0; rep < 2; ++rep) {  // first pass warms the variant; the second is timed
      cudaEventRecord(e0, st);
      for (int a0 = 0; a0 < n_alpha; a0 += B) {
        const int nb = std::min(B, n_alpha - a0);
        cudaError_t e = which == 0
                            ? OPS(p, p1, N, p->d_phi, Ta, Tb, lut, p->d_phitab[0], nm1, a0, nb, batch, p->d_tw, v, st)
                            : OPS(p, p2, N, Ta, Tb, p->d_work, n_alpha, a0, nb, batch, p->d_tw, v << 2, st);
        if (e != cudaSuccess) return cuda_fail(p, e, "autotune launch");
      }
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(ms, e0, e1) != cudaSuccess)
        return cuda_fail(p, cudaGetLastError(), "autotune timing");
    }
    return SIGW_OK;
  };
  // first-pass candidates: the two radix forms and, where it exists, the radix-16 form with its tile in TMEM
  const bool p1tm = p->opts.precision == 32 && (N == 128 || N == 256 || N == 512);
  const int p1bits[3] = {0, 1, 16};
  const int np1 = nvar + (p1tm ? 1 : 0);
  for (int B : cands) {
    if (p->opts.alpha_batch > 0) B = bmax;  // terms per launch fixed by the options: tune the radices only
    if (B > bmax || status != SIGW_OK) continue;
    float t1[3] = {1e30f, 1e30f, 1e30f}, t2[2] = {1e30f, 1e30f};
    for (int v = 0; v < np1 && status == SIGW_OK; ++v) {
      const int bits = (v == nvar) ? 16 : p1bits[v];
      status = time_pass(0, B, bits, &t1[v]);  // P1 writes the T that P2 reads next
      if (status == SIGW_OK && v < nvar) status = time_pass(1, B, v, &t2[v]);
    }
    if (status != SIGW_OK) break;
    int v1 = 0;
    for (int v = 1; v < np1; ++v)
      if (t1[v] < t1[v1]) v1 = v;
    const int v2 = t2[1] < t2[0] ? 1 : 0;
    const double ms = (double)t1[v1] + (double)t2[v2];
    if (ms < best) {
      best = ms;
      bestB = B;
      bestV = (v1 == nvar ? 16 : p1bits[v1]) | (v2 << 2);
    }
    if (p->opts.alpha_batch > 0) break;
  }
  // last inverse pass: radix variants on the W just produced by the best strided choice
  int bestP3 = 0;
  if (status == SIGW_OK && OPS(p, p3_variants, N) > 1) {
    {
      void* Ta = p->d_T;
      void* Tb = (char*)p->d_T + (size_t)batch * bestB * NN * H * cel;
      for (int a0 = 0; a0 < n_alpha && status == SIGW_OK; a0 += bestB) {
        const int nb = std::min(bestB, n_alpha - a0);
        cudaError_t e = OPS(p, p1, N, p->d_phi, Ta, Tb, lut, p->d_phitab[0], nm1, a0, nb, batch, p->d_tw, bestV, st);
        if (e == cudaSuccess) e = OPS(p, p2, N, Ta, Tb, p->d_work, n_alpha, a0, nb, batch, p->d_tw, bestV, st);
        if (e != cudaSuccess) status = cuda_fail(p, e, "autotune launch");
      }
    }
    const int np3 = OPS(p, p3_variants, N);  // 2: radix 8 / 16; 3: also radix 16 with TMEM accumulators
    const int p3bits[3] = {0, 2, 8};
    float t3[3] = {1e30f, 1e30f, 1e30f};
    for (int v3 = 0; v3 < np3 && status == SIGW_OK; ++v3) {
      for (int rep = 0; rep < 2; ++rep) {
        cudaEventRecord(e0, st);
        cudaError_t e = OPS(p, p3, N, p->d_work, p->d_sigma[0], n_alpha, p->d_F, n_c, batch, p->d_tw, p->d_err,
                            sigw::kDefaultWaitLimit, p3bits[v3], st);
        cudaEventRecord(e1, st);
        if (e != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&t3[v3], e0, e1) != cudaSuccess) {
          status = cuda_fail(p, e != cudaSuccess ? e : cudaGetLastError(), "autotune last pass");
          break;
        }
      }
    }
    int bv = 0;
    for (int v3 = 1; v3 < np3; ++v3)
      if (t3[v3] < t3[bv]) bv = v3;
    if (status == SIGW_OK) {
      bestP3 = p3bits[bv];
      best += t3[bv];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (status != SIGW_OK) return status;
  p->B = bestB;
  p->variant = bestV | bestP3;
  if (p->graph) {  // the captured loop used the old choice
    cudaGraphExecDestroy(p->graph);
    p->graph = nullptr;
  }
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[TuneKey{N, p->opts.precision, p->opts.max_batch, n_alpha}] = {bestB, bestV | bestP3};
  }
  if (out_alpha_batch) *out_alpha_batch = bestB;
  if (out_variant) *out_variant = bestV | bestP3;
  if (out_ms) *out_ms = best;
  return SIGW_OK;
}

// ---- per-target box (Sec. sec_numerical)
static double erfinv_bisect(double x) {  // erf(y) = x for x in (-1, 1), by bisection on the monotone erf
  double lo = -7.0, hi = 7.0;
  for (int i = 0; i < 200 && hi - lo > 1e-16; ++i) {
    const double mid = 0.5 * (lo + hi);
    (std::erf(mid) < x ? lo : hi) = mid;
  }
  return 0.5 * (lo + hi);
}

sigw_status sigw_target_box(int N, double k, const sigw_pzeta* pz, double eps, double* L, int* n_c) {
  if (!pz || !L || !n_c || !is_pow2_in_range(N) || !(k > 0) || !(eps > 0 && eps < 1) || !(pz->kstar > 0) ||
      !(pz->sigma > 0))
    return SIGW_EINVAL;
  const double kbar = pz->kstar * std::exp(pz->sigma * std::sqrt(2.0) * erfinv_bisect(1.0 - 2.0 * eps));
  const double kmax = 3.0 * std::max(k, kbar);
  const double Lrule = kPi * N / kmax;
  long nc = std::lround(k * Lrule / (2.0 * kPi));
  nc = std::max(1L, std::min((long)(N / 2), nc));
  *n_c = (int)nc;
  *L = 2.0 * kPi * (double)nc / k;
  return SIGW_OK;
}

sigw_status sigw_plan_set_box(sigw_plan p, double L) {
  if (!p) return SIGW_EINVAL;
  if (!(L > 0) || !std::isfinite(L)) return fail(p, SIGW_EINVAL, "sigw_plan_set_box: L must be positive");
  CKP(p, cudaSetDevice(p->dev), "cudaSetDevice");
  CKP(p, cudaStreamSynchronize(p->st), "set_box");
  p->L = L;
  p->generated = 0;
  if (p->graph) {  // the captured finalisation holds the old L
    cudaGraphExecDestroy(p->graph);
    p->graph = nullptr;
  }
  return SIGW_OK;
}

sigw_status sigw_target_scan(sigw_plan p, const sigw_pzeta* pz, const sigw_ngmap* map, uint64_t seed,
                             const double* k, int n_k, double eps, double* omega, double* L_out, int* nc_out) {
  if (!p) return SIGW_EINVAL;
  if (!pz || !map || !k || n_k < 1) return fail(p, SIGW_EINVAL, "sigw_target_scan: bad arguments");
  for (int i = 0; i < n_k; ++i) {
    double L = 0.0;
    int nc = 0;
    if (sigw_target_box(p->N, k[i], pz, eps, &L, &nc) != SIGW_OK)
      return fail(p, SIGW_EINVAL, "sigw_target_scan: bad target or P_zeta");
    sigw_status s = sigw_plan_set_box(p, L);
    if (s == SIGW_OK) s = sigw_generate(p, pz, map, &seed, 1, nullptr);
    double om = 0.0;
    if (s == SIGW_OK) s = sigw_spectrum(p, &nc, 1, &om, nullptr, nullptr, nullptr);
    if (s != SIGW_OK) return s;
    if (omega) omega[i] = om;
    if (L_out) L_out[i] = L;
    if (nc_out) nc_out[i] = nc;
  }
  return SIGW_OK;
}

sigw_status sigw_plan_set_tuning(sigw_plan p, int alpha_batch, int variant) {
  if (!p) return SIGW_EINVAL;
  if (alpha_batch < 1 || alpha_batch > max_alpha_batch(p->opts) || variant < 0 || variant > 31)
    return fail(p, SIGW_EINVAL, "sigw_plan_set_tuning: alpha_batch or variant out of range");
  CKP(p, cudaSetDevice(p->dev), "cudaSetDevice");
  CKP(p, cudaStreamSynchronize(p->st), "set_tuning");
  p->B = alpha_batch;
  p->variant = variant;
  if (p->graph) {  // the captured loop used the old choice
    cudaGraphExecDestroy(p->graph);
    p->graph = nullptr;
  }
  return SIGW_OK;
}

sigw_status sigw_plan_debug_wait_limit(sigw_plan p, long long cycles) {
  if (!p || cycles < 0) return SIGW_EINVAL;
  p->wait_limit = cycles > 0 ? cycles : sigw::kDefaultWaitLimit;
  if (p->graph) {  // a captured graph holds the old limit in its kernel arguments
    cudaGraphExecDestroy(p->graph);
    p->graph = nullptr;
  }
  return SIGW_OK;
}

sigw_status sigw_plan_profile(sigw_plan p, int enable) {
  if (!p) return SIGW_EINVAL;
  CKP(p, cudaSetDevice(p->dev), "cudaSetDevice");
  CKP(p, cudaStreamSynchronize(p->st), "profile");
  prof_reset(p);
  p->prof_on = enable != 0;
  return SIGW_OK;
}

sigw_status sigw_plan_profile_read(sigw_plan p, sigw_profile* out) {
  if (!p || !out) return SIGW_EINVAL;
  CKP(p, cudaSetDevice(p->dev), "cudaSetDevice");
  CKP(p, cudaStreamSynchronize(p->st), "profile read");
  std::memset(out, 0, sizeof(*out));
  for (auto& r : p->recs) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) out->ms[r.kind] += ms;
    (void)cudaGetLastError();
  }
  for (int k = 0; k < SIGW_NKINDS; ++k) {
    out->bytes[k] = p->kbytes[k];
    out->launches[k] = p->launches[k];
  }
  out->h2d_bytes = p->h2d;
  out->d2h_bytes = p->d2h;
  prof_reset(p);
  return SIGW_OK;
}

}  // extern "C"
