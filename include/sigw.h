/*
 * sigw.h -- C ABI of the GB300 (sm_103a) lattice SIGW library.
 *
 * The library evaluates the scalar-induced gravitational-wave spectrum of a
 * (possibly non-Gaussian) curvature field on a periodic N^3 lattice by the
 * method of arXiv 2605.27231 (Piccoli, "A Fast Method to Compute Scalar Induced
 * Gravitational Waves on a Lattice with Primordial Non-Gaussianities"):
 *
 *   1. a Gaussian field zeta_g with the log-normal Delta^2_zeta of Eq. eq_lognormal
 *      (Sec. sec_numerical) is drawn on the lattice;
 *   2. a pointwise map zeta = F(zeta_g) (local F_NL/G_NL of Sec. "Local
 *      Non-Gaussianities", or the USR tail -1/3 ln(1-3 zeta_g)) gives
 *      Phi = 2 zeta / 3 (Sec. sec_sigw);
 *   3. for each target shell k_c the envelopes A, B of Eq. eq_final_envelopes are
 *      evaluated as a sum of N_alpha separable FFT convolutions built from the
 *      eigen-decomposition of the kernels I_s, I_c (Eqs. eq_kernels,
 *      eq_decomposition, eq_diagonalization, eq_C_matrix_discrete,
 *      eq_grid_density), projected on the TT polarisations (Sec. sec_sigw);
 *   4. |A|^2 and |B|^2 are shell-averaged into P_A, P_B and
 *      Omega(k_c) = k_c^3 / (48 pi^2) sum_l [P_A,l + P_B,l] (Sec. sec_envelope_obs).
 *
 * Conventions shared by every entry point
 *   - N is a power of two, 8 <= N <= 512; L > 0 is the box side; k_f = 2 pi / L.
 *   - Shells are n_c = 1..N/2 (k_c = n_c k_f), a shell holding the modes with
 *     |n| in [n_c - 1/2, n_c + 1/2) of the full lattice n in (-N/2, N/2]^3.
 *   - Every call returns a sigw_status and never aborts the process.  The text
 *     of the last failure on a plan is kept (sigw_plan_last_error).
 *   - The library owns all device memory it allocates (cudaMalloc at
 *     sigw_plan_create, freed by sigw_plan_destroy).  Host arrays passed in are
 *     owned by the caller and only read or written during the call.
 *   - A plan is used from one host thread at a time; its work is queued on the
 *     CUDA stream given at creation (or one it creates).  A server is thread-safe.
 *   - Arrays indexed [batch][shell] are row-major.
 */
#ifndef SIGW_H
#define SIGW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SIGW_ABI_VERSION 1

typedef enum sigw_status {
  SIGW_OK = 0,
  SIGW_EINVAL = 1,    /* an argument is out of range or NULL where required */
  SIGW_ENOMEM = 2,    /* a device or host allocation failed */
  SIGW_ECUDA = 3,     /* a CUDA runtime call or kernel failed (text in last_error) */
  SIGW_EDOMAIN = 4,   /* USR map argument 1 - 3 zeta_g fell below the floor (strict mode only) */
  SIGW_ETIMEOUT = 5,  /* a bounded wait ran out */
  SIGW_EBUSY = 6,     /* server admission refused: the request does not fit the HBM budget */
  SIGW_ENOTREADY = 7, /* result not available yet (sigw_poll) */
  SIGW_ESTATE = 8     /* call out of order (e.g. sigw_spectrum before sigw_generate) */
} sigw_status;

typedef struct sigw_plan_s* sigw_plan;
typedef struct sigw_server_s* sigw_server;

/* Log-normal peak of Eq. eq_lognormal: Delta^2(k) = A / sqrt(2 pi sigma^2) exp(-ln^2(k/kstar) / (2 sigma^2)).
 * kstar is an absolute wave number (units 1/length, same length unit as L). */
typedef struct sigw_pzeta {
  double A, sigma, kstar;
} sigw_pzeta;

typedef enum sigw_mapkind {
  SIGW_MAP_GAUSS = 0, /* zeta = zeta_g (no FFT round trip) */
  SIGW_MAP_LOCAL = 1, /* zeta = zeta_g + F_NL (zeta_g^2 - <zeta_g^2>) + G_NL zeta_g^3, <.> the box mean */
  SIGW_MAP_USR = 2,   /* zeta = -1/3 ln(max(1 - 3 zeta_g, usr_floor)); hits below the floor are counted */
  SIGW_MAP_NONLOCAL = 3 /* Eq. eq_nonlocal: zeta = zeta_g + alpha_NL / k*^2 lap(zeta_g^2) + beta_NL / k*^2 zeta_g
                         * lap(zeta_g), k* the peak of P_zeta; lap is the spectral Laplacian -|k|^2 with
                         * n_j = +N/2 on Nyquist indices (two extra FFT round trips) */
} sigw_mapkind;

/* F_NL is the coefficient of zeta_g^2 (F_NL = 3/5 f_NL); alpha_NL, beta_NL are used by SIGW_MAP_NONLOCAL only. */
typedef struct sigw_ngmap {
  int kind;
  double F_NL, G_NL;
  double usr_floor; /* > 0; 1e-6 if 0 is given */
  double alpha_NL, beta_NL;
} sigw_ngmap;

/* Plan options.  sigw_opts_default fills the paper's decomposition meta-parameters
 * (Fig. fig_eigenvalues caption, Sec. sec_numerical): n_modes = 200, n_alpha = 50,
 * umin = 1e-3, umax = 15, upiv = 1, sigp = 0.5, Ap = 10; precision 32; alpha_batch 0 (auto);
 * max_batch 1; strict_domain 0. */
typedef struct sigw_opts {
  int n_modes;        /* cells of the u-grid (N_modes) */
  int n_alpha;        /* separable terms kept (N_alpha), 1 <= n_alpha <= n_modes */
  double umin, umax;  /* u-grid range */
  double upiv, sigp, Ap; /* grid density bump of Eq. eq_grid_density */
  int precision;      /* 32: FP32 fields and FFTs (FP64 plan, twiddles and bin sums); 64: FP64 throughout */
  int alpha_batch;    /* terms per first/second-pass launch; 0 picks a value */
  int max_batch;      /* most realisations handled by one sigw_generate / sigw_spectrum call */
  int strict_domain;  /* nonzero: USR floor hits make sigw_generate return SIGW_EDOMAIN */
} sigw_opts;

/* Fill *o with the defaults above.  Returns SIGW_EINVAL if o is NULL. */
sigw_status sigw_opts_default(sigw_opts* o);

/* Device memory (bytes) a plan with these arguments allocates.  opts may be NULL (defaults). */
sigw_status sigw_plan_footprint(int N, const sigw_opts* opts, size_t* bytes);

/* "sigw_plan": build the kernel decomposition (Sec. sec_decomposition: u-grid, C matrices,
 * Jacobi eigen-decomposition, truncation to n_alpha by |sigma|), the per-shell cell tables,
 * the FFT twiddles (FP64 generated) and the device buffers for up to opts->max_batch
 * realisations.  cuda_stream is a cudaStream_t (NULL: the plan creates its own stream).
 * Errors: SIGW_EINVAL (N not a power of two in [8, 512], L <= 0, bad opts),
 * SIGW_ENOMEM (device allocation), SIGW_ECUDA. */
sigw_status sigw_plan_create(int N, double L, const sigw_opts* opts, void* cuda_stream, sigw_plan* out);
sigw_status sigw_plan_destroy(sigw_plan plan);
const char* sigw_plan_last_error(sigw_plan plan);

/* The truncated separable terms of kernel m (0: I_s / envelope A, 1: I_c / envelope B), Eq. eq_decomposition:
 * sigma[n_alpha] eigenvalues sorted by |sigma| descending, phi[n_alpha * n_modes] the value of phi_a on
 * each cell (row-major [a][cell]), edges[n_modes + 1] the cell edges of the u-grid.  Any pointer may be NULL. */
sigw_status sigw_plan_kernel_terms(sigw_plan plan, int m, double* sigma, double* phi, double* edges);

/* Synthesis (steps 1-2 above) for `batch` realisations, seeds[b] the Philox4x32-10 key of realisation b
 * (noise g(x) ~ N(0,1) per cell from counter (cell, 0, 0, 0), Box-Muller in FP64).  Leaves Phi~ resident
 * on the device.  usr_hits (nullable, host, [batch]) receives the USR floor-hit counts.  Waits for the stream.
 * Errors: SIGW_EINVAL (batch out of [1, max_batch], bad parameters), SIGW_EDOMAIN (strict mode), SIGW_ECUDA. */
sigw_status sigw_generate(sigw_plan plan, const sigw_pzeta* pz, const sigw_ngmap* map, const uint64_t* seeds,
                          int batch, int64_t* usr_hits);

/* As sigw_generate, with its own P_zeta parameters and map per realisation: pz[batch], maps[batch].  A batch that
 * mixes Gaussian and non-Gaussian members sends the Gaussian ones through the identity map (their Phi~ then
 * differs from the Gaussian-only route by round-off).  Same errors as sigw_generate. */
sigw_status sigw_generate_batch(sigw_plan plan, const sigw_pzeta* pz, const sigw_ngmap* maps, const uint64_t* seeds,
                                int batch, int64_t* usr_hits);

/* Envelopes, TT projection and shell binning (steps 3-4) for the realisations of the last sigw_generate.
 * shells: n_shells shell indices in [1, N/2] (NULL: all N/2 in order).  Host outputs, [batch][n_shells],
 * any may be NULL: omega (Omega_GW), PA, PB (P_A, P_B summed over polarisations), Nk (modes per shell).
 * Waits for the stream.  Errors: SIGW_ESTATE (no generated field), SIGW_EINVAL, SIGW_ECUDA. */
sigw_status sigw_spectrum(sigw_plan plan, const int* shells, int n_shells, double* omega, double* PA, double* PB,
                          int64_t* Nk);

/* Jackknife error bars (Sec. sec_envelope_obs): as sigw_spectrum, and for every shell the TT fields A_l, B_l on
 * the shell modes are transformed to real space, the box is split into M^3 equal sub-volumes (M = 4 in the
 * paper; N must be a multiple of M), and M^3 leave-one-out estimates P^(i) = (E - E_i) / ((1 - M^-3) V N_k) are
 * formed from the real-space energies (E_i: sub-volume i, E: total).  sigma^2 = (M^3 - 1)/M^3 sum_i
 * (P^(i) - P_bar)^2 for P_A, P_B and Omega.  The replica means equal the plain shell estimates (Parseval).
 * shells: 1..N/2-1 (the Nyquist shell is not offered), NULL for all of them.  Host outputs [batch][n_shells], any
 * may be NULL.  Allocates a partials buffer for the call (2 x 2 batch x M^3 x N/M doubles per shell).
 * Errors: SIGW_ESTATE, SIGW_EINVAL, SIGW_ENOMEM, SIGW_ECUDA. */
sigw_status sigw_spectrum_jackknife(sigw_plan plan, const int* shells, int n_shells, int M, double* omega,
                                    double* sigma_omega, double* PA, double* sigma_PA, double* PB, double* sigma_PB);

/* As sigw_spectrum, but only queues the work on the plan's stream and writes device memory:
 * dev_out (device, [batch][n_shells][4] doubles: P_A, P_B, N_k, Omega).  n_shells <= N/2. */
sigw_status sigw_spectrum_async(sigw_plan plan, const int* shells, int n_shells, double* dev_out);

/* ---- The paper's per-target box (Sec. sec_numerical) ----
 * The paper evaluates each target frequency k in its own box: L = pi N / k_max with k_max = 3 max(k, k_bar),
 * where k_bar is the (1 - eps) quantile of the integral of Delta^2_zeta over ln k (eps = 0.1 in the paper).
 * Reading used here (the paper is silent on placing k on the lattice): the target shell is
 * n_c = round(k L / 2 pi) clamped to [1, N/2], and the box is then set to L = 2 pi n_c / k so that k_c = k exactly.
 * For the log-normal of Eq. eq_lognormal, ln k_bar = ln k* + sigma sqrt(2) erfinv(1 - 2 eps).
 * Host only.  Outputs: *L (box side), *n_c (target shell).  Errors: SIGW_EINVAL (N, k <= 0, eps not in (0, 1),
 * bad P_zeta). */
sigw_status sigw_target_box(int N, double k, const sigw_pzeta* pz, double eps, double* L, int* n_c);

/* Changes the plan's box side to L > 0 (the lattice size N stays).  The next sigw_spectrum needs a new
 * sigw_generate, since P_zeta on the lattice depends on L.  Errors: SIGW_EINVAL. */
sigw_status sigw_plan_set_box(sigw_plan plan, double L);

/* The paper's frequency scan: for each of n_k target wavenumbers k[i] (absolute, 1/length), its own box
 * (sigw_target_box with eps), one realisation with the given seed, and Omega_GW at k[i] (the one shell n_c).
 * Host outputs [n_k], any may be NULL: omega, L_out (box side used), nc_out (shell).  The plan's box is left at
 * the last target's.  Same errors as sigw_generate / sigw_spectrum. */
sigw_status sigw_target_scan(sigw_plan plan, const sigw_pzeta* pz, const sigw_ngmap* map, uint64_t seed,
                             const double* k, int n_k, double eps, double* omega, double* L_out, int* nc_out);

/* Copy Phi~ of realisation b to host memory in the standard half-spectrum layout
 * [k0][k1][k2], k2 = 0..N/2 (N*N*(N/2+1) complex values of the plan precision: float or double pairs),
 * continuum normalisation X~(k) = dx^3 sum_x X(x) e^{-ik.x}. */
sigw_status sigw_copy_phi(sigw_plan plan, int b, void* host_out);

/* The library's 3-D real FFT on device buffers of the plan precision (test and utility entry point).
 * direction -1: real in[N][N][N] -> complex out[N][N][N/2+1] (unnormalised forward DFT);
 * direction +1: complex in -> real out (unnormalised inverse DFT; in is not modified).  Queued on the
 * plan's stream; does not wait. */
sigw_status sigw_fft3d(sigw_plan plan, int direction, const void* in_dev, void* out_dev);

/* Block the calling thread until the plan's stream is idle. */
sigw_status sigw_synchronize(sigw_plan plan);

/* Human-readable text of a status code. */
const char* sigw_strerror(sigw_status s);

/* ---------------------------------------------------------------- serving
 * A server keeps plans resident on the current device and batches spectrum requests as they arrive
 * (continuous batching): max_slots worker threads each take the oldest admissible request together with
 * queued requests of the same size class (N, L), up to opts->max_batch, and run them as one batch on a plan of
 * a shared pool; plans own their streams, so slots overlap on the device.  A plan is created only if its
 * footprint (sigw_plan_footprint) fits hbm_budget_bytes beside the resident plans.  Only the oldest queued
 * request may evict idle plans (least-recently-used first, and only if that frees enough); later requests may
 * allocate only budget that is free and not needed by the oldest one, and start nothing while the oldest one
 * cannot be admitted even by eviction (no starvation).
 * All server calls are thread-safe.  No counterpart in the paper (which reports single timings,
 * Sec. sec_conclusions); this is the serving layer around its method. */
typedef struct sigw_server_stats {
  uint64_t submitted, completed, failed, queued, batches, plans_created, plans_evicted, plans_resident;
  size_t hbm_in_use, hbm_peak, hbm_budget;
  uint64_t express_batches; /* batches run by express slots */
} sigw_server_stats;

/* opts: plan options of every plan (NULL: defaults; max_batch is the per-batch cap).  Errors: SIGW_EINVAL. */
sigw_status sigw_server_create(size_t hbm_budget_bytes, int max_slots, const sigw_opts* opts, sigw_server* out);

/* "sigw_submit": queue one request (one seed); *ticket identifies it.  SIGW_EBUSY if a plan for N alone does not
 * fit the budget (the request could never run); SIGW_EINVAL for bad arguments. */
sigw_status sigw_submit(sigw_server srv, int N, double L, const sigw_pzeta* pz, const sigw_ngmap* map, uint64_t seed,
                        uint64_t* ticket);

/* Non-blocking: SIGW_ENOTREADY until the request is done; then copies Omega (N/2 doubles, nullable) and the
 * latency (seconds from submission to completion, nullable), returns the request's status and forgets the
 * ticket.  SIGW_EINVAL for an unknown ticket. */
sigw_status sigw_poll(sigw_server srv, uint64_t ticket, double* omega, double* latency_s);

/* As sigw_poll, but waits up to timeout_s seconds; SIGW_ETIMEOUT if the request is still not done.  If another
 * thread takes the result first (sigw_poll or sigw_wait on the same ticket), this call returns SIGW_EINVAL. */
sigw_status sigw_wait(sigw_server srv, uint64_t ticket, double timeout_s, double* omega, double* latency_s);

sigw_status sigw_server_stats_read(sigw_server srv, sigw_server_stats* out);

/* Adds `slots` express worker slots (once per server) that take only requests with N <= max_N, in arrival order,
 * under the same pool, budget and admission rule; small requests then need not wait for a general slot held by
 * batches of large lattices (their kernels also run on higher-priority streams).  Errors: SIGW_EINVAL
 * (slots not in [1, 16], max_N not in [8, 512]), SIGW_ESTATE (already set). */
sigw_status sigw_server_set_express(sigw_server srv, int slots, int max_N);

/* Finishes running batches, drops queued requests, frees every plan. */
sigw_status sigw_server_destroy(sigw_server srv);

/* Autotuner (no counterpart in the paper).  On the plan's current field, times the two strided inverse passes of
 * one target shell (n_c; 0 picks N/4) for every candidate choice: terms per launch in {4, 5, 8, 10, 16} (at most
 * n_alpha; exactly opts->alpha_batch when that is set) and, where two exist (FP32, N >= 128), both radix
 * variants of the strided passes.  Keeps the fastest in the plan and in a process-wide table keyed by
 * (N, precision, max_batch, n_alpha) from which later plans with alpha_batch = 0 start; then times both radix
 * forms of the last inverse pass (FP32, N = 128, 256, 512) on the terms just produced; at FP32 N = 128, 256, 512 it
 * also times the first pass with its Phi~ tile and cells in tensor memory and the radix-16 last pass with its
 * accumulators in tensor memory.  An untuned FP32 plan starts from the bits measured fastest on GB300 (26 at
 * N = 128 and 256, 15 at N = 512).  Outputs nullable: chosen terms per launch, variant bits (1: alternative radix of
 * the first strided pass, 2: radix-16 last pass, 4: alternative radix of the second strided pass, 8: radix-16 last
 * pass with its accumulators in tensor memory, 16: first pass with its tile in tensor memory) and the time in ms of the
 * chosen strided passes plus last pass for one kernel (m = s).  Waits for the stream.
 * Errors: SIGW_ESTATE (no field), SIGW_EINVAL, SIGW_ECUDA. */
sigw_status sigw_plan_autotune(sigw_plan plan, int n_c, int* out_alpha_batch, int* out_variant, double* out_ms);

/* Sets the tuned choices directly (for example to replay a choice sigw_plan_autotune made in another process):
 * terms per launch in [1, the plan's maximum] and the variant bits of sigw_plan_autotune (bits for variants the
 * plan's N and precision lack are ignored).  Errors: SIGW_EINVAL. */
sigw_status sigw_plan_set_tuning(sigw_plan plan, int alpha_batch, int variant);

/* Per-kernel accounting of a plan.  Kernel kinds: 0 synthesis chain, 1 first inverse pass (filter,
 * gradient), 2 second inverse pass, 3 last inverse pass + product + first forward pass, 4 second forward
 * pass, 5 last forward pass + TT projection + shell sum, 6 bin finalisation. */
#define SIGW_NKINDS 7
typedef struct sigw_profile {
  double ms[SIGW_NKINDS];        /* summed CUDA-event durations (only while event timing is on) */
  double bytes[SIGW_NKINDS];     /* algorithmic bytes: each input element read once, each output written once */
  int64_t launches[SIGW_NKINDS]; /* kernel launches (always counted) */
  double h2d_bytes, d2h_bytes;   /* host<->device bytes copied by the library */
} sigw_profile;

/* enable != 0: bracket every kernel launch with CUDA events on the plan's stream (adds a few microseconds
 * per launch).  Both enabling and disabling reset the counters. */
sigw_status sigw_plan_profile(sigw_plan plan, int enable);

/* Wait for the plan's stream, fill *out with the counters accumulated since the last reset, and reset them. */
sigw_status sigw_plan_profile_read(sigw_plan plan, sigw_profile* out);

/* Host-only (no GPU needed): the truncated decomposition a plan with these options uses, for kernel m
 * (0: I_s, 1: I_c).  Same outputs as sigw_plan_kernel_terms; opts may be NULL (defaults).
 * Also reports all n_modes eigenvalues (sigma_all[n_modes], sorted by |sigma| descending) when non-NULL. */
sigw_status sigw_decompose(const sigw_opts* opts, int m, double* sigma, double* phi, double* edges, double* sigma_all);

/* Host-only decomposition study (the paper leaves the choice of grid meta-parameters open, Sec. sec_conclusions;
 * Fig. fig_eigenvalues, Fig. fig_reconstruction).  For kernel m and the grid of opts, compares the rank-n_alpha
 * truncation C_k = sum_{a < n_alpha} sigma_a q_a q_a^T with the full matrix C_ij = sqrt(L_i L_j) I_m(u_i, u_j)
 * on the strip (Eq. eq_C_matrix_discrete).  Outputs (nullable): *frob = ||C - C_k||_F / ||C||_F,
 * *maxrel = max_ij |C - C_k|_ij / max_ij |C_ij|, *gap = |sigma_{n_alpha}| / |sigma_{n_alpha - 1}| (0-based; the
 * spectral gap at the cut, 0 when n_alpha = n_modes).  Errors: SIGW_EINVAL. */
sigw_status sigw_decomposition_error(const sigw_opts* opts, int m, double* frob, double* maxrel, double* gap);

/* Host-only: the cell table of target shell n_c, lut[msq] for msq = 0..msq_max: the u-grid cell holding
 * u = sqrt(msq)/n_c, decided on squares ((e_i n_c)^2 <= msq in FP64), or n_modes outside [umin, umax). */
sigw_status sigw_cell_table(const sigw_opts* opts, int n_c, int msq_max, int16_t* lut);

/* The paper has no counterpart to this entry point: it is a library utility.
 * sigw_fft3d without a plan and without any device allocation, for callers that cannot call cudaMalloc
 * (for example a host program whose own pool allocator already owns all device memory, or a latency-critical
 * path where a synchronising cudaMalloc is not acceptable).  Same transforms and layouts as sigw_fft3d:
 * direction -1 real in[N][N][N] -> complex out[N][N][N/2+1], +1 the unnormalised inverse; precision 32 or 64.
 * Scratch: file-scope device arrays of fixed size (8 MiB for the packed half spectrum, N*N*(N/2) complex
 * values, plus 248-entry twiddle tables per precision), held by every GPU that loads the library until the
 * process exits.  Limit: N*N*(N/2) complex values must fit in 8 MiB, i.e. N <= 128 in FP32 and N <= 64 in
 * FP64 (N a power of two >= 8); larger N returns SIGW_EINVAL.  The first call on a device sets that device up
 * (looks up the arrays' device addresses, fills the twiddles and waits for the whole device, so that a
 * non-blocking stream sees the tables); make that first call before any stream capture.  The set-up is cached
 * for the life of the process: resetting the device (cudaDeviceReset) after its first call is not supported.  Work is queued on cuda_stream (NULL: the legacy default stream); the call does not
 * wait.  All calls share the one scratch array, which keeps the last call's contents (every call overwrites
 * all of what it reads, so nothing needs clearing): calls that overlap on the GPU (different streams, or a
 * second call before the first finished on another stream) race and give wrong results.
 * Errors: SIGW_EINVAL (arguments or size limit), SIGW_ECUDA (set-up or launch failed). */
sigw_status sigw_fft3d_noalloc(int N, int precision, int direction, const void* in_dev, void* out_dev,
                               void* cuda_stream);

/* Test hook for failure handling (no counterpart in the paper): the bounded waits in the main loop of the last
 * inverse pass (the bulk-copy ring) give up after `cycles` clock cycles instead of about a second (cycles = 0
 * restores the default).  A tiny limit makes waits give up while every copy still completes normally: the
 * spectrum call then returns SIGW_ETIMEOUT (results invalid), every copy in flight has landed before its CTA
 * exits, and the plan stays usable.  Applies to launches queued after the call (a captured all-shells graph is
 * dropped and captured again).  Errors: SIGW_EINVAL (NULL plan, cycles < 0). */
sigw_status sigw_plan_debug_wait_limit(sigw_plan plan, long long cycles);

/* Test hook for failure handling: the next `n`-th device allocation made by the library fails with
 * SIGW_ENOMEM (n = 1: the next one; n <= 0 disables).  Affects the calling process only. */
sigw_status sigw_debug_fail_alloc(int n);

#ifdef __cplusplus
}
#endif
#endif /* SIGW_H */
