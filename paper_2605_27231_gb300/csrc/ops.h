// Host-callable launchers of the device kernels, one instantiation per working
// precision (float in ops_f32.cu, double in ops_f64.cu).  All pointers are device
// pointers; each launcher queues work on `st` and returns the launch status.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace sigw {

// Tile shapes chosen per (precision, N); exposed so the host can size buffers.
constexpr long long kDefaultWaitLimit = 1ll << 31;  // clock cycles of a bounded wait, about one second

struct LaunchShape {
  int tc_strided;   // columns per CTA in strided passes
  int tc_f3;        // columns per CTA in the forward-axis-0 / TT / bin pass
  int maxblk_f3;    // upper bound on CTAs of one forward-axis-0 / TT / bin launch
};

struct MapArgs {
  int kind;  // 0 gauss, 1 local, 2 usr, 3 non-local (F = alpha_NL / k*^2, G = beta_NL / k*^2)
  double F, G, floor;
};

template <typename T>
struct OpsRT {
  // ---- synthesis chain (packed layout [b][a0][a1][N/2], standard layout [b][k0][k1][N/2+1])
  static cudaError_t rows_r2c_noise(int N, void* Y, const uint64_t* seeds, int batch, const void* tw, cudaStream_t st);
  static cudaError_t rows_r2c_real(int N, const void* R, void* Y, int batch, const void* tw, cudaStream_t st);
  // map: device array of per-realisation MapArgs; R2 = lap(zeta_g), R3 = lap(zeta_g^2) for the non-local map
  static cudaError_t rows_r2c_map(int N, const void* R, void* Y, int batch, const MapArgs* map, const double* mean,
                                  unsigned long long* hits, const void* tw, cudaStream_t st, const void* R2 = nullptr,
                                  const void* R3 = nullptr);
  // rows of R squared, R2C
  static cudaError_t rows_r2c_square(int N, const void* R, void* Y, int batch, const void* tw, cudaStream_t st);
  static cudaError_t rows_c2r(int N, const void* Y, void* R, int batch, double scale, double* sq_partial,
                              const void* tw, cudaStream_t st);
  static cudaError_t pass(int N, void* Y, int axis, int dir, int batch, const void* tw, cudaStream_t st);
  // mode 0: times amp[b * amp_bstride + |n|^2] * factor and zero on k = 0 and the Nyquist planes;
  // mode 1: times factor
  static cudaError_t unpack(int N, const void* Y, void* X, int batch, const void* amp, long amp_bstride, double factor,
                            int mode, cudaStream_t st);
  // lap != 0: times -lap |n|^2 (spectral Laplacian for lap = k_f^2)
  static cudaError_t pack(int N, const void* X, void* Y, int batch, cudaStream_t st, double lap = 0.0);
  static int rows_blocks(int N);  // CTAs per realisation of rows_c2r (entries of sq_partial per realisation)
  static LaunchShape shape(int N);

  // ---- hot path
  // variant: radix choice of the two strided inverse passes (0 default; 1 the alternative, where variants(N) == 2)
  static int variants(int N);
  // first inverse pass (axis 0) with the filter phi_a(cell) and the i n_0 gradient factor
  static cudaError_t p1(int N, const void* phi, void* Ta, void* Tb, const int16_t* lut, const void* phitab, int nm1,
                        int alpha0, int nb, int batch, const void* tw, int variant, cudaStream_t st);
  // second inverse pass (axis 1), three outputs per term
  static cudaError_t p2(int N, const void* Ta, const void* Tb, void* W, int n_alpha, int alpha0, int nb, int batch,
                        const void* tw, int variant, cudaStream_t st);
  // last inverse pass (axis 2, C2R) + sum_a sigma_a g_i g_j + forward R2C along axis 2 keeping k2 <= n_c
  // err: device int, OR-ed with 1 when a bounded wait of the bulk-copy pipeline gives up; wait_limit: clock
  // cycles after which a wait of the main loop gives up (kDefaultWaitLimit unless a test shrinks it).
  // variant bit 2 selects the radix-16 form where p3_variants(N) >= 2; bit 8 the radix-16 form with its
  // accumulators in tensor memory where p3_variants(N) == 3 (FP32, N = 128, 256, 512).
  static int p3_variants(int N);
  static cudaError_t p3(int N, const void* W, const void* sigma, int n_alpha, void* F, int n_c, int batch,
                        const void* tw, int* err, long long wait_limit, int variant, cudaStream_t st);
  // forward pass along axis 1 keeping |n1| <= n_c
  static cudaError_t f2(int N, const void* F, void* F2, int n_c, int batch, const void* tw, cudaStream_t st);
  // forward pass along axis 0 + TT projection + shell sum -> per-CTA FP64 partials; with Xj (nullable) also the
  // two TT amplitudes of every stored shell mode into the zeroed standard half spectra Xj[batch][2]
  static cudaError_t f3(int N, const void* F2, int n_c, double* partial, long pbstride, int batch, const void* tw,
                        cudaStream_t st, void* Xj = nullptr);
  // jackknife: sum of R^2 over each x0-plane of each of the M^3 sub-volumes, out[field][M^3][N/M]
  static cudaError_t subvol(int N, int M, const void* R, int nfields, double* out, cudaStream_t st);
};

extern template struct OpsRT<float>;
extern template struct OpsRT<double>;

// precision-independent kernels (defined in ops_f64.cu)
cudaError_t launch_reduce_mean(const double* part, int nblk, double* mean, int batch, double inv, cudaStream_t st);
cudaError_t launch_fin(const double* partial, long pbstride, int maxblk, int n_shells, const int* shells,
                       const double* Nk, int N, double L, int tc3, double* out, int batch, cudaStream_t st);

}  // namespace sigw
