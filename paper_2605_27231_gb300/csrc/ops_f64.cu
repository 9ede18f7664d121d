// FP64 instantiation of the device kernels and their launchers, plus the precision-independent kernels.
#define SIGW_COMMON_KERNELS
#include "ops_impl.cuh"
namespace sigw {
template struct OpsRT<double>;

cudaError_t launch_reduce_mean(const double* part, int nblk, double* mean, int batch, double inv, cudaStream_t st) {
  k_reduce_mean<<<batch, 32, 0, st>>>(part, nblk, mean, inv);
  return cudaGetLastError();
}

cudaError_t launch_fin(const double* partial, long pbstride, int maxblk, int n_shells, const int* shells,
                       const double* Nk, int N, double L, int tc3, double* out, int batch, cudaStream_t st) {
  const int n = batch * n_shells;
  k_fin<<<(n + 127) / 128, 128, 0, st>>>(partial, pbstride, maxblk, n_shells, shells, Nk, N, L, tc3, out, batch);
  return cudaGetLastError();
}
}  // namespace sigw
