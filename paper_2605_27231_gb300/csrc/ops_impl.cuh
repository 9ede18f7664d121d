// Launchers of the kernels in kernels.cuh for one precision T (instantiated by ops_f32.cu / ops_f64.cu).
#pragma once
#include "kernels.cuh"
#include "ops.h"

namespace sigw {

// Opt in to more than the default 48 KB of shared memory per CTA.  The default limit covers static and dynamic
// shared memory together, so the opt-in starts a little below 48 KB of dynamic memory (kernels here declare at
// most 1 KB of static shared memory).
template <typename Kern>
static cudaError_t allow_smem(Kern k, size_t bytes) {
  if (bytes <= 47 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

#define SIGW_CHECK_LAUNCH(...)            \
  do {                                    \
    cudaError_t _e = (__VA_ARGS__);       \
    if (_e != cudaSuccess) return _e;     \
  } while (0)

template <typename T>
struct OpsT {
  using C = cx<T>;

  template <int N>
  static size_t row_bytes(int count) { return (size_t)count * RowLayout<T, N>::SIZE * sizeof(C); }
  template <int N, int TC, int E>
  static size_t col_bytes() { return (size_t)ColLayout<T, N, TC, E>::SIZE * sizeof(C); }
  template <int N, int TC, int E>
  static size_t strided_bytes() { return (size_t)StridedLay<T, N, TC, E>::SIZE * sizeof(C); }

  // ------------------------------------------------------------ synthesis
  template <int N, int MODE>
  static cudaError_t rows_r2c_n(const void* R, void* Y, const uint64_t* seeds, const MapArgs* map, const double* mean,
                                unsigned long long* hits, int batch, const void* tw, cudaStream_t st,
                                const void* R2 = nullptr, const void* R3 = nullptr) {
    using SH = Shape<T, N>;
    const size_t sm = row_bytes<N>(SH::RPC);
    auto k = k_rows_r2c<T, N, MODE>;
    SIGW_CHECK_LAUNCH(allow_smem(k, sm));
    dim3 grid((N * N / 2) / SH::RPC, batch);
    k<<<grid, SH::RPC * SH::PR, sm, st>>>((const T*)R, (C*)Y, (const C*)tw, seeds, map, mean, hits, (const T*)R2,
                                          (const T*)R3);
    return cudaGetLastError();
  }
  template <int N, bool SQ>
  static cudaError_t rows_c2r_n(const void* Y, void* R, int batch, double scale, double* sqp, const void* tw,
                                cudaStream_t st) {
    using SH = Shape<T, N>;
    const size_t sm = row_bytes<N>(SH::RPC);
    auto k = k_rows_c2r<T, N, SQ>;
    SIGW_CHECK_LAUNCH(allow_smem(k, sm));
    dim3 grid((N * N / 2) / SH::RPC, batch);
    k<<<grid, SH::RPC * SH::PR, sm, st>>>((const C*)Y, (T*)R, (T)scale, sqp, (const C*)tw);
    return cudaGetLastError();
  }
  template <int N, int DIR, int AX>
  static cudaError_t pass_n(void* Y, int batch, const void* tw, cudaStream_t st) {
    using SH = Shape<T, N>;
    const size_t sm = col_bytes<N, SH::TC, SH::ES>();
    auto k = k_pass<T, N, DIR, AX>;
    SIGW_CHECK_LAUNCH(allow_smem(k, sm));
    dim3 grid((N / 2) / SH::TC, N, batch);
    k<<<grid, SH::TC * SH::PS, sm, st>>>((C*)Y, (const C*)tw);
    return cudaGetLastError();
  }
  // ------------------------------------------------------------ hot path
  template <int N, int E, int TC>
  static cudaError_t p1_v(const void* phi, void* Ta, void* Tb, const int16_t* lut, const void* phitab, int nm1,
                          int alpha0, int nb, int batch, const void* tw, cudaStream_t st) {
    const size_t sm = strided_bytes<N, TC, E>() + N * sizeof(C) + N * sizeof(int) + (size_t)nb * nm1 * sizeof(T);
    auto k = k_p1<T, N, E, TC>;
    SIGW_CHECK_LAUNCH(allow_smem(k, 227 * 1024));
    dim3 grid((N / 2) / TC, N, batch);
    k<<<grid, TC * (N / E), sm, st>>>((const C*)phi, (C*)Ta, (C*)Tb, lut, (const T*)phitab, nm1, alpha0, nb,
                                      (const C*)tw);
    return cudaGetLastError();
  }
  template <int N>
  static cudaError_t p1_tm_v(const void* phi, void* Ta, void* Tb, const int16_t* lut, const void* phitab, int nm1,
                             int alpha0, int nb, int batch, const void* tw, cudaStream_t st) {
    using CF = P1TCfg<N>;
    const size_t sm = CF::smem(nb, nm1);
    auto k = k_p1_tm<N>;
    SIGW_CHECK_LAUNCH(allow_smem(k, 227 * 1024));
    dim3 grid((N / 2) / CF::TC, N, batch);
    k<<<grid, CF::THREADS, sm, st>>>((const float2*)phi, (float2*)Ta, (float2*)Tb, lut, (const float*)phitab, nm1,
                                     alpha0, nb, (const float2*)tw);
    return cudaGetLastError();
  }
  template <int N>
  static cudaError_t p1_n(const void* phi, void* Ta, void* Tb, const int16_t* lut, const void* phitab, int nm1,
                          int alpha0, int nb, int batch, const void* tw, int variant, cudaStream_t st) {
    using SH = Shape<T, N>;
    using AL = AltStrided<T, N>;
    if constexpr (sizeof(T) == 4 && (N == 128 || N == 256 || N == 512)) {  // Phi~ tile and cells in tensor memory
      if (variant & 16) return p1_tm_v<N>(phi, Ta, Tb, lut, phitab, nm1, alpha0, nb, batch, tw, st);
    }
    if constexpr (AL::exists) {
      if (variant & 1)
        return p1_v<N, AL::E, AL::TC>(phi, Ta, Tb, lut, phitab, nm1, alpha0, nb, batch, tw, st);
    }
    return p1_v<N, SH::ES, SH::TC>(phi, Ta, Tb, lut, phitab, nm1, alpha0, nb, batch, tw, st);
  }
  template <int N, int E, int TC>
  static cudaError_t p2_v(const void* Ta, const void* Tb, void* W, int n_alpha, int alpha0, int nb, int batch,
                          const void* tw, cudaStream_t st) {
    const size_t sm = strided_bytes<N, TC, E>();
    auto k = k_p2<T, N, E, TC>;
    SIGW_CHECK_LAUNCH(allow_smem(k, sm));
    dim3 grid((N / 2) / TC, N, batch * nb);
    k<<<grid, TC * (N / E), sm, st>>>((const C*)Ta, (const C*)Tb, (C*)W, n_alpha, alpha0, nb, (const C*)tw);
    return cudaGetLastError();
  }
  template <int N>
  static cudaError_t p2_n(const void* Ta, const void* Tb, void* W, int n_alpha, int alpha0, int nb, int batch,
                          const void* tw, int variant, cudaStream_t st) {
    using SH = Shape<T, N>;
    using AL = AltStrided2<T, N>;
    if constexpr (AL::exists) {
      if (variant & 4) return p2_v<N, AL::E, AL::TC>(Ta, Tb, W, n_alpha, alpha0, nb, batch, tw, st);
    }
    return p2_v<N, SH::ES, SH::TC>(Ta, Tb, W, n_alpha, alpha0, nb, batch, tw, st);
  }
  template <int N, int E>
  static cudaError_t p3_v(const void* W, const void* sigma, int n_alpha, void* F, int n_c, int batch, const void* tw,
                          int* err, long long wait_limit, cudaStream_t st) {
    using CF = P3Cfg<T, N, E>;
    auto k = k_p3<T, N, E>;
    SIGW_CHECK_LAUNCH(allow_smem(k, CF::SMEM));
    dim3 grid((N * N) / CF::RPC, batch);
    k<<<grid, CF::THREADS, CF::SMEM, st>>>((const C*)W, (const T*)sigma, n_alpha, (C*)F, n_c, (const C*)tw, err,
                                           wait_limit);
    return cudaGetLastError();
  }
  template <int N>
  static cudaError_t p3_tm_v(const void* W, const void* sigma, int n_alpha, void* F, int n_c, int batch,
                             const void* tw, int* err, long long wait_limit, cudaStream_t st) {
    using CF = P3TCfg<N>;
    auto k = k_p3_tm<N>;
    SIGW_CHECK_LAUNCH(allow_smem(k, CF::SMEM));
    dim3 grid((N * N) / CF::RPC, batch);
    k<<<grid, CF::THREADS, CF::SMEM, st>>>((const float2*)W, (const float*)sigma, n_alpha, (float2*)F, n_c,
                                           (const float2*)tw, err, wait_limit);
    return cudaGetLastError();
  }
  template <int N>
  static cudaError_t p3_n(const void* W, const void* sigma, int n_alpha, void* F, int n_c, int batch, const void* tw,
                          int* err, long long wait_limit, int variant, cudaStream_t st) {
    if constexpr (sizeof(T) == 4 && (N == 128 || N == 256 || N == 512)) {  // accumulators in tensor memory
      if (variant & 8) return p3_tm_v<N>(W, sigma, n_alpha, F, n_c, batch, tw, err, wait_limit, st);
    }
    if constexpr (AltP3<T, N>::exists) {
      if (variant & 2) return p3_v<N, AltP3<T, N>::E>(W, sigma, n_alpha, F, n_c, batch, tw, err, wait_limit, st);
    }
    return p3_v<N, ((N >= 16) ? 8 : 4)>(W, sigma, n_alpha, F, n_c, batch, tw, err, wait_limit, st);
  }
  static void n1_range(int N, int n_c, int* lo, int* nk1) {
    const int H = N / 2;
    const int a = n_c < H - 1 ? -n_c : -H + 1;
    const int bhi = n_c < H ? n_c : H;
    *lo = a;
    *nk1 = bhi - a + 1;
  }
  template <int N>
  static cudaError_t f2_n(const void* F, void* F2, int n_c, int batch, const void* tw, cudaStream_t st) {
    using SH = Shape<T, N>;
    const size_t sm = (size_t)ColLayout<T, N, SH::TC, SH::ES, true>::SIZE * sizeof(C);  // single exchange buffer
    auto k = k_f2<T, N>;
    SIGW_CHECK_LAUNCH(allow_smem(k, sm));
    int lo, nk1;
    n1_range(N, n_c, &lo, &nk1);
    dim3 grid((n_c + 1 + SH::TC - 1) / SH::TC, N, batch * 6);
    k<<<grid, SH::TC * SH::PS, sm, st>>>((const C*)F, (C*)F2, n_c, lo, nk1, (const C*)tw);
    return cudaGetLastError();
  }
  template <int N>
  static cudaError_t f3_n(const void* F2, int n_c, double* partial, long pbs, int batch, const void* tw,
                          cudaStream_t st, void* Xj) {
    using SH = Shape<T, N>;
    const size_t sm = col_bytes<N, SH::TC3, SH::E3>();
    auto k = k_f3<T, N>;
    SIGW_CHECK_LAUNCH(allow_smem(k, sm));
    int lo, nk1;
    n1_range(N, n_c, &lo, &nk1);
    dim3 grid((n_c + 1 + SH::TC3 - 1) / SH::TC3, nk1, batch);
    k<<<grid, SH::TC3 * SH::P3, sm, st>>>((const C*)F2, n_c, lo, nk1, partial, pbs, (const C*)tw, (C*)Xj);
    return cudaGetLastError();
  }
  template <int N>
  static LaunchShape shape_n() {
    using SH = Shape<T, N>;
    LaunchShape s;
    s.tc_strided = SH::TC;
    s.tc_f3 = SH::TC3;
    s.maxblk_f3 = ((N / 2 + 1 + SH::TC3 - 1) / SH::TC3) * N;
    return s;
  }
  template <int N>
  static int rows_blocks_n() { return (N * N / 2) / Shape<T, N>::RPC; }
};

// Runtime switch on N (powers of two 8..512).
#define SIGW_DISPATCH_N(N, CALL)          \
  switch (N) {                            \
    case 8: { constexpr int NN = 8; CALL; } \
    case 16: { constexpr int NN = 16; CALL; } \
    case 32: { constexpr int NN = 32; CALL; } \
    case 64: { constexpr int NN = 64; CALL; } \
    case 128: { constexpr int NN = 128; CALL; } \
    case 256: { constexpr int NN = 256; CALL; } \
    case 512: { constexpr int NN = 512; CALL; } \
    default: return cudaErrorInvalidValue; \
  }

template <typename T>
cudaError_t OpsRT<T>::rows_r2c_noise(int N, void* Y, const uint64_t* seeds, int batch, const void* tw, cudaStream_t st) {
  SIGW_DISPATCH_N(N, return (OpsT<T>::template rows_r2c_n<NN, 1>(nullptr, Y, seeds, nullptr, nullptr, nullptr, batch, tw, st)));
}
template <typename T>
cudaError_t OpsRT<T>::rows_r2c_real(int N, const void* R, void* Y, int batch, const void* tw, cudaStream_t st) {
  SIGW_DISPATCH_N(N, return (OpsT<T>::template rows_r2c_n<NN, 0>(R, Y, nullptr, nullptr, nullptr, nullptr, batch, tw, st)));
}
template <typename T>
cudaError_t OpsRT<T>::rows_r2c_map(int N, const void* R, void* Y, int batch, const MapArgs* map, const double* mean,
                                unsigned long long* hits, const void* tw, cudaStream_t st, const void* R2,
                                const void* R3) {
  SIGW_DISPATCH_N(N, return (OpsT<T>::template rows_r2c_n<NN, 2>(R, Y, nullptr, map, mean, hits, batch, tw, st, R2, R3)));
}
template <typename T>
cudaError_t OpsRT<T>::rows_r2c_square(int N, const void* R, void* Y, int batch, const void* tw, cudaStream_t st) {
  SIGW_DISPATCH_N(N, return (OpsT<T>::template rows_r2c_n<NN, 3>(R, Y, nullptr, nullptr, nullptr, nullptr, batch, tw, st)));
}
template <typename T>
cudaError_t OpsRT<T>::rows_c2r(int N, const void* Y, void* R, int batch, double scale, double* sqp, const void* tw,
                            cudaStream_t st) {
  if (sqp) {
    SIGW_DISPATCH_N(N, return (OpsT<T>::template rows_c2r_n<NN, true>(Y, R, batch, scale, sqp, tw, st)));
  } else {
    SIGW_DISPATCH_N(N, return (OpsT<T>::template rows_c2r_n<NN, false>(Y, R, batch, scale, sqp, tw, st)));
  }
}
template <typename T>
cudaError_t OpsRT<T>::pass(int N, void* Y, int axis, int dir, int batch, const void* tw, cudaStream_t st) {
  if (axis == 0 && dir < 0) { SIGW_DISPATCH_N(N, return (OpsT<T>::template pass_n<NN, -1, 0>(Y, batch, tw, st))); }
  if (axis == 0 && dir > 0) { SIGW_DISPATCH_N(N, return (OpsT<T>::template pass_n<NN, +1, 0>(Y, batch, tw, st))); }
  if (axis == 1 && dir < 0) { SIGW_DISPATCH_N(N, return (OpsT<T>::template pass_n<NN, -1, 1>(Y, batch, tw, st))); }
  if (axis == 1 && dir > 0) { SIGW_DISPATCH_N(N, return (OpsT<T>::template pass_n<NN, +1, 1>(Y, batch, tw, st))); }
  return cudaErrorInvalidValue;
}
template <typename T>
cudaError_t OpsRT<T>::unpack(int N, const void* Y, void* X, int batch, const void* amp, long amp_bstride,
                          double factor, int mode, cudaStream_t st) {
  const long total = (long)batch * N * N * (N / 2 + 1);
  const int thr = 256;
  long blocks = (total + thr - 1) / thr;
  if (blocks > 152 * 32) blocks = 152 * 32;
  if (mode == 0)
    k_unpack<T, 0><<<(int)blocks, thr, 0, st>>>((const cx<T>*)Y, (cx<T>*)X, N, (const T*)amp, amp_bstride, (T)factor,
                                               total);
  else
    k_unpack<T, 1><<<(int)blocks, thr, 0, st>>>((const cx<T>*)Y, (cx<T>*)X, N, nullptr, 0, (T)factor, total);
  return cudaGetLastError();
}
template <typename T>
cudaError_t OpsRT<T>::pack(int N, const void* X, void* Y, int batch, cudaStream_t st, double lap) {
  const long total = (long)batch * N * N * (N / 2);
  const int thr = 256;
  long blocks = (total + thr - 1) / thr;
  if (blocks > 152 * 32) blocks = 152 * 32;
  k_pack<T><<<(int)blocks, thr, 0, st>>>((const cx<T>*)X, (cx<T>*)Y, N, total, lap);
  return cudaGetLastError();
}
template <typename T>
int OpsRT<T>::rows_blocks(int N) {
  switch (N) {
    case 8: return OpsT<T>::template rows_blocks_n<8>();
    case 16: return OpsT<T>::template rows_blocks_n<16>();
    case 32: return OpsT<T>::template rows_blocks_n<32>();
    case 64: return OpsT<T>::template rows_blocks_n<64>();
    case 128: return OpsT<T>::template rows_blocks_n<128>();
    case 256: return OpsT<T>::template rows_blocks_n<256>();
    case 512: return OpsT<T>::template rows_blocks_n<512>();
  }
  return 0;
}
template <typename T>
int OpsRT<T>::p3_variants(int N) {
  if (N == 128) return AltP3<T, 128>::exists ? 3 : 1;  // FP32: radix 8, radix 16, radix 16 with TMEM accumulators
  if (N == 256) return AltP3<T, 256>::exists ? 3 : 1;
  if (N == 512) return AltP3<T, 512>::exists ? 3 : 1;
  return 1;
}
template <typename T>
int OpsRT<T>::variants(int N) {
  switch (N) {
    case 128: return AltStrided<T, 128>::exists ? 2 : 1;
    case 256: return AltStrided<T, 256>::exists ? 2 : 1;
    case 512: return AltStrided<T, 512>::exists ? 2 : 1;
  }
  return 1;
}
template <typename T>
LaunchShape OpsRT<T>::shape(int N) {
  switch (N) {
    case 8: return OpsT<T>::template shape_n<8>();
    case 16: return OpsT<T>::template shape_n<16>();
    case 32: return OpsT<T>::template shape_n<32>();
    case 64: return OpsT<T>::template shape_n<64>();
    case 128: return OpsT<T>::template shape_n<128>();
    case 256: return OpsT<T>::template shape_n<256>();
    default: return OpsT<T>::template shape_n<512>();
  }
}
template <typename T>
cudaError_t OpsRT<T>::p1(int N, const void* phi, void* Ta, void* Tb, const int16_t* lut, const void* phitab, int nm1,
                      int alpha0, int nb, int batch, const void* tw, int variant, cudaStream_t st) {
  SIGW_DISPATCH_N(N, return (OpsT<T>::template p1_n<NN>(phi, Ta, Tb, lut, phitab, nm1, alpha0, nb, batch, tw, variant, st)));
}
template <typename T>
cudaError_t OpsRT<T>::p2(int N, const void* Ta, const void* Tb, void* W, int n_alpha, int alpha0, int nb, int batch,
                      const void* tw, int variant, cudaStream_t st) {
  SIGW_DISPATCH_N(N, return (OpsT<T>::template p2_n<NN>(Ta, Tb, W, n_alpha, alpha0, nb, batch, tw, variant, st)));
}
template <typename T>
cudaError_t OpsRT<T>::p3(int N, const void* W, const void* sigma, int n_alpha, void* F, int n_c, int batch,
                      const void* tw, int* err, long long wait_limit, int variant, cudaStream_t st) {
  SIGW_DISPATCH_N(N, return (OpsT<T>::template p3_n<NN>(W, sigma, n_alpha, F, n_c, batch, tw, err, wait_limit,
                                                       variant, st)));
}
template <typename T>
cudaError_t OpsRT<T>::f2(int N, const void* F, void* F2, int n_c, int batch, const void* tw, cudaStream_t st) {
  SIGW_DISPATCH_N(N, return (OpsT<T>::template f2_n<NN>(F, F2, n_c, batch, tw, st)));
}
template <typename T>
cudaError_t OpsRT<T>::f3(int N, const void* F2, int n_c, double* partial, long pbs, int batch, const void* tw,
                      cudaStream_t st, void* Xj) {
  SIGW_DISPATCH_N(N, return (OpsT<T>::template f3_n<NN>(F2, n_c, partial, pbs, batch, tw, st, Xj)));
}
template <typename T>
cudaError_t OpsRT<T>::subvol(int N, int M, const void* R, int nfields, double* out, cudaStream_t st) {
  if (M < 2 || N % M) return cudaErrorInvalidValue;
  dim3 grid(M * M * M * (N / M), nfields);
  k_subvol<T><<<grid, 256, 0, st>>>((const T*)R, N, M, out);
  return cudaGetLastError();
}


}  // namespace sigw
