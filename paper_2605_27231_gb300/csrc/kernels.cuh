// Device kernels of the lattice SIGW path, templated on the working precision T
// (float or double) and the lattice size N.  Included by one translation unit per
// precision, which instantiates them and defines the sigw::Ops launchers.
//
// Layouts (b = realisation in the batch, H = N/2, NH = N/2 + 1):
//   real       R[b][a0][a1][a2]                      N^3 values
//   standard   X[b][k0][k1][k2], k2 = 0..H           the usual half spectrum (Phi~ is kept this way)
//   packed     Y[b][a0|k0][a1|k1][c], c = 0..H-1     column 0 holds (k2 = 0) + i (k2 = H); this is
//              exact because both planes are transforms of real 2-D fields, and it makes every
//              strided pass run over exactly H columns.
// Lattice wave numbers: index k -> n = k for k <= H, k - N otherwise (index H is +N/2).
// The derivative factor uses n^D = 0 on the Nyquist index H.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <type_traits>

#include "fft.cuh"
#include "ops.h"

namespace sigw {

__device__ __forceinline__ int wrapn(int k, int N) { return k <= (N >> 1) ? k : k - N; }
__device__ __forceinline__ int derivn(int k, int N) { return k == (N >> 1) ? 0 : wrapn(k, N); }

// ---------------------------------------------------------------- Philox4x32-10 (SC'11)
// counter (c0, c1, c2, c3), key (k0, k1); 10 rounds, Weyl key schedule between rounds.
__device__ __forceinline__ void philox10(uint32_t& c0, uint32_t& c1, uint32_t& c2, uint32_t& c3, uint32_t k0,
                                         uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
}

// N(0,1) draw for lattice cell `cell` (row-major linear index) and key `seed`: Box-Muller in FP64 on
// two 53-bit uniforms made from the four output words, u1 in (0, 1], u2 in [0, 1).
__device__ __forceinline__ double gauss_draw(uint32_t cell, uint64_t seed) {
  uint32_t c0 = cell, c1 = 0u, c2 = 0u, c3 = 0u;
  philox10(c0, c1, c2, c3, (uint32_t)(seed & 0xffffffffull), (uint32_t)(seed >> 32));
  const uint64_t a = ((((uint64_t)c0) << 32) | c1) >> 11;
  const uint64_t bb = ((((uint64_t)c2) << 32) | c3) >> 11;
  const double u1 = ((double)a + 1.0) * 1.1102230246251565404e-16;  // 2^-53
  const double u2 = (double)bb * 1.1102230246251565404e-16;
  return sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
}

// ---------------------------------------------------------------- shapes
template <typename T, int N> struct Shape {
  static constexpr int H = N / 2;
  // strided passes: E values per thread, TC columns per CTA
  static constexpr int ES = (sizeof(T) == 4) ? (N >= 256 ? 16 : (N >= 16 ? 8 : 4)) : (N >= 16 ? 8 : 4);
  static constexpr int PS = N / ES;
  static constexpr int TC0 = 256 / PS;
  static constexpr int TC = TC0 < 1 ? 1 : (TC0 > H ? H : TC0);
  // row passes: E values per thread, RPC rows per CTA
  static constexpr int ER = (N >= 16) ? 8 : 4;
  static constexpr int PR = N / ER;
  static constexpr int RPC0 = 256 / PR;
  static constexpr int RPC = RPC0 > (N * N / 2) ? (N * N / 2) : RPC0;
  // forward-a0 + TT pass keeps six spectra per thread: fewer values per thread
  static constexpr int E3 = (sizeof(T) == 4) ? (N >= 16 ? 8 : 4) : 4;
  static constexpr int P3 = N / E3;
  static constexpr int TC3_0 = 256 / P3;
  static constexpr int TC3_1 = TC3_0 < 1 ? 1 : (TC3_0 > 8 ? 8 : TC3_0);
  static constexpr int TC3 = TC3_1 * P3 < 32 ? 32 / P3 : TC3_1;  // whole warps (the partial sum uses shuffles)
};

// Alternative radix of the strided inverse passes (variant bit 1 for the first pass; the second pass uses
// AltStrided2 with bit 4): FP32, N >= 128 only.  At N = 512 the
// alternative is radix 32 (two stages, one exchange, 16-column tiles) instead of radix 16 (three stages).
template <typename T, int N> struct AltStrided {
  static constexpr bool exists = sizeof(T) == 4 && N >= 128;
  static constexpr int E = N == 512 ? 32 : (Shape<T, N>::ES == 16 ? 8 : 16);
  static constexpr int P = N / E;
  static constexpr int TC0 = 256 / P;
  static constexpr int TC = TC0 > N / 2 ? N / 2 : TC0;
};

// Column-tile exchange layout of the strided passes: one buffer when E >= 32 (a radix-32 pencil of 512
// points would otherwise need 128 KB for a 16-column tile).
template <typename T, int N, int TC, int E> using StridedLay = ColLayout<T, N, TC, E, (E >= 32)>;

// Alternative of the second strided pass (variant bit 4): as AltStrided, except at N = 512, where a 512-thread
// CTA runs 16 columns of radix 16 (full 128-byte row segments, 16 warps per SM, no spills).
template <typename T, int N> struct AltStrided2 {
  static constexpr bool exists = sizeof(T) == 4 && N >= 128;
  static constexpr int E = N == 512 ? 16 : AltStrided<T, N>::E;
  static constexpr int TC = N == 512 ? 16 : AltStrided<T, N>::TC;
};

template <int P> struct RowSync { using type = SyncWarp; };
template <> struct RowSync<64> { using type = SyncBlock; };
template <> struct RowSync<128> { using type = SyncBlock; };

// ================================================================ synthesis chain
// Two real rows (2q, 2q+1) share one complex FFT: z = x1 + i x2, Z = DFT z,
// X1(k) = (Z(k) + Z*(N-k))/2, X2(k) = -i/2 (Z(k) - Z*(N-k)).
// MODE 0: rows from R;  MODE 1: Philox noise;  MODE 2: R through the NG map;  MODE 3: R squared.
// The non-local map (kind 3) also reads lap(zeta_g) from R2 and lap(zeta_g^2) from R3 (same layout as R).
template <typename T, int N, int MODE>
__global__ void __launch_bounds__(256) k_rows_r2c(const T* __restrict__ R, cx<T>* __restrict__ Y,
                                                  const cx<T>* __restrict__ tw, const uint64_t* __restrict__ seeds,
                                                  const MapArgs* __restrict__ maps, const double* __restrict__ mean,
                                                  unsigned long long* __restrict__ hits, const T* __restrict__ R2,
                                                  const T* __restrict__ R3) {
  using SH = Shape<T, N>;
  constexpr int E = SH::ER, P = SH::PR, H = N / 2;
  constexpr int PPC = SH::RPC;  // row pairs per CTA
  using Sync = typename RowSync<P>::type;
  using Lay = RowLayout<T, N>;
  extern __shared__ __align__(16) unsigned char smraw[];
  const Lay L{reinterpret_cast<cx<T>*>(smraw) + (threadIdx.x / P) * Lay::SIZE};
  const int j = threadIdx.x % P;
  const int b = blockIdx.y;
  const long pair = (long)blockIdx.x * PPC + threadIdx.x / P;
  const bool live = pair < (long)N * N / 2;
  const long row0 = 2 * pair;
  cx<T> v[E];
  unsigned long long myhits = 0;
  double mu = 0.0;
  MapArgs map{0, 0.0, 0.0, 0.0};
  if (MODE == 2) {
    mu = mean[b];
    map = maps[b];
  }
#pragma unroll
  for (int r = 0; r < E; ++r) {
    const int x = j + r * P;
    T x1 = 0, x2 = 0;
    if (live) {
      if (MODE == 1) {
        const uint64_t sd = seeds[b];
        x1 = (T)gauss_draw((uint32_t)(row0 * N + x), sd);
        x2 = (T)gauss_draw((uint32_t)((row0 + 1) * N + x), sd);
      } else {
        const long ro = ((long)b * N * N + row0) * N;
        const T* rb = R + ro;
        x1 = rb[x];
        x2 = rb[N + x];
        if (MODE == 3) {
          x1 = x1 * x1;
          x2 = x2 * x2;
        }
        if (MODE == 2) {
          T z[2] = {x1, x2};
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            const T g = z[q];
            if (map.kind == 1) {
              z[q] = g + (T)map.F * (g * g - (T)mu) + (T)map.G * g * g * g;
            } else if (map.kind == 3) {
              const long o = ro + (long)q * N + x;
              z[q] = g + (T)map.F * R3[o] + (T)map.G * g * R2[o];
            } else if (map.kind == 2) {
              T arg = (T)1 - (T)3 * g;
              if (arg < (T)map.floor) {
                ++myhits;
                arg = (T)map.floor;
              }
              z[q] = -log(arg) / (T)3;
            }
          }
          x1 = z[0];
          x2 = z[1];
        }
      }
    }
    v[r] = mk<T>(x1, x2);
  }
  if (MODE == 2 && map.kind == 2) {
    // warp-reduce the hit count, one atomic per warp
    for (int o = 16; o > 0; o >>= 1) myhits += __shfl_down_sync(0xffffffffu, myhits, o);
    if ((threadIdx.x & 31) == 0 && myhits) atomicAdd(hits + b, myhits);
  }
  fft_pencil<T, N, E, -1, Lay, Sync>(v, j, L, tw, Sync());
  cx<T>* zb = L.buf(0);
#pragma unroll
  for (int r = 0; r < E; ++r) zb[L.idx(j + r * P)] = v[r];
  Sync()();
  if (live) {
    cx<T>* y1 = Y + ((long)b * N * N + row0) * H;
    cx<T>* y2 = y1 + H;
#pragma unroll
    for (int r = 0; r < E / 2; ++r) {
      const int c = j + r * P;
      if (c == 0) {
        const cx<T> z0 = zb[L.idx(0)];
        const cx<T> zh = zb[L.idx(H)];
        y1[0] = mk<T>(z0.x, zh.x);
        y2[0] = mk<T>(z0.y, zh.y);
      } else {
        const cx<T> zc = zb[L.idx(c)];
        const cx<T> zm = conjg<T>(zb[L.idx(N - c)]);
        y1[c] = mk<T>((T)0.5 * (zc.x + zm.x), (T)0.5 * (zc.y + zm.y));
        y2[c] = mk<T>((T)0.5 * (zc.y - zm.y), (T)-0.5 * (zc.x - zm.x));
      }
    }
  }
}

// Packed half rows -> real rows (two rows per complex inverse FFT), scaled by `scale`.
// With SQ, per-CTA FP64 partial sums of the squared outputs go to sq_partial[b][blockIdx.x].
template <typename T, int N, bool SQ>
__global__ void __launch_bounds__(256) k_rows_c2r(const cx<T>* __restrict__ Y, T* __restrict__ R, T scale,
                                                  double* __restrict__ sq_partial, const cx<T>* __restrict__ tw) {
  using SH = Shape<T, N>;
  constexpr int E = SH::ER, P = SH::PR, H = N / 2;
  constexpr int PPC = SH::RPC;
  using Sync = typename RowSync<P>::type;
  using Lay = RowLayout<T, N>;
  extern __shared__ __align__(16) unsigned char smraw[];
  const Lay L{reinterpret_cast<cx<T>*>(smraw) + (threadIdx.x / P) * Lay::SIZE};
  __shared__ double red[32];
  const int j = threadIdx.x % P;
  const int b = blockIdx.y;
  const long pair = (long)blockIdx.x * PPC + threadIdx.x / P;
  const bool live = pair < (long)N * N / 2;
  const long row0 = 2 * pair;
  const cx<T>* y1 = Y + ((long)b * N * N + row0) * H;
  const cx<T>* y2 = y1 + H;
  cx<T> v[E];
#pragma unroll
  for (int r = 0; r < E; ++r) {
    const int k = j + r * P;
    cx<T> a = mk<T>(0, 0), c = mk<T>(0, 0);
    if (live) {
      if (k == 0) {
        a = mk<T>(y1[0].x, 0);
        c = mk<T>(y2[0].x, 0);
      } else if (k == H) {
        a = mk<T>(y1[0].y, 0);
        c = mk<T>(y2[0].y, 0);
      } else if (k < H) {
        a = y1[k];
        c = y2[k];
      } else {
        a = conjg<T>(y1[N - k]);
        c = conjg<T>(y2[N - k]);
      }
    }
    v[r] = mk<T>(a.x - c.y, a.y + c.x);  // a + i c
  }
  fft_pencil<T, N, E, +1, Lay, Sync>(v, j, L, tw, Sync());
  double sq = 0.0;
  if (live) {
    T* r1 = R + ((long)b * N * N + row0) * N;
#pragma unroll
    for (int r = 0; r < E; ++r) {
      const int x = j + r * P;
      const T u = v[r].x * scale, w = v[r].y * scale;
      r1[x] = u;
      r1[N + x] = w;
      if (SQ) sq += (double)u * (double)u + (double)w * (double)w;
    }
  }
  if (SQ) {
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_down_sync(0xffffffffu, sq, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sq;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) t += red[w];
      sq_partial[(long)b * gridDim.x + blockIdx.x] = t;
    }
  }
}

// In-place C2C transforms along axis 0 (AX = 0, stride N*H) or axis 1 (AX = 1, stride H) of a packed array.
template <typename T, int N, int DIR, int AX>
__global__ void __launch_bounds__(256) k_pass(cx<T>* __restrict__ Y, const cx<T>* __restrict__ tw) {
  using SH = Shape<T, N>;
  constexpr int E = SH::ES, P = SH::PS, TC = SH::TC, H = N / 2;
  using Lay = ColLayout<T, N, TC, E>;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int c = threadIdx.x % TC, j = threadIdx.x / TC;
  const Lay L{reinterpret_cast<cx<T>*>(smraw), c};
  const int col = blockIdx.x * TC + c;
  const int o = blockIdx.y;
  const int b = blockIdx.z;
  const long stride = AX == 0 ? (long)N * H : (long)H;
  const long ostride = AX == 0 ? (long)H : (long)N * H;
  cx<T>* base = Y + (long)b * N * N * H + o * ostride + col;
  cx<T> v[E];
#pragma unroll
  for (int r = 0; r < E; ++r) v[r] = base[(j + r * P) * stride];
  fft_pencil<T, N, E, DIR, Lay, SyncBlock, false>(v, j, L, tw, SyncBlock());
#pragma unroll
  for (int r = 0; r < E; ++r) base[(j + r * P) * stride] = v[r];
}

// Packed -> standard.  MODE 0 (synthesis): times amp[|n|^2] * factor, zero on k = 0 and the Nyquist planes.
// MODE 1: times factor.
template <typename T, int MODE>
__global__ void k_unpack(const cx<T>* __restrict__ Y, cx<T>* __restrict__ X, int N, const T* __restrict__ amp,
                         long amp_bstride, T factor, long total) {
  const int H = N / 2, NH = H + 1;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const int k2 = (int)(i % NH);
    const long q = i / NH;
    const int k1 = (int)(q % N);
    const long q2 = q / N;
    const int k0 = (int)(q2 % N);
    const long b = q2 / N;
    cx<T> val;
    if (k2 >= 1 && k2 < H) {
      val = Y[((b * N + k0) * N + k1) * H + k2];
    } else {
      const cx<T> yk = Y[((b * N + k0) * N + k1) * H];
      const cx<T> ym = Y[((b * N + ((N - k0) & (N - 1))) * N + ((N - k1) & (N - 1))) * H];
      if (k2 == 0)
        val = mk<T>((T)0.5 * (yk.x + ym.x), (T)0.5 * (yk.y - ym.y));
      else
        val = mk<T>((T)0.5 * (yk.y + ym.y), (T)-0.5 * (yk.x - ym.x));
    }
    if (MODE == 0) {
      const int n0 = wrapn(k0, N), n1 = wrapn(k1, N);
      const int msq = n0 * n0 + n1 * n1 + k2 * k2;
      const bool zero = (k0 == H) || (k1 == H) || (k2 == H) || msq == 0;
      const T a = zero ? (T)0 : amp[b * amp_bstride + msq] * factor;
      val = mk<T>(val.x * a, val.y * a);
    } else {
      val = mk<T>(val.x * factor, val.y * factor);
    }
    X[i] = val;
  }
}

// Standard -> packed.  With lap != 0 each value is first multiplied by -lap |n|^2 (the spectral Laplacian for
// lap = k_f^2; a Nyquist index counts as n = +N/2, which is exact for the second derivative).
template <typename T>
__global__ void k_pack(const cx<T>* __restrict__ X, cx<T>* __restrict__ Y, int N, long total, double lap) {
  const int H = N / 2, NH = H + 1;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const int c = (int)(i % H);
    const long q = i / H;
    const cx<T>* xr = X + q * NH;
    T f0 = (T)1, fh = (T)1;
    if (lap != 0.0) {
      const int k1 = (int)(q % N), k0 = (int)((q / N) % N);
      const int n0 = wrapn(k0, N), n1 = wrapn(k1, N);
      const long m01 = (long)n0 * n0 + (long)n1 * n1;
      f0 = (T)(-lap * (double)(m01 + (long)c * c));
      fh = (T)(-lap * (double)(m01 + (long)H * H));
    }
    if (c == 0) {
      const cx<T> x0 = xr[0], xh = xr[H];
      Y[i] = mk<T>(f0 * x0.x - fh * xh.y, f0 * x0.y + fh * xh.x);  // f0 X(0) + i fH X(H)
    } else {
      const cx<T> v = xr[c];
      Y[i] = mk<T>(f0 * v.x, f0 * v.y);
    }
  }
}

#ifdef SIGW_COMMON_KERNELS
__global__ void k_reduce_mean(const double* __restrict__ part, int nblk, double* __restrict__ mean, double inv) {
  const int b = blockIdx.x;
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < nblk; ++i) t += part[(long)b * nblk + i];
    mean[b] = t * inv;
  }
}
#endif

// ================================================================ hot path
// P1: first inverse pass along axis 0 for a tile of TC packed columns at fixed k1.
//   V_a(n) = phi_a(cell(|n|^2)) Phi~(n)          (column 0: V(k2=0) + i V(k2=H), each with its own cell)
//   Ta_a = IDFT_0[V_a],  Tb_a = IDFT_0[i n0^D V_a]
template <typename T, int N, int E_ = Shape<T, N>::ES, int TC_ = Shape<T, N>::TC>
__global__ void __launch_bounds__(256) k_p1(const cx<T>* __restrict__ phi, cx<T>* __restrict__ Ta,
                                            cx<T>* __restrict__ Tb, const int16_t* __restrict__ lut,
                                            const T* __restrict__ phitab, int nm1, int alpha0, int nb,
                                            const cx<T>* __restrict__ tw) {
  constexpr int E = E_, P = N / E_, TC = TC_, H = N / 2, NH = H + 1;
  using Lay = StridedLay<T, N, TC, E>;
  extern __shared__ __align__(16) unsigned char smraw[];
  cx<T>* sm_nyq = reinterpret_cast<cx<T>*>(smraw) + Lay::SIZE;  // N values (column 0 only)
  int* sm_cn = reinterpret_cast<int*>(sm_nyq + N);              // N cells
  T* sm_tab = reinterpret_cast<T*>(sm_cn + N);                  // nb * nm1
  const int c = threadIdx.x % TC, j = threadIdx.x / TC;
  const Lay L{reinterpret_cast<cx<T>*>(smraw), c};
  const int cc = blockIdx.x * TC + c;
  const int k1 = blockIdx.y;
  const int b = blockIdx.z;
  const int n1 = wrapn(k1, N);
  for (int i = threadIdx.x; i < nb * nm1; i += blockDim.x) sm_tab[i] = phitab[(long)alpha0 * nm1 + i];
  const cx<T>* pb = phi + ((long)b * N * N + k1) * NH;  // + k0 * N * NH + k2
  if (blockIdx.x == 0) {
    for (int k0 = threadIdx.x; k0 < N; k0 += blockDim.x) {
      const int n0 = wrapn(k0, N);
      sm_nyq[k0] = pb[(long)k0 * N * NH + H];
      sm_cn[k0] = lut[n0 * n0 + n1 * n1 + H * H];
    }
  }
  cx<T> ph[E];
  int cell[E];
#pragma unroll
  for (int r = 0; r < E; ++r) {
    const int k0 = j + r * P;
    const int n0 = wrapn(k0, N);
    ph[r] = pb[(long)k0 * N * NH + cc];
    cell[r] = lut[n0 * n0 + n1 * n1 + cc * cc];
  }
  __syncthreads();
  const long fstride = (long)N * N * H;  // one field
  const T fj = (T)j;
  for (int a = 0; a < nb; ++a) {
    const T* tab = sm_tab + a * nm1;
    // D = 0: V_a; D = 1: i n0 V_a.  V_a is formed again for the second transform instead of being kept,
    // so only one value array is live next to the Phi~ tile.
#pragma unroll 1
    for (int D = 0; D < 2; ++D) {
      cx<T> v[E];
#pragma unroll
      for (int r = 0; r < E; ++r) {
        const T f = tab[cell[r]];
        cx<T> x = mk<T>(f * ph[r].x, f * ph[r].y);
        if (cc == 0) {
          const int k0 = j + r * P;
          const T fn = tab[sm_cn[k0]];
          const cx<T> yn = sm_nyq[k0];
          x = mk<T>(x.x - fn * yn.y, x.y + fn * yn.x);
        }
        if (D) {  // n^D(k0) for k0 = j + r P: j < P, so k0 < N/2 exactly when r < E/2 (Nyquist: r = E/2, j = 0)
          const T nd = r < E / 2 ? fj + (T)(r * P) : ((r == E / 2 && j == 0) ? (T)0 : fj + (T)(r * P - N));
          x = mk<T>(-nd * x.y, nd * x.x);
        }
        v[r] = x;
      }
      fft_pencil<T, N, E, +1, Lay, SyncBlock>(v, j, L, tw, SyncBlock());
      cx<T>* dst = (D ? Tb : Ta) + ((long)b * nb + a) * fstride + (long)k1 * H + cc;
#pragma unroll
      for (int r = 0; r < E; ++r) dst[(long)(j + r * P) * N * H] = v[r];
    }
  }
}

// P2: second inverse pass along axis 1 at fixed a0.  For term a:
//   W[0] = IDFT_1[Ta]            (G_2 after i n2 and the last pass)
//   W[1] = IDFT_1[i n1^D Ta]     (G_1)
//   W[2] = IDFT_1[Tb]            (G_0)
// One value array is live at a time (the Ta tile is reloaded through L1 for the second transform).
template <typename T, int N, int E_ = Shape<T, N>::ES, int TC_ = Shape<T, N>::TC>
__global__ void __launch_bounds__(TC_ * (N / E_), ((E_ >= 32 || TC_ * (N / E_) > 256) ? 1 : 2)) k_p2(const cx<T>* __restrict__ Ta, const cx<T>* __restrict__ Tb,
                                               cx<T>* __restrict__ W, int n_alpha, int alpha0, int nb,
                                               const cx<T>* __restrict__ tw) {
  constexpr int E = E_, P = N / E_, TC = TC_, H = N / 2;
  using Lay = StridedLay<T, N, TC, E>;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int c = threadIdx.x % TC, j = threadIdx.x / TC;
  const Lay L{reinterpret_cast<cx<T>*>(smraw), c};
  const int cc = blockIdx.x * TC + c;
  const int a0 = blockIdx.y;
  const int b = blockIdx.z / nb, a = blockIdx.z % nb;
  const long fstride = (long)N * N * H;
  const long off = (long)a0 * N * H + cc;
  const cx<T>* ta = Ta + ((long)b * nb + a) * fstride + off;
  const cx<T>* tb = Tb + ((long)b * nb + a) * fstride + off;
  auto wout = [&](int f) { return W + (((long)b * 3 + f) * n_alpha + alpha0 + a) * fstride + off; };
  cx<T> v[E];
#pragma unroll
  for (int r = 0; r < E; ++r) v[r] = __ldg(ta + (long)(j + r * P) * H);
  fft_pencil<T, N, E, +1, Lay, SyncBlock>(v, j, L, tw, SyncBlock());
  cx<T>* o0 = wout(0);
#pragma unroll
  for (int r = 0; r < E; ++r) o0[(long)(j + r * P) * H] = v[r];
#pragma unroll
  for (int r = 0; r < E; ++r) {
    const cx<T> x = __ldg(ta + (long)(j + r * P) * H);
    const T nd = (T)derivn(j + r * P, N);
    v[r] = mk<T>(-nd * x.y, nd * x.x);
  }
  fft_pencil<T, N, E, +1, Lay, SyncBlock>(v, j, L, tw, SyncBlock());
  cx<T>* o1 = wout(1);
#pragma unroll
  for (int r = 0; r < E; ++r) o1[(long)(j + r * P) * H] = v[r];
#pragma unroll
  for (int r = 0; r < E; ++r) v[r] = __ldg(tb + (long)(j + r * P) * H);
  fft_pencil<T, N, E, +1, Lay, SyncBlock, false>(v, j, L, tw, SyncBlock());
  cx<T>* o2 = wout(2);
#pragma unroll
  for (int r = 0; r < E; ++r) o2[(long)(j + r * P) * H] = v[r];
}

// ---------------------------------------------------------------- bulk-copy pipeline helpers
// cp.async.bulk (TMA, 1-D) global -> shared with mbarrier completion.  Waits are bounded: after `limit` clock
// cycles (about a second by default) the wait sets *err and gives up, so a lost copy can never hang the GPU.
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// With the default limit the wait uses try_wait, which may suspend the thread for a while inside the instruction;
// with a shorter limit (a test's) it polls with the non-blocking test_wait, so the limit is what decides.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err,
                                          long long limit = kDefaultWaitLimit) {
  const uint32_t a = smem_u32(bar);
  const long long t0 = clock64();
  const bool poll = limit < kDefaultWaitLimit;
  while (true) {
    uint32_t done;
    if (poll) {
      asm volatile(
          "{ .reg .pred p; mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
          : "=r"(done)
          : "r"(a), "r"(parity)
          : "memory");
    } else {
      asm volatile(
          "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
          : "=r"(done)
          : "r"(a), "r"(parity)
          : "memory");
    }
    if (done) return true;
    if (clock64() - t0 > limit) {
      atomicOr(err, 1);
      return false;
    }
  }
}

template <typename T, int N, int E_ = ((N >= 16) ? 8 : 4)> struct P3Cfg {
  static constexpr int H = N / 2;
  static constexpr int E = E_;
  static constexpr int P = N / E;
  static constexpr int STAGES = 2;
  using Lay = RowLayout<T, N, true, 4>;  // single exchange buffer per row
  static constexpr size_t smem_for(int rpc) {
    return (size_t)STAGES * 6 * rpc * H * sizeof(cx<T>) + (size_t)rpc * Lay::SIZE * sizeof(cx<T>) +
           STAGES * sizeof(uint64_t);
  }
  static constexpr int RPC0 = 16384 / (H * (int)sizeof(cx<T>));  // one 16 KB bulk copy per (field, term)
  static constexpr int RPC1 = RPC0 > N * N ? N * N : RPC0;
  static constexpr int RPC = smem_for(RPC1) <= 227 * 1024 ? RPC1 : RPC1 / 2;
  static constexpr int THREADS = RPC * P;
  static constexpr int STAGE_ELEMS = 6 * RPC * H;  // three fields of two terms
  static constexpr size_t SMEM = smem_for(RPC);
  static_assert(SMEM <= 227 * 1024, "shared memory");
};

// Radix-16 alternative of the last inverse pass (autotuner variant bit 2), FP32.  N = 128, 256: one
// shared-memory exchange per transform instead of two.  N = 512: two exchanges either way, but a row is one
// warp (P = 32), so the exchanges need warp barriers only (the radix-8 form uses 64 threads and block barriers).
template <typename T, int N> struct AltP3 {
  static constexpr bool exists = sizeof(T) == 4 && (N == 128 || N == 256 || N == 512);
  static constexpr int E = 16;
};

// 1-D Hermitian spectrum value of a packed row held in shared memory, at the element k = j + r P that thread j
// (0 <= j < P) holds in its r-th register (r unrolled).  plain: k = 0 -> Re row[0], k = N/2 -> Im row[0], else
// row[k] or conj(row[N-k]); grad: i n^D(k) times the plain value, zero at k = 0 and k = N/2.
// With P E = N, k < N/2 exactly when r < E/2, so only j = 0 needs a run-time test (k = 0 and k = N/2 come from
// the packed column 0), and the wave number of the gradient is (T) j plus a compile-time offset.
template <typename T, int N, int E>
__device__ __forceinline__ cx<T> herm_plain_r(const cx<T>* row, int j, int r) {
  constexpr int P = N / E;
  if (r < E / 2) {
    const cx<T> v = row[j + r * P];
    return (r == 0 && j == 0) ? mk<T>(v.x, (T)0) : v;
  }
  const bool hz = (r == E / 2) && (j == 0);
  const cx<T> v = row[hz ? 0 : (E - r) * P - j];
  return hz ? mk<T>(v.y, (T)0) : conjg<T>(v);
}
template <typename T, int N, int E>
__device__ __forceinline__ cx<T> herm_grad_r(const cx<T>* row, int j, int r, T fj) {
  constexpr int P = N / E;
  if (r < E / 2) {
    const cx<T> x = row[j + r * P];
    const T n = fj + (T)(r * P);
    return mk<T>(-n * x.y, n * x.x);
  }
  const bool hz = (r == E / 2) && (j == 0);
  const cx<T> x = conjg<T>(row[hz ? 0 : (E - r) * P - j]);
  const T n = hz ? (T)0 : fj + (T)(r * P - N);
  return mk<T>(-n * x.y, n * x.x);
}

// The same values by a run-time test on k = j + r P.  At N = 512 this form measured faster in the radix-16 last
// pass (the specialised form above costs registers there, where the kernel already spills).
template <typename T, int N, int E>
__device__ __forceinline__ cx<T> herm_plain_k(const cx<T>* row, int j, int r) {
  constexpr int H = N / 2;
  const int k = j + r * (N / E);
  if (k == 0) return mk<T>(row[0].x, (T)0);
  if (k == H) return mk<T>(row[0].y, (T)0);
  if (k < H) return row[k];
  return conjg<T>(row[N - k]);
}
template <typename T, int N, int E>
__device__ __forceinline__ cx<T> herm_grad_k(const cx<T>* row, int j, int r) {
  constexpr int H = N / 2;
  const int k = j + r * (N / E);
  if (k == 0 || k == H) return mk<T>((T)0, (T)0);
  cx<T> x;
  T n;
  if (k < H) {
    x = row[k];
    n = (T)k;
  } else {
    x = conjg<T>(row[N - k]);
    n = (T)(k - N);
  }
  return mk<T>(-n * x.y, n * x.x);
}
template <typename T, int N, int E>
__device__ __forceinline__ cx<T> row_plain(const cx<T>* row, int j, int r) {
  if constexpr (N <= 256) return herm_plain_r<T, N, E>(row, j, r);
  else return herm_plain_k<T, N, E>(row, j, r);
}
template <typename T, int N, int E>
__device__ __forceinline__ cx<T> row_grad(const cx<T>* row, int j, int r, T fj) {
  if constexpr (N <= 256) return herm_grad_r<T, N, E>(row, j, r, fj);
  else return herm_grad_k<T, N, E>(row, j, r);
}

// One term's contribution sigma g_i g_j to the six product components at one point, with zz = (g2, g1):
// a0 = s_00, a21 = (s_22, s_11), a43 = (s_02, s_01), a5 = s_12.  PAIRED (FP32, N <= 256) uses paired (FP32x2)
// multiply-adds; at N = 512 their aligned register pairs made the radix-16 last pass spill, so it stays scalar.
template <typename T, bool PAIRED>
__device__ __forceinline__ void accum6(T sa, T g0, cx<T> zz, T& a0, cx<T>& a21, cx<T>& a43, T& a5) {
  const T s0 = sa * g0;
  const cx<T> t = mk<T>(sa * zz.x, sa * zz.y);
  a21 = mk<T>(fma(t.x, zz.x, a21.x), fma(t.y, zz.y, a21.y));
  a43 = mk<T>(fma(s0, zz.x, a43.x), fma(s0, zz.y, a43.y));
  a0 = fma(s0, g0, a0);
  a5 = fma(t.y, zz.x, a5);
}
template <>
__device__ __forceinline__ void accum6<float, true>(float sa, float g0, float2 zz, float& a0, float2& a21,
                                                    float2& a43, float& a5) {
  const float s0 = sa * g0;
  const float2 t = __fmul2_rn(zz, make_float2(sa, sa));
  a21 = __ffma2_rn(t, zz, a21);
  a43 = __ffma2_rn(make_float2(s0, s0), zz, a43);
  a0 = __fmaf_rn(s0, g0, a0);
  a5 = __fmaf_rn(t.y, zz.x, a5);
}

// P3: last inverse pass (axis 2, C2R) of all terms for RPC consecutive rows, the product
//   s_ij(x) = sum_a sigma_a g^a_i(x) g^a_j(x)  (six components in registers),
// then the forward R2C of s_ij along axis 2 keeping k2 = 0..n_c, written to F[b][comp][a0][a1][k2].
// Term pair (a, a+1) uses three complex transforms: (g2^a + i g1^a), (g0^a + i g0^{a+1}), (g2^{a+1} + i g1^{a+1}).
// The six packed rows of a term pair stream into a STAGES-deep shared-memory ring by cp.async.bulk,
// issued STAGES-1 pairs ahead by thread 0.  Bounded waits: the main loop's waits give up after wait_limit cycles
// (normally kDefaultWaitLimit; a test passes a tiny limit, so that waits give up while the copies still land).
// A thread whose wait gave up sets *err, stops waiting and (thread 0) stops issuing copies; before the CTA exits,
// thread 0 waits, with the default limit, for the last copy issued into each stage, so no bulk copy can still be
// writing into the CTA's shared memory after it has exited.  The results of a launch that set *err are invalid.
template <typename T, int N, int E_ = ((N >= 16) ? 8 : 4)>
__global__ void __launch_bounds__(P3Cfg<T, N, E_>::THREADS, 1) k_p3(const cx<T>* __restrict__ W,
                                                                   const T* __restrict__ sigma, int n_alpha,
                                                                   cx<T>* __restrict__ F, int n_c,
                                                                   const cx<T>* __restrict__ tw,
                                                                   int* __restrict__ err, long long wait_limit) {
  using CF = P3Cfg<T, N, E_>;
  constexpr int E = CF::E, P = CF::P, H = N / 2, RPC = CF::RPC, STAGES = CF::STAGES;
  using Sync = typename RowSync<P>::type;
  using Lay = typename CF::Lay;
  extern __shared__ __align__(128) unsigned char smraw[];
  cx<T>* ring = reinterpret_cast<cx<T>*>(smraw);
  cx<T>* xch = ring + STAGES * CF::STAGE_ELEMS;
  uint64_t* bars = reinterpret_cast<uint64_t*>(xch + RPC * Lay::SIZE);
  const int rr = threadIdx.x / P, j = threadIdx.x % P;
  const Lay L{xch + rr * Lay::SIZE};
  const long row0 = (long)blockIdx.x * RPC;
  const long row = row0 + rr;
  const int b = blockIdx.y;
  const long fstride = (long)N * N * H;
  const int npairs = (n_alpha + 1) / 2;
  constexpr uint32_t COPY = RPC * H * sizeof(cx<T>);
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) mbar_init(bars + s, 1);
    mbar_init_fence();
  }
  __syncthreads();
  auto issue = [&](int pr) {  // thread 0: the six rows blocks of term pair pr into stage pr % STAGES
    const int s = pr % STAGES, a = 2 * pr;
    const bool two = a + 1 < n_alpha;
    cx<T>* dst = ring + s * CF::STAGE_ELEMS;
    fence_proxy_async();
    mbar_expect_tx(bars + s, (two ? 6u : 3u) * COPY);
    for (int f = 0; f < 3; ++f) {
      bulk_g2s(dst + f * RPC * H, W + (((long)b * 3 + f) * n_alpha + a) * fstride + row0 * H, COPY, bars + s);
      if (two) bulk_g2s(dst + (3 + f) * RPC * H, W + (((long)b * 3 + f) * n_alpha + a + 1) * fstride + row0 * H, COPY,
                        bars + s);
    }
  };
  if (threadIdx.x == 0)
    for (int pr = 0; pr < STAGES - 1 && pr < npairs; ++pr) issue(pr);
  T a0[E], a5[E];
  cx<T> a21[E], a43[E];
#pragma unroll
  for (int r = 0; r < E; ++r) {
    a0[r] = a5[r] = (T)0;
    a21[r] = a43[r] = mk<T>((T)0, (T)0);
  }
  const T fj = (T)j;
  bool ok = true;
  int issued = STAGES - 1 < npairs ? STAGES - 1 : npairs;  // term pairs whose copies thread 0 has issued
  for (int pr = 0; pr < npairs; ++pr) {
    const int s = pr % STAGES;
    if (threadIdx.x == 0 && ok && pr + STAGES - 1 < npairs) {
      issue(pr + STAGES - 1);
      issued = pr + STAGES;
    }
    if (ok) ok = mbar_wait(bars + s, (uint32_t)((pr / STAGES) & 1), err, wait_limit);
    const int a = 2 * pr;
    const bool two = a + 1 < n_alpha;
    const cx<T>* st = ring + s * CF::STAGE_ELEMS + rr * H;
    const cx<T>* wb0 = st;
    const cx<T>* w10 = st + RPC * H;
    const cx<T>* w20 = st + 2 * RPC * H;
    const cx<T>* wb1 = st + 3 * RPC * H;
    const cx<T>* w11 = st + 4 * RPC * H;
    const cx<T>* w21 = st + 5 * RPC * H;
    // (g0^a + i g0^{a+1}) first; its two real parts are kept while the other two transforms run
    cx<T> zB[E], z[E];
#pragma unroll
    for (int r = 0; r < E; ++r) {
      const cx<T> g0 = row_plain<T, N, E>(w20, j, r);
      const cx<T> g0b = two ? row_plain<T, N, E>(w21, j, r) : mk<T>((T)0, (T)0);
      zB[r] = mk<T>(g0.x - g0b.y, g0.y + g0b.x);
    }
    fft_pencil<T, N, E, +1, Lay, Sync>(zB, j, L, tw, Sync());
    const T sa = sigma[a];
#pragma unroll
    for (int r = 0; r < E; ++r) {
      const cx<T> g2 = row_grad<T, N, E>(wb0, j, r, fj), g1 = row_plain<T, N, E>(w10, j, r);
      z[r] = mk<T>(g2.x - g1.y, g2.y + g1.x);
    }
    fft_pencil<T, N, E, +1, Lay, Sync>(z, j, L, tw, Sync());
#pragma unroll
    for (int r = 0; r < E; ++r) accum6<T, (sizeof(T) == 4 && N <= 256)>(sa, zB[r].x, z[r], a0[r], a21[r], a43[r], a5[r]);
    if (two) {  // uniform across the CTA
      const T sb = sigma[a + 1];
#pragma unroll
      for (int r = 0; r < E; ++r) {
        const cx<T> h2 = row_grad<T, N, E>(wb1, j, r, fj), h1 = row_plain<T, N, E>(w11, j, r);
        z[r] = mk<T>(h2.x - h1.y, h2.y + h1.x);
      }
      fft_pencil<T, N, E, +1, Lay, Sync>(z, j, L, tw, Sync());
#pragma unroll
      for (int r = 0; r < E; ++r) accum6<T, (sizeof(T) == 4 && N <= 256)>(sb, zB[r].y, z[r], a0[r], a21[r], a43[r], a5[r]);
    }
    __syncthreads();  // stage s fully read before it is refilled
  }
  if (threadIdx.x == 0) {
    // The last copy issued into each stage has landed before the CTA may exit (immediate when every wait
    // succeeded; after a wait gave up, the copies still in flight are waited for with the default limit).
    for (int s = 0; s < STAGES && s < issued; ++s) {
      const int last = s + ((issued - 1 - s) / STAGES) * STAGES;
      mbar_wait(bars + s, (uint32_t)((last / STAGES) & 1), err);
    }
  }
  // forward R2C of the six real rows (00, 11 | 22, 01 | 02, 12), two per complex transform
  cx<T>* zb = L.buf(0);
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    cx<T> z[E];
#pragma unroll
    for (int r = 0; r < E; ++r)
      z[r] = q == 0 ? mk<T>(a0[r], a21[r].y) : (q == 1 ? mk<T>(a21[r].x, a43[r].y) : mk<T>(a43[r].x, a5[r]));
    fft_pencil<T, N, E, -1, Lay, Sync>(z, j, L, tw, Sync());
#pragma unroll
    for (int r = 0; r < E; ++r) zb[L.idx(j + r * P)] = z[r];
    Sync()();
    const int ncp = n_c + 1;
    cx<T>* f1 = F + (((long)b * 6 + 2 * q) * N * N + row) * ncp;
    cx<T>* f2 = F + (((long)b * 6 + 2 * q + 1) * N * N + row) * ncp;
    for (int k = j; k <= n_c; k += P) {
      const cx<T> zk = zb[L.idx(k)];
      const cx<T> zm = conjg<T>(zb[L.idx((N - k) & (N - 1))]);
      f1[k] = mk<T>((T)0.5 * (zk.x + zm.x), (T)0.5 * (zk.y + zm.y));
      f2[k] = mk<T>((T)0.5 * (zk.y - zm.y), (T)-0.5 * (zk.x - zm.x));
    }
    Sync()();
  }
}

// ---------------------------------------------------------------- tensor memory (TMEM) helpers
// A CTA allocates NCOLS 32-bit columns of the SM's tensor memory (128 lanes x 512 columns) with one warp, keeps
// per-thread values in its own lane (warp w may access lanes 32 (w mod 4) .. 32 (w mod 4) + 31), and frees them
// with the same warp before it exits.  No tensor-core instruction is involved: the memory is used as storage.
__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {  // whole warp
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {  // whole warp
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// 16 consecutive columns of this thread's lane into registers; the load and its completion wait are one
// statement, so no use of the values can be scheduled before the wait.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16};" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
      "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
      "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
      "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])), "r"(__float_as_uint(v[15]))
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Two-stage inverse pencil transform of N = 16 R points (R = 8, 16: N = 128, 256), radix 16 then radix R, with the
// last stage's twiddles held in tensor memory.  Thread j of a pencil needs the same NB (R - 1) twiddles
// W^{-r k}, k = (j + t P) mod 16 (t < NB = 16 / R, 0 < r < R), in every transform of a launch; tw_tm_store writes
// them once into 32 columns of its lane (twiddle q = t (R - 1) + r - 1 in columns 2q, 2q + 1), and
// fft_pencil_tw_tm reads them with two tensor-memory loads instead of NB (R - 1) table loads.  Its first stage
// writes the exchange row as 16-byte pairs (RowLayoutV).  Same arithmetic, in the same order, as
// fft_pencil<float, N, 16, +1>.
template <int N> struct TwTm {
  static constexpr int E = 16, P = N / E, R = N / E, NB = E / R;
  static_assert(R >= 2 && R <= E && NB * (R - 1) <= 16, "two stages, at most 16 twiddles");
};
template <int N>
__device__ __forceinline__ void tw_tm_store(uint32_t taddr, int j, const float2* __restrict__ tw) {
  using C = TwTm<N>;
  float w[2][16];
#pragma unroll
  for (int i = 0; i < 16; ++i) w[0][i] = w[1][i] = 0.f;
#pragma unroll
  for (int t = 0; t < C::NB; ++t) {
    const int k = (j + t * C::P) & 15;
#pragma unroll
    for (int r = 1; r < C::R; ++r) {
      const int q = t * (C::R - 1) + r - 1;
      const float2 x = conjg<float>(__ldg(tw + r * k));  // stride N / (16 R) = 1
      w[q >> 3][2 * (q & 7)] = x.x;
      w[q >> 3][2 * (q & 7) + 1] = x.y;
    }
  }
  tmem_st16(taddr, w[0]);
  tmem_st16(taddr + 16, w[1]);
}
template <int N, typename Lay, typename Sync>
__device__ __forceinline__ void fft_pencil_tw_tm(float2 (&v)[16], int j, const Lay& L, uint32_t tw_taddr, Sync sync) {
  using C = TwTm<N>;
  constexpr int E = C::E, P = C::P, R = C::R, NB = C::NB;
  static_assert(Lay::VEC && Lay::SINGLE, "one exchange row with 16-byte pairs");
  float2* x = L.buf(0);
  dftR<float, +1, E>(v);
#pragma unroll
  for (int m = 0; m < E / 2; ++m)
    *reinterpret_cast<float4*>(x + L.idx(j * E + 2 * m)) =
        make_float4(v[2 * m].x, v[2 * m].y, v[2 * m + 1].x, v[2 * m + 1].y);
  sync();
  float w[2][16];
  tmem_ld16(tw_taddr, w[0]);
  tmem_ld16(tw_taddr + 16, w[1]);
#pragma unroll
  for (int t = 0; t < NB; ++t) {
    const int jj = j + t * P;
    float2 a[R];
#pragma unroll
    for (int r = 0; r < R; ++r) a[r] = x[L.idx(jj + r * (N / R))];
#pragma unroll
    for (int r = 1; r < R; ++r) {
      const int q = t * (R - 1) + r - 1;
      a[r] = mul<float>(a[r], make_float2(w[q >> 3][2 * (q & 7)], w[q >> 3][2 * (q & 7) + 1]));
    }
    dftR<float, +1, R>(a);
#pragma unroll
    for (int r = 0; r < R; ++r) v[t + r * NB] = a[r];
  }
  sync();  // the row may be rewritten at once
}
// As fft_pencil<float, N, 16, +1> for a two-stage transform, with the first 8 of the thread's last-stage twiddles
// (q = t (R - 1) + r - 1 < 8, same order as TwTm) taken from 16 columns of its tensor-memory lane (written once by
// tw8_tm_store) and the others from the table.  Any exchange layout.
template <int N>
__device__ __forceinline__ void tw8_tm_store(uint32_t taddr, int j, const float2* __restrict__ tw) {
  using C = TwTm<N>;
  float w[16];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int t = q / (C::R - 1), r = q % (C::R - 1) + 1;
    const float2 x = conjg<float>(__ldg(tw + r * ((j + t * C::P) & 15)));
    w[2 * q] = x.x;
    w[2 * q + 1] = x.y;
  }
  tmem_st16(taddr, w);
}
template <int N, typename Lay, typename Sync>
__device__ __forceinline__ void fft_pencil_tw8_tm(float2 (&v)[16], int j, const Lay& L, const float2* __restrict__ tw,
                                                  uint32_t tw_taddr, Sync sync) {
  using C = TwTm<N>;
  constexpr int E = C::E, P = C::P, R = C::R, NB = C::NB;
  float2* x = L.buf(0);
  dftR<float, +1, E>(v);
#pragma unroll
  for (int r = 0; r < E; ++r) x[L.idx(j * E + r)] = v[r];
  sync();
  float w[16];
  tmem_ld16(tw_taddr, w);
#pragma unroll
  for (int t = 0; t < NB; ++t) {
    const int jj = j + t * P;
    const int k = jj & 15;
    float2 a[R];
#pragma unroll
    for (int r = 0; r < R; ++r) a[r] = x[L.idx(jj + r * (N / R))];
#pragma unroll
    for (int r = 1; r < R; ++r) {
      const int q = t * (R - 1) + r - 1;
      const float2 wr = q < 8 ? make_float2(w[2 * q], w[2 * q + 1]) : twiddle<float, +1>(tw, r * k);
      a[r] = mul<float>(a[r], wr);
    }
    dftR<float, +1, R>(a);
#pragma unroll
    for (int r = 0; r < R; ++r) v[t + r * NB] = a[r];
  }
  sync();  // the exchange buffer may be rewritten at once
}

// P3 with its accumulators in tensor memory (autotuner variant bit 8; FP32, radix 16, N = 128, 256, 512).  The last pass
// above keeps the six product components of its 16 points per thread in registers (96 of its 254), which holds
// it to one CTA of 8 warps per SM.  Here they live in TMEM, in the thread's lane: s00 in columns 0-15, s12 in
// 16-31, (s22, s11) interleaved in 32-63 and (s02, s01) interleaved in 64-95, so a thread needs ~170 registers and
// three CTAs of 128 threads (4 warps; 16, 8 or 4 rows) share an SM.  At N <= 256 (two-stage transforms) columns
// 96-127 hold the thread's last-stage twiddles, and the exchange rows take 16-byte first-stage stores (RowLayoutV).
// One ring stage per CTA: the three transforms' inputs of a term pair are read into registers, the stage is
// refilled for the next pair while the transforms run, and the other CTAs of the SM cover the copy.
// Bounded waits, error flag and the drain before exit as in k_p3.
template <int N>
struct P3TCfg {
  static constexpr int H = N / 2, E = 16, P = N / E, RPC = 128 / P, THREADS = RPC * P;  // 16 / 8 / 4 rows at N = 128 / 256 / 512
  static_assert(THREADS == 128 && P <= 32, "one warp per TMEM lane quarter; a row inside one warp");
  // two-stage transforms (N <= 256): twiddles in TMEM columns 96-127 and 16-byte exchange stores
  static constexpr bool TWTM = N <= 256;
  using Lay = std::conditional_t<TWTM, RowLayoutV<float, N>, RowLayout<float, N, true, 4>>;
  static constexpr int STAGE_ELEMS = 6 * RPC * H;  // three fields of two terms
  static constexpr uint32_t NCOLS = 128;           // TMEM columns per CTA (96, or 128 with the twiddles)
  static constexpr size_t SMEM = (size_t)STAGE_ELEMS * 8 + (size_t)RPC * Lay::SIZE * 8 + 16;
};

template <int N>
__global__ void __launch_bounds__(P3TCfg<N>::THREADS, 3) k_p3_tm(const float2* __restrict__ W,
                                                                  const float* __restrict__ sigma, int n_alpha,
                                                                  float2* __restrict__ F, int n_c,
                                                                  const float2* __restrict__ tw,
                                                                  int* __restrict__ err, long long wait_limit) {
  using CF = P3TCfg<N>;
  constexpr int E = CF::E, P = CF::P, H = CF::H, RPC = CF::RPC;
  using Sync = typename RowSync<P>::type;
  using Lay = typename CF::Lay;
  extern __shared__ __align__(128) unsigned char smraw[];
  float2* ring = reinterpret_cast<float2*>(smraw);
  float2* xch = ring + CF::STAGE_ELEMS;
  uint64_t* bar = reinterpret_cast<uint64_t*>(xch + RPC * Lay::SIZE);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  const int rr = threadIdx.x / P, j = threadIdx.x % P;
  const Lay L{xch + rr * Lay::SIZE};
  const long row0 = (long)blockIdx.x * RPC;
  const long row = row0 + rr;
  const int b = blockIdx.y;
  const long fstride = (long)N * N * H;
  const int npairs = (n_alpha + 1) / 2;
  constexpr uint32_t COPY = RPC * H * sizeof(float2);
  const int warp = threadIdx.x >> 5;
  if (warp == 0) tmem_alloc(tslot, CF::NCOLS);
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    mbar_init_fence();
  }
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  const uint32_t tbase = *tslot + ((uint32_t)(32 * (warp & 3)) << 16);  // this warp's lane quarter
  auto tcol = [&](int c) { return tbase + (uint32_t)(16 * c); };
  {
    float z0[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) z0[i] = 0.f;
#pragma unroll
    for (int c = 0; c < 6; ++c) tmem_st16(tcol(c), z0);
    if constexpr (CF::TWTM) tw_tm_store<N>(tcol(6), j, tw);
    tmem_wait_st();
  }
  auto issue = [&](int pr) {  // thread 0: the six row blocks of term pair pr into the stage
    const int a = 2 * pr;
    const bool two = a + 1 < n_alpha;
    fence_proxy_async();
    mbar_expect_tx(bar, (two ? 6u : 3u) * COPY);
    for (int f = 0; f < 3; ++f) {
      bulk_g2s(ring + f * RPC * H, W + (((long)b * 3 + f) * n_alpha + a) * fstride + row0 * H, COPY, bar);
      if (two) bulk_g2s(ring + (3 + f) * RPC * H, W + (((long)b * 3 + f) * n_alpha + a + 1) * fstride + row0 * H, COPY,
                        bar);
    }
  };
  if (threadIdx.x == 0) issue(0);
  int issued = 1;  // term pairs whose copies thread 0 has issued
  const float fj = (float)j;
  bool ok = true;
  for (int pr = 0; pr < npairs; ++pr) {
    if (ok) ok = mbar_wait(bar, (uint32_t)(pr & 1), err, wait_limit);
    const int a = 2 * pr;
    const bool two = a + 1 < n_alpha;
    const float2* wb0 = ring + rr * H;
    const float2* w10 = wb0 + RPC * H;
    const float2* w20 = wb0 + 2 * RPC * H;
    const float2* wb1 = wb0 + 3 * RPC * H;
    const float2* w11 = wb0 + 4 * RPC * H;
    const float2* w21 = wb0 + 5 * RPC * H;
    // inputs of the three transforms: (g0^a + i g0^{a+1}), (g2^a + i g1^a), (g2^{a+1} + i g1^{a+1}); whether the
    // pair has a second term (all but an odd last pair) is chosen once, not per value
    float2 zB[E], za[E], zb[E];
    auto assemble = [&](auto second) {
      constexpr bool TWO = decltype(second)::value;
#pragma unroll
      for (int r = 0; r < E; ++r) {
        const float2 g0 = row_plain<float, N, E>(w20, j, r);
        const float2 g0b = TWO ? row_plain<float, N, E>(w21, j, r) : make_float2(0.f, 0.f);
        zB[r] = make_float2(g0.x - g0b.y, g0.y + g0b.x);
        const float2 g2 = row_grad<float, N, E>(wb0, j, r, fj), g1 = row_plain<float, N, E>(w10, j, r);
        za[r] = make_float2(g2.x - g1.y, g2.y + g1.x);
        if constexpr (TWO) {
          const float2 h2 = row_grad<float, N, E>(wb1, j, r, fj), h1 = row_plain<float, N, E>(w11, j, r);
          zb[r] = make_float2(h2.x - h1.y, h2.y + h1.x);
        } else {
          zb[r] = make_float2(0.f, 0.f);
        }
      }
    };
    if (two) assemble(std::true_type{});
    else assemble(std::false_type{});
    __syncthreads();  // the stage has been read: refill it for the next pair while the transforms run
    if (threadIdx.x == 0 && ok && pr + 1 < npairs) {
      issue(pr + 1);
      issued = pr + 2;
    }
    if constexpr (CF::TWTM) {
      fft_pencil_tw_tm<N, Lay, Sync>(zB, j, L, tcol(6), Sync());
      fft_pencil_tw_tm<N, Lay, Sync>(za, j, L, tcol(6), Sync());
      fft_pencil_tw_tm<N, Lay, Sync>(zb, j, L, tcol(6), Sync());
    } else {
      fft_pencil<float, N, E, +1, Lay, Sync>(zB, j, L, tw, Sync());
      fft_pencil<float, N, E, +1, Lay, Sync>(za, j, L, tw, Sync());
      fft_pencil<float, N, E, +1, Lay, Sync>(zb, j, L, tw, Sync());
    }
    const float sa = sigma[a], sb = two ? sigma[a + 1] : 0.f;
    // za = (g2a, g1a), zb = (g2b, g1b), zB = (g0a, g0b).  Chunks: s00 and s12 (16 columns each), (s22, s11) and
    // (s02, s01) interleaved (32 columns each), so the pair updates are paired (FP32x2) multiply-adds.
    {
      float u[16];
      tmem_ld16(tcol(0), u);  // s00 += sa g0a^2 + sb g0b^2
#pragma unroll
      for (int r = 0; r < E; ++r) u[r] = fmaf(sb * zB[r].y, zB[r].y, fmaf(sa * zB[r].x, zB[r].x, u[r]));
      tmem_st16(tcol(0), u);
      tmem_ld16(tcol(1), u);  // s12 += sa g1a g2a + sb g1b g2b
#pragma unroll
      for (int r = 0; r < E; ++r) u[r] = fmaf(sb * zb[r].y, zb[r].x, fmaf(sa * za[r].y, za[r].x, u[r]));
      tmem_st16(tcol(1), u);
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {  // points 8 h .. 8 h + 7 of the interleaved chunks
      float u[16], w[16];
      tmem_ld16(tcol(2) + 16 * h, u);  // (s22, s11) += sa (g2a, g1a)^2 + sb (g2b, g1b)^2
      tmem_ld16(tcol(4) + 16 * h, w);  // (s02, s01) += sa g0a (g2a, g1a) + sb g0b (g2b, g1b)
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int r = 8 * h + i;
        float2 c = make_float2(u[2 * i], u[2 * i + 1]);
        c = __ffma2_rn(__fmul2_rn(za[r], make_float2(sa, sa)), za[r], c);
        c = __ffma2_rn(__fmul2_rn(zb[r], make_float2(sb, sb)), zb[r], c);
        u[2 * i] = c.x;
        u[2 * i + 1] = c.y;
        float2 d = make_float2(w[2 * i], w[2 * i + 1]);
        const float t0a = sa * zB[r].x, t0b = sb * zB[r].y;
        d = __ffma2_rn(make_float2(t0a, t0a), za[r], d);
        d = __ffma2_rn(make_float2(t0b, t0b), zb[r], d);
        w[2 * i] = d.x;
        w[2 * i + 1] = d.y;
      }
      tmem_st16(tcol(2) + 16 * h, u);
      tmem_st16(tcol(4) + 16 * h, w);
    }
    tmem_wait_st();
  }
  if (threadIdx.x == 0 && issued > 0) mbar_wait(bar, (uint32_t)((issued - 1) & 1), err);  // drain the last copy
  // forward R2C of the six real rows, two per complex transform: (s00, s11), (s22, s01), (s02, s12)
  float2* zo = L.buf(0);
#pragma unroll 1
  for (int q = 0; q < 3; ++q) {
    float2 z[E];
    {
      float u[16], w[16];
      if (q == 0) {  // s00 and the odd columns of (s22, s11)
        tmem_ld16(tcol(0), u);
#pragma unroll
        for (int r = 0; r < E; ++r) z[r].x = u[r];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          tmem_ld16(tcol(2) + 16 * h, w);
#pragma unroll
          for (int i = 0; i < 8; ++i) z[8 * h + i].y = w[2 * i + 1];
        }
      } else if (q == 1) {  // the even columns of (s22, s11) and the odd ones of (s02, s01)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          tmem_ld16(tcol(2) + 16 * h, u);
          tmem_ld16(tcol(4) + 16 * h, w);
#pragma unroll
          for (int i = 0; i < 8; ++i) z[8 * h + i] = make_float2(u[2 * i], w[2 * i + 1]);
        }
      } else {  // the even columns of (s02, s01) and s12
        tmem_ld16(tcol(1), u);
#pragma unroll
        for (int r = 0; r < E; ++r) z[r].y = u[r];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          tmem_ld16(tcol(4) + 16 * h, w);
#pragma unroll
          for (int i = 0; i < 8; ++i) z[8 * h + i].x = w[2 * i];
        }
      }
    }
    fft_pencil<float, N, E, -1, Lay, Sync>(z, j, L, tw, Sync());
#pragma unroll
    for (int r = 0; r < E; ++r) zo[L.idx(j + r * P)] = z[r];
    Sync()();
    const int ncp = n_c + 1;
    const int c1 = q == 0 ? 0 : (q == 1 ? 2 : 4), c2 = q == 0 ? 1 : (q == 1 ? 3 : 5);
    // stored component order of F: (00, 11, 22, 01, 02, 12) = c = 0..5
    float2* f1 = F + (((long)b * 6 + c1) * N * N + row) * ncp;
    float2* f2 = F + (((long)b * 6 + c2) * N * N + row) * ncp;
    for (int k = j; k <= n_c; k += P) {
      const float2 zk = zo[L.idx(k)];
      const float2 zm = conjg<float>(zo[L.idx((N - k) & (N - 1))]);
      f1[k] = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y + zm.y));
      f2[k] = make_float2(0.5f * (zk.y - zm.y), -0.5f * (zk.x - zm.x));
    }
    Sync()();
  }
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  if (warp == 0) tmem_dealloc(*tslot, CF::NCOLS);
}

// P1 with its Phi~ tile and cell indices in tensor memory (autotuner variant bit 16; FP32, radix 16, 256 threads
// per CTA: 32, 16 or 8 columns at N = 128, 256, 512).  k_p1 keeps each thread's 16 Phi~ values and cells in registers for all the terms of a launch
// (125 registers: two CTAs of 8 warps per SM, latency-bound).  Here they sit in the thread's TMEM lane (columns
// 0-31: Phi~ as (re, im) pairs, 32-47: cells; warps w and w + 4 share a lane quarter, the latter at column 64) and are read back for every transform;
// with a single exchange buffer (free for a two-stage transform; a three-stage
// one syncs between a stage's reads and writes) three CTAs share an SM at 80 registers (measured faster than four at
// 64).  At N <= 256, 8 of each thread's 15 last-stage twiddles also sit in its lane (columns 48-63).  Same arithmetic
// as k_p1.
template <int N>
struct P1TCfg {
  static constexpr int H = N / 2, E = 16, P = N / E, TC = 256 / P, THREADS = TC * P;  // 32 / 16 / 8 columns
  static_assert(THREADS == 256, "two warps per TMEM lane quarter");
  using Lay = ColLayout<float, N, TC, E, true>;
  static constexpr uint32_t NCOLS = 128;  // per warp group: Phi~ 0-31, cells 32-47, 8 twiddles 48-63 (N <= 256)
  static size_t smem(int nb, int nm1) {
    return (size_t)Lay::SIZE * 8 + (size_t)N * 8 + (size_t)N * 4 + (size_t)nb * nm1 * 4 + 16;
  }
};

template <int N>
__global__ void __launch_bounds__(P1TCfg<N>::THREADS, 3) k_p1_tm(const float2* __restrict__ phi, float2* __restrict__ Ta,
                                                                  float2* __restrict__ Tb, const int16_t* __restrict__ lut,
                                                                  const float* __restrict__ phitab, int nm1, int alpha0,
                                                                  int nb, const float2* __restrict__ tw) {
  using CF = P1TCfg<N>;
  constexpr int E = CF::E, P = CF::P, TC = CF::TC, H = CF::H, NH = H + 1;
  using Lay = typename CF::Lay;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* sm_nyq = reinterpret_cast<float2*>(smraw) + Lay::SIZE;  // N values (column 0 only)
  int* sm_cn = reinterpret_cast<int*>(sm_nyq + N);                // N cells
  float* sm_tab = reinterpret_cast<float*>(sm_cn + N);            // nb * nm1
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm_tab + nb * nm1);
  const int c = threadIdx.x % TC, j = threadIdx.x / TC;
  const Lay L{reinterpret_cast<float2*>(smraw), c};
  const int cc = blockIdx.x * TC + c;
  const int k1 = blockIdx.y;
  const int b = blockIdx.z;
  const int n1 = wrapn(k1, N);
  const int warp = threadIdx.x >> 5;
  if (warp == 0) tmem_alloc(tslot, CF::NCOLS);
  for (int i = threadIdx.x; i < nb * nm1; i += blockDim.x) sm_tab[i] = phitab[(long)alpha0 * nm1 + i];
  const float2* pb = phi + ((long)b * N * N + k1) * NH;  // + k0 * N * NH + k2
  if (blockIdx.x == 0) {
    for (int k0 = threadIdx.x; k0 < N; k0 += blockDim.x) {
      const int n0 = wrapn(k0, N);
      sm_nyq[k0] = pb[(long)k0 * N * NH + H];
      sm_cn[k0] = lut[n0 * n0 + n1 * n1 + H * H];
    }
  }
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  const uint32_t tbase = *tslot + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(64 * (warp >> 2));
  {
    float u[16];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int k0 = j + (8 * h + i) * P;
        const float2 v = pb[(long)k0 * N * NH + cc];
        u[2 * i] = v.x;
        u[2 * i + 1] = v.y;
      }
      tmem_st16(tbase + 16 * h, u);
    }
#pragma unroll
    for (int r = 0; r < E; ++r) {
      const int n0 = wrapn(j + r * P, N);
      u[r] = __int_as_float((int)lut[n0 * n0 + n1 * n1 + cc * cc]);
    }
    tmem_st16(tbase + 32, u);
    if constexpr (N <= 256) tw8_tm_store<N>(tbase + 48, j, tw);  // 8 last-stage twiddles in columns 48-63
    tmem_wait_st();
  }
  const long fstride = (long)N * N * H;  // one field
  const float fj = (float)j;
  for (int a = 0; a < nb; ++a) {
    const float* tab = sm_tab + a * nm1;
#pragma unroll 1
    for (int D = 0; D < 2; ++D) {
      float2 v[E];
      {
        // the filter values of this term, looked up from the cells (keeping them in tensor memory for the second
        // field was measured slower)
        float fl[16], u[16];
        tmem_ld16(tbase + 32, fl);
#pragma unroll
        for (int r = 0; r < E; ++r) fl[r] = tab[__float_as_int(fl[r])];
        // the 8 inputs of half h.  DER: times i n0^D(k0), k0 = j + r P (k0 < N/2 exactly when r < E/2; zero on the
        // Nyquist index r = E/2, j = 0), folded into the filter value.  NYQ: the CTA holds packed column 0, whose
        // thread c = 0 adds i V(k2 = N/2) with its own cell.  Both are compile-time, so the other CTAs' loops carry
        // no per-value branches.
        auto fill = [&](auto der, auto nyq, int h) {
          constexpr bool DER = decltype(der)::value, NYQ = decltype(nyq)::value;
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int r = 8 * h + i;
            const float nd = r < E / 2 ? fj + (float)(r * P) : ((r == E / 2 && j == 0) ? 0.f : fj + (float)(r * P - N));
            float2 x;
            if (NYQ && cc == 0) {
              const float f = fl[r];
              x = make_float2(f * u[2 * i], f * u[2 * i + 1]);
              const int k0 = j + r * P;
              const float fn = tab[sm_cn[k0]];
              const float2 yn = sm_nyq[k0];
              x = make_float2(x.x - fn * yn.y, x.y + fn * yn.x);
              if constexpr (DER) x = make_float2(-nd * x.y, nd * x.x);
            } else if constexpr (DER) {
              const float g = fl[r] * nd;
              x = make_float2(-g * u[2 * i + 1], g * u[2 * i]);
            } else {
              const float f = fl[r];
              x = make_float2(f * u[2 * i], f * u[2 * i + 1]);
            }
            v[r] = x;
          }
        };
        const std::true_type yes{};
        const std::false_type no{};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          tmem_ld16(tbase + 16 * h, u);
          if (blockIdx.x == 0) {
            if (D) fill(yes, yes, h);
            else fill(no, yes, h);
          } else {
            if (D) fill(yes, no, h);
            else fill(no, no, h);
          }
        }
      }
      if constexpr (N <= 256) fft_pencil_tw8_tm<N, Lay, SyncBlock>(v, j, L, tw, tbase + 48, SyncBlock());
      else fft_pencil<float, N, E, +1, Lay, SyncBlock>(v, j, L, tw, SyncBlock());
      float2* dst = (D ? Tb : Ta) + ((long)b * nb + a) * fstride + (long)k1 * H + cc;
#pragma unroll
      for (int r = 0; r < E; ++r) dst[(long)(j + r * P) * N * H] = v[r];
    }
  }
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  if (warp == 0) tmem_dealloc(*tslot, CF::NCOLS);
}

// F2: forward DFT along axis 1 of F[b][comp][a0][a1][k2] (k2 = 0..n_c), keeping n1 in [n1lo, n1lo + nk1).
template <typename T, int N>
__global__ void __launch_bounds__(256) k_f2(const cx<T>* __restrict__ F, cx<T>* __restrict__ F2, int n_c, int n1lo,
                                            int nk1, const cx<T>* __restrict__ tw) {
  using SH = Shape<T, N>;
  constexpr int E = SH::ES, P = SH::PS, TC = SH::TC;
  // one exchange buffer (a CTA runs one transform): half the shared memory of two, so more CTAs share an SM
  using Lay = ColLayout<T, N, TC, E, true>;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int c = threadIdx.x % TC, j = threadIdx.x / TC;
  const Lay L{reinterpret_cast<cx<T>*>(smraw), c};
  const int ncp = n_c + 1;
  const int cc = blockIdx.x * TC + c;
  const bool valid = cc < ncp;
  const int a0 = blockIdx.y;
  const long bc = blockIdx.z;  // b * 6 + comp
  const cx<T>* in = F + (bc * N + a0) * (long)N * ncp + cc;
  cx<T> v[E];
#pragma unroll
  for (int r = 0; r < E; ++r) v[r] = valid ? in[(long)(j + r * P) * ncp] : mk<T>((T)0, (T)0);
  fft_pencil<T, N, E, -1, Lay, SyncBlock, false>(v, j, L, tw, SyncBlock());
  if (valid) {
    cx<T>* out = F2 + (bc * N + a0) * (long)nk1 * ncp + cc;
#pragma unroll
    for (int r = 0; r < E; ++r) {
      const int idx = wrapn(j + r * P, N) - n1lo;
      if (idx >= 0 && idx < nk1) out[(long)idx * ncp] = v[r];
    }
  }
}

// The two TT amplitudes e^+_ij(k_hat) S_ij and e^x_ij(k_hat) S_ij (Sec. sec_sigw basis: u = k x e0 / |k x e0|,
// e1 in place of e0 when k is parallel to e0, v = k x u; e^+ = (uu - vv)/sqrt2, e^x = (uv + vu)/sqrt2).
// S = (00, 11, 22, 01, 02, 12).
__device__ __forceinline__ void tt_amp(int n0, int n1, int n2, const double2* S, double2& ap, double2& ax) {
  const double nn = sqrt((double)(n0 * n0 + n1 * n1 + n2 * n2));
  const double k0 = n0 / nn, k1 = n1 / nn, k2 = n2 / nn;
  double u0 = 0.0, u1 = k2, u2 = -k1;  // k x e0
  double un = sqrt(u1 * u1 + u2 * u2);
  if (un < 1e-12) {  // k x e1
    u0 = -k2;
    u1 = 0.0;
    u2 = k0;
    un = sqrt(u0 * u0 + u2 * u2);
  }
  u0 /= un;
  u1 /= un;
  u2 /= un;
  const double v0 = k1 * u2 - k2 * u1, v1 = k2 * u0 - k0 * u2, v2 = k0 * u1 - k1 * u0;
  // S u and S v
  const double2 s00 = S[0], s11 = S[1], s22 = S[2], s01 = S[3], s02 = S[4], s12 = S[5];
  auto sdot = [&](double a0, double a1, double a2, double c0, double c1, double c2) {
    // a . S . c
    double re = a0 * (s00.x * c0 + s01.x * c1 + s02.x * c2) + a1 * (s01.x * c0 + s11.x * c1 + s12.x * c2) +
                a2 * (s02.x * c0 + s12.x * c1 + s22.x * c2);
    double im = a0 * (s00.y * c0 + s01.y * c1 + s02.y * c2) + a1 * (s01.y * c0 + s11.y * c1 + s12.y * c2) +
                a2 * (s02.y * c0 + s12.y * c1 + s22.y * c2);
    return make_double2(re, im);
  };
  const double2 uu = sdot(u0, u1, u2, u0, u1, u2), vv = sdot(v0, v1, v2, v0, v1, v2), uv = sdot(u0, u1, u2, v0, v1, v2);
  ap = make_double2((uu.x - vv.x) * 0.70710678118654752440, (uu.y - vv.y) * 0.70710678118654752440);
  ax = make_double2(uv.x * 1.41421356237309504880, uv.y * 1.41421356237309504880);
}
// Sum over the two polarisations of |e^l_ij(k_hat) S_ij|^2, written with the TT projector instead of the basis:
// sum_l e^l_ij e^l_lm = (P_il P_jm + P_im P_jl - P_ij P_lm) / 2 with P = I - n n^T / |n|^2, which annihilates the
// identity, so S may first lose its trace (S' = S - tr(S) I / 3; that also removes most of the cancellation when S
// is near-isotropic).  For symmetric S':
//   |S'|^2 - 2 |S' n|^2 / |n|^2 + |n.S'.n|^2 / (2 |n|^4),
// rational in the integer mode (one division, no square root) and the same for n and -n.
// R is the arithmetic type (FP64 for the FP64 path).
template <typename R>
__device__ __forceinline__ R tt_power(int n0, int n1, int n2, const cx<R>* S) {
  const R m0 = (R)n0, m1 = (R)n1, m2 = (R)n2;
  const R inv = (R)1 / (m0 * m0 + m1 * m1 + m2 * m2);
  const R third = (R)1 / (R)3;
  const R tx = (S[0].x + S[1].x + S[2].x) * third, ty = (S[0].y + S[1].y + S[2].y) * third;
  const cx<R> s00 = mk<R>(S[0].x - tx, S[0].y - ty), s11 = mk<R>(S[1].x - tx, S[1].y - ty),
              s22 = mk<R>(S[2].x - tx, S[2].y - ty), s01 = S[3], s02 = S[4], s12 = S[5];
  const cx<R> a0 = mk<R>(s00.x * m0 + s01.x * m1 + s02.x * m2, s00.y * m0 + s01.y * m1 + s02.y * m2);
  const cx<R> a1 = mk<R>(s01.x * m0 + s11.x * m1 + s12.x * m2, s01.y * m0 + s11.y * m1 + s12.y * m2);
  const cx<R> a2 = mk<R>(s02.x * m0 + s12.x * m1 + s22.x * m2, s02.y * m0 + s12.y * m1 + s22.y * m2);
  const R qx = m0 * a0.x + m1 * a1.x + m2 * a2.x, qy = m0 * a0.y + m1 * a1.y + m2 * a2.y;
  const R ss = s00.x * s00.x + s00.y * s00.y + s11.x * s11.x + s11.y * s11.y + s22.x * s22.x + s22.y * s22.y +
               (R)2 * (s01.x * s01.x + s01.y * s01.y + s02.x * s02.x + s02.y * s02.y + s12.x * s12.x +
                       s12.y * s12.y);
  const R aa = a0.x * a0.x + a0.y * a0.y + a1.x * a1.x + a1.y * a1.y + a2.x * a2.x + a2.y * a2.y;
  return ss - (R)2 * aa * inv + (R)0.5 * (qx * qx + qy * qy) * inv * inv;
}
// The same power from FP32 components, evaluated in FP32 (the FP32 path's S carries FP32 rounding already; the
// shell sums stay FP64, and their relative error is of order eps_32 |S|^2 / power, ~1e-6).  S is first scaled by an
// exact power of two that brings its largest component near 1, so neither the squares nor the |n|^2 factors leave
// the FP32 range, and the factor is put back in FP64.
__device__ __forceinline__ double tt_power_f32(int n0, int n1, int n2, const float2* S) {
  uint32_t mb = 0;
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    mb = max(mb, __float_as_uint(S[q].x) & 0x7fffffffu);
    mb = max(mb, __float_as_uint(S[q].y) & 0x7fffffffu);
  }
  if (mb == 0) return 0.0;
  const int e = min(max((int)(mb >> 23) - 127, -126), 126);  // exponent of the largest component
  const float sc = __uint_as_float((uint32_t)(127 - e) << 23);  // 2^-e
  float2 T[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) T[q] = make_float2(S[q].x * sc, S[q].y * sc);
  const double back = __longlong_as_double((long long)(1023 + 2 * e) << 52);  // 2^(2e)
  return (double)tt_power<float>(n0, n1, n2, T) * back;
}

// F3: forward DFT along axis 0 of the six components for a tile of columns (n1 fixed, n2 = k2),
// TT projection on the modes of shell n_c and the FP64 sum, one partial per CTA.
// Half-spectrum weight: a stored mode with 0 < k2 < H also stands for its partner wrap(-n), whose
// direction is -n_hat except on Nyquist indices; the partner is projected with its own direction.
// With Xj (jackknife), the amplitudes of the stored shell modes are also written to the standard half spectra
// Xj[b][0] = e^+ : S and Xj[b][1] = -i e^x : S (both Hermitian in this basis away from the Nyquist shell),
// [b][f][k0][k1][k2], k2 = 0..N/2; every other entry is left as it is (zero).
template <typename T, int N>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1) k_f3(const cx<T>* __restrict__ F2, int n_c, int n1lo, int nk1,
                                            double* __restrict__ partial, long pbstride,
                                            const cx<T>* __restrict__ tw, cx<T>* __restrict__ Xj) {
  using SH = Shape<T, N>;
  constexpr int E = SH::E3, P = SH::P3, TC = SH::TC3, H = N / 2;
  using Lay = ColLayout<T, N, TC, E>;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double red[32];
  const int c = threadIdx.x % TC, j = threadIdx.x / TC;
  const Lay L{reinterpret_cast<cx<T>*>(smraw), c};
  const int ncp = n_c + 1;
  const int k1i = blockIdx.y;
  const int n1 = n1lo + k1i;
  const int b = blockIdx.z;
  const long blk = (long)blockIdx.y * gridDim.x + blockIdx.x;
  const int cc0 = blockIdx.x * TC;
  const int rmax = n_c * n_c + n_c;  // |n|^2 < (n_c + 1/2)^2
  const int rmin = n_c * n_c - n_c + 1;  // |n|^2 >= (n_c - 1/2)^2
  if (!(cc0 < ncp && n1 * n1 + cc0 * cc0 <= rmax)) {  // no column of this tile reaches the shell
    if (threadIdx.x == 0) partial[(long)b * pbstride + blk] = 0.0;
    return;
  }
  const int cc = cc0 + c;
  const bool valid = cc < ncp && n1 * n1 + cc * cc <= rmax;
  // all six components are loaded before the first transform, so their latencies overlap (a barrier inside a
  // transform would otherwise hold back the loads of the next component)
  cx<T> X[6][E];
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    const cx<T>* in = F2 + (((long)b * 6 + q) * N * nk1 + k1i) * (long)ncp + (valid ? cc : 0);
#pragma unroll
    for (int r = 0; r < E; ++r) X[q][r] = valid ? in[(long)(j + r * P) * nk1 * ncp] : mk<T>((T)0, (T)0);
  }
#pragma unroll
  for (int q = 0; q < 6; ++q) fft_pencil<T, N, E, -1, Lay, SyncBlock>(X[q], j, L, tw, SyncBlock());
  double acc = 0.0;
  if (valid) {
    const int n2 = cc;
#pragma unroll
    for (int r = 0; r < E; ++r) {
      const int n0 = wrapn(j + r * P, N);
      const int msq = n0 * n0 + n1 * n1 + n2 * n2;
      if (msq >= rmin && msq <= rmax) {
        cx<T> St[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) St[q] = X[q][r];
        auto power = [&](int a0, int a1, int a2) -> double {
          if constexpr (sizeof(T) == 4) return tt_power_f32(a0, a1, a2, St);
          else return tt_power<T>(a0, a1, a2, St);
        };
        const double pw = power(n0, n1, n2);
        acc += pw;
        if (Xj) {
          double2 S[6];
#pragma unroll
          for (int q = 0; q < 6; ++q) S[q] = make_double2((double)X[q][r].x, (double)X[q][r].y);
          double2 ap, ax;
          tt_amp(n0, n1, n2, S, ap, ax);
          constexpr long NNH = (long)N * N * (H + 1);
          const long o = ((long)b * 2 * N + (j + r * P)) * N * (H + 1) + (long)((n1 + N) % N) * (H + 1) + n2;
          Xj[o] = mk<T>((T)ap.x, (T)ap.y);
          Xj[o + NNH] = mk<T>((T)ax.y, (T)-ax.x);
        }
        if (n2 > 0 && n2 < H) {  // the partner -n has the same projector unless n0 or n1 is a Nyquist index
          if (n0 == H || n1 == H) {
            const int p0 = (n0 == H) ? H : -n0, p1 = (n1 == H) ? H : -n1;
            acc += power(p0, p1, -n2);
          } else {
            acc += pw;
          }
        }
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) t += red[w];
    partial[(long)b * pbstride + blk] = t;
  }
}

// Jackknife sub-volume energies: for field f (blockIdx.y) of R[f][x0][x1][x2] and sub-volume `sub` of the M^3
// blocks of s = N/M cells per side, CTA (sub, t) sums R^2 over the plane x0 = a s + t of that block in FP64:
// out[(f * M^3 + sub) * s + t].
template <typename T>
__global__ void __launch_bounds__(256) k_subvol(const T* __restrict__ R, int N, int M, double* __restrict__ out) {
  __shared__ double red[8];
  const int s = N / M;
  const int t = blockIdx.x % s, sub = blockIdx.x / s;
  const int a = sub / (M * M), bb = (sub / M) % M, c = sub % M;
  const long f = blockIdx.y;
  const T* plane = R + (f * N + (long)a * s + t) * N * N;
  double acc = 0.0;
  for (int e = threadIdx.x; e < s * s; e += blockDim.x) {
    const int x1 = bb * s + e / s, x2 = c * s + e % s;
    const double v = (double)plane[(long)x1 * N + x2];
    acc += v * v;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) tot += red[w];
    out[(f * M * M * M + sub) * s + t] = tot;
  }
}

#ifdef SIGW_COMMON_KERNELS
// Deterministic second-stage reduction and the Omega constants:
//   P_X = C^2 sum / (V N_k), C = 4 dx^3 / (n_c^2 V^2), Omega = k_c^3 / (48 pi^2) (P_A + P_B).
__global__ void k_fin(const double* __restrict__ partial, long pbstride, int maxblk, int n_shells,
                      const int* __restrict__ shells, const double* __restrict__ Nk, int N, double L, int tc3,
                      double* __restrict__ out, int batch) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= batch * n_shells) return;
  const int b = i / n_shells, s = i % n_shells;
  const int n_c = shells[s];
  const int H = N / 2;
  const int n1lo = max(-n_c, -H + 1), n1hi = min(n_c, H);
  const int nk1 = n1hi - n1lo + 1;
  const int nblk = ((n_c + 1 + tc3 - 1) / tc3) * nk1;
  double sum[2];
  for (int m = 0; m < 2; ++m) {
    const double* p = partial + (long)b * pbstride + ((long)s * 2 + m) * maxblk;
    double t = 0.0;
    for (int k = 0; k < nblk; ++k) t += p[k];
    sum[m] = t;
  }
  const double pi = 3.14159265358979323846;
  const double V = L * L * L, dx = L / N;
  const double C = 4.0 * dx * dx * dx / ((double)n_c * n_c * V * V);
  const double nk = Nk[s];
  const double PA = C * C * sum[0] / (V * nk), PB = C * C * sum[1] / (V * nk);
  const double kc = n_c * 2.0 * pi / L;
  double* o = out + (long)i * 4;
  o[0] = PA;
  o[1] = PB;
  o[2] = nk;
  o[3] = kc * kc * kc / (48.0 * pi * pi) * (PA + PB);
}

#endif

}  // namespace sigw
