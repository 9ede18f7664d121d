// Fused first and second inverse passes (axes 0 and 1) of the hot loop, FP32, N = 256.
//
// The unfused path runs the first inverse pass (filter x derivative, axis 0) and the second (axis 1) as two
// kernels with a two-field intermediate per term in HBM (written once, read once).  Both passes work on one
// packed k2 column at a time, so a column's whole (k0, k1) plane can stay on chip if it is spread over a thread
// block cluster: CL CTAs each transform N/CL k1-pencils along axis 0 (phase A), write every output value straight
// into the shared memory of the CTA that owns its a0 (distributed shared memory), and after a cluster barrier
// each CTA transforms its N/CL a0-rows along axis 1 (phase B) and writes the three output fields of the term.
// Per term and realisation the HBM traffic falls from ten field passes (two written and read by the first pass,
// three written and read by the second and the last) to six.
//
// Term a, k2 column c, realisation b (Eq. eq_final_envelopes):
//   phase A, D = 0, 1:  T_D(a0, k1) = IDFT_0[(i n0^D)^D phi_a(cell(|n|^2)) Phi~(k0, k1, c)]   (k1 of this CTA)
//   phase B:  W0 = IDFT_1[T_0],  W1 = IDFT_1[i n1^D T_0],  W2 = IDFT_1[T_1]                   (a0 of this CTA)
// with n^D = 0 on the Nyquist index and the packed column 0 holding V(k2 = 0) + i V(k2 = N/2), as in the unfused
// passes.  The input is Phi~ in k2-major order, Phi~T[b][k2][k0][k1] (k2 = 0..N/2), so that the pencils of one
// column are contiguous in k1.
//
// Output layout (swizzled tiles): W[b][f][a][a0][a1 / 16][tile], where a tile holds the 16 rows a1 = 16 t..16 t+15
// for every packed column c (16 KB at N = 256), each 128-byte segment (c, rows 0..15) stored as eight 16-byte
// chunks (2 rows each) in the order chunk' = (rr / 2) xor (c mod 8).  A tile therefore sits at exactly the bytes
// rows 16 t..16 t+15 of the row-major layout occupy, the last pass loads it with one bulk copy as before, and its
// shared-memory reads of one row across c hit distinct banks.
//
// Launch: clusters of CL = 8 CTAs along x (one cluster per packed column), y = realisation; 256 threads, two CTAs
// per SM (about 101 KB of shared memory each).  Every CTA runs the same sequence of cluster barriers (no early
// exit); the barriers are hardware barriers, not spin loops.
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.cuh"
#include "ops.h"

namespace sigw {
namespace {

constexpr int kCL = 8;  // CTAs per cluster

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Address of the same shared-memory location in CTA `rank` of this cluster.
__device__ __forceinline__ uint32_t dsmem_map(const void* local, uint32_t rank) {
  uint32_t ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(smem_u32(local)), "r"(rank));
  return ra;
}
__device__ __forceinline__ void dsmem_st(uint32_t ra, float2 v) {
  asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(ra), "f"(v.x), "f"(v.y) : "memory");
}

template <int N, int CL>
struct P12Cfg {
  static constexpr int H = N / 2;
  static constexpr int E = 16, P = N / E;  // 16 threads per pencil
  static constexpr int TC = 16;             // pencils per round
  static constexpr int THREADS = TC * P;    // 256
  static constexpr int K1C = N / CL;        // k1 pencils (phase A) and a0 rows (phase B) of one CTA
  static constexpr int ROUNDS = K1C / TC;
  static_assert(K1C % TC == 0, "rounds");
  static_assert(P * E == N && P <= 32, "a phase-B row must live in one warp");
  using LayA = ColLayout<float, N, TC, E, true>;
  using LayB = RowLayout<float, N, true, 3>;
  static constexpr size_t RECV = (size_t)K1C * N;  // complex values: one field, [a0 local][k1]
  static constexpr size_t XA = LayA::SIZE, XB = (size_t)TC * LayB::SIZE;
  static constexpr size_t XCH = XA > XB ? XA : XB;
  static size_t smem(int nm1) { return (RECV + XCH) * sizeof(float2) + (size_t)nm1 * sizeof(float); }
};

// Offset (in complex values) of element (row rr = a1 mod 16, packed column c) inside a swizzled 16-row tile.
__device__ __forceinline__ int tile_off(int rr, int c) { return (((c << 3) + ((rr >> 1) ^ (c & 7))) << 1) + (rr & 1); }

template <int N, int CL>
__global__ void __launch_bounds__(P12Cfg<N, CL>::THREADS, 2)
    k_p12(const float2* __restrict__ phiT, float2* __restrict__ W, const int16_t* __restrict__ lut,
          const float* __restrict__ phitab, int nm1, int n_alpha, int alpha0, int nb, const float2* __restrict__ tw) {
  using CF = P12Cfg<N, CL>;
  constexpr int H = CF::H, E = CF::E, P = CF::P, TC = CF::TC, K1C = CF::K1C;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* recv = reinterpret_cast<float2*>(smraw);
  float2* xch = recv + CF::RECV;
  float* sm_tab = reinterpret_cast<float*>(xch + CF::XCH);
  const uint32_t rank = cluster_rank();
  const int c = blockIdx.x / CL;  // packed column
  const int b = blockIdx.y;
  const int t = threadIdx.x;
  // phase A: pencil p of a round, thread j of the pencil (column-tile convention: t = j TC + p)
  const int pA = t % TC, jA = t / TC;
  const typename CF::LayA LA{xch, pA};
  // phase B: row of a round, thread j of the row (row convention: t = row P + j)
  const int rB = t / P, jB = t % P;
  const typename CF::LayB LB{xch + rB * CF::LayB::SIZE};
  const long plane = (long)N * N;
  const float2* col0 = phiT + ((long)b * (H + 1) + c) * plane;
  const float2* colH = phiT + ((long)b * (H + 1) + H) * plane;  // k2 = N/2 plane (packed into column 0)
  const long fstride = (long)N * N * H;
  const float fj = (float)jB;
  cluster_sync();  // every CTA of the cluster is running before any distributed shared-memory store
  for (int ai = 0; ai < nb; ++ai) {
    const int a = alpha0 + ai;
    for (int i = t; i < nm1; i += CF::THREADS) sm_tab[i] = phitab[(long)a * nm1 + i];
    __syncthreads();
    for (int D = 0; D < 2; ++D) {
      // ---- phase A: axis-0 transforms of this CTA's k1 pencils, scattered to the a0 owners
#pragma unroll 1
      for (int q = 0; q < CF::ROUNDS; ++q) {
        const int k1 = K1C * (int)rank + TC * q + pA;
        const int n1 = wrapn(k1, N);
        float2 v[E];
#pragma unroll
        for (int s = 0; s < E; ++s) {
          const int k0 = jA + s * P;
          const int n0 = wrapn(k0, N);
          const int m01 = n0 * n0 + n1 * n1;
          const float2 ph = __ldg(col0 + (long)k0 * N + k1);
          const float f = sm_tab[lut[m01 + c * c]];
          float2 x = make_float2(f * ph.x, f * ph.y);
          if (c == 0) {  // + i V(k2 = N/2), with its own cell
            const float2 yh = __ldg(colH + (long)k0 * N + k1);
            const float fn = sm_tab[lut[m01 + H * H]];
            x = make_float2(x.x - fn * yh.y, x.y + fn * yh.x);
          }
          if (D) {  // i n0^D, zero on the Nyquist index (s = E/2 with j = 0)
            const float nd = (float)derivn(k0, N);
            x = make_float2(-nd * x.y, nd * x.x);
          }
          v[s] = x;
        }
        fft_pencil<float, N, E, +1, typename CF::LayA, SyncBlock>(v, jA, LA, tw, SyncBlock());
        // value s is a0 = j + s P: owner CTA a0 / K1C, row a0 mod K1C of its receive buffer, column k1
#pragma unroll
        for (int s = 0; s < E; ++s) {
          const int a0 = jA + s * P;
          dsmem_st(dsmem_map(recv + (long)(a0 % K1C) * N + k1, (uint32_t)(a0 / K1C)), v[s]);
        }
      }
      cluster_sync();  // the field is complete in every CTA's receive buffer
      // ---- phase B: axis-1 transforms of this CTA's a0 rows; D = 0 gives W0 and W1, D = 1 gives W2
#pragma unroll 1
      for (int q = 0; q < CF::ROUNDS; ++q) {
        const int la0 = TC * q + rB;
        const int a0 = K1C * (int)rank + la0;
        const float2* row = recv + (long)la0 * N;
#pragma unroll 1
        for (int g = 0; g < (D ? 1 : 2); ++g) {
          float2 v[E];
#pragma unroll
          for (int s = 0; s < E; ++s) {
            const float2 x = row[jB + s * P];
            if (g) {  // i n1^D: k1 = j + s P < N/2 exactly when s < E/2; the Nyquist index is s = E/2, j = 0
              const float nd = s < E / 2 ? fj + (float)(s * P)
                                         : ((s == E / 2 && jB == 0) ? 0.f : fj + (float)(s * P - N));
              v[s] = make_float2(-nd * x.y, nd * x.x);
            } else {
              v[s] = x;
            }
          }
          fft_pencil<float, N, E, +1, typename CF::LayB, SyncWarp>(v, jB, LB, tw, SyncWarp());
          const int f = D ? 2 : g;
          float2* dst = W + (((long)b * 3 + f) * n_alpha + a) * fstride + (long)a0 * N * H;
          // value s is a1 = j + s P: tile a1 / 16, row a1 mod 16
#pragma unroll
          for (int s = 0; s < E; ++s) {
            const int a1 = jB + s * P;
            dst[(long)(a1 >> 4) * (16 * H) + tile_off(a1 & 15, c)] = v[s];
          }
        }
      }
      cluster_sync();  // every receive buffer has been read before the next scatter
    }
  }
}

// Phi~ (standard half spectrum X[b][k0][k1][k2], k2 = 0..N/2) to k2-major order XT[b][k2][k0][k1]: a 32 x 32
// shared-memory tile transpose of (k1, k2) per (b, k0).
__global__ void __launch_bounds__(256) k_phi_k2major(const float2* __restrict__ X, float2* __restrict__ XT, int N) {
  __shared__ float2 tile[32][33];
  const int NH = N / 2 + 1;
  const int k2b = blockIdx.x * 32, k1b = blockIdx.y * 32;
  const long bk0 = blockIdx.z;  // b * N + k0
  const long b = bk0 / N, k0 = bk0 % N;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  for (int y = ty; y < 32; y += 8) {
    const int k1 = k1b + y, k2 = k2b + tx;
    if (k1 < N && k2 < NH) tile[y][tx] = X[(bk0 * N + k1) * NH + k2];
  }
  __syncthreads();
  for (int y = ty; y < 32; y += 8) {
    const int k2 = k2b + y, k1 = k1b + tx;
    if (k1 < N && k2 < NH) XT[((b * NH + k2) * N + k0) * N + k1] = tile[tx][y];
  }
}

}  // namespace

bool fused_supported(int N, int precision) { return precision == 32 && N == 256; }

cudaError_t fused_phi_k2major(int N, const void* X, void* XT, int batch, cudaStream_t st) {
  if (N < 32) return cudaErrorInvalidValue;
  const int NH = N / 2 + 1;
  dim3 grid((NH + 31) / 32, (N + 31) / 32, batch * N);
  k_phi_k2major<<<grid, 256, 0, st>>>((const float2*)X, (float2*)XT, N);
  return cudaGetLastError();
}

cudaError_t fused_p12(int N, const void* phiT, void* W, const int16_t* lut, const void* phitab, int nm1, int n_alpha,
                      int alpha0, int nb, int batch, const void* tw, cudaStream_t st) {
  if (N != 256) return cudaErrorInvalidValue;
  constexpr int NN = 256;
  using CF = P12Cfg<NN, kCL>;
  auto k = k_p12<NN, kCL>;
  const size_t sm = CF::smem(nm1);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kCL * (NN / 2), batch, 1);
  cfg.blockDim = dim3(CF::THREADS, 1, 1);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = kCL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, (const float2*)phiT, (float2*)W, lut, (const float*)phitab, nm1, n_alpha, alpha0,
                            nb, (const float2*)tw);
}

}  // namespace sigw
