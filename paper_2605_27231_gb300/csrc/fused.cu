// Fused first and second inverse passes (axes 0 and 1) of the hot loop, FP32, N = 256 (autotuner variant bit 32).
//
// The unfused path runs the first inverse pass (filter x derivative, axis 0) and the second (axis 1) as two
// kernels with a two-field intermediate per term in HBM (written once, read once).  Both passes work on one
// packed k2 column at a time, so a column's whole (k0, k1) plane can stay on chip when it is spread over a thread
// block cluster: CL CTAs each transform N/CL k1-pencils along axis 0 (phase A) and store every output value
// straight into the shared memory of the CTA that owns its a0 (distributed shared memory); each CTA then
// transforms its N/CL a0-rows along axis 1 (phase B) and writes the term's three output fields.  Per term and
// realisation the HBM traffic falls from ten field passes to six.
//
// Term a, k2 column c, realisation b (Eq. eq_final_envelopes):
//   phase A, D = 0, 1:  T_D(a0, k1) = IDFT_0[(i n0^D)^D phi_a(cell(|n|^2)) Phi~(k0, k1, c)]   (k1 of this CTA)
//   phase B:  W0 = IDFT_1[T_0],  W1 = IDFT_1[i n1^D T_0],  W2 = IDFT_1[T_1]                   (a0 of this CTA)
// with n^D = 0 on the Nyquist index and the packed column 0 holding V(k2 = 0) + i V(k2 = N/2), as in the unfused
// passes.  The input is Phi~ in k2-major order, Phi~T[b][k2][k0][k1] (k2 = 0..N/2), so that the pencils of one
// column are contiguous in k1.
//
// On-chip state and synchronisation (no cluster barrier inside the term loop):
//  * each thread's Phi~ values and cells of its two phase-A pencils sit in its tensor-memory lane for the whole
//    launch (96 of the CTA's 256 TMEM columns per warp group), so a term reads no Phi~ from L2;
//  * a phase-A value goes to its owner with st.async, which completes on the owner's `full` mbarrier (the owner arms
//    it with the 64 KB its receive buffer takes); the owner waits on `full` before phase B;
//  * after phase B an owner arrives (relaxed, cluster scope) on every CTA's `done` mbarrier (8 arrivals per
//    phase); a CTA waits on its `done` before it scatters the next field into the others' buffers.
//  Both waits are bounded (they set *err and give up; the results of such a launch are invalid).  Cluster barriers
//  are used only at the start (every CTA running, barriers initialised) and at the end (no CTA exits while a
//  remote store or arrival may still target it).
//
// Output layout (swizzled tiles): W[b][f][a][a0][a1 / 8][tile], where a tile holds the 8 rows a1 = 8 t..8 t+7 for
// every packed column c (8 KB), each 64-byte segment (c, rows 0..7) stored as four 16-byte chunks (2 rows each) in
// the order chunk' = (rr / 2) xor ((c / 2) mod 4).  A tile sits at exactly the bytes rows 8 t..8 t+7 of the
// row-major layout occupy, so the last pass bulk-copies it as before (8 rows per CTA at 256^3); its reads of one row
// across c hit distinct banks.
//
// Launch: clusters of 8 CTAs along x (one cluster per packed column), y = realisation; 256 threads, two CTAs per SM
// (about 101 KB of shared memory and 256 TMEM columns each).
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
// Address of the same shared-memory location (32-bit shared::cta address) in CTA `rank` of this cluster.
__device__ __forceinline__ uint32_t dsmem_map(uint32_t local, uint32_t rank) {
  uint32_t ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(local), "r"(rank));
  return ra;
}
// Remote store that completes (8 bytes) on the remote CTA's mbarrier.
__device__ __forceinline__ void st_async_tx(uint32_t ra, float2 v, uint32_t rbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];" ::"r"(ra),
               "f"(v.x), "f"(v.y), "r"(rbar)
               : "memory");
}
__device__ __forceinline__ void remote_arrive(uint32_t rbar) {
  asm volatile("mbarrier.arrive.relaxed.cluster.shared::cluster.b64 _, [%0];" ::"r"(rbar) : "memory");
}

template <int N, int CL>
struct P12Cfg {
  static constexpr int H = N / 2;
  static constexpr int E = 16, P = N / E;  // 16 threads per pencil
  static constexpr int TC = 16;             // pencils per round
  static constexpr int THREADS = TC * P;    // 256
  static constexpr int K1C = N / CL;        // k1 pencils (phase A) and a0 rows (phase B) of one CTA
  static constexpr int ROUNDS = K1C / TC;
  static_assert(K1C % TC == 0 && ROUNDS == 2, "two rounds of 16 pencils");
  static_assert(P * E == N && P <= 32, "a phase-B row must live in one warp");
  using LayA = ColLayout<float, N, TC, E, true>;
  using LayB = RowLayout<float, N, true, 4>;  // one pad per 16: keeps the CTA under 100 KiB of shared memory
  static constexpr size_t RECV = (size_t)K1C * N;  // complex values: one field, [a0 local][k1]
  static constexpr uint32_t RECV_BYTES = (uint32_t)(RECV * sizeof(float2));
  static constexpr size_t XA = LayA::SIZE, XB = (size_t)TC * LayB::SIZE;
  static constexpr size_t XCH = XA > XB ? XA : XB;
  static constexpr uint32_t NCOLS = 256;  // TMEM columns per CTA: 2 warp groups x 2 rounds x 48
  static size_t smem(int nm1) {
    return (RECV + XCH) * sizeof(float2) + (((size_t)nm1 * sizeof(float) + 15) & ~(size_t)15) + 32;
  }
};

// Offset (in complex values) of element (row rr = a1 mod 8, packed column c) inside a swizzled 8-row tile.
__device__ __forceinline__ int tile_off8(int rr, int c) { return (c << 3) + (((rr >> 1) ^ ((c >> 1) & 3)) << 1) + (rr & 1); }

template <int N, int CL>
__global__ void __launch_bounds__(P12Cfg<N, CL>::THREADS, 2)
    k_p12(const float2* __restrict__ phiT, float2* __restrict__ W, const int16_t* __restrict__ lut,
          const float* __restrict__ phitab, int nm1, int n_alpha, int alpha0, int nb, const float2* __restrict__ tw,
          int* __restrict__ err, long long wait_limit) {
  using CF = P12Cfg<N, CL>;
  constexpr int H = CF::H, E = CF::E, P = CF::P, TC = CF::TC, K1C = CF::K1C;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* recv = reinterpret_cast<float2*>(smraw);
  float2* xch = recv + CF::RECV;
  float* sm_tab = reinterpret_cast<float*>(xch + CF::XCH);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smraw + (CF::RECV + CF::XCH) * sizeof(float2) +
                                                (((size_t)nm1 * sizeof(float) + 15) & ~(size_t)15));
  uint64_t* full = bars;
  uint64_t* done = bars + 1;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 2);
  const uint32_t rank = cluster_rank();
  const int c = blockIdx.x / CL;  // packed column
  const int b = blockIdx.y;
  const int t = threadIdx.x;
  const int warp = t >> 5;
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
  if (warp == 0) tmem_alloc(tslot, CF::NCOLS);
  if (t == 0) {
    mbar_init(full, 1);
    mbar_init(done, CL);
    mbar_init_fence();
  }
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  const uint32_t tbase = *tslot + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(96 * (warp >> 2));
  // this thread's Phi~ values (columns 48 q .. 48 q + 31) and cells (48 q + 32 ..) of its two phase-A pencils
#pragma unroll
  for (int q = 0; q < CF::ROUNDS; ++q) {
    const int k1 = K1C * (int)rank + TC * q + pA;
    const int n1 = wrapn(k1, N);
    float u[16];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int k0 = jA + (8 * h + i) * P;
        const float2 v = __ldg(col0 + (long)k0 * N + k1);
        u[2 * i] = v.x;
        u[2 * i + 1] = v.y;
      }
      tmem_st16(tbase + 48 * q + 16 * h, u);
    }
#pragma unroll
    for (int s = 0; s < E; ++s) {
      const int n0 = wrapn(jA + s * P, N);
      u[s] = __int_as_float((int)lut[n0 * n0 + n1 * n1 + c * c]);
    }
    tmem_st16(tbase + 48 * q + 32, u);
  }
  tmem_wait_st();
  const uint32_t recv_l = smem_u32(recv), full_l = smem_u32(full), done_l = smem_u32(done);
  cluster_sync();  // every CTA runs and has initialised its barriers before any remote operation
  bool ok = true;
  int phase = 0;
  for (int ai = 0; ai < nb; ++ai) {
    const int a = alpha0 + ai;
    __syncthreads();  // the previous term's phase-A reads of the table are done
    for (int i = t; i < nm1; i += CF::THREADS) sm_tab[i] = phitab[(long)a * nm1 + i];
    __syncthreads();
    for (int D = 0; D < 2; ++D, ++phase) {
      // every owner has read its receive buffer of the previous phase
      if (phase > 0 && ok) ok = mbar_wait(done, (uint32_t)((phase - 1) & 1), err, wait_limit);
      if (t == 0) mbar_expect_tx(full, CF::RECV_BYTES);  // arm this phase: the 64 KB the others store here
      // ---- phase A: axis-0 transforms of this CTA's k1 pencils, stored to the a0 owners
#pragma unroll 1
      for (int q = 0; q < CF::ROUNDS; ++q) {
        const int k1 = K1C * (int)rank + TC * q + pA;
        const int n1 = wrapn(k1, N);
        float2 v[E];
        {
          float cl[16], u[16];
          tmem_ld16(tbase + 48 * q + 32, cl);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            tmem_ld16(tbase + 48 * q + 16 * h, u);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const int s = 8 * h + i;
              const float f = sm_tab[__float_as_int(cl[s])];
              float2 x = make_float2(f * u[2 * i], f * u[2 * i + 1]);
              const int k0 = jA + s * P;
              if (c == 0) {  // + i V(k2 = N/2), with its own cell
                const int n0 = wrapn(k0, N);
                const float2 yh = __ldg(colH + (long)k0 * N + k1);
                const float fn = sm_tab[lut[n0 * n0 + n1 * n1 + H * H]];
                x = make_float2(x.x - fn * yh.y, x.y + fn * yh.x);
              }
              if (D) {  // i n0^D, zero on the Nyquist index
                const float nd = (float)derivn(k0, N);
                x = make_float2(-nd * x.y, nd * x.x);
              }
              v[s] = x;
            }
          }
        }
        fft_pencil<float, N, E, +1, typename CF::LayA, SyncBlock>(v, jA, LA, tw, SyncBlock());
        // value s is a0 = j + s P: owner CTA a0 / K1C, row a0 mod K1C of its receive buffer, column k1
        static_assert(K1C == 2 * P, "a0 = j + s P: owner s / 2, row j + P (s mod 2)");
#pragma unroll
        for (int s = 0; s < E; ++s) {
          const uint32_t owner = (uint32_t)(s >> 1);
          const uint32_t off = (uint32_t)(((jA + P * (s & 1)) * N + k1) * sizeof(float2));
          st_async_tx(dsmem_map(recv_l + off, owner), v[s], dsmem_map(full_l, owner));
        }
      }
      // ---- phase B: axis-1 transforms of this CTA's a0 rows once its buffer is complete
      if (ok) ok = mbar_wait(full, (uint32_t)(phase & 1), err, wait_limit);
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
          // value s is a1 = j + s P: tile a1 / 8, row a1 mod 8
#pragma unroll
          for (int s = 0; s < E; ++s) {
            const int a1 = jB + s * P;
            dst[(long)(a1 >> 3) * (8 * H) + tile_off8(a1 & 7, c)] = v[s];
          }
        }
      }
      __syncthreads();  // every thread of this CTA has read its receive buffer
      if (t < CL) remote_arrive(dsmem_map(done_l, (uint32_t)t));  // tell CTA t its stores may begin
    }
  }
  cluster_sync();  // no remote store or arrival can still target an exited CTA
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  if (warp == 0) tmem_dealloc(*tslot, CF::NCOLS);
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
                      int alpha0, int nb, int batch, const void* tw, int* err, long long wait_limit,
                      cudaStream_t st) {
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
                            nb, (const float2*)tw, err, wait_limit);
}

}  // namespace sigw
