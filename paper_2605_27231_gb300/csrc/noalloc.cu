// sigw_fft3d_noalloc: the library's 3-D real FFT for callers that cannot allocate device memory.
//
// The plan-based sigw_fft3d keeps its intermediate (the packed half spectrum) in memory the plan
// allocated with cudaMalloc.  Some callers cannot make that allocation: a host application that has
// already handed all device memory to its own pool allocator, or a latency-critical path where a
// cudaMalloc (which may synchronise the device) is not acceptable.  This entry point takes its
// scratch from file-scope __device__ arrays instead, so it calls no cudaMalloc, cudaFree or other
// allocating routine.
//
// The arrays live in every GPU that loads the library until the process exits:
//   g_scratch   8 MiB: the packed half spectrum, N*N*(N/2) complex values of the requested precision;
//               this bounds N to <= 128 for FP32 and <= 64 for FP64.
//   g_tw_f32 / g_tw_f64: the FP64-generated twiddle tables of every supported N (8..128), 248 entries each.
// Host code cannot use a __device__ array's name as a device address (in host code it names a host-side
// stand-in), so the first call on each device looks the addresses up with cudaGetSymbolAddress while that
// device is current, fills the twiddle tables, waits for the device, and caches the addresses for that device.
// The cache lives as long as the process: resetting a device (cudaDeviceReset) after its first call here is
// not supported, because the reloaded module would hold empty tables, possibly at other addresses.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <vector>

#include "../../include/sigw.h"
#include "ops.h"
#include "plan.h"

namespace {

constexpr size_t kScratchBytes = 8u << 20;  // 8 MiB
constexpr int kMaxDevices = 64;
constexpr int kTwEntries = 8 + 16 + 32 + 64 + 128;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];
static __device__ __align__(256) float2 g_tw_f32[kTwEntries];
static __device__ __align__(256) double2 g_tw_f64[kTwEntries];

struct DevState {
  bool ready = false;
  void* scratch = nullptr;
  float2* tw32 = nullptr;
  double2* tw64 = nullptr;
};

std::mutex g_mu;
DevState g_dev[kMaxDevices];

int tw_offset(int N) {  // offset of the table of N in the concatenated tables (8, 16, ..., 128)
  int off = 0;
  for (int n = 8; n < N; n *= 2) off += n;
  return off;
}

// Set-up on the current device (once): look up the arrays' device addresses and fill the twiddles.
cudaError_t setup(int dev, DevState** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  DevState& s = g_dev[dev];
  if (!s.ready) {
    cudaError_t e;
    if ((e = cudaGetSymbolAddress(&s.scratch, g_scratch)) != cudaSuccess) return e;
    if ((e = cudaGetSymbolAddress((void**)&s.tw32, g_tw_f32)) != cudaSuccess) return e;
    if ((e = cudaGetSymbolAddress((void**)&s.tw64, g_tw_f64)) != cudaSuccess) return e;
    std::vector<float2> t32(kTwEntries);
    std::vector<double2> t64(kTwEntries);
    for (int N = 8; N <= 128; N *= 2) {
      std::vector<double> tw;
      sigw::build_twiddles(N, tw);
      const int o = tw_offset(N);
      for (int k = 0; k < N; ++k) {
        t64[o + k] = make_double2(tw[2 * k], tw[2 * k + 1]);
        t32[o + k] = make_float2((float)tw[2 * k], (float)tw[2 * k + 1]);
      }
    }
    if ((e = cudaMemcpy(s.tw32, t32.data(), sizeof(float2) * kTwEntries, cudaMemcpyHostToDevice)) != cudaSuccess)
      return e;
    if ((e = cudaMemcpy(s.tw64, t64.data(), sizeof(double2) * kTwEntries, cudaMemcpyHostToDevice)) != cudaSuccess)
      return e;
    // A copy from pageable host memory may return before the data has reached the device, and the caller's
    // stream may be a non-blocking one that is not ordered after these copies: wait for the device before
    // any kernel can read the tables.
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return e;
    s.ready = true;
  }
  *out = &s;
  return cudaSuccess;
}

template <typename T>
cudaError_t run_fft(int N, int direction, const void* in, void* out, void* scratch, const void* tw, cudaStream_t st) {
  using O = sigw::OpsRT<T>;
  cudaError_t e;
  if (direction < 0) {
    if ((e = O::rows_r2c_real(N, in, scratch, 1, tw, st)) != cudaSuccess) return e;
    if ((e = O::pass(N, scratch, 1, -1, 1, tw, st)) != cudaSuccess) return e;
    if ((e = O::pass(N, scratch, 0, -1, 1, tw, st)) != cudaSuccess) return e;
    return O::unpack(N, scratch, out, 1, nullptr, 0, 1.0, 1, st);
  }
  if ((e = O::pack(N, in, scratch, 1, st)) != cudaSuccess) return e;
  if ((e = O::pass(N, scratch, 0, +1, 1, tw, st)) != cudaSuccess) return e;
  if ((e = O::pass(N, scratch, 1, +1, 1, tw, st)) != cudaSuccess) return e;
  return O::rows_c2r(N, scratch, out, 1, 1.0, nullptr, tw, st);
}

}  // namespace

extern "C" sigw_status sigw_fft3d_noalloc(int N, int precision, int direction, const void* in_dev, void* out_dev,
                                          void* cuda_stream) {
  if (!in_dev || !out_dev || (direction != -1 && direction != 1) || (precision != 32 && precision != 64))
    return SIGW_EINVAL;
  if (N < 8 || N > 128 || (N & (N - 1)) != 0) return SIGW_EINVAL;
  const size_t need = (size_t)N * N * (N / 2) * (precision == 64 ? sizeof(double2) : sizeof(float2));
  if (need > kScratchBytes) return SIGW_EINVAL;  // FP32: N <= 128; FP64: N <= 64
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    (void)cudaGetLastError();
    return SIGW_ECUDA;
  }
  DevState* s = nullptr;
  if (setup(dev, &s) != cudaSuccess) {
    (void)cudaGetLastError();
    return SIGW_ECUDA;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int o = tw_offset(N);
  const cudaError_t e = precision == 64 ? run_fft<double>(N, direction, in_dev, out_dev, s->scratch, s->tw64 + o, st)
                                        : run_fft<float>(N, direction, in_dev, out_dev, s->scratch, s->tw32 + o, st);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return SIGW_ECUDA;
  }
  return SIGW_OK;
}
