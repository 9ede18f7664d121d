// Device FFT building blocks: in-register radix-2/4/8/16 DFTs and a mixed-radix
// Stockham pencil transform with shared-memory exchanges between stages.
//
// A length-N pencil (N = 2^p, 8 <= N <= 512) is owned by P = N/E threads, each
// holding E complex values.  On entry thread j holds x[j + r*P] in v[r]; on exit
// it holds X[j + r*P] in v[r].  That convention makes global loads and stores of
// a pencil coalesced whether the pencil is contiguous (consecutive j -> consecutive
// addresses) or one column of a tile of adjacent pencils.
//
// Stage s (radix R, span Ns = product of the earlier radices) is the Stockham
// autosort step: butterfly jj reads in[jj + r N/R], multiplies by W_{Ns R}^{r (jj mod Ns)},
// applies DFT_R and writes out[(jj/Ns) Ns R + jj mod Ns + r Ns].  All stages but the
// last have radix E; the last has radix N / E^(S-1).  Twiddles come from a table of
// the N-th roots of unity built on the host in FP64 (stored in the working precision).
// DIR = -1 is the forward transform e^{-2 pi i k n / N}, DIR = +1 the unnormalised inverse.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace sigw {

template <typename T> struct vec2;
template <> struct vec2<float> { using type = float2; };
template <> struct vec2<double> { using type = double2; };
template <typename T> using cx = typename vec2<T>::type;

template <typename T> __host__ __device__ __forceinline__ cx<T> mk(T a, T b) { cx<T> r; r.x = a; r.y = b; return r; }
template <typename T> __device__ __forceinline__ cx<T> add(cx<T> a, cx<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ cx<T> sub(cx<T> a, cx<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
// FP32: one paired (FP32x2) instruction per complex add / subtract (a - b as fma(b, -1, a), exact).
template <> __device__ __forceinline__ cx<float> add<float>(cx<float> a, cx<float> b) { return __fadd2_rn(a, b); }
template <> __device__ __forceinline__ cx<float> sub<float>(cx<float> a, cx<float> b) {
  return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}
template <typename T> __device__ __forceinline__ cx<T> mul(cx<T> a, cx<T> b) {
  return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T> __device__ __forceinline__ cx<T> conjg(cx<T> a) { return mk<T>(a.x, -a.y); }
template <typename T> __device__ __forceinline__ cx<T> scale(cx<T> a, T s) { return mk<T>(a.x * s, a.y * s); }
// multiply by i*DIR (DIR = +1: i, DIR = -1: -i)
template <typename T, int DIR> __device__ __forceinline__ cx<T> mul_i(cx<T> a) {
  return DIR > 0 ? mk<T>(-a.y, a.x) : mk<T>(a.y, -a.x);
}
// multiply by the root W = (c + i DIR s)
template <typename T, int DIR> __device__ __forceinline__ cx<T> rot(cx<T> a, T c, T s) {
  return DIR > 0 ? mk<T>(a.x * c - a.y * s, a.x * s + a.y * c) : mk<T>(a.x * c + a.y * s, a.y * c - a.x * s);
}

// ---------------------------------------------------------------- in-register DFTs
template <typename T, int DIR> __device__ __forceinline__ void dft2(cx<T>& a, cx<T>& b) {
  cx<T> t = a;
  a = add<T>(t, b);
  b = sub<T>(t, b);
}

template <typename T, int DIR> __device__ __forceinline__ void dft4(cx<T>* v) {
  cx<T> s0 = add<T>(v[0], v[2]), d0 = sub<T>(v[0], v[2]);
  cx<T> s1 = add<T>(v[1], v[3]), d1 = mul_i<T, DIR>(sub<T>(v[1], v[3]));
  v[0] = add<T>(s0, s1);
  v[2] = sub<T>(s0, s1);
  v[1] = add<T>(d0, d1);
  v[3] = sub<T>(d0, d1);
}

// radix-2 split of an 8-point DFT into two 4-point DFTs
template <typename T, int DIR> __device__ __forceinline__ void dft8(cx<T>* v) {
  const T h = (T)0.70710678118654752440;  // sqrt(2)/2
  cx<T> e[4] = {v[0], v[2], v[4], v[6]};
  cx<T> o[4] = {v[1], v[3], v[5], v[7]};
  dft4<T, DIR>(e);
  dft4<T, DIR>(o);
  o[1] = rot<T, DIR>(o[1], h, h);
  o[2] = mul_i<T, DIR>(o[2]);
  o[3] = rot<T, DIR>(o[3], -h, h);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    v[k] = add<T>(e[k], o[k]);
    v[k + 4] = sub<T>(e[k], o[k]);
  }
}

template <typename T, int DIR> __device__ __forceinline__ void dft16(cx<T>* v) {
  const T c1 = (T)0.92387953251128675613, s1 = (T)0.38268343236508977173;  // cos, sin (pi/8)
  const T h = (T)0.70710678118654752440;
  cx<T> e[8], o[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) { e[k] = v[2 * k]; o[k] = v[2 * k + 1]; }
  dft8<T, DIR>(e);
  dft8<T, DIR>(o);
  o[1] = rot<T, DIR>(o[1], c1, s1);
  o[2] = rot<T, DIR>(o[2], h, h);
  o[3] = rot<T, DIR>(o[3], s1, c1);
  o[4] = mul_i<T, DIR>(o[4]);
  o[5] = rot<T, DIR>(o[5], -s1, c1);
  o[6] = rot<T, DIR>(o[6], -h, h);
  o[7] = rot<T, DIR>(o[7], -c1, s1);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    v[k] = add<T>(e[k], o[k]);
    v[k + 8] = sub<T>(e[k], o[k]);
  }
}

// radix-2 split of a 32-point DFT into two 16-point DFTs; the odd half is rotated by W_32^k (k = 1..15),
// written with the cos/sin of k pi / 16 and the symmetries of the first octant.
template <typename T, int DIR> __device__ __forceinline__ void dft32(cx<T>* v) {
  const T c1 = (T)0.98078528040323044913, s1 = (T)0.19509032201612826785;  // pi/16
  const T c2 = (T)0.92387953251128675613, s2 = (T)0.38268343236508977173;  // pi/8
  const T c3 = (T)0.83146961230254523708, s3 = (T)0.55557023301960222474;  // 3 pi/16
  const T h = (T)0.70710678118654752440;                                    // pi/4
  cx<T> e[16], o[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) { e[k] = v[2 * k]; o[k] = v[2 * k + 1]; }
  dft16<T, DIR>(e);
  dft16<T, DIR>(o);
  // o[k] times W_32^k = e^{i DIR k pi / 16}: rot<T, DIR>(a, c, s) multiplies by c + i DIR s
  o[1] = rot<T, DIR>(o[1], c1, s1);
  o[2] = rot<T, DIR>(o[2], c2, s2);
  o[3] = rot<T, DIR>(o[3], c3, s3);
  o[4] = rot<T, DIR>(o[4], h, h);
  o[5] = rot<T, DIR>(o[5], s3, c3);
  o[6] = rot<T, DIR>(o[6], s2, c2);
  o[7] = rot<T, DIR>(o[7], s1, c1);
  o[8] = mul_i<T, DIR>(o[8]);
  o[9] = rot<T, DIR>(o[9], -s1, c1);
  o[10] = rot<T, DIR>(o[10], -s2, c2);
  o[11] = rot<T, DIR>(o[11], -s3, c3);
  o[12] = rot<T, DIR>(o[12], -h, h);
  o[13] = rot<T, DIR>(o[13], -c3, s3);
  o[14] = rot<T, DIR>(o[14], -c2, s2);
  o[15] = rot<T, DIR>(o[15], -c1, s1);
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    v[k] = add<T>(e[k], o[k]);
    v[k + 16] = sub<T>(e[k], o[k]);
  }
}

template <typename T, int DIR, int R> __device__ __forceinline__ void dftR(cx<T>* v) {
  if constexpr (R == 1) {
  } else if constexpr (R == 2) {
    dft2<T, DIR>(v[0], v[1]);
  } else if constexpr (R == 4) {
    dft4<T, DIR>(v);
  } else if constexpr (R == 8) {
    dft8<T, DIR>(v);
  } else if constexpr (R == 16) {
    dft16<T, DIR>(v);
  } else if constexpr (R == 32) {
    dft32<T, DIR>(v);
  } else {
    static_assert(R == 16, "unsupported radix");
  }
}

// ---------------------------------------------------------------- Stockham pencil
__host__ __device__ constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n / 2); }
__host__ __device__ constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }

template <int N, int E> struct StockPlan {
  static_assert((N & (N - 1)) == 0 && (E & (E - 1)) == 0, "powers of two");
  static constexpr int P = N / E;
  static constexpr int LE = ilog2c(E);
  static constexpr int LN = ilog2c(N);
  static constexpr int S = (LN + LE - 1) / LE;           // number of stages
  static constexpr int RLAST = N / ipow(E, S - 1);       // radix of the last stage
  static_assert(RLAST >= 2 && RLAST <= E, "bad factorisation");
};

// ---------------------------------------------------------------- exchange layouts
// Exchange buffers hold complex values (one 64-bit (FP32) or 128-bit (FP64) access per element) in two
// ping-pong buffers, so a stage reads one buffer and writes the other with one barrier per stage.
//
// RowLayout: one pencil per group of P consecutive threads, private buffer, element p at p + p/2^PADSH.
//   With PADSH = 3, stage-0 writes (stride E = 8 between threads), the span-8 writes of the middle stage
//   and unit-stride reads fall in distinct banks within each 128-byte access phase; PADSH = 4 saves space
//   at the cost of two-way conflicts on the middle-stage writes.
// ColLayout<TC, E>: TC adjacent pencils (thread = j * TC + c) interleaved as [p][c]; rows are permuted
//   within aligned groups of G = (128 B / element) / TC positions by g(p) = (p + p/E) mod G, so the G
//   positions touched by one access phase of a warp (stride 1 or stride E) land on distinct banks.
template <typename T, int N, bool ONE = false, int PADSH = 3> struct RowLayout {
  static constexpr bool SINGLE = ONE;                       // one buffer: a stage syncs between its reads and writes
  static constexpr bool VEC = false;                        // first-stage values stored one by one
  static constexpr int BUF = N + (N - 1) / (1 << PADSH) + 1;  // elements per buffer
  static constexpr int SIZE = ONE ? BUF : 2 * BUF;          // elements per pencil
  cx<T>* base;
  __device__ __forceinline__ cx<T>* buf(int which) const { return ONE ? base : base + which * BUF; }
  __device__ __forceinline__ int idx(int p) const { return p + (p >> PADSH); }
};

// RowLayoutV: one buffer per pencil with two pad elements after every 16, so the 16 consecutive outputs of a
//   thread's first radix-16 stage form 16-byte aligned pairs (one 128-bit store per two values); unit-stride reads
//   of 16 threads cover 128 contiguous bytes.  The pitch N + N/8 + 8 puts consecutive rows 64 bytes apart in the
//   128-byte bank cycle, so two rows of 8 threads each also read conflict-free.
template <typename T, int N> struct RowLayoutV {
  static constexpr bool SINGLE = true;
  static constexpr bool VEC = true;
  static constexpr int BUF = N + N / 8 + 8;
  static constexpr int SIZE = BUF;
  static_assert(N % 16 == 0 && (BUF * (int)sizeof(cx<T>)) % 16 == 0, "16-byte aligned rows");
  cx<T>* base;
  __device__ __forceinline__ cx<T>* buf(int) const { return base; }
  __device__ __forceinline__ int idx(int p) const { return p + 2 * (p >> 4); }
};

// ONE: a single buffer (a stage syncs between its reads and writes), for tiles whose two buffers would not
// leave room for a second CTA per SM.
template <typename T, int N, int TC, int E, bool ONE = false> struct ColLayout {
  static constexpr bool SINGLE = ONE;
  static constexpr bool VEC = false;
  static constexpr int PER_PHASE = 128 / (int)sizeof(cx<T>);
  static constexpr int G0 = PER_PHASE / TC;
  // (p + p/E) mod G permutes each aligned group of G positions only while G <= E (p/E is then constant in the
  // group); a larger G would make two rows collide.
  static constexpr int G1 = G0 < 1 ? 1 : G0;
  static constexpr int G = G1 > E ? E : G1;
  static constexpr int BUF = N * TC;
  static constexpr int SIZE = ONE ? BUF : 2 * BUF;  // elements for all TC pencils
  cx<T>* base;  // shared by the TC pencils of the CTA
  int c;
  __device__ __forceinline__ cx<T>* buf(int which) const { return ONE ? base : base + which * BUF; }
  __device__ __forceinline__ int idx(int p) const {
    if constexpr (G == 1) {
      return p * TC + c;
    } else {
      const int q = (p & ~(G - 1)) + ((p + p / E) & (G - 1));
      return q * TC + c;
    }
  }
};

struct SyncBlock { __device__ __forceinline__ void operator()() const { __syncthreads(); } };
struct SyncWarp { __device__ __forceinline__ void operator()() const { __syncwarp(); } };

// tw[k] = exp(-2 pi i k / N), k = 0..N-1 (FP64-generated, stored in T)
template <typename T, int DIR>
__device__ __forceinline__ cx<T> twiddle(const cx<T>* __restrict__ tw, int idx) {
  cx<T> w = __ldg(tw + idx);
  return DIR > 0 ? conjg<T>(w) : w;
}

// Stage s >= 1 of the Stockham recursion: reads buffer (s-1)&1, writes buffer s&1.
template <typename T, int N, int E, int DIR, int s, typename Lay, typename Sync>
__device__ __forceinline__ void stock_stage(cx<T> (&v)[E], int j, const Lay& L, const cx<T>* __restrict__ tw,
                                            Sync sync) {
  using PL = StockPlan<N, E>;
  constexpr int P = PL::P;
  constexpr int S = PL::S;
  constexpr int Ns = ipow(E, s);
  const cx<T>* rd = L.buf((s - 1) & 1);
  if constexpr (s < S - 1) {
    cx<T>* wr = L.buf(s & 1);
    const int jj = j;
    const int k = jj & (Ns - 1);
#pragma unroll
    for (int r = 0; r < E; ++r) v[r] = rd[L.idx(jj + r * P)];
    if constexpr (Lay::SINGLE) sync();
    constexpr int stride = N / (Ns * E);
#pragma unroll
    for (int r = 1; r < E; ++r) v[r] = mul<T>(v[r], twiddle<T, DIR>(tw, r * k * stride));
    dftR<T, DIR, E>(v);
    const int base = (jj / Ns) * Ns * E + k;
#pragma unroll
    for (int r = 0; r < E; ++r) wr[L.idx(base + r * Ns)] = v[r];
    sync();
    stock_stage<T, N, E, DIR, s + 1, Lay, Sync>(v, j, L, tw, sync);
  } else {
    constexpr int R = PL::RLAST;
    constexpr int NB = E / R;
#pragma unroll
    for (int t = 0; t < NB; ++t) {
      const int jj = j + t * P;
      const int k = jj & (Ns - 1);
      cx<T> a[R];
#pragma unroll
      for (int r = 0; r < R; ++r) a[r] = rd[L.idx(jj + r * (N / R))];
      constexpr int stride = N / (Ns * R);
#pragma unroll
      for (int r = 1; r < R; ++r) a[r] = mul<T>(a[r], twiddle<T, DIR>(tw, r * k * stride));
      dftR<T, DIR, R>(a);
#pragma unroll
      for (int r = 0; r < R; ++r) v[t + r * NB] = a[r];
    }
  }
}

// Full pencil transform (see the file header for the data convention).  Every thread of the
// synchronisation group must call it (no divergent early exit).  With TRAIL, a final barrier lets
// the caller reuse the exchange buffers at once.
template <typename T, int N, int E, int DIR, typename Lay, typename Sync, bool TRAIL = true>
__device__ __forceinline__ void fft_pencil(cx<T> (&v)[E], int j, const Lay& L, const cx<T>* __restrict__ tw,
                                           Sync sync) {
  using PL = StockPlan<N, E>;
  if constexpr (PL::S == 1) {
    dftR<T, DIR, E>(v);
  } else {
    cx<T>* wr = L.buf(0);
    dftR<T, DIR, E>(v);
    const int base = j * E;  // Ns = 1
    if constexpr (Lay::VEC) {  // 16-byte pairs (RowLayoutV, FP32)
      static_assert(E % 2 == 0 && sizeof(cx<T>) == 8, "pairs of FP32 complex values");
#pragma unroll
      for (int m = 0; m < E / 2; ++m)
        *reinterpret_cast<float4*>(wr + L.idx(base + 2 * m)) =
            make_float4(v[2 * m].x, v[2 * m].y, v[2 * m + 1].x, v[2 * m + 1].y);
    } else {
#pragma unroll
      for (int r = 0; r < E; ++r) wr[L.idx(base + r)] = v[r];
    }
    sync();
    stock_stage<T, N, E, DIR, 1, Lay, Sync>(v, j, L, tw, sync);
    if constexpr (TRAIL) sync();
  }
}

}  // namespace sigw
