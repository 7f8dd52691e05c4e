// Register-resident small DFTs and the two-pass line-FFT decomposition used by every
// transform kernel of libshearlet. Internal header.
//
// A length-L line is split as L = A * B (powers of two, 384 = 24 * 16 or 192 = 16 * 12).
// With
// n = a + A b and
// k = kb + B ka,
//   X[kb + B ka] = sum_a W_A^{a ka} * ( W_L^{a kb} * sum_b x[a + A b] W_B^{b kb} ).
// Pass 1 gives each thread the B samples x[a + A b] of one (line, a): a DFT of length
// B in registers, then the twiddle W_L^{a kb}. One exchange through shared memory
// regroups the values by kb. Pass 2 gives each thread the A values of one (line, kb):
// a DFT of length A in registers yields the outputs kb + B ka in natural order.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <utility>

namespace sl {
namespace dev {

// ------------------------------------------------------------------ complex ops ---

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * w for DIR < 0 (forward, w = e^{-i t}) and a * conj(w) for DIR > 0 (inverse).
template <int DIR>
__device__ __forceinline__ float2 ctw(float2 a, float2 w) {
  if constexpr (DIR < 0) return cmul(a, w);
  else return make_float2(a.x * w.x + a.y * w.y, a.y * w.x - a.x * w.y);
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }

// ------------------------------------------------------- compile-time twiddles ---

constexpr double kPiD = 3.14159265358979323846264338327950288;

// Taylor series, |x| <= pi: the truncation error of 20 terms is below 1e-25.
constexpr double cx_sin(double x) {
  double t = x, s = x;
  for (int n = 1; n < 20; ++n) { t *= -x * x / ((2.0 * n) * (2.0 * n + 1.0)); s += t; }
  return s;
}
constexpr double cx_cos(double x) {
  double t = 1.0, s = 1.0;
  for (int n = 1; n < 20; ++n) { t *= -x * x / ((2.0 * n - 1.0) * (2.0 * n)); s += t; }
  return s;
}

// W_N^K = exp(-2 pi i K / N) for 0 <= K < 3N/4 (angle in (-3pi/2, 0]; the series
// error there is still below 1e-21).
template <int N, int K>
struct Tw {
  static constexpr float re = (float)cx_cos(-2.0 * kPiD * K / N);
  static constexpr float im = (float)cx_sin(-2.0 * kPiD * K / N);
};

// ------------------------------------------------------------ register DFTs ---
// In place, natural order in and out. DIR = -1: forward (e^{-i}), +1: inverse
// (unnormalised). Decimation in time (radix 4 where N is a multiple of 4 and at
// least 16, else radix 3 or 2), fully unrolled at compile time.

template <int N, int DIR>
struct Dft;

template <int N, int DIR, int K>
__device__ __forceinline__ void dft_bfly(float2 (&x)[N], const float2 (&e)[N / 2],
                                         const float2 (&o)[N / 2]) {
  float2 t;
  if constexpr (K == 0) {
    t = o[0];
  } else if constexpr (4 * K == N) {  // W = -i (forward) or +i (inverse)
    if constexpr (DIR < 0) t = make_float2(o[K].y, -o[K].x);
    else t = make_float2(-o[K].y, o[K].x);
  } else {
    constexpr float wr = Tw<N, K>::re;
    constexpr float wi = DIR < 0 ? Tw<N, K>::im : -Tw<N, K>::im;
    t = make_float2(o[K].x * wr - o[K].y * wi, o[K].x * wi + o[K].y * wr);
  }
  x[K] = cadd(e[K], t);
  x[K + N / 2] = csub(e[K], t);
}

template <int N, int DIR, int... K>
__device__ __forceinline__ void dft_combine(float2 (&x)[N], const float2 (&e)[N / 2],
                                            const float2 (&o)[N / 2],
                                            std::integer_sequence<int, K...>) {
  (dft_bfly<N, DIR, K>(x, e, o), ...);
}

// Radix-3 decimation in time for N divisible by 3:
//   X[k + r N/3] = E0[k] + w^r W^k E1[k] + w^{2r} W^{2k} E2[k],  w = W_3, W = W_N,
// with E_m the length-N/3 DFT of x[3n + m].
template <int N, int DIR, int K>
__device__ __forceinline__ void dft3_bfly(float2 (&x)[N], const float2 (&e0)[N / 3],
                                          const float2 (&e1)[N / 3], const float2 (&e2)[N / 3]) {
  constexpr int M = N / 3;
  float2 t1 = e1[K], t2 = e2[K];
  if constexpr (K != 0) {
    constexpr float c1 = Tw<N, K>::re, s1 = DIR < 0 ? Tw<N, K>::im : -Tw<N, K>::im;
    constexpr float c2 = Tw<N, 2 * K>::re, s2 = DIR < 0 ? Tw<N, 2 * K>::im : -Tw<N, 2 * K>::im;
    t1 = make_float2(t1.x * c1 - t1.y * s1, t1.x * s1 + t1.y * c1);
    t2 = make_float2(t2.x * c2 - t2.y * s2, t2.x * s2 + t2.y * c2);
  }
  // w = cos(2pi/3) -+ i sin(2pi/3): t1 w + t2 w^2 and t1 w^2 + t2 w
  constexpr float h = 0.8660254037844386f;  // sin(2 pi / 3)
  const float2 sum = cadd(t1, t2), dif = csub(t1, t2);
  const float2 base = make_float2(e0[K].x - 0.5f * sum.x, e0[K].y - 0.5f * sum.y);
  // -i h dif for the forward direction (+i h dif for the inverse)
  const float2 rot = DIR < 0 ? make_float2(h * dif.y, -h * dif.x) : make_float2(-h * dif.y, h * dif.x);
  x[K] = cadd(e0[K], sum);
  x[K + M] = cadd(base, rot);
  x[K + 2 * M] = csub(base, rot);
}

template <int N, int DIR, int... K>
__device__ __forceinline__ void dft3_combine(float2 (&x)[N], const float2 (&e0)[N / 3],
                                             const float2 (&e1)[N / 3], const float2 (&e2)[N / 3],
                                             std::integer_sequence<int, K...>) {
  (dft3_bfly<N, DIR, K>(x, e0, e1, e2), ...);
}

// Radix-4 decimation in time for N divisible by 4 (N >= 16): with E_r the length-N/4
// DFT of x[4n + r] and t_r = W_N^{r k} E_r[k],
//   X[k] = (t0 + t2) + (t1 + t3),            X[k + N/2]  = (t0 + t2) - (t1 + t3),
//   X[k + N/4] = (t0 - t2) + w (t1 - t3),    X[k + 3N/4] = (t0 - t2) - w (t1 - t3),
// w = W_4 = -i (forward) or +i (inverse): three twiddle products per four outputs
// instead of the four of two radix-2 levels.
template <int N, int DIR, int K, int R>
__device__ __forceinline__ float2 tw_r4(float2 v) {
  constexpr int m = R * K;  // exponent of W_N, 0 <= m < 3N/4
  if constexpr (m == 0) {
    return v;
  } else if constexpr (4 * m == N) {  // W = -i (forward) or +i (inverse)
    if constexpr (DIR < 0) return make_float2(v.y, -v.x);
    else return make_float2(-v.y, v.x);
  } else if constexpr (2 * m == N) {  // W = -1
    return make_float2(-v.x, -v.y);
  } else {
    constexpr float wr = Tw<N, m>::re;
    constexpr float wi = DIR < 0 ? Tw<N, m>::im : -Tw<N, m>::im;
    return make_float2(v.x * wr - v.y * wi, v.x * wi + v.y * wr);
  }
}

template <int N, int DIR, int K>
__device__ __forceinline__ void dft4_bfly(float2 (&x)[N], const float2 (&e0)[N / 4],
                                          const float2 (&e1)[N / 4], const float2 (&e2)[N / 4],
                                          const float2 (&e3)[N / 4]) {
  constexpr int M = N / 4;
  const float2 t0 = e0[K];
  const float2 t1 = tw_r4<N, DIR, K, 1>(e1[K]);
  const float2 t2 = tw_r4<N, DIR, K, 2>(e2[K]);
  const float2 t3 = tw_r4<N, DIR, K, 3>(e3[K]);
  const float2 a = cadd(t0, t2), b = csub(t0, t2), c = cadd(t1, t3), d = csub(t1, t3);
  // w d with w = -i (forward) or +i (inverse)
  const float2 wd = DIR < 0 ? make_float2(d.y, -d.x) : make_float2(-d.y, d.x);
  x[K] = cadd(a, c);
  x[K + 2 * M] = csub(a, c);
  x[K + M] = cadd(b, wd);
  x[K + 3 * M] = csub(b, wd);
}

template <int N, int DIR, int... K>
__device__ __forceinline__ void dft4_combine(float2 (&x)[N], const float2 (&e0)[N / 4],
                                             const float2 (&e1)[N / 4], const float2 (&e2)[N / 4],
                                             const float2 (&e3)[N / 4],
                                             std::integer_sequence<int, K...>) {
  (dft4_bfly<N, DIR, K>(x, e0, e1, e2, e3), ...);
}

template <int N, int DIR>
struct Dft {
  static __device__ __forceinline__ void run(float2 (&x)[N]) {
    if constexpr (N % 4 == 0 && N >= 16) {
      constexpr int M = N / 4;
      float2 e0[M], e1[M], e2[M], e3[M];
#pragma unroll
      for (int i = 0; i < M; ++i) {
        e0[i] = x[4 * i];
        e1[i] = x[4 * i + 1];
        e2[i] = x[4 * i + 2];
        e3[i] = x[4 * i + 3];
      }
      Dft<M, DIR>::run(e0);
      Dft<M, DIR>::run(e1);
      Dft<M, DIR>::run(e2);
      Dft<M, DIR>::run(e3);
      dft4_combine<N, DIR>(x, e0, e1, e2, e3, std::make_integer_sequence<int, M>{});
    } else if constexpr (N % 3 == 0) {
      constexpr int M = N / 3;
      float2 e0[M], e1[M], e2[M];
#pragma unroll
      for (int i = 0; i < M; ++i) {
        e0[i] = x[3 * i];
        e1[i] = x[3 * i + 1];
        e2[i] = x[3 * i + 2];
      }
      Dft<M, DIR>::run(e0);
      Dft<M, DIR>::run(e1);
      Dft<M, DIR>::run(e2);
      dft3_combine<N, DIR>(x, e0, e1, e2, std::make_integer_sequence<int, M>{});
    } else {
      float2 e[N / 2], o[N / 2];
#pragma unroll
      for (int i = 0; i < N / 2; ++i) {
        e[i] = x[2 * i];
        o[i] = x[2 * i + 1];
      }
      Dft<N / 2, DIR>::run(e);
      Dft<N / 2, DIR>::run(o);
      dft_combine<N, DIR>(x, e, o, std::make_integer_sequence<int, N / 2>{});
    }
  }
};

template <int DIR>
struct Dft<1, DIR> {
  static __device__ __forceinline__ void run(float2 (&)[1]) {}
};

// ------------------------------------------------------------- line split ---

template <int L>
struct Split;
template <> struct Split<8> { static constexpr int A = 4, B = 2; };
template <> struct Split<16> { static constexpr int A = 4, B = 4; };
template <> struct Split<32> { static constexpr int A = 8, B = 4; };
template <> struct Split<64> { static constexpr int A = 8, B = 8; };
template <> struct Split<128> { static constexpr int A = 16, B = 8; };
template <> struct Split<256> { static constexpr int A = 16, B = 16; };
template <> struct Split<512> { static constexpr int A = 32, B = 16; };
template <> struct Split<1024> { static constexpr int A = 32, B = 32; };
template <> struct Split<384> { static constexpr int A = 24, B = 16; };  // 3 * 2^7
template <> struct Split<192> { static constexpr int A = 16, B = 12; };  // 3 * 2^6 (3D)

// Offset of the twiddle table of length L inside the concatenated table: lengths
// 8, 16, ..., 1024 back to back (8 + 16 + ... + L/2 = L - 8), then 384, then 192.
__host__ __device__ constexpr int twiddle_offset(int L) {
  return L == 384 ? 2040 : L == 192 ? 2040 + 384 : L - 8;
}
constexpr int kTwiddleTotal = 2040 + 384 + 192;

}  // namespace dev
}  // namespace sl
