// 3D plane passes: transforms along axes 1 and 2 of one n1 x n2 plane held entirely in
// shared memory (half spectrum along axis 2). Internal header.
#pragma once

#include "kernels2d.cuh"

namespace sl {
namespace dev {

// 17 warps: the plane phases have 1040, 520, 1024, 512 and 4160 work items at 128 x 128,
// so 544 threads take the column FFT in two rounds and its second pass in one.
constexpr int kPlaneThreads = 544;

template <int L1, int L2>
struct PlaneGeom {
  static constexpr int NH = L2 / 2 + 1;
  static constexpr int HALF = L1 * NH;                                    // half plane
  static constexpr int XROW = (L1 / 2) * Split<L2>::B * (Split<L2>::A + 1);  // row exchange
  static constexpr int FULL = (L1 / 2) * L2;                               // row pairs, natural
  static constexpr int S0 = HALF > XROW ? HALF : XROW;
  static constexpr int S = S0 > FULL ? S0 : FULL;                         // one buffer
  static constexpr int bytes = 2 * S * (int)sizeof(float2);
};

// FFT along axis 1 of a half plane [L1][NH] (columns), src -> wk (exchange) -> dst
// (natural). src may equal dst. Ends with a __syncthreads().
template <int L1, int NH, int DIR>
__device__ __forceinline__ void plane_col_fft(const float2* src, float2* wk, float2* dst) {
  constexpr int A = Split<L1>::A, B = Split<L1>::B;
  const float2* tw = g_twiddle + twiddle_offset(L1);
  for (int it = threadIdx.x; it < NH * A; it += kPlaneThreads) {
    const int col = it % NH, a = it / NH;
    float2 v[B];
#pragma unroll
    for (int b = 0; b < B; ++b) v[b] = src[(a + A * b) * NH + col];
    Dft<B, DIR>::run(v);
#pragma unroll
    for (int kb = 1; kb < B; ++kb) v[kb] = ctw<DIR>(v[kb], tw[kb * A + a]);
#pragma unroll
    for (int kb = 0; kb < B; ++kb) wk[(kb * A + a) * NH + col] = v[kb];
  }
  __syncthreads();
  for (int it = threadIdx.x; it < NH * B; it += kPlaneThreads) {
    const int col = it % NH, kb = it / NH;
    float2 w[A];
#pragma unroll
    for (int a = 0; a < A; ++a) w[a] = wk[(kb * A + a) * NH + col];
    Dft<A, DIR>::run(w);
#pragma unroll
    for (int ka = 0; ka < A; ++ka) dst[(kb + B * ka) * NH + col] = w[ka];
  }
  __syncthreads();
}

// Plane pass, persistent: work item i = (slot i / L0, plane i0 = i % L0); CTA c takes
// items c, c + gridDim.x, ... (one plane in shared memory at a time).
//   ROW_C2R  half-spectrum plane -> real plane * scale (optional threshold)
//   ROW_R2C  real plane -> half-spectrum plane
//   ROW_RT   half -> real * scale -> threshold -> half
// The next item's input is loaded into registers while the current plane is
// transformed (C2R: during the axis-1 FFT and the first row pass, then parked in the
// plane buffer once that is free; R2C: during everything after the first row pass).
// in/out slot strides are in elements of their own type. Spectra are tile-major
// (p.tm): point p = k1 * NH + k2 of plane i0 lives at p.tm.at(i0, p); real planes are
// row-major and plane i0 starts at i0 * (L1 * L2).
template <int L1, int L2, int MODE>
__global__ void __launch_bounds__(kPlaneThreads) k_plane(RowArgs p, int nslots) {
  using G = PlaneGeom<L1, L2>;
  constexpr int NH = G::NH;
  constexpr int A = Split<L2>::A, B = Split<L2>::B;
  constexpr int LS = B * (A + 1);
  constexpr int PAIRS = L1 / 2;
  constexpr int H = L2 / 2;
  constexpr int NIT = (G::HALF + kPlaneThreads - 1) / kPlaneThreads;  // gather loads
  constexpr int NI = (PAIRS * A + kPlaneThreads - 1) / kPlaneThreads;  // row items
  extern __shared__ float2 sm[];
  float2* P = sm;
  float2* W = sm + G::S;
  const int tid = threadIdx.x;
  const int L0 = p.n_rows;
  const int nitems = nslots * L0;
  const float2* tw = g_twiddle + twiddle_offset(L2);

  // half-spectrum plane gather (C2R, RT) into registers
  auto gather = [&](int item, float2 (&ld)[NIT]) {
    const int slot = item / L0, i0 = item % L0;
    const float2* in = p.in_half + (int64_t)slot * p.in_stride;
#pragma unroll
    for (int r = 0; r < NIT; ++r) {
      const int i = tid + r * kPlaneThreads;
      ld[r] = i < G::HALF ? in[p.tm.at(i0, i)] : make_float2(0.f, 0.f);
    }
  };
  auto park = [&](const float2 (&ld)[NIT]) {
#pragma unroll
    for (int r = 0; r < NIT; ++r) {
      const int i = tid + r * kPlaneThreads;
      if (i < G::HALF) P[i] = ld[r];
    }
  };
  // this thread's real row items (a, q) of a plane (R2C)
  auto load_rows = [&](int item, float2 (&v)[NI][B]) {
    const int slot = item / L0, i0 = item % L0;
    const float* inr = p.in_real + (int64_t)slot * p.in_stride + (int64_t)i0 * (L1 * L2);
#pragma unroll
    for (int r = 0; r < NI; ++r) {
      const int it = tid + r * kPlaneThreads;
      const int a = it % A, q = it / A;
#pragma unroll
      for (int b = 0; b < B; ++b) {
        const int n = a + A * b;
        v[r][b] = it < PAIRS * A ? make_float2(inr[(2 * q) * L2 + n], inr[(2 * q + 1) * L2 + n])
                                 : make_float2(0.f, 0.f);
      }
    }
  };

  int item = blockIdx.x;
  float2 ld[MODE == ROW_R2C ? 1 : NIT];
  float2 v[NI][B];
  if (item < nitems) {
    if constexpr (MODE == ROW_R2C) {
      load_rows(item, v);
    } else {
      gather(item, ld);
      park(ld);
    }
  }
  for (; item < nitems; item += gridDim.x) {
    const int slot = item / L0, i0 = item % L0;
    const int next = item + gridDim.x;
    if constexpr (MODE == ROW_C2R || MODE == ROW_RT) {
      __syncthreads();  // the parked plane is in P
      if constexpr (MODE == ROW_C2R) {
        if (next < nitems) gather(next, ld);
      }
      plane_col_fft<L1, NH, 1>(P, W, P);
      // rows (2q, 2q+1): complex inverse DFT of the Hermitian-extended pair
      for (int it = tid; it < PAIRS * A; it += kPlaneThreads) {
        const int a = it % A, q = it / A;
        const float2* r0 = P + (2 * q) * NH;
        const float2* r1 = r0 + NH;
        float2 u[B];
#pragma unroll
        for (int b = 0; b < B; ++b) {
          const int n = a + A * b;
          float2 ya, yb;
          if (n <= H) {
            ya = r0[n];
            yb = r1[n];
          } else {
            ya = cconj(r0[L2 - n]);
            yb = cconj(r1[L2 - n]);
          }
          u[b] = make_float2(ya.x - yb.y, ya.y + yb.x);
        }
        Dft<B, 1>::run(u);
#pragma unroll
        for (int kb = 1; kb < B; ++kb) u[kb] = ctw<1>(u[kb], tw[kb * A + a]);
#pragma unroll
        for (int kb = 0; kb < B; ++kb) W[q * LS + kb * (A + 1) + a] = u[kb];
      }
      __syncthreads();
      if constexpr (MODE == ROW_C2R) {
        if (next < nitems) park(ld);  // P is free: the rows are in W
      }
      const float thr = p.use_thr ? p.thr.v[slot] : 0.f;
      float* outr = nullptr;
      if constexpr (MODE == ROW_C2R)
        outr = p.out_real + (int64_t)slot * p.out_stride + (int64_t)i0 * (L1 * L2);
      for (int it = tid; it < PAIRS * B; it += kPlaneThreads) {
        const int kb = it % B, q = it / B;
        float2 w[A];
#pragma unroll
        for (int a = 0; a < A; ++a) w[a] = W[q * LS + kb * (A + 1) + a];
        Dft<A, 1>::run(w);
#pragma unroll
        for (int ka = 0; ka < A; ++ka) {
          const int k = kb + B * ka;
          float c0 = w[ka].x * p.scale, c1 = w[ka].y * p.scale;
          if (p.use_thr) {
            if (fabsf(c0) < thr) c0 = 0.f;
            if (fabsf(c1) < thr) c1 = 0.f;
          }
          if constexpr (MODE == ROW_C2R) {
            outr[(2 * q) * L2 + k] = c0;
            outr[(2 * q + 1) * L2 + k] = c1;
          } else {
            P[q * L2 + k] = make_float2(c0, c1);  // natural pairs for the forward pass
          }
        }
      }
      if constexpr (MODE == ROW_C2R) continue;
      __syncthreads();
      // RT: this plane's rows, from P
#pragma unroll
      for (int r = 0; r < NI; ++r) {
        const int it = tid + r * kPlaneThreads;
        const int a = it % A, q = it / A;
#pragma unroll
        for (int b = 0; b < B; ++b)
          v[r][b] = it < PAIRS * A ? P[q * L2 + a + A * b] : make_float2(0.f, 0.f);
      }
      if (next < nitems) gather(next, ld);  // in flight during the forward half
    } else {
      __syncthreads();  // the previous item is done with the shared buffers
    }

    // real rows (pairs) in v -> half rows in W -> FFT along axis 1 -> out
#pragma unroll
    for (int r = 0; r < NI; ++r) {
      const int it = tid + r * kPlaneThreads;
      if (it >= PAIRS * A) continue;
      const int a = it % A, q = it / A;
      Dft<B, -1>::run(v[r]);
#pragma unroll
      for (int kb = 1; kb < B; ++kb) v[r][kb] = ctw<-1>(v[r][kb], tw[kb * A + a]);
#pragma unroll
      for (int kb = 0; kb < B; ++kb) W[q * LS + kb * (A + 1) + a] = v[r][kb];
    }
    if constexpr (MODE == ROW_R2C) {
      if (next < nitems) load_rows(next, v);  // v is free: in flight during the rest
    }
    __syncthreads();
    // Pass 2, and the split of each row pair's spectrum Z = FFT(x0 + i x1) into the two
    // half rows in registers: the thread of (q, kb) holds Z[kb + B ka], and Z[L2 - k]
    // sits in the thread of (q, (B - kb) mod B) at index A - 1 - ka (in this thread at
    // (A - ka) mod A when kb = 0). Whole warps iterate (the B-thread groups never
    // straddle a warp: B divides 32), so the shuffles see every lane. The half rows go
    // to P (free: its natural pairs, in RT mode, were read before pass 1).
    static_assert(32 % B == 0 && (A & (A - 1)) == 0, "partner lanes within a warp");
    {
      const int lane = tid & 31;
      for (int it0 = tid & ~31; it0 < PAIRS * B; it0 += kPlaneThreads) {
        const int it = it0 + lane;
        const bool valid = it < PAIRS * B;
        const int kb = it % B, q = it / B;
        float2 w[A];
#pragma unroll
        for (int a = 0; a < A; ++a)
          w[a] = valid ? W[q * LS + kb * (A + 1) + a] : make_float2(0.f, 0.f);
        Dft<A, -1>::run(w);
        const int partner = (lane & ~(B - 1)) | ((B - kb) & (B - 1));
#pragma unroll
        for (int ka = 0; ka <= A / 2; ++ka) {
          const float2 far = w[A - 1 - ka];
          const float2 oth = make_float2(__shfl_sync(0xffffffffu, far.x, partner),
                                         __shfl_sync(0xffffffffu, far.y, partner));
          const float2 wz = kb == 0 ? w[(A - ka) & (A - 1)] : oth;
          const float2 z = w[ka];
          if (valid && (ka < A / 2 || kb == 0)) {  // k <= L2 / 2
            const int k = kb + B * ka;
            P[(2 * q) * NH + k] = make_float2(0.5f * (z.x + wz.x), 0.5f * (z.y - wz.y));
            P[(2 * q + 1) * NH + k] = make_float2(0.5f * (z.y + wz.y), 0.5f * (wz.x - z.x));
          }
        }
      }
    }
    __syncthreads();
    plane_col_fft<L1, NH, -1>(P, W, P);
    float2* out = p.out_half + (int64_t)slot * p.out_stride;
    for (int i = tid; i < G::HALF; i += kPlaneThreads) out[p.tm.at(i0, i)] = P[i];
    if constexpr (MODE == ROW_RT) {
      __syncthreads();  // P is free once the last axis-1 pass has read it
      if (next < nitems) park(ld);
    }
  }
}

// ------------------------------------------------ planes too large to double-buffer ---
// Plane pass for L x L planes whose half spectrum [L][L/2 + 1] leaves room for only one
// plane buffer and a partial exchange in one CTA's shared memory (L = 192: 149 KB plane,
// 78 KB exchange, 227 KB in total). Persistent, one plane at a time, no prefetch:
//   * the axis-1 (column) FFT runs on the plane in place, half of the columns at a time
//     through the exchange;
//   * the axis-2 row FFTs run on QC row pairs at a time: real rows are read from (R2C)
//     or written to (C2R) global memory directly, so the plane buffer only ever holds
//     half spectra (RT keeps each chunk's thresholded rows in the chunk's own part of the
//     plane buffer until their forward row FFT).
// Modes as k_plane (ROW_C2R, ROW_R2C, ROW_RT); spectra tile-major (p.tm), real planes
// row-major. Input half planes arrive by 16-byte cp.async copies (pairs of elements
// never straddle a tile run: TC is even); in ROW_C2R mode the next plane's copies are
// issued into each half of the plane buffer as soon as that half has been consumed, so
// they overlap the rest of the current plane.
constexpr int kBigThreads = 768;

template <int L>
struct BigPlane {
  static constexpr int A = Split<L>::A, B = Split<L>::B;
  static constexpr int NH = L / 2 + 1, H = L / 2;
  static constexpr int HALF = L * NH;            // plane buffer (half spectrum)
  static constexpr int LS = B * (A + 1);         // padded row exchange per pair
  static constexpr int QC = L / 4;               // row pairs per chunk (two chunks)
  static constexpr int CW = (NH + 1) / 2;        // columns per chunk (two chunks)
  static constexpr int WROW = QC * LS, WCOL = L * CW;
  static constexpr int WSZ = WROW > WCOL ? WROW : WCOL;
  static constexpr int bytes = (HALF + WSZ) * (int)sizeof(float2);
  static_assert(QC * L <= (L / 2) * NH, "a chunk's natural pairs fit its part of the plane");
  static_assert(QC * 2 * NH <= WSZ, "a chunk's half rows fit the exchange");
};

// FFT along axis 1 of columns [c0, c0 + cw) of the half plane P (in place through W).
// If out is not null the transformed columns go to the tile-major spectrum out (plane
// i0) instead of back into P; then `consumed` runs once the chunk's columns of P have
// been read (after the barrier between the two passes). Ends with a CTA barrier.
struct NoHook {
  __device__ void operator()() const {}
};
template <int L, int DIR, typename Hook = NoHook>
__device__ __forceinline__ void big_col_chunk(float2* P, float2* W, int c0, int cw,
                                              float2* out, const TileMap& tm, int i0,
                                              Hook consumed = Hook()) {
  using G = BigPlane<L>;
  constexpr int A = G::A, B = G::B, NH = G::NH;
  const float2* tw = g_twiddle + twiddle_offset(L);
  for (int it = threadIdx.x; it < cw * A; it += kBigThreads) {
    const int c = it % cw, a = it / cw;
    float2 v[B];
#pragma unroll
    for (int b = 0; b < B; ++b) v[b] = P[(a + A * b) * NH + c0 + c];
    Dft<B, DIR>::run(v);
#pragma unroll
    for (int kb = 1; kb < B; ++kb) v[kb] = ctw<DIR>(v[kb], tw[kb * A + a]);
#pragma unroll
    for (int kb = 0; kb < B; ++kb) W[(kb * A + a) * cw + c] = v[kb];
  }
  __syncthreads();
  if (out) consumed();
  for (int it = threadIdx.x; it < cw * B; it += kBigThreads) {
    const int c = it % cw, kb = it / cw;
    float2 w[A];
#pragma unroll
    for (int a = 0; a < A; ++a) w[a] = W[(kb * A + a) * cw + c];
    Dft<A, DIR>::run(w);
#pragma unroll
    for (int ka = 0; ka < A; ++ka) {
      const int k = kb + B * ka;
      if (out) out[tm.at(i0, k * NH + c0 + c)] = w[ka];
      else P[k * NH + c0 + c] = w[ka];
    }
  }
  __syncthreads();
}

// cp.async copies of elements [e0, e1) (even bounds) of plane i0 of the tile-major half
// spectrum `in` into P, one 16-byte pair per copy; committed as one group.
template <int L>
__device__ __forceinline__ void big_load(float2* P, const float2* in, const TileMap& tm, int i0,
                                         int e0, int e1) {
  for (int e = e0 + 2 * (int)threadIdx.x; e < e1; e += 2 * kBigThreads)
    cp_async16(P + e, in + tm.at(i0, e));
  cp_async_commit();
}

template <int L, int MODE>
__global__ void __launch_bounds__(kBigThreads, 1) k_plane_big(RowArgs p, int nslots) {
  using G = BigPlane<L>;
  constexpr int A = G::A, B = G::B, NH = G::NH, H = G::H, LS = G::LS, QC = G::QC, CW = G::CW;
  extern __shared__ float2 sm[];
  float2* P = sm;             // [L][NH] half spectrum of the plane
  float2* W = sm + G::HALF;   // exchange
  const int tid = threadIdx.x;
  const int L0 = p.n_rows;
  const int nitems = nslots * L0;
  const float2* tw = g_twiddle + twiddle_offset(L);

  static_assert(G::HALF % 2 == 0 && (2 * QC * NH) % 2 == 0, "copies move element pairs");
  bool prefetched = false;  // this item's plane was copied during the previous one
  for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
    const int slot = item / L0, i0 = item % L0;
    __syncthreads();  // the previous plane is done with P and W
    if constexpr (MODE == ROW_C2R || MODE == ROW_RT) {
      if (!prefetched)
        big_load<L>(P, p.in_half + (int64_t)slot * p.in_stride, p.tm, i0, 0, G::HALF);
      cp_async_wait<0>();
      __syncthreads();
      const int next = item + gridDim.x;  // C2R: its plane is copied half by half below
      const bool pre = MODE == ROW_C2R && next < nitems;
      const float2* in_next = p.in_half + (int64_t)(next / L0) * p.in_stride;
      for (int c0 = 0; c0 < NH; c0 += CW) big_col_chunk<L, 1>(P, W, c0, min(CW, NH - c0), nullptr, p.tm, i0);
      const float thr = p.use_thr ? p.thr.v[slot] : 0.f;
      float* outr = nullptr;
      if constexpr (MODE == ROW_C2R)
        outr = p.out_real + (int64_t)slot * p.out_stride + (int64_t)i0 * (L * L);
      for (int q0 = 0; q0 < L / 2; q0 += QC) {
        // rows (2q, 2q+1), q in [q0, q0 + QC): inverse DFT of the Hermitian-extended pair
        for (int it = tid; it < QC * A; it += kBigThreads) {
          const int a = it % A, qq = it / A, q = q0 + qq;
          const float2* r0 = P + (2 * q) * NH;
          const float2* r1 = r0 + NH;
          float2 u[B];
#pragma unroll
          for (int b = 0; b < B; ++b) {
            const int n = a + A * b;
            float2 ya, yb;
            if (n <= H) {
              ya = r0[n];
              yb = r1[n];
            } else {
              ya = cconj(r0[L - n]);
              yb = cconj(r1[L - n]);
            }
            u[b] = make_float2(ya.x - yb.y, ya.y + yb.x);
          }
          Dft<B, 1>::run(u);
#pragma unroll
          for (int kb = 1; kb < B; ++kb) u[kb] = ctw<1>(u[kb], tw[kb * A + a]);
#pragma unroll
          for (int kb = 0; kb < B; ++kb) W[qq * LS + kb * (A + 1) + a] = u[kb];
        }
        __syncthreads();  // the chunk's half rows are consumed: its part of P is free
        if (pre) big_load<L>(P, in_next, p.tm, next % L0, (2 * q0) * NH, (2 * q0 + 2 * QC) * NH);
        float2* nat = P + (2 * q0) * NH;  // RT: the chunk's natural pairs [QC][L]
        for (int it = tid; it < QC * B; it += kBigThreads) {
          const int kb = it % B, qq = it / B, q = q0 + qq;
          float2 w[A];
#pragma unroll
          for (int a = 0; a < A; ++a) w[a] = W[qq * LS + kb * (A + 1) + a];
          Dft<A, 1>::run(w);
#pragma unroll
          for (int ka = 0; ka < A; ++ka) {
            const int k = kb + B * ka;
            float c0 = w[ka].x * p.scale, c1 = w[ka].y * p.scale;
            if (p.use_thr) {
              if (fabsf(c0) < thr) c0 = 0.f;
              if (fabsf(c1) < thr) c1 = 0.f;
            }
            if constexpr (MODE == ROW_C2R) {
              outr[(2 * q) * L + k] = c0;
              outr[(2 * q + 1) * L + k] = c1;
            } else {
              nat[qq * L + k] = make_float2(c0, c1);
            }
          }
        }
        __syncthreads();  // W free for the next chunk
      }
      prefetched = pre;
      if constexpr (MODE == ROW_C2R) continue;
    }

    // real row pairs (R2C: staged from global into each chunk's own part of P, both
    // chunks' copies issued at once so the second's overlap the first chunk; RT: each
    // chunk's natural pairs in P) -> half rows in P -> FFT along axis 1 -> out
    // copies of plane (sl, pl)'s real rows into the chunks' parts of P, one group per chunk
    auto stage_rows = [&](int sl, int pl) {
      const float* inr = p.in_real + (int64_t)sl * p.in_stride + (int64_t)pl * (L * L);
      for (int q0 = 0; q0 < L / 2; q0 += QC) {
        float* dst = reinterpret_cast<float*>(P + (2 * q0) * NH);
        const float* src = inr + (2 * q0) * L;
        for (int o = 4 * tid; o < 2 * QC * L; o += 4 * kBigThreads) cp_async16(dst + o, src + o);
        cp_async_commit();
      }
    };
    if constexpr (MODE == ROW_R2C) {
      static_assert(2 * QC * L * 4 <= 2 * QC * NH * 8, "a chunk's real rows fit its part of P");
      if (!prefetched) stage_rows(slot, i0);
    }
    for (int q0 = 0; q0 < L / 2; q0 += QC) {
      float2* chunk = P + (2 * q0) * NH;  // the chunk's part of P
      if constexpr (MODE == ROW_R2C) {
        if (q0 == 0) cp_async_wait<1>();
        else cp_async_wait<0>();
        __syncthreads();  // the chunk's real rows have landed
      }
      for (int it = tid; it < QC * A; it += kBigThreads) {
        const int a = it % A, qq = it / A;
        float2 v[B];
        if constexpr (MODE == ROW_R2C) {
          const float* rows = reinterpret_cast<const float*>(chunk);  // [2 QC][L]
#pragma unroll
          for (int b = 0; b < B; ++b) {
            const int n = a + A * b;
            v[b] = make_float2(rows[(2 * qq) * L + n], rows[(2 * qq + 1) * L + n]);
          }
        } else {
#pragma unroll
          for (int b = 0; b < B; ++b) v[b] = chunk[qq * L + a + A * b];
        }
        Dft<B, -1>::run(v);
#pragma unroll
        for (int kb = 1; kb < B; ++kb) v[kb] = ctw<-1>(v[kb], tw[kb * A + a]);
#pragma unroll
        for (int kb = 0; kb < B; ++kb) W[qq * LS + kb * (A + 1) + a] = v[kb];
      }
      __syncthreads();  // the chunk's inputs are consumed
      // full spectra Z of the chunk's pairs -> the chunk's part of P (natural, [QC][L])
      for (int it = tid; it < QC * B; it += kBigThreads) {
        const int kb = it % B, qq = it / B;
        float2 w[A];
#pragma unroll
        for (int a = 0; a < A; ++a) w[a] = W[qq * LS + kb * (A + 1) + a];
        Dft<A, -1>::run(w);
#pragma unroll
        for (int ka = 0; ka < A; ++ka) chunk[qq * L + kb + B * ka] = w[ka];
      }
      __syncthreads();
      // split Z = FFT(x0 + i x1) into the two half rows, through W, then into P
      for (int it = tid; it < QC * NH; it += kBigThreads) {
        const int qq = it / NH, k = it % NH;
        const float2 z = chunk[qq * L + k];
        const float2 w = chunk[qq * L + (k == 0 ? 0 : L - k)];
        W[(2 * qq) * NH + k] = make_float2(0.5f * (z.x + w.x), 0.5f * (z.y - w.y));
        W[(2 * qq + 1) * NH + k] = make_float2(0.5f * (z.y + w.y), 0.5f * (w.x - z.x));
      }
      __syncthreads();
      for (int i = tid; i < QC * 2 * NH; i += kBigThreads) chunk[i] = W[i];
      __syncthreads();
    }
    float2* out = p.out_half + (int64_t)slot * p.out_stride;
    const int next = item + gridDim.x;
    // the next plane's input is copied once the last column chunk has read P: R2C its
    // real rows, RT its half spectrum
    const bool pre = MODE != ROW_C2R && next < nitems;
    for (int c0 = 0; c0 < NH; c0 += CW) {
      const bool last = c0 + CW >= NH;
      big_col_chunk<L, -1>(P, W, c0, min(CW, NH - c0), out, p.tm, i0, [&]() {
        if (pre && last) {
          if constexpr (MODE == ROW_R2C)
            stage_rows(next / L0, next % L0);
          else
            big_load<L>(P, p.in_half + (int64_t)(next / L0) * p.in_stride, p.tm, next % L0, 0,
                        G::HALF);
        }
      });
    }
    prefetched = pre;
  }
}

}  // namespace dev
}  // namespace sl
