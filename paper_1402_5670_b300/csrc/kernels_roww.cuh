// Warp-synchronous row passes for rows of 512 and 1024 points. Internal header.
//
// The CTA-wide row kernels (k_row_pipe) share each item's shared-memory stage and
// exchange among all warps of a CTA, so every item costs several CTA barriers, and for
// 512 = 32 x 16 their second pass keeps only half of the threads busy. Here every
// warp is an independent pipeline: it owns one row pair per work item, streams its own
// rows into its own two shared-memory stages with cp.async, and exchanges values only
// among its own lanes (__syncwarp, no CTA barrier). Both passes use all 32 lanes:
//   pass 1: lane a in [0, 32) takes the B values x[a + 32 b] (a length-B DFT);
//   pass 2: L = 1024 (B = 32): lane kb takes the 32 values of line kb;
//           L =  512 (B = 16): lanes 2 kb and 2 kb + 1 share line kb: each takes the
//           length-16 DFT of the even or the odd samples, and one radix-2 step across
//           the lane pair (shuffles) yields the 32 outputs, 16 per lane.
// Row pair (r0, r0 + 1) is transformed as the complex line Z = row r0 + i row r0+1
// (two real FFTs for the price of one complex FFT), as in k_row_pipe.
#pragma once

#include "kernels2d.cuh"

namespace sl {
namespace dev {


template <int L>
struct RowW {
  static constexpr int A = Split<L>::A, B = Split<L>::B;
  static_assert(A == 32 && (B == 16 || B == 32), "one row pair per warp needs A = 32");
  static constexpr int SF = 32 / B;                 // lanes per pass-2 line
  static constexpr int LS = SF == 2 ? A + 2 : A + 1;  // padded line stride of the exchange
  static constexpr int EXB = B * LS * 8;            // exchange bytes (>= L * 8)
  static_assert(EXB >= L * 8, "the exchange also holds a natural-order line");
};

// out[kb + B * ka] of the length-L line whose twiddled pass-1 values sit in ex
// ([kb][LS]); this lane's outputs are X[kb + B * (16 h + m)] (SF = 2, kb = lane / 2,
// h = lane % 2) or X[kb + B * m] (SF = 1, kb = lane), m < 32 / SF.
template <int L, int DIR>
__device__ __forceinline__ void roww_pass2(const float2* ex, int lane, float2 (&r)[32 / RowW<L>::SF]) {
  using RW = RowW<L>;
  constexpr int A = RW::A, LS = RW::LS;
  if constexpr (RW::SF == 1) {
#pragma unroll
    for (int aa = 0; aa < A; ++aa) r[aa] = ex[lane * LS + aa];
    Dft<A, DIR>::run(r);
  } else {
    const int kb = lane >> 1, h = lane & 1;
#pragma unroll
    for (int i = 0; i < 16; ++i) r[i] = ex[kb * LS + 2 * i + h];
    Dft<16, DIR>::run(r);  // E_h[m]
    // u[m] = W_32^m E_1[m] on the odd lane; X[m] = E_0 + u, X[m + 16] = E_0 - u
    constexpr float tr[16] = {Tw<32, 0>::re, Tw<32, 1>::re, Tw<32, 2>::re, Tw<32, 3>::re,
                              Tw<32, 4>::re, Tw<32, 5>::re, Tw<32, 6>::re, Tw<32, 7>::re,
                              Tw<32, 8>::re, Tw<32, 9>::re, Tw<32, 10>::re, Tw<32, 11>::re,
                              Tw<32, 12>::re, Tw<32, 13>::re, Tw<32, 14>::re, Tw<32, 15>::re};
    constexpr float ti[16] = {Tw<32, 0>::im, Tw<32, 1>::im, Tw<32, 2>::im, Tw<32, 3>::im,
                              Tw<32, 4>::im, Tw<32, 5>::im, Tw<32, 6>::im, Tw<32, 7>::im,
                              Tw<32, 8>::im, Tw<32, 9>::im, Tw<32, 10>::im, Tw<32, 11>::im,
                              Tw<32, 12>::im, Tw<32, 13>::im, Tw<32, 14>::im, Tw<32, 15>::im};
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      if (h) r[m] = ctw<DIR>(r[m], make_float2(tr[m], ti[m]));
      const float2 o = make_float2(__shfl_xor_sync(0xffffffffu, r[m].x, 1),
                                   __shfl_xor_sync(0xffffffffu, r[m].y, 1));
      r[m] = h ? csub(o, r[m]) : cadd(r[m], o);
    }
  }
}

// Output index of r[m] for this lane.
template <int L>
__device__ __forceinline__ int roww_k(int lane, int m) {
  using RW = RowW<L>;
  if constexpr (RW::SF == 1) return lane + RW::B * m;
  else return (lane >> 1) + RW::B * (16 * (lane & 1) + m);
}

// Persistent, warp-pipelined row pass: item i = (slot i / G, row pair i % G) with
// G = n_rows / 2; warp w of CTA c (W warps per CTA) takes items c W + w,
// + gridDim.x W, ...
// Modes and I/O as k_row_pipe (ROW_R2C, ROW_C2R, ROW_RT).
template <int L, int MODE, int W>
__global__ void __launch_bounds__(32 * W)
    k_row_warp(RowArgs p, int nslots, int NPp, int stage_bytes) {
  using RW = RowW<L>;
  constexpr int A = RW::A, B = RW::B, LS = RW::LS, NR = 32 / RW::SF;
  constexpr int H = L / 2;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* stg = smraw + (size_t)warp * (2 * stage_bytes + RW::EXB);  // [2][stage]
  float2* ex = reinterpret_cast<float2*>(stg + 2 * stage_bytes);
  const float2* tw = g_twiddle + twiddle_offset(L);
  const TileMap tm = p.tm;
  const int pairs = p.n_rows / 2;
  const int nitems = pairs * nslots;
  const int gstride = gridDim.x * W;
  const int tc = tm_tc(tm);
  const int nrun = NPp / tc;

  auto issue = [&](int item, int stage) {
    if (item < nitems) {
      const int slot = item / pairs, r0 = (item % pairs) * 2;
      unsigned char* dst = stg + stage * stage_bytes;
      if constexpr (MODE == ROW_R2C) {
        const char* src = reinterpret_cast<const char*>(p.in_real + (int64_t)slot * p.in_stride +
                                                        (int64_t)r0 * L);
        for (int o = lane * 16; o < 2 * L * 4; o += 32 * 16) cp_async16(dst + o, src + o);
      } else {
        const float2* src = p.in_half + (int64_t)slot * p.in_stride;
        const int chunks = tc / 2;  // 16-byte chunks per tile run
        const int per_row = nrun * chunks;
        for (int c = lane; c < 2 * per_row; c += 32) {
          const int rr = c / per_row, rem = c % per_row;
          const int t = rem / chunks, ch = rem % chunks;
          const float2* g = src + (((int64_t)t * tm.L0 + r0 + rr) << tm.lg) + 2 * ch;
          cp_async16(dst + ((int64_t)rr * NPp + t * tc + 2 * ch) * 8, g);
        }
      }
    }
    cp_async_commit();
  };

  int item = blockIdx.x * W + warp;
  issue(item, 0);
  issue(item + gstride, 1);
  for (int k = 0; item < nitems; ++k, item += gstride) {
    const int stage = k & 1;
    const int slot = item / pairs, r0 = (item % pairs) * 2;
    const unsigned char* in = stg + stage * stage_bytes;
    cp_async_wait<1>();
    __syncwarp();
    float2 r[NR];
    if constexpr (MODE == ROW_C2R || MODE == ROW_RT) {
      const float2* hin = reinterpret_cast<const float2*>(in);
      float2 v[B];
#pragma unroll
      for (int b = 0; b < B; ++b) {
        const int n = lane + A * b;
        const int m = n <= H ? n : L - n;
        float2 ya = hin[m], yb = hin[NPp + m];
        if (n > H) {
          ya = cconj(ya);
          yb = cconj(yb);
        }
        v[b] = make_float2(ya.x - yb.y, ya.y + yb.x);
      }
      __syncwarp();                    // stage read by every lane
      issue(item + 2 * gstride, stage);  // prefetch two items ahead
      Dft<B, 1>::run(v);
#pragma unroll
      for (int kb = 0; kb < B; ++kb) ex[kb * LS + lane] = kb ? ctw<1>(v[kb], tw[kb * A + lane]) : v[0];
      __syncwarp();
      roww_pass2<L, 1>(ex, lane, r);
      const float thr = p.use_thr ? p.thr.v[slot] : 0.f;
#pragma unroll
      for (int m = 0; m < NR; ++m) {
        float c0 = r[m].x * p.scale, c1 = r[m].y * p.scale;
        if (p.use_thr) {
          if (fabsf(c0) < thr) c0 = 0.f;
          if (fabsf(c1) < thr) c1 = 0.f;
        }
        r[m] = make_float2(c0, c1);
      }
      if constexpr (MODE == ROW_C2R) {
        float* o0 = p.out_real + (int64_t)slot * p.out_stride + (int64_t)r0 * L;
#pragma unroll
        for (int m = 0; m < NR; ++m) {
          const int kk = roww_k<L>(lane, m);
          o0[kk] = r[m].x;
          o0[L + kk] = r[m].y;
        }
        __syncwarp();  // exchange reads done before the next item's pass 1
        continue;
      }
      __syncwarp();  // pass-2 reads of the exchange done
#pragma unroll
      for (int m = 0; m < NR; ++m) ex[roww_k<L>(lane, m)] = r[m];  // natural order
      __syncwarp();
    }
    // real row pair -> half spectra
    {
      float2 v[B];
#pragma unroll
      for (int b = 0; b < B; ++b) {
        const int n = lane + A * b;
        if constexpr (MODE == ROW_R2C) {
          const float* rin = reinterpret_cast<const float*>(in);
          v[b] = make_float2(rin[n], rin[L + n]);
        } else {
          v[b] = ex[n];
        }
      }
      __syncwarp();  // stage (R2C) or natural line (RT) read by every lane
      if constexpr (MODE == ROW_R2C) issue(item + 2 * gstride, stage);
      Dft<B, -1>::run(v);
#pragma unroll
      for (int kb = 0; kb < B; ++kb) ex[kb * LS + lane] = kb ? ctw<-1>(v[kb], tw[kb * A + lane]) : v[0];
      __syncwarp();
      roww_pass2<L, -1>(ex, lane, r);
      __syncwarp();
#pragma unroll
      for (int m = 0; m < NR; ++m) ex[roww_k<L>(lane, m)] = r[m];
      __syncwarp();
    }
    // Z = FFT(x0 + i x1) -> half spectra of x0 and x1
    float2* out = p.out_half + (int64_t)slot * p.out_stride;
    for (int kk = lane; kk <= H; kk += 32) {
      const float2 z = ex[kk];
      const float2 w = ex[kk == 0 ? 0 : L - kk];
      out[tm.at(r0, kk)] = make_float2(0.5f * (z.x + w.x), 0.5f * (z.y - w.y));
      out[tm.at(r0 + 1, kk)] = make_float2(0.5f * (z.y + w.y), 0.5f * (w.x - z.x));
    }
    __syncwarp();  // exchange reads done before the next item's pass 1
  }
  cp_async_wait<0>();
}

template <int L>
constexpr int roww_exchange_bytes() { return RowW<L>::EXB; }

}  // namespace dev
}  // namespace sl
