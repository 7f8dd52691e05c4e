// Tensor-core pencil passes (mixed precision). Internal header.
//
// The DFT along axis 0 (length L = n0, a power of two in [64, 1024]) of a tile of TC
// pencils is computed in shared memory as a sequence of radix-8 stages, each one a
// real 16 x 16 matrix product on the tensor cores (mma.sync m16n8k16, BF16 operands,
// FP32 accumulation), preceded by one radix-2 or radix-4 stage in FP32 when L is not a
// power of 8. A complex DFT of length 8, Y = W x with W = exp(DIR 2 pi i k n / 8), is
// the real product
//     [Yr]   [ C  -DIR S ] [xr]        C[k][n] = cos(2 pi k n / 8)
//     [Yi] = [ DIR S   C ] [xi],       S[k][n] = sin(2 pi k n / 8),
// with the 16 x 16 matrix as operand A and 8 columns (independent length-8 DFTs) as
// operand B. Split precision: every FP32 operand v is carried as v_hi = bf16(v) and
// v_lo = bf16(v - v_hi), and the product is accumulated in FP32 as
// A_lo B_hi + A_hi B_lo + A_hi B_hi (the A_lo B_lo term, ~2^-18 relative, is dropped),
// which keeps each stage within about 1e-5 of FP32.
//
// FP16 operands (TC_OP_F16) carry 11 significant bits per part instead of BF16's 8,
// so the split keeps about 22 bits, but FP16's range ends at 65504: before the split,
// each warp scales its 16 x 8 block of operand B by a power of two 2^s that brings
// the block's largest magnitude to [2^12, 2^13), and multiplies the FP32 products by
// 2^-s (both exact). Values far below the block's largest lose relative precision in
// the lo part (subnormal FP16), which bounds the error relative to the block maximum,
// near 2^-22.
//
// Stage structure (decimation in time, in place). For a sub-length Ls = 8 Lr the data
// of outer block o is x[o Ls + n'' + Lr n1] (n'' < Lr, digit n1 < 8). A stage takes
// the length-8 DFT over n1 for every (o, n'', pencil), multiplies output digit k1 by
// the twiddle W_Ls^{n'' k1} and stores it back in the slot of n1. After the last stage
// X[k] sits at the digit-reversed position tc_pos<L>(k).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "kernels2d.cuh"

namespace sl {
namespace dev {

// Full twiddle tables: g_wfull[twiddle_offset(L) + m] = exp(-2 pi i m / L), m < L, for
// L = 8..1024 (powers of two). Filled by the host from FP64 values.
__device__ float2 g_wfull[kTwiddleTotal];

// L = r * 8^m with r in {1, 2, 4}
template <int L>
struct TcRadix {
  static constexpr int m = L >= 512 ? 3 : L >= 64 ? 2 : 1;
  static constexpr int pow8 = m == 3 ? 512 : m == 2 ? 64 : 8;
  static constexpr int r = L / pow8;
  static_assert(r == 1 || r == 2 || r == 4, "L must be r * 8^m");
};

constexpr int kTcThreads = 128;  // four warps per CTA

template <int L>
__device__ __forceinline__ int tc_pos(int k) {
  int pos = 0, Ls = L;
  if constexpr (TcRadix<L>::r > 1) {
    constexpr int r = TcRadix<L>::r;
    Ls = L / r;
    pos += Ls * (k % r);
    k /= r;
  }
#pragma unroll
  for (int i = 0; i < TcRadix<L>::m; ++i) {
    Ls >>= 3;
    pos += Ls * (k & 7);
    k >>= 3;
  }
  return pos;
}

__device__ __forceinline__ uint32_t bf16x2_bits(__nv_bfloat162 v) {
  return *reinterpret_cast<uint32_t*>(&v);
}

// (x0, x1) -> packed bf16 pairs hi = bf16(x), lo = bf16(x - hi); x0 in the low half.
__device__ __forceinline__ void split_bf16x2(float x0, float x1, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
  const float2 hf = __bfloat1622float2(h);
  hi = bf16x2_bits(h);
  lo = bf16x2_bits(__floats2bfloat162_rn(x0 - hf.x, x1 - hf.y));
}

__device__ __forceinline__ void mma_bf16_16x8x16(float (&d)[4], const uint32_t (&a)[4],
                                                 const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// (x0, x1) -> packed FP16 pairs hi = f16(x), lo = f16(x - hi); x0 in the low half.
__device__ __forceinline__ void split_f16x2(float x0, float x1, uint32_t& hi, uint32_t& lo) {
  const __half2 h = __floats2half2_rn(x0, x1);
  const float2 hf = __half22float2(h);
  const __half2 l = __floats2half2_rn(x0 - hf.x, x1 - hf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

__device__ __forceinline__ void mma_f16_16x8x16(float (&d)[4], const uint32_t (&a)[4],
                                                const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Operand type of the tensor-core stages (both operands of one product share it).
enum TcOp { TC_OP_BF16 = 0, TC_OP_F16 = 1 };

template <int OP>
__device__ __forceinline__ void split_x2(float x0, float x1, uint32_t& hi, uint32_t& lo) {
  if constexpr (OP == TC_OP_F16) split_f16x2(x0, x1, hi, lo);
  else split_bf16x2(x0, x1, hi, lo);
}

template <int OP>
__device__ __forceinline__ void mma_16x8x16(float (&d)[4], const uint32_t (&a)[4],
                                            const uint32_t (&b)[2]) {
  if constexpr (OP == TC_OP_F16) mma_f16_16x8x16(d, a, b);
  else mma_bf16_16x8x16(d, a, b);
}

// Power-of-two scale of a warp's operand block for FP16 (header comment): returns
// 2^s with s = 12 - floor(log2(max |v|)) clamped to [-126, 126], and 2^-s in *inv.
// m is this lane's largest magnitude; every lane of the warp must call it.
__device__ __forceinline__ float f16_block_scale(float m, float* inv) {
  const uint32_t bits = __reduce_max_sync(0xffffffffu, __float_as_uint(m));  // m >= 0
  const int e = (int)((bits >> 23) & 0xFF) - 127;
  const int s = max(-126, min(126, 12 - e));
  *inv = __uint_as_float((uint32_t)(127 - s) << 23);
  return __uint_as_float((uint32_t)(127 + s) << 23);
}

// Entry (row, col) of the real 16 x 16 form of the length-8 DFT (header comment).
template <int DIR>
__device__ __forceinline__ float dft8_real_entry(int row, int col) {
  constexpr float s = 0.70710678118654752f;
  const float cs8[8] = {1.f, s, 0.f, -s, -1.f, -s, 0.f, s};
  const float sn8[8] = {0.f, s, 1.f, s, 0.f, -s, -1.f, -s};
  const int m = ((row & 7) * (col & 7)) & 7;
  if ((row < 8) == (col < 8)) return cs8[m];
  return row < 8 ? -DIR * sn8[m] : DIR * sn8[m];
}

// A fragments (hi and lo) of the length-8 DFT matrix for this lane.
template <int DIR, int OP = TC_OP_BF16>
struct Dft8Frag {
  uint32_t hi[4], lo[4];
  __device__ __forceinline__ void init(int lane) {
    const int g = lane >> 2, q = lane & 3;
    const int rows[4] = {g, g + 8, g, g + 8};
    const int cols[4] = {2 * q, 2 * q, 2 * q + 8, 2 * q + 8};
#pragma unroll
    for (int i = 0; i < 4; ++i)
      split_x2<OP>(dft8_real_entry<DIR>(rows[i], cols[i]),
                   dft8_real_entry<DIR>(rows[i], cols[i] + 1), hi[i], lo[i]);
  }
};

// One radix-8 stage over sub-length Ls on wk ([L][TC] complex, element (n, p) at
// n * TC + p), in place; warps take n-tiles of 8 columns in turn.
template <int L, int TC, int DIR, int OP>
__device__ __forceinline__ void tc_radix8_stage(float2* wk, int Ls, const float2* wtab,
                                                const Dft8Frag<DIR, OP>& F, int warp, int lane) {
  constexpr int NT = L * TC / 64;
  constexpr int NW = kTcThreads / 32;
  const int Lr = Ls >> 3;
  const int dstride = Lr * TC;
  const int g = lane >> 2, q = lane & 3;
  const int tscale = L / Ls;
  for (int nt = warp; nt < NT; nt += NW) {
    const int c = nt * 8 + g;
    const int p = c % TC, rest = c / TC;
    const int base = ((rest / Lr) * Ls + rest % Lr) * TC + p;
    float2 x0 = wk[base + (2 * q) * dstride];
    float2 x1 = wk[base + (2 * q + 1) * dstride];
    float inv = 1.f;
    if constexpr (OP == TC_OP_F16) {
      const float sc = f16_block_scale(
          fmaxf(fmaxf(fabsf(x0.x), fabsf(x0.y)), fmaxf(fabsf(x1.x), fabsf(x1.y))), &inv);
      x0 = make_float2(x0.x * sc, x0.y * sc);
      x1 = make_float2(x1.x * sc, x1.y * sc);
    }
    uint32_t bh[2], bl[2];
    split_x2<OP>(x0.x, x1.x, bh[0], bl[0]);
    split_x2<OP>(x0.y, x1.y, bh[1], bl[1]);
    float d[4] = {0.f, 0.f, 0.f, 0.f};
    mma_16x8x16<OP>(d, F.lo, bh);
    mma_16x8x16<OP>(d, F.hi, bl);
    mma_16x8x16<OP>(d, F.hi, bh);
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int c2 = nt * 8 + 2 * q + e;
      const int p2 = c2 % TC, rest2 = c2 / TC;
      const int nlo = rest2 % Lr;
      float2 y = make_float2(d[e], d[2 + e]);
      if constexpr (OP == TC_OP_F16) y = make_float2(y.x * inv, y.y * inv);
      if (Lr > 1 && g != 0) y = ctw<DIR>(y, wtab[nlo * g * tscale]);
      wk[((rest2 / Lr) * Ls + nlo + g * Lr) * TC + p2] = y;
    }
  }
}

// The whole DFT of the tile in wk (in place, digit-reversed output), CTA-wide.
// Starts and ends with a barrier.
template <int L, int TC, int DIR, int OP>
__device__ __forceinline__ void tc_dft_tile(float2* wk, const float2* wtab,
                                            const Dft8Frag<DIR, OP>& F) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr int r = TcRadix<L>::r;
  int Ls = L;
  __syncthreads();
  if constexpr (r > 1) {
    constexpr int Lp = L / r;  // leading FP32 stage over the top digit
    for (int it = tid; it < Lp * TC; it += kTcThreads) {
      const int p = it % TC, n = it / TC;
      float2 v[r];
#pragma unroll
      for (int j = 0; j < r; ++j) v[j] = wk[(n + Lp * j) * TC + p];
      Dft<r, DIR>::run(v);
#pragma unroll
      for (int k1 = 0; k1 < r; ++k1) {
        const float2 y = k1 ? ctw<DIR>(v[k1], wtab[n * k1]) : v[0];
        wk[(n + Lp * k1) * TC + p] = y;
      }
    }
    Ls = Lp;
    __syncthreads();
  }
#pragma unroll 1
  for (; Ls >= 8; Ls >>= 3) {
    tc_radix8_stage<L, TC, DIR, OP>(wk, Ls, wtab, F, warp, lane);
    __syncthreads();
  }
}

template <int L>
__device__ __forceinline__ void tc_load_twiddles(float2* wtab) {
  const float2* src = g_wfull + twiddle_offset(L);
  for (int i = threadIdx.x; i < L; i += kTcThreads) wtab[i] = src[i];
}

// Forward filter pass on the tensor cores: the contract of k_col_fwd_pipe (item i is
// (tile i / nfilt, filter j0 + i % nfilt); out[s] = IFFT_0(in * psi[j0 + s])), with the
// product formed and transformed in place in the item's shared-memory stage.
template <int L, int OP>
__global__ void __launch_bounds__(kTcThreads) k_col_fwd_tc(ColArgs p) {
  constexpr int TC = col_tile_of(L), T = kTcThreads;
  constexpr int TILE = L * TC;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* xs = reinterpret_cast<float2*>(smraw);        // [2][TILE]
  float* ps = reinterpret_cast<float*>(xs + 2 * TILE);  // [2][TILE]
  float2* wtab = reinterpret_cast<float2*>(ps + 2 * TILE);
  const int tid = threadIdx.x;
  const int nitems = (int)(p.Nhp / TILE) * p.nfilt;
  Dft8Frag<1, OP> F;
  F.init(tid & 31);
  tc_load_twiddles<L>(wtab);

  auto issue = [&](int item, int stage) {
    if (item < nitems) {
      const int tile = item / p.nfilt, j = p.j0 + item % p.nfilt;
      cp_async_block<T>(xs + stage * TILE, p.in + (int64_t)tile * TILE, TILE * 8);
      cp_async_block<T>(ps + stage * TILE, p.psi + (int64_t)j * p.Nhp + (int64_t)tile * TILE,
                        TILE * 4);
    }
    cp_async_commit();
  };

  int item = blockIdx.x;
  issue(item, 0);
  issue(item + gridDim.x, 1);
  for (int k = 0; item < nitems; ++k, item += gridDim.x) {
    const int stage = k & 1;
    float2* wk = xs + stage * TILE;
    const float* pk = ps + stage * TILE;
    cp_async_wait<1>();
    __syncthreads();
    for (int e = tid; e < TILE; e += T) wk[e] = cscale(wk[e], pk[e]);
    tc_dft_tile<L, TC, 1, OP>(wk, wtab, F);
    const int tile = item / p.nfilt, s = item % p.nfilt;
    float2* o = p.out + (int64_t)s * p.Nhp + (int64_t)tile * TILE;
    for (int e = tid; e < TILE; e += T) o[e] = wk[tc_pos<L>(e / TC) * TC + e % TC];
    __syncthreads();  // stage consumed
    issue(item + 2 * gridDim.x, stage);
  }
  cp_async_wait<0>();
}

// Inverse accumulation on the tensor cores: the contract of k_col_inv_pipe (item i is
// (tile i % ntiles, split i / ntiles); out[part0 + split] = sum over the split's
// filters of psi_j * FFT_0(in[j - j0])), one (item, filter) load per stage.
template <int L, int OP>
__global__ void __launch_bounds__(kTcThreads) k_col_inv_tc(ColArgs p) {
  constexpr int TC = col_tile_of(L), T = kTcThreads;
  constexpr int TILE = L * TC, PER = TILE / T;
  static_assert(TILE % T == 0, "tile must split evenly over the threads");
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* zs = reinterpret_cast<float2*>(smraw);        // [2][TILE]
  float* ps = reinterpret_cast<float*>(zs + 2 * TILE);  // [2][TILE]
  float2* wtab = reinterpret_cast<float2*>(ps + 2 * TILE);
  const int tid = threadIdx.x;
  const int ntiles = (int)(p.Nhp / TILE);
  const int nsplit = (p.nfilt + p.fps - 1) / p.fps;
  const int nitems = ntiles * nsplit;
  Dft8Frag<-1, OP> F;
  F.init(tid & 31);
  tc_load_twiddles<L>(wtab);

  auto first_filter = [&](int item) { return (item / ntiles) * p.fps; };
  auto last_filter = [&](int item) { return min(first_filter(item) + p.fps, p.nfilt); };
  auto issue = [&](int item, int f, int stage) {
    if (item < nitems) {
      const int tile = item % ntiles;
      cp_async_block<T>(zs + stage * TILE, p.in + (int64_t)f * p.Nhp + (int64_t)tile * TILE,
                        TILE * 8);
      cp_async_block<T>(ps + stage * TILE,
                        p.psi + (int64_t)(p.j0 + f) * p.Nhp + (int64_t)tile * TILE, TILE * 4);
    }
    cp_async_commit();
  };
  auto advance = [&](int& item, int& f) {
    if (++f >= last_filter(item)) {
      item += gridDim.x;
      f = item < nitems ? first_filter(item) : 0;
    }
  };

  int cur_item = blockIdx.x, cur_f = cur_item < nitems ? first_filter(cur_item) : 0;
  int pre_item = cur_item, pre_f = cur_f;
  issue(pre_item, pre_f, 0);
  advance(pre_item, pre_f);
  issue(pre_item, pre_f, 1);
  advance(pre_item, pre_f);
  float2 acc[PER];
#pragma unroll
  for (int i = 0; i < PER; ++i) acc[i] = make_float2(0.f, 0.f);
  for (int k = 0; cur_item < nitems; ++k) {
    const int stage = k & 1;
    float2* wk = zs + stage * TILE;
    const float* pk = ps + stage * TILE;
    cp_async_wait<1>();
    tc_dft_tile<L, TC, -1, OP>(wk, wtab, F);
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int e = tid + T * i;
      const float f = pk[e];
      const float2 z = wk[tc_pos<L>(e / TC) * TC + e % TC];
      acc[i].x = fmaf(f, z.x, acc[i].x);
      acc[i].y = fmaf(f, z.y, acc[i].y);
    }
    __syncthreads();  // stage consumed
    issue(pre_item, pre_f, stage);
    advance(pre_item, pre_f);
    const int done_item = cur_item;
    advance(cur_item, cur_f);
    if (cur_item != done_item) {
      const int tile = done_item % ntiles, split = done_item / ntiles;
      float2* o = p.out + (int64_t)(p.part0 + split) * p.Nhp + (int64_t)tile * TILE;
#pragma unroll
      for (int i = 0; i < PER; ++i) {
        o[tid + T * i] = acc[i];
        acc[i] = make_float2(0.f, 0.f);
      }
    }
  }
  cp_async_wait<0>();
}

template <int L>
constexpr int tc_col_smem_bytes() {
  return 2 * L * col_tile_of(L) * (8 + 4) + L * 8;
}

}  // namespace dev
}  // namespace sl
