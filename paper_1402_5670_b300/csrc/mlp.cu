// Learned shrinkage: a small MLP that predicts a gain g in [0, 1] per shearlet
// coefficient from the coefficient, its neighbourhood magnitudes and a learned
// subband embedding, replacing the hard threshold of the paper's denoiser
// (eq. hard_tresholding, Sec. 5.3). Training (forward, backward, Adam) and inference
// run in these kernels; the products run on the tensor cores in BF16 with FP32
// accumulation: tcgen05.mma on 128-row tiles with the accumulators in tensor memory
// (the default engine, training and inference), or warp-level mma.sync with the
// activations in registers (the second engine); master weights stay FP32.
//
// Network (F = 1 + 3^ndim + 8 features, padded to KP = F rounded up to 16):
//   x = [c/s, |c(m+d)|/s for d in {-1,0,1}^ndim (row-major, periodic), E_j]
//   h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), g = sigmoid(w3 . h2 + b3), c_hat = g c
// with s = sigma ||psi_j||_2. Loss on a sample: mean(((g c - c_clean) / s)^2).
//
// mma.sync engine tiles: a warp handles 16 coefficients (the M = 16 rows of m16n8k16); the hidden
// width 64 is 8 n-tiles of 8. Fragment layouts (lane = 4 * gid + tig):
//   A 16x16: a0 = (gid, 2tig..+1), a1 = (gid+8, 2tig..+1), a2 = (gid, 2tig+8..+9),
//            a3 = (gid+8, 2tig+8..+9);   B 16x8: b0 = (k 2tig..+1, n gid), b1 = (k 2tig+8..+9, n gid)
//   C 16x8 : c0,c1 = (gid, 2tig..+1), c2,c3 = (gid+8, 2tig..+1).
// Two adjacent C n-tiles of one layer are exactly the A fragment of one k-slice of
// the next product, so activations stay in registers.

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/shearlet.h"

namespace {

constexpr int H = 64;   // hidden width
constexpr int EMB = 8;  // subband embedding
constexpr int WARPS = 8;
constexpr int ROWS = 16 * WARPS;  // coefficients per CTA tile

template <int NDIM>
struct Net {
  static constexpr int NB = NDIM == 2 ? 9 : 27;
  static constexpr int F = 1 + NB + EMB;
  static constexpr int KP = (F + 15) / 16 * 16;
  static constexpr int KS = KP / 16;
  // flat parameter offsets
  static constexpr int oW1 = 0, ob1 = oW1 + H * F, oW2 = ob1 + H, ob2 = oW2 + H * H,
                       ow3 = ob2 + H, ob3 = ow3 + H, oE = ob3 + 1;
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Shared-memory weights of one CTA: BF16 copies, row-major with padded rows.
template <int NDIM>
struct SmemW {
  static constexpr int KP = Net<NDIM>::KP;
  static constexpr int P1 = KP + 8;  // row pitch (bf16) of W1 [H][KP]
  static constexpr int P2 = H + 8;   // row pitch of W2 [H][H] and its transpose
  __nv_bfloat16 W1[H * P1];          // W1[o][k]
  __nv_bfloat16 W1T[KP * (H + 8)];   // W1T[k][o]
  __nv_bfloat16 W2[H * P2];          // W2[o][i]
  __nv_bfloat16 W2T[H * P2];         // W2T[i][o]
  float b1[H], b2[H], w3[H];
  float b3;
};

template <int NDIM>
__device__ void load_weights(SmemW<NDIM>& s, const float* __restrict__ prm) {
  using N = Net<NDIM>;
  constexpr int F = N::F, KP = N::KP;
  for (int i = threadIdx.x; i < H * KP; i += blockDim.x) {
    const int o = i / KP, k = i % KP;
    const float w = k < F ? prm[N::oW1 + o * F + k] : 0.f;
    s.W1[o * SmemW<NDIM>::P1 + k] = __float2bfloat16_rn(w);
    s.W1T[k * (H + 8) + o] = __float2bfloat16_rn(w);
  }
  for (int i = threadIdx.x; i < H * H; i += blockDim.x) {
    const int o = i / H, k = i % H;
    const float w = prm[N::oW2 + i];
    s.W2[o * SmemW<NDIM>::P2 + k] = __float2bfloat16_rn(w);
    s.W2T[k * SmemW<NDIM>::P2 + o] = __float2bfloat16_rn(w);
  }
  for (int i = threadIdx.x; i < H; i += blockDim.x) {
    s.b1[i] = prm[N::ob1 + i];
    s.b2[i] = prm[N::ob2 + i];
    s.w3[i] = prm[N::ow3 + i];
  }
  if (threadIdx.x == 0) s.b3 = prm[N::ob3];
}

struct Geom {
  int dims[3];  // grid
  int lg[3];    // log2 of dims
  int64_t N;    // points per subband
};

// Flat coefficient index q = j * N + m; the neighbour of m at offset index t
// (row-major over {-1, 0, 1}^ndim) with periodic wrap.
template <int NDIM>
__device__ __forceinline__ int64_t neighbour(const Geom& g, int64_t q, int t) {
  const int64_t m = q & (g.N - 1);
  const int64_t base = q - m;
  if constexpr (NDIM == 2) {
    const int i0 = (int)(m >> g.lg[1]), i1 = (int)(m & (g.dims[1] - 1));
    const int d0 = t / 3 - 1, d1 = t % 3 - 1;
    const int n0 = (i0 + d0) & (g.dims[0] - 1), n1 = (i1 + d1) & (g.dims[1] - 1);
    return base + ((int64_t)n0 << g.lg[1]) + n1;
  } else {
    const int i0 = (int)(m >> (g.lg[1] + g.lg[2]));
    const int i1 = (int)((m >> g.lg[2]) & (g.dims[1] - 1));
    const int i2 = (int)(m & (g.dims[2] - 1));
    const int d0 = t / 9 - 1, d1 = (t / 3) % 3 - 1, d2 = t % 3 - 1;
    const int n0 = (i0 + d0) & (g.dims[0] - 1), n1 = (i1 + d1) & (g.dims[1] - 1),
              n2 = (i2 + d2) & (g.dims[2] - 1);
    return base + ((((int64_t)n0 << g.lg[1]) + n1) << g.lg[2]) + n2;
  }
}

// Feature k of coefficient q (subband j, scale s), in FP32.
template <int NDIM>
__device__ __forceinline__ float feature(const Geom& g, const float* __restrict__ C, int64_t q,
                                         int j, float inv_s, const float* __restrict__ E, int k) {
  using N = Net<NDIM>;
  if (k == 0) return C[q] * inv_s;
  if (k <= N::NB) return fabsf(C[neighbour<NDIM>(g, q, k - 1)]) * inv_s;
  if (k <= N::NB + EMB) return E[j * EMB + (k - N::NB - 1)];
  return 0.f;
}

// Forward of one warp tile (16 coefficients, rows gid and gid+8 of this thread).
// Outputs: g for both rows; optionally the intermediates for backward.
template <int NDIM, bool TRAIN>
struct Fwd {
  uint32_t A1[Net<NDIM>::KS][4];  // features (bf16 A fragments)
  uint32_t A2[4][4];              // h1 (bf16 A fragments, 4 k-slices of 16)
  float z1[8][4], z2[8][4];       // pre-activations (C layout)
  float z3[2], g[2];
};

template <int NDIM, bool TRAIN>
__device__ __forceinline__ void mlp_forward(const SmemW<NDIM>& s, Fwd<NDIM, TRAIN>& f,
                                            const Geom& geo, const float* __restrict__ C,
                                            const int64_t (&q)[2], const int (&j)[2],
                                            const float (&inv_s)[2],
                                            const float* __restrict__ E) {
  using N = Net<NDIM>;
  const int lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;
  // features -> A fragments
#pragma unroll
  for (int ks = 0; ks < N::KS; ++ks) {
    float v[2][4];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int e = 0; e < 2; ++e)
          v[r][2 * h + e] = feature<NDIM>(geo, C, q[r], j[r], inv_s[r], E, 16 * ks + 8 * h + 2 * tig + e);
    f.A1[ks][0] = pack_bf16(v[0][0], v[0][1]);
    f.A1[ks][1] = pack_bf16(v[1][0], v[1][1]);
    f.A1[ks][2] = pack_bf16(v[0][2], v[0][3]);
    f.A1[ks][3] = pack_bf16(v[1][2], v[1][3]);
  }
  // layer 1
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const int n0 = 8 * nt + 2 * tig;
    float d[4] = {s.b1[n0], s.b1[n0 + 1], s.b1[n0], s.b1[n0 + 1]};
#pragma unroll
    for (int ks = 0; ks < N::KS; ++ks) {
      const __nv_bfloat16* w = s.W1 + (8 * nt + gid) * SmemW<NDIM>::P1 + 16 * ks + 2 * tig;
      mma16816(d, f.A1[ks], *reinterpret_cast<const uint32_t*>(w),
               *reinterpret_cast<const uint32_t*>(w + 8));
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) f.z1[nt][i] = d[i];
  }
  // h1 = relu(z1) -> A fragments of layer 2
#pragma unroll
  for (int ks = 0; ks < 4; ++ks) {
    const float(&lo)[4] = f.z1[2 * ks];
    const float(&hi)[4] = f.z1[2 * ks + 1];
    f.A2[ks][0] = pack_bf16(fmaxf(lo[0], 0.f), fmaxf(lo[1], 0.f));
    f.A2[ks][1] = pack_bf16(fmaxf(lo[2], 0.f), fmaxf(lo[3], 0.f));
    f.A2[ks][2] = pack_bf16(fmaxf(hi[0], 0.f), fmaxf(hi[1], 0.f));
    f.A2[ks][3] = pack_bf16(fmaxf(hi[2], 0.f), fmaxf(hi[3], 0.f));
  }
  // layer 2 and the dot with w3
  float part[2] = {0.f, 0.f};
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const int n0 = 8 * nt + 2 * tig;
    float d[4] = {s.b2[n0], s.b2[n0 + 1], s.b2[n0], s.b2[n0 + 1]};
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {
      const __nv_bfloat16* w = s.W2 + (8 * nt + gid) * SmemW<NDIM>::P2 + 16 * ks + 2 * tig;
      mma16816(d, f.A2[ks], *reinterpret_cast<const uint32_t*>(w),
               *reinterpret_cast<const uint32_t*>(w + 8));
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) f.z2[nt][i] = d[i];
    part[0] += fmaxf(d[0], 0.f) * s.w3[n0] + fmaxf(d[1], 0.f) * s.w3[n0 + 1];
    part[1] += fmaxf(d[2], 0.f) * s.w3[n0] + fmaxf(d[3], 0.f) * s.w3[n0 + 1];
  }
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    float z = part[r];
    z += __shfl_xor_sync(0xffffffffu, z, 1);
    z += __shfl_xor_sync(0xffffffffu, z, 2);
    f.z3[r] = z + s.b3;
    f.g[r] = 1.f / (1.f + expf(-f.z3[r]));
  }
}

struct MlpArgs {
  const float* prm;   // master parameters (FP32, flat)
  const float* C;     // noisy coefficients [R][N]
  const float* Cc;    // clean coefficients (training)
  float* out;         // inference output [R][N] (never aliases C)
  const int* idx;     // training sample: flat indices q = j N + m, j >= 1
  int n;              // samples (multiple of 128) or tiles
  const float* inv_s; // [R] 1 / (sigma ||psi_j||)
  float* grad;        // gradient accumulators (FP32, flat, zeroed by the caller)
  float* loss;        // loss accumulator (device scalar)
  Geom geo;
  int R;
};

// Inference over all subbands j >= 1: out[j][m] = g * C[j][m]; out[0] = C[0].
template <int NDIM>
__global__ void __launch_bounds__(32 * WARPS) k_mlp_apply(MlpArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  SmemW<NDIM>& s = *reinterpret_cast<SmemW<NDIM>*>(smraw);
  load_weights<NDIM>(s, a.prm);
  __syncthreads();
  const int lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;
  const int warp = threadIdx.x >> 5;
  const float* E = a.prm + Net<NDIM>::oE;
  const int64_t tiles = (int64_t)(a.R - 1) * (a.geo.N / 16);
  for (int64_t t = (int64_t)blockIdx.x * WARPS + warp; t < tiles; t += (int64_t)gridDim.x * WARPS) {
    const int64_t q0 = a.geo.N + t * 16;  // subbands 1.. are contiguous after subband 0
    const int jj = (int)(q0 / a.geo.N);
    int64_t q[2] = {q0 + gid, q0 + gid + 8};
    int j[2] = {jj, jj};
    float is[2] = {a.inv_s[jj], a.inv_s[jj]};
    Fwd<NDIM, false> f;
    mlp_forward<NDIM, false>(s, f, a.geo, a.C, q, j, is, E);
    if (tig == 0) {
      a.out[q[0]] = f.g[0] * a.C[q[0]];
      a.out[q[1]] = f.g[1] * a.C[q[1]];
    }
  }
  // the lowpass passes through
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.geo.N;
         i += (int64_t)gridDim.x * blockDim.x)
      a.out[i] = a.C[i];
}

// ---------------------------------------------- inference on tcgen05 tensor cores ---
// Tiles of 128 coefficients: one CTA of 4 warps, thread t builds the features of row t
// (BF16, in shared memory), one thread issues tcgen05.mma for the two dense layers
// with the accumulator in tensor memory (128 lanes = rows, 64 FP32 columns, reused by
// both layers), and every warp reads its 32 rows back with tcgen05.ld for bias, ReLU,
// the output dot and the gain. The raw neighbourhood of the next tile is loaded into
// registers while the current tile is in the tensor cores, so global-memory latency
// overlaps the products and the epilogues.
// Operands are K-major without swizzle: 8 x 16-byte core matrices, element (r, k) of a
// [rows][K] tile at ((r / 8) (K / 8) + k / 8) 128 + (r % 8) 16 + (k % 8) 2 bytes, so the
// descriptors' leading (K) offset is 128 B and the stride (row block) offset (K / 8) 128 B.
constexpr int TC_ROWS = 128;
constexpr int TC_THREADS = 128;
constexpr int TC_TMEM_COLS = 64;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ int kmajor(int r, int k, int K) {
  return ((r >> 3) * (K >> 3) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// tcgen05 shared-memory matrix descriptor: start, leading and stride byte offsets
// (all >> 4), the fixed descriptor version 1 at bit 46, no swizzle.
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// kind::f16 instruction descriptor: FP32 accumulator, BF16 A and B, both K-major,
// M = 128 and N (a multiple of 16, 16..256).
__host__ __device__ constexpr uint32_t idesc_m128(uint32_t n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((128u >> 4) << 24);
}
constexpr uint32_t kIdesc = idesc_m128(64);

__device__ __forceinline__ void umma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc,
                                          uint32_t idesc = kIdesc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.u32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
      smem_addr(bar)));
}

// Default limit of a tensor-core wait: about two seconds of SM clock.
constexpr long long kTcWaitCycles = 4000000000LL;

// Bounded wait for the mbarrier phase with the given parity; false once `limit`
// cycles have passed without the phase completing.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity,
                                          long long limit = kTcWaitCycles) {
  if (limit <= 0) return false;  // a zero budget gives up at once (test hook)
  uint32_t done = 0;
  const long long t0 = clock64();
  while (!done) {
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity));
    if (!done && clock64() - t0 > limit) return false;
  }
  return true;
}

// 32 FP32 accumulator columns of this thread's TMEM lane (warp w owns lanes 32w..).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
        "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
        "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// 16 FP32 accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tc_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// generic-proxy shared-memory writes -> visible to the tensor cores' reads
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ReLU and round to BF16, two values packed (lo in the low half)
__device__ __forceinline__ uint32_t relu_pack_bf16(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}

// The biases ride in the products: b = hi + lo (two BF16 parts, |b - hi - lo| <=
// 2^-16 |b|) occupy two extra K columns of W1 and W2, against two constant-one
// columns of the activations, so the epilogues read no bias.
constexpr int K2 = H + 16;  // layer-2 K: h1, [1, 1], zero padding

// The weights of one CTA as its shared memory holds them, packed once per call by
// k_mlp_pack_tc and copied by every CTA with 16-byte loads.
template <int NDIM>
struct TcWeights {
  static constexpr int KP = Net<NDIM>::KP;
  static_assert(Net<NDIM>::F + 2 <= KP, "two bias columns after the features");
  // operand tiles without swizzle need only 16-byte alignment
  alignas(16) unsigned char w1[H * KP * 2];  // [W1, b1 hi, b1 lo, 0..] [64][KP]
  alignas(16) unsigned char w2[H * K2 * 2];  // [W2, b2 hi, b2 lo, 0..] [64][K2]
  alignas(16) float w3[H];
  alignas(16) float b3[4];
};

template <int NDIM>
struct TcApplySmem {
  static_assert(Net<NDIM>::KP <= K2, "the layer-1 operand shares the layer-2 buffer");
  static_assert(sizeof(TcWeights<NDIM>) % 16 == 0, "copied in 16-byte pieces");
  TcWeights<NDIM> w;
  // act holds the features [128][KP] for layer 1, then [h1, 1, 1, 0..] [128][K2]
  alignas(16) unsigned char act[TC_ROWS * K2 * 2];
  alignas(8) uint64_t bar;
  uint32_t tmem;
};

// FP32 master parameters -> the BF16 K-major weight tiles of TcWeights, one element
// per thread over w1, w2, w3 and b3 in turn.
template <int NDIM>
__host__ __device__ constexpr int tc_pack_elems() { return H * Net<NDIM>::KP + H * K2 + H + 4; }

template <int NDIM>
__device__ __forceinline__ void pack_tc_one(const float* __restrict__ prm,
                                            TcWeights<NDIM>* __restrict__ out, int i) {
  using NN = Net<NDIM>;
  constexpr int F = NN::F, KP = NN::KP;
  auto split = [](float b, bool lo_part) {
    const __nv_bfloat16 hi = __float2bfloat16_rn(b);
    return lo_part ? __float2bfloat16_rn(b - __bfloat162float(hi)) : hi;
  };
  if (i < H * KP) {
    const int o = i / KP, k = i % KP;
    __nv_bfloat16 w = __float2bfloat16_rn(0.f);
    if (k < F) w = __float2bfloat16_rn(prm[NN::oW1 + o * F + k]);
    else if (k < F + 2) w = split(prm[NN::ob1 + o], k == F + 1);
    *reinterpret_cast<__nv_bfloat16*>(out->w1 + kmajor(o, k, KP)) = w;
    return;
  }
  i -= H * KP;
  if (i < H * K2) {
    const int o = i / K2, k = i % K2;
    __nv_bfloat16 w = __float2bfloat16_rn(0.f);
    if (k < H) w = __float2bfloat16_rn(prm[NN::oW2 + o * H + k]);
    else if (k < H + 2) w = split(prm[NN::ob2 + o], k == H + 1);
    *reinterpret_cast<__nv_bfloat16*>(out->w2 + kmajor(o, k, K2)) = w;
    return;
  }
  i -= H * K2;
  if (i < H) {
    out->w3[i] = prm[NN::ow3 + i];
    return;
  }
  i -= H;
  if (i < 4) out->b3[i] = i == 0 ? prm[NN::ob3] : 0.f;
}

template <int NDIM>
__global__ void __launch_bounds__(256) k_mlp_pack_tc(const float* __restrict__ prm,
                                                     TcWeights<NDIM>* __restrict__ out) {
  pack_tc_one<NDIM>(prm, out, blockIdx.x * blockDim.x + threadIdx.x);
}

// Read-only global load that the compiler keeps where it is written (a prefetch a
// tile ahead must not sink to its first use).
__device__ __forceinline__ float ld_early(const float* p) {
  float v;
  asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}

// The raw neighbourhood of point m of one subband (nb in the row-major order of
// {-1, 0, 1}^ndim that neighbour() uses), with the periodic wrap taken once per axis.
template <int NDIM>
__device__ __forceinline__ void gather_nb(const Geom& g, const float* __restrict__ sub, uint32_t m,
                                          float (&nb)[Net<NDIM>::NB]) {
  if constexpr (NDIM == 2) {
    const uint32_t m0 = g.dims[0] - 1, m1 = g.dims[1] - 1;
    const uint32_t i0 = m >> g.lg[1], i1 = m & m1;
    const uint32_t r[3] = {((i0 - 1) & m0) << g.lg[1], i0 << g.lg[1], ((i0 + 1) & m0) << g.lg[1]};
    const uint32_t c[3] = {(i1 - 1) & m1, i1, (i1 + 1) & m1};
#pragma unroll
    for (int a0 = 0; a0 < 3; ++a0)
#pragma unroll
      for (int a1 = 0; a1 < 3; ++a1) nb[3 * a0 + a1] = ld_early(sub + (r[a0] + c[a1]));
  } else {
    const uint32_t m0 = g.dims[0] - 1, m1 = g.dims[1] - 1, m2 = g.dims[2] - 1;
    const int s0 = g.lg[1] + g.lg[2];
    const uint32_t i0 = m >> s0, i1 = (m >> g.lg[2]) & m1, i2 = m & m2;
    const uint32_t pl[3] = {((i0 - 1) & m0) << s0, i0 << s0, ((i0 + 1) & m0) << s0};
    const uint32_t r[3] = {((i1 - 1) & m1) << g.lg[2], i1 << g.lg[2], ((i1 + 1) & m1) << g.lg[2]};
    const uint32_t c[3] = {(i2 - 1) & m2, i2, (i2 + 1) & m2};
#pragma unroll
    for (int a0 = 0; a0 < 3; ++a0)
#pragma unroll
      for (int a1 = 0; a1 < 3; ++a1) {
        const uint32_t pr = pl[a0] + r[a1];
#pragma unroll
        for (int a2 = 0; a2 < 3; ++a2) nb[9 * a0 + 3 * a1 + a2] = ld_early(sub + (pr + c[a2]));
      }
  }
}

template <int NDIM>
__global__ void __launch_bounds__(TC_THREADS)
    k_mlp_apply_tc(MlpArgs a, const TcWeights<NDIM>* __restrict__ wg, int* err,
                   long long wait_limit) {
  using NN = Net<NDIM>;
  constexpr int F = NN::F, KP = NN::KP, NB = NN::NB;
  constexpr int CENTRE = NB / 2;  // offset (0, .., 0) in the row-major neighbourhood
  extern __shared__ __align__(16) unsigned char smraw[];
  TcApplySmem<NDIM>& S = *reinterpret_cast<TcApplySmem<NDIM>*>(smraw);
  const int tid = threadIdx.x, warp = tid >> 5;
  // Tensor memory first: the SM starts its next CTA only once this one has given up
  // its allocation permit.
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(&S.tmem)),
                 "n"(TC_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  {
    constexpr int n16 = (int)(sizeof(TcWeights<NDIM>) / 16);
    const uint4* src = reinterpret_cast<const uint4*>(wg);
    uint4* dst = reinterpret_cast<uint4*>(&S.w);
    for (int i = tid; i < n16; i += TC_THREADS) dst[i] = __ldg(src + i);
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&S.bar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  fence_async_smem();  // the weight tiles are read by the tensor cores
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  const uint32_t tmem = S.tmem;
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  const float* E = a.prm + NN::oE;
  const int64_t total = (int64_t)(a.R - 1) * a.geo.N;
  const int64_t tiles = (total + TC_ROWS - 1) / TC_ROWS;
  const uint32_t act = smem_addr(S.act), w1 = smem_addr(S.w.w1), w2 = smem_addr(S.w.w2);
  const int lgN = a.geo.lg[0] + a.geo.lg[1] + a.geo.lg[2];
  constexpr uint32_t kOnes = 0x3F803F80u;  // two BF16 ones
  // raw neighbourhood of this thread's row, gathered one tile ahead (rows past the
  // end read coefficient N); N = 2^lgN points per subband (sizes are powers of two)
  float nb[NB];
  auto gather = [&](int64_t t) {
    const int64_t idx = t * TC_ROWS + tid;
    const int64_t q = a.geo.N + (t < tiles && idx < total ? idx : 0);
    gather_nb<NDIM>(a.geo, a.C + ((q >> lgN) << lgN), (uint32_t)(q & (a.geo.N - 1)), nb);
  };
  gather(blockIdx.x);
  // Each tile completes two phases of the mbarrier: layer 1 (parity 0), layer 2
  // (parity 1). Every thread waits on both, so none lags a phase behind; a wait that
  // runs out is made CTA-uniform at the next barrier, and the loop ends there.
  int timed_out = 0;     // CTA-uniform
  uint32_t pending = 0;  // parity of the phase a timed-out wait left in flight
  bool late = false;     // this warp's last wait ran out (warp-uniform)
  for (int64_t t = blockIdx.x;; t += gridDim.x) {
    const bool more = t < tiles;
    const int64_t idx = t * TC_ROWS + tid;
    const bool valid = more && idx < total;
    const int64_t q = a.geo.N + (valid ? idx : 0);  // other rows compute on coefficient N
    float c = 0.f;
    if (more) {
      const int j = (int)(q >> lgN);
      c = nb[CENTRE];
      const float is = a.inv_s[j];
      // features of this thread's row, the two bias ones -> act (8 BF16 per store)
      float x[KP];
      x[0] = c * is;
#pragma unroll
      for (int d = 0; d < NB; ++d) x[1 + d] = fabsf(nb[d]) * is;
#pragma unroll
      for (int e = 0; e < EMB; ++e) x[1 + NB + e] = __ldg(E + j * EMB + e);
      x[F] = 1.f;
      x[F + 1] = 1.f;
#pragma unroll
      for (int k = F + 2; k < KP; ++k) x[k] = 0.f;
#pragma unroll
      for (int k8 = 0; k8 < KP / 8; ++k8)
        *reinterpret_cast<uint4*>(S.act + kmajor(tid, 8 * k8, KP)) =
            make_uint4(pack_bf16(x[8 * k8], x[8 * k8 + 1]), pack_bf16(x[8 * k8 + 2], x[8 * k8 + 3]),
                       pack_bf16(x[8 * k8 + 4], x[8 * k8 + 5]),
                       pack_bf16(x[8 * k8 + 6], x[8 * k8 + 7]));
    }
    fence_async_smem();
    tc_before_sync();
    // features written, previous tile's TMEM reads done; any earlier timeout seen
    if (__syncthreads_or(late)) {
      timed_out = 1;
      pending = 1;
      break;
    }
    tc_after_sync();
    if (!more) break;
    if (tid == 0) {
#pragma unroll
      for (int ks = 0; ks < KP / 16; ++ks)
        umma_bf16(tmem, umma_desc(act + ks * 256, 128, (KP / 8) * 128),
                  umma_desc(w1 + ks * 256, 128, (KP / 8) * 128), ks > 0);
      umma_commit(&S.bar);
    }
    late = __any_sync(0xffffffffu, !mbar_wait(&S.bar, 0, wait_limit));
    tc_after_sync();
    if (!late) {
      // h1 = relu(z1) -> act, 32 columns at a time, then the bias ones
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float z[32];
        tmem_ld32(tmem + lane_base + 32 * h, z);
#pragma unroll
        for (int k8 = 0; k8 < 4; ++k8)
          *reinterpret_cast<uint4*>(S.act + kmajor(tid, 32 * h + 8 * k8, K2)) =
              make_uint4(relu_pack_bf16(z[8 * k8], z[8 * k8 + 1]),
                         relu_pack_bf16(z[8 * k8 + 2], z[8 * k8 + 3]),
                         relu_pack_bf16(z[8 * k8 + 4], z[8 * k8 + 5]),
                         relu_pack_bf16(z[8 * k8 + 6], z[8 * k8 + 7]));
      }
      *reinterpret_cast<uint4*>(S.act + kmajor(tid, H, K2)) = make_uint4(kOnes, 0u, 0u, 0u);
      *reinterpret_cast<uint4*>(S.act + kmajor(tid, H + 8, K2)) = make_uint4(0u, 0u, 0u, 0u);
    }
    fence_async_smem();
    tc_before_sync();
    if (__syncthreads_or(late)) {
      timed_out = 1;
      pending = 0;
      break;
    }
    tc_after_sync();
    gather(t + gridDim.x);  // the next tile's loads overlap layer 2
    if (tid == 0) {
#pragma unroll
      for (int ks = 0; ks < K2 / 16; ++ks)
        umma_bf16(tmem, umma_desc(act + ks * 256, 128, (K2 / 8) * 128),
                  umma_desc(w2 + ks * 256, 128, (K2 / 8) * 128), ks > 0);
      umma_commit(&S.bar);
    }
    late = __any_sync(0xffffffffu, !mbar_wait(&S.bar, 1, wait_limit));
    tc_after_sync();
    if (!late) {
      float acc[4] = {S.w.b3[0], 0.f, 0.f, 0.f};  // four chains of 16
      const float4* w3 = reinterpret_cast<const float4*>(S.w.w3);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float z[32];
        tmem_ld32(tmem + lane_base + 32 * h, z);
#pragma unroll
        for (int k4 = 0; k4 < 8; ++k4) {
          const float4 w = w3[8 * h + k4];
          acc[0] += fmaxf(z[4 * k4], 0.f) * w.x;
          acc[1] += fmaxf(z[4 * k4 + 1], 0.f) * w.y;
          acc[2] += fmaxf(z[4 * k4 + 2], 0.f) * w.z;
          acc[3] += fmaxf(z[4 * k4 + 3], 0.f) * w.w;
        }
      }
      const float g = 1.f / (1.f + expf(-((acc[0] + acc[1]) + (acc[2] + acc[3]))));
      if (valid) a.out[q] = g * c;
    }
  }
  if (timed_out) {
    if (tid == 0) {
      atomicExch(err, 1);
      // let the MMAs in flight finish (bounded by the default limit, whatever the
      // per-tile limit was) before the tensor memory is freed
      mbar_wait(&S.bar, pending);
    }
    __syncthreads();
  }
  // the lowpass passes through
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.geo.N;
       i += (int64_t)gridDim.x * blockDim.x)
    a.out[i] = a.C[i];
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "n"(TC_TMEM_COLS));
}

// Persistent grid: every SM holds as many CTAs as its registers, shared memory and
// tensor memory (TC_TMEM_COLS of 512 columns each) allow. (The occupancy calculator
// is not used: for this kernel it reports one CTA per SM, below what runs.)
static int sm_count() {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

template <int NDIM>
static int apply_tc_grid() {
  static int grid[64] = {0};  // per device
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!grid[dev]) {
    int smem_sm = 228 * 1024, regs_sm = 65536;
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    cudaFuncAttributes fa{};
    cudaFuncGetAttributes(&fa, k_mlp_apply_tc<NDIM>);
    const int regs = std::max(1, (fa.numRegs + 7) / 8 * 8) * TC_THREADS;
    const int smem = (int)sizeof(TcApplySmem<NDIM>) + 1024;  // + the per-CTA reserve
    int per_sm = std::min({512 / TC_TMEM_COLS, smem_sm / smem, regs_sm / regs});
    grid[dev] = std::max(1, per_sm) * sm_count();
  }
  return grid[dev];
}

// ---------------------------------------------- training on tcgen05 tensor cores ---
// One CTA of 8 warps per SM walks tiles of 128 samples; row r of a tile is TMEM lane
// r, read by warps r / 32 and 4 + r / 32, which split the 64 columns of every layer
// between them (warps 0-3 take columns 0-31, warps 4-7 columns 32-63). Per tile, one
// thread issues six products, each accumulating in tensor memory:
//   z1  = [x, 1, 1] [W1, b1]^T            (128 x 64, K = KP)     -> columns 0..63
//   z2  = [h1, 1, 1] [W2, b2]^T           (128 x 64, K = K2)     -> columns 0..63
//   dh1 = dz2 W2                          (128 x 64, K = 64)     -> columns 0..63
//   D1 += [dz2 ; dz1]^T [x ; h1]          (128 x (KP + 64), K = the tile's 128 rows)
//   D2 += [h2 ; x ; h1]^T [dz3, 0 ..]     (128 x 16, K = 128)
//   DE  = dz1 [W1 embedding columns, 0 ..] (128 x 16, K = 64)
// D1 and D2 carry the weight gradients across the CTA's tiles: D1 holds dW2 (dz2 rows x
// h1 columns), dW1 (dz1 rows x feature columns), and through the constant-one feature
// column b2's and b1's gradients; D2 holds w3's gradient (h2 rows) and b3's (the
// one-row of x). The cross blocks (dz2 x features, dz1 x h1, ...) are computed and
// ignored: they keep both products at M = 128. DE is each row's gradient with respect
// to its subband embedding, added into a per-CTA table in shared memory (read at the
// start of the next tile, while that tile's features are built). At the end every CTA
// writes its gradients and its loss as one row of a partial-sum table; k_mlp_reduce
// adds the rows in a fixed order (and applies Adam).
// The weight-gradient operands are K-major over the tile's rows (element (m, r) of a
// [M][128] tile), written with one 2-byte store per value; their core matrices sit
// 144 bytes apart along K (128 + 16 of padding) so that the four 8-lane groups of a
// warp store into different banks.
constexpr int TT_THREADS = 256;
constexpr int TT_TMEM_COLS = 256;
constexpr int KR = 128;                  // rows per tile = K of the weight-gradient products
constexpr int KR_LBO = 144;              // K-direction core-matrix stride of those operands
constexpr int KR_SBO = (KR / 8) * KR_LBO;  // 8-row block stride

__host__ __device__ __forceinline__ int kmajor_r(int m, int r) {
  return (m >> 3) * KR_SBO + (r >> 3) * KR_LBO + (m & 7) * 16 + (r & 7) * 2;
}

// Weights of one training CTA: the inference tiles plus W2 transposed (the B operand of
// dz2 W2: element (i, o) = W2[o][i], K-major over o) and W1's embedding columns
// transposed (the B operand of DE: element (e, o) = W1[o][1 + NB + e] for e < 8, zero
// rows 8..15).
template <int NDIM>
struct TcTrainWeights {
  TcWeights<NDIM> base;
  alignas(16) unsigned char w2t[H * H * 2];
  alignas(16) unsigned char w1et[16 * H * 2];
};

template <int NDIM>
__host__ __device__ constexpr int tc_train_pack_elems() {
  return tc_pack_elems<NDIM>() + H * H + 16 * H;
}

template <int NDIM>
__global__ void __launch_bounds__(256) k_mlp_pack_train(const float* __restrict__ prm,
                                                        TcTrainWeights<NDIM>* __restrict__ out) {
  using NN = Net<NDIM>;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < tc_pack_elems<NDIM>()) {
    pack_tc_one<NDIM>(prm, &out->base, i);
    return;
  }
  i -= tc_pack_elems<NDIM>();
  if (i < H * H) {
    const int n = i / H, o = i % H;  // row n = hidden unit of h1, K index o
    *reinterpret_cast<__nv_bfloat16*>(out->w2t + kmajor(n, o, H)) =
        __float2bfloat16_rn(prm[NN::oW2 + o * H + n]);
    return;
  }
  i -= H * H;
  if (i < 16 * H) {
    const int e = i / H, o = i % H;
    const float w = e < EMB ? prm[NN::oW1 + o * NN::F + 1 + NN::NB + e] : 0.f;
    *reinterpret_cast<__nv_bfloat16*>(out->w1et + kmajor(e, o, H)) = __float2bfloat16_rn(w);
  }
}

template <int NDIM>
struct TcTrainSmem {
  static constexpr int KP = Net<NDIM>::KP;
  static constexpr int TR = 128 + KP;  // rows of tt
  TcTrainWeights<NDIM> w;
  // features [128][KP], then [h1, 1, 1, 0..] [128][K2], then dz2 [128][64], then dz1
  // [128][64] (K-major)
  alignas(16) unsigned char act[TC_ROWS * K2 * 2];
  alignas(16) unsigned char aw1[(128 / 8) * KR_SBO];  // [dz2^T ; dz1^T]      [128][KR]
  alignas(16) unsigned char tt[(TR / 8) * KR_SBO];    // [h2^T ; x^T ; h1^T]  [TR][KR]
  alignas(16) unsigned char bw2[(16 / 8) * KR_SBO];   // [dz3 ; 0 x 15]       [16][KR]
  alignas(8) uint64_t bar;
  uint32_t tmem;
  float red[TT_THREADS / 32];
  float z3half[2][TC_ROWS];  // each column half's part of the output dot
  int jrow[TC_ROWS];         // subband of each row of the tile
  // followed by the CTA's embedding-gradient table, R x EMB floats
};

template <int NDIM>
constexpr size_t tc_train_smem_bytes(int R) {
  return sizeof(TcTrainSmem<NDIM>) + (size_t)R * EMB * sizeof(float);
}

__device__ __forceinline__ void st_bf16(unsigned char* base, int off, float v) {
  *reinterpret_cast<__nv_bfloat16*>(base + off) = __float2bfloat16_rn(v);
}

template <int NDIM>
__global__ void __launch_bounds__(TT_THREADS, 1)
    k_mlp_train_tc(MlpArgs a, const TcTrainWeights<NDIM>* __restrict__ wg, float* __restrict__ parts,
                   int stride, int* err, long long wait_limit) {
  using NN = Net<NDIM>;
  using SM = TcTrainSmem<NDIM>;
  constexpr int F = NN::F, KP = NN::KP, NB = NN::NB;
  constexpr int CENTRE = NB / 2;
  constexpr int NW1 = KP + H;                 // columns of D1: features, then h1
  constexpr int C_D1 = H, C_D2 = H + NW1, C_E = C_D2 + 16;  // tensor-memory columns
  static_assert(C_E + 16 <= TT_TMEM_COLS, "tensor-memory budget");
  static_assert(NW1 % 16 == 0 && NW1 <= 256, "N of the D1 product");
  static_assert(64 + F < 128, "the one-row of x lies inside D2's 128 rows");
  extern __shared__ __align__(16) unsigned char smraw[];
  SM& S = *reinterpret_cast<SM*>(smraw);
  float* sE = reinterpret_cast<float*>(smraw + sizeof(SM));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int half = warp >> 2;   // column half of every layer: 32 * half ..
  const int r = tid & 127;      // row of the tile = TMEM lane
  const int col0 = 32 * half;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(&S.tmem)),
                 "n"(TT_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  {
    constexpr int n16 = (int)(sizeof(TcTrainWeights<NDIM>) / 16);
    const uint4* src = reinterpret_cast<const uint4*>(wg);
    uint4* dst = reinterpret_cast<uint4*>(&S.w);
    for (int i = tid; i < n16; i += TT_THREADS) dst[i] = __ldg(src + i);
  }
  for (int i = tid; i < a.R * EMB; i += TT_THREADS) sE[i] = 0.f;
  // rows that never change: x^T's two bias ones and its zero padding, bw2's zero rows
  if (half == 0) {
#pragma unroll
    for (int k = F; k < KP; ++k) st_bf16(S.tt, kmajor_r(64 + k, r), k < F + 2 ? 1.f : 0.f);
  } else {
#pragma unroll
    for (int m = 1; m < 16; ++m) st_bf16(S.bw2, kmajor_r(m, r), 0.f);
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&S.bar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  fence_async_smem();
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  const uint32_t tmem = S.tmem;
  const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
  const float* E = a.prm + NN::oE;
  const int lgN = a.geo.lg[0] + a.geo.lg[1] + a.geo.lg[2];
  const int tiles = a.n / TC_ROWS;
  const float inv_n = 1.f / (float)a.n;
  const uint32_t act = smem_addr(S.act), w1 = smem_addr(S.w.base.w1), w2 = smem_addr(S.w.base.w2),
                 w2t = smem_addr(S.w.w2t), w1et = smem_addr(S.w.w1et), aw1 = smem_addr(S.aw1),
                 tt = smem_addr(S.tt), bw2 = smem_addr(S.bw2);
  constexpr uint32_t kOnes = 0x3F803F80u;  // two BF16 ones
  const float* w3 = S.w.base.w3;
  // sample indices are clamped to subbands 1..R-1 so that a bad index cannot read
  // outside the stacks (the API requires valid indices)
  const int64_t qlo = a.geo.N, qhi = (int64_t)a.R * a.geo.N - 1;
  float nb[NB];  // row r's neighbourhood (the first half's threads), loaded a tile ahead
#pragma unroll
  for (int d = 0; d < NB; ++d) nb[d] = 0.f;
  float cc_next = 0.f, is_next = 0.f, e_next[EMB];
#pragma unroll
  for (int e = 0; e < EMB; ++e) e_next[e] = 0.f;
  int64_t q_next = qlo;
  auto gather = [&](int t) {  // with the row's 1/s and (first half) its embedding
    if (t < tiles) {
      const int64_t q = min(max((int64_t)__ldg(a.idx + (int64_t)t * TC_ROWS + r), qlo), qhi);
      const int jn = (int)(q >> lgN);
      q_next = q;
      if (half == 0) {
        gather_nb<NDIM>(a.geo, a.C + ((q >> lgN) << lgN), (uint32_t)(q & (a.geo.N - 1)), nb);
#pragma unroll
        for (int e = 0; e < EMB; ++e) e_next[e] = ld_early(E + jn * EMB + e);
      } else {
        nb[CENTRE] = ld_early(a.C + q);
      }
      cc_next = ld_early(a.Cc + q);
      is_next = ld_early(a.inv_s + jn);
    }
  };
  gather(blockIdx.x);
  // The mbarrier completes four phases per tile: layer 1 (parity 0), layer 2 (1), dh1
  // (0), the gradient products (1, waited for at the next tile's start). A wait that
  // runs out is made CTA-uniform at the next barrier and ends the loop there.
  float loss_acc = 0.f;
  int jprev = 0;         // subband of row r in the previous tile (second half)
  int timed_out = 0;     // CTA-uniform
  uint32_t pending = 0;  // parity of the phase a timed-out wait left in flight
  bool late = false;     // this warp's last wait ran out (warp-uniform)
  bool first = true;     // no gradient product issued yet (CTA-uniform)
  // the previous tile's embedding gradients (DE) into the CTA's table
  auto take_de = [&]() {
    float v[16];
    tmem_ld16(tmem + lane_base + C_E, v);
#pragma unroll
    for (int e = 0; e < EMB; ++e) atomicAdd(sE + jprev * EMB + e, v[e]);
  };
  for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
    // the previous tile's gradient products read aw1, tt, bw2 and act
    if (!first) late = __any_sync(0xffffffffu, !mbar_wait(&S.bar, 1, wait_limit));
    tc_after_sync();
    const int64_t q = q_next;
    const int j = (int)(q >> lgN);
    const float c = nb[CENTRE], cc = cc_next;
    const float is = is_next;
    if (!late) {
      if (half == 0) {
        float x[KP];
        x[0] = c * is;
#pragma unroll
        for (int d = 0; d < NB; ++d) x[1 + d] = fabsf(nb[d]) * is;
#pragma unroll
        for (int e = 0; e < EMB; ++e) x[1 + NB + e] = e_next[e];
        x[F] = 1.f;
        x[F + 1] = 1.f;
#pragma unroll
        for (int k = F + 2; k < KP; ++k) x[k] = 0.f;
#pragma unroll
        for (int k8 = 0; k8 < KP / 8; ++k8)
          *reinterpret_cast<uint4*>(S.act + kmajor(r, 8 * k8, KP)) =
              make_uint4(pack_bf16(x[8 * k8], x[8 * k8 + 1]), pack_bf16(x[8 * k8 + 2], x[8 * k8 + 3]),
                         pack_bf16(x[8 * k8 + 4], x[8 * k8 + 5]),
                         pack_bf16(x[8 * k8 + 6], x[8 * k8 + 7]));
#pragma unroll
        for (int k = 0; k < F; ++k) st_bf16(S.tt, kmajor_r(64 + k, r), x[k]);
      } else if (!first) {
        take_de();
      }
    }
    fence_async_smem();
    tc_before_sync();
    if (__syncthreads_or(late)) {
      timed_out = 1;
      pending = 1;
      break;
    }
    tc_after_sync();
    // z1 = [x, 1, 1] [W1, b1]^T
    if (tid == 0) {
#pragma unroll
      for (int ks = 0; ks < KP / 16; ++ks)
        umma_bf16(tmem, umma_desc(act + ks * 256, 128, (KP / 8) * 128),
                  umma_desc(w1 + ks * 256, 128, (KP / 8) * 128), ks > 0);
      umma_commit(&S.bar);
    }
    late = __any_sync(0xffffffffu, !mbar_wait(&S.bar, 0, wait_limit));
    tc_after_sync();
    uint32_t mask = 0u;  // z1 > 0 on this half's columns
    if (!late) {
      float z[32];
      tmem_ld32(tmem + lane_base + col0, z);
#pragma unroll
      for (int i = 0; i < 32; ++i) mask |= (z[i] > 0.f ? 1u : 0u) << i;
#pragma unroll
      for (int k8 = 0; k8 < 4; ++k8)
        *reinterpret_cast<uint4*>(S.act + kmajor(r, col0 + 8 * k8, K2)) =
            make_uint4(relu_pack_bf16(z[8 * k8], z[8 * k8 + 1]),
                       relu_pack_bf16(z[8 * k8 + 2], z[8 * k8 + 3]),
                       relu_pack_bf16(z[8 * k8 + 4], z[8 * k8 + 5]),
                       relu_pack_bf16(z[8 * k8 + 6], z[8 * k8 + 7]));
#pragma unroll
      for (int i = 0; i < 32; ++i) st_bf16(S.tt, kmajor_r(64 + KP + col0 + i, r), fmaxf(z[i], 0.f));
      if (half == 0) {
        *reinterpret_cast<uint4*>(S.act + kmajor(r, H, K2)) = make_uint4(kOnes, 0u, 0u, 0u);
        *reinterpret_cast<uint4*>(S.act + kmajor(r, H + 8, K2)) = make_uint4(0u, 0u, 0u, 0u);
      }
    }
    fence_async_smem();
    tc_before_sync();
    if (__syncthreads_or(late)) {
      timed_out = 1;
      pending = 0;
      break;
    }
    tc_after_sync();
    gather(t + gridDim.x);  // the next tile's loads overlap the rest of this one
    // z2 = [h1, 1, 1] [W2, b2]^T
    if (tid == 0) {
#pragma unroll
      for (int ks = 0; ks < K2 / 16; ++ks)
        umma_bf16(tmem, umma_desc(act + ks * 256, 128, (K2 / 8) * 128),
                  umma_desc(w2 + ks * 256, 128, (K2 / 8) * 128), ks > 0);
      umma_commit(&S.bar);
    }
    late = __any_sync(0xffffffffu, !mbar_wait(&S.bar, 1, wait_limit));
    tc_after_sync();
    float z[32];
    if (!late) {
      tmem_ld32(tmem + lane_base + col0, z);
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int i = 0; i < 32; i += 4) {
        acc[0] += fmaxf(z[i], 0.f) * w3[col0 + i];
        acc[1] += fmaxf(z[i + 1], 0.f) * w3[col0 + i + 1];
        acc[2] += fmaxf(z[i + 2], 0.f) * w3[col0 + i + 2];
        acc[3] += fmaxf(z[i + 3], 0.f) * w3[col0 + i + 3];
      }
      S.z3half[half][r] = (acc[0] + acc[1]) + (acc[2] + acc[3]);
    }
    __syncthreads();  // both halves of the output dot
    if (!late) {
      const float g =
          1.f / (1.f + expf(-(S.w.base.b3[0] + (S.z3half[0][r] + S.z3half[1][r]))));
      const float res = (g * c - cc) * is;
      const float dz3 = 2.f * res * c * is * inv_n * g * (1.f - g);
      if (half == 0) {
        loss_acc += res * res;
        st_bf16(S.bw2, kmajor_r(0, r), dz3);
      }
      // dz2 on this half's columns: the A operand of dh1 (act is free: layer 2 is
      // done) and rows of aw1; h2 as rows of tt
      float dz2[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) dz2[i] = z[i] > 0.f ? dz3 * w3[col0 + i] : 0.f;
#pragma unroll
      for (int k8 = 0; k8 < 4; ++k8)
        *reinterpret_cast<uint4*>(S.act + kmajor(r, col0 + 8 * k8, H)) =
            make_uint4(pack_bf16(dz2[8 * k8], dz2[8 * k8 + 1]),
                       pack_bf16(dz2[8 * k8 + 2], dz2[8 * k8 + 3]),
                       pack_bf16(dz2[8 * k8 + 4], dz2[8 * k8 + 5]),
                       pack_bf16(dz2[8 * k8 + 6], dz2[8 * k8 + 7]));
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        st_bf16(S.aw1, kmajor_r(col0 + i, r), dz2[i]);
        st_bf16(S.tt, kmajor_r(col0 + i, r), fmaxf(z[i], 0.f));
      }
    }
    fence_async_smem();
    tc_before_sync();
    if (__syncthreads_or(late)) {
      timed_out = 1;
      pending = 1;
      break;
    }
    tc_after_sync();
    // dh1 = dz2 W2
    if (tid == 0) {
#pragma unroll
      for (int ks = 0; ks < H / 16; ++ks)
        umma_bf16(tmem, umma_desc(act + ks * 256, 128, (H / 8) * 128),
                  umma_desc(w2t + ks * 256, 128, (H / 8) * 128), ks > 0);
      umma_commit(&S.bar);
    }
    late = __any_sync(0xffffffffu, !mbar_wait(&S.bar, 0, wait_limit));
    tc_after_sync();
    if (!late) {
      // dz1 = dh1 [z1 > 0], rounded to BF16 as the products see it: rows of aw1 and
      // the A operand of DE (act is free: dh1 is done)
      tmem_ld32(tmem + lane_base + col0, z);
      uint32_t pk[16];
#pragma unroll
      for (int i = 0; i < 32; i += 2) {
        const float v0 = (mask >> i) & 1u ? z[i] : 0.f;
        const float v1 = (mask >> (i + 1)) & 1u ? z[i + 1] : 0.f;
        pk[i / 2] = pack_bf16(v0, v1);
        const __nv_bfloat162 p2 = *reinterpret_cast<const __nv_bfloat162*>(&pk[i / 2]);
        *reinterpret_cast<__nv_bfloat16*>(S.aw1 + kmajor_r(64 + col0 + i, r)) = p2.x;
        *reinterpret_cast<__nv_bfloat16*>(S.aw1 + kmajor_r(64 + col0 + i + 1, r)) = p2.y;
      }
#pragma unroll
      for (int k8 = 0; k8 < 4; ++k8)
        *reinterpret_cast<uint4*>(S.act + kmajor(r, col0 + 8 * k8, H)) =
            make_uint4(pk[4 * k8], pk[4 * k8 + 1], pk[4 * k8 + 2], pk[4 * k8 + 3]);
      if (half == 0) S.jrow[r] = j;
    }
    fence_async_smem();
    tc_before_sync();
    if (__syncthreads_or(late)) {
      timed_out = 1;
      pending = 0;
      break;
    }
    tc_after_sync();
    if (half == 1) jprev = S.jrow[r];
    // D1 += [dz2 ; dz1]^T [x ; h1],  D2 += [h2 ; x ; h1]^T [dz3, 0 ..],  DE = dz1 W1e^T
    if (tid == 0) {
#pragma unroll
      for (int ks = 0; ks < KR / 16; ++ks)
        umma_bf16(tmem + C_D1, umma_desc(aw1 + ks * 2 * KR_LBO, KR_LBO, KR_SBO),
                  umma_desc(tt + 8 * KR_SBO + ks * 2 * KR_LBO, KR_LBO, KR_SBO),
                  (!first || ks > 0) ? 1u : 0u, idesc_m128(NW1));
#pragma unroll
      for (int ks = 0; ks < KR / 16; ++ks)
        umma_bf16(tmem + C_D2, umma_desc(tt + ks * 2 * KR_LBO, KR_LBO, KR_SBO),
                  umma_desc(bw2 + ks * 2 * KR_LBO, KR_LBO, KR_SBO),
                  (!first || ks > 0) ? 1u : 0u, idesc_m128(16));
#pragma unroll
      for (int ks = 0; ks < H / 16; ++ks)
        umma_bf16(tmem + C_E, umma_desc(act + ks * 256, 128, (H / 8) * 128),
                  umma_desc(w1et + ks * 256, 128, (H / 8) * 128), ks > 0, idesc_m128(16));
      umma_commit(&S.bar);
    }
    first = false;
  }
  if (!timed_out && !first) {
    late = __any_sync(0xffffffffu, !mbar_wait(&S.bar, 1, wait_limit));
    tc_after_sync();
    if (!late && half == 1) take_de();
    if (__syncthreads_or(late)) {
      timed_out = 1;
      pending = 1;
    }
  }
  if (timed_out) {
    if (tid == 0) {
      atomicExch(err, 1);
      // let the products in flight finish (bounded by the default limit) before the
      // tensor memory is freed
      mbar_wait(&S.bar, pending);
    }
    // this CTA's share is dropped (a zero row): the call reports the timeout
    float* row = parts + (size_t)blockIdx.x * stride;
    for (int i = tid; i <= NN::oE + a.R * EMB; i += TT_THREADS) row[i] = 0.f;
    __syncthreads();
  } else {
    // this CTA's row of the partial-sum table: every gradient entry and the loss
    float* row = parts + (size_t)blockIdx.x * stride;
    const int m = r;  // TMEM lane = row of D1 and D2
    if (first) {      // no tile: zero gradients
      for (int i = tid; i < NN::oE; i += TT_THREADS) row[i] = 0.f;
    } else {
      for (int c0 = 16 * half; c0 < NW1; c0 += 32) {  // the halves take alternate chunks
        float v[16];
        tmem_ld16(tmem + lane_base + C_D1 + c0, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int n = c0 + i;
          if (m < H) {  // dz2 rows: b2 through the first one-column, W2 through h1
            if (n == F) row[NN::ob2 + m] = v[i];
            else if (n >= KP) row[NN::oW2 + m * H + (n - KP)] = v[i];
          } else {      // dz1 rows: W1 through the features, b1 through the one-column
            const int o = m - H;
            if (n < F) row[NN::oW1 + o * F + n] = v[i];
            else if (n == F) row[NN::ob1 + o] = v[i];
          }
        }
      }
      if (half == 0) {
        float v[16];
        tmem_ld16(tmem + lane_base + C_D2, v);
        if (m < H) row[NN::ow3 + m] = v[0];
        if (m == H + F) row[NN::ob3] = v[0];
      }
    }
    float l = loss_acc;
#pragma unroll
    for (int sft = 16; sft > 0; sft >>= 1) l += __shfl_xor_sync(0xffffffffu, l, sft);
    if (lane == 0) S.red[warp] = l;
    __syncthreads();  // also orders the embedding table's atomics before its copy
    const int P = NN::oE + a.R * EMB;
    if (tid == 0) {
      float s = 0.f;
#pragma unroll
      for (int w = 0; w < TT_THREADS / 32; ++w) s += S.red[w];
      row[P] = s * inv_n;
    }
    for (int i = tid; i < a.R * EMB; i += TT_THREADS) row[NN::oE + i] = sE[i];
  }
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "n"(TT_TMEM_COLS));
}

// Sum of the training CTAs' partial rows, in row order (the same sum on every run for
// the same rows): grad[i] for i < P and the loss from column P; with adam != 0 also
// the Adam update of parameter i (as k_adam). A CTA covers 32 columns, its 8 warps
// stride over the rows.
__global__ void __launch_bounds__(256) k_mlp_reduce(const float* __restrict__ parts, int nparts,
                                                    int stride, int P, float* __restrict__ grad,
                                                    float* __restrict__ loss, float* __restrict__ p,
                                                    float* __restrict__ m, float* __restrict__ v,
                                                    float lr, float c1, float c2, int adam) {
  __shared__ float sh[8][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int i = blockIdx.x * 32 + lane;
  float s = 0.f;
  if (i <= P)
    for (int r = w; r < nparts; r += 8) s += parts[(size_t)r * stride + i];
  sh[w][lane] = s;
  __syncthreads();
  if (w != 0 || i > P) return;
  float t = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) t += sh[k][lane];
  if (i == P) {
    *loss = t;
    return;
  }
  grad[i] = t;
  if (adam) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float mi = b1 * m[i] + (1.f - b1) * t;
    const float vi = b2 * v[i] + (1.f - b2) * t * t;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// Training: forward and backward on a sample; gradients accumulate into a.grad.
// Each CTA takes tiles of ROWS = 128 samples (16 per warp). The weight gradients
// dW2 = sum dz2^T h1 and dW1 = sum dz1^T x are products over the sample dimension:
// every warp stages its tile transposed in shared memory, and after a barrier the 8
// warps multiply the CTA's 128 rows on the tensor cores, each warp owning a slice of
// the output tiles and accumulating it over all tiles of the CTA in registers.
template <int NDIM>
struct TrainSmem {
  static constexpr int KP = Net<NDIM>::KP;
  static constexpr int PB = ROWS + 8;   // pitch (bf16) of the staged [.][ROWS] tiles
  SmemW<NDIM> w;
  __nv_bfloat16 dz2T[H * PB];           // dz2T[o][b]
  __nv_bfloat16 h1T[H * PB];            // h1T[i][b]
  __nv_bfloat16 dz1T[H * PB];           // dz1T[o][b]
  __nv_bfloat16 xT[KP * PB];            // xT[k][b]
};

template <int NDIM>
__global__ void __launch_bounds__(32 * WARPS) k_mlp_train(MlpArgs a) {
  using N = Net<NDIM>;
  using TS = TrainSmem<NDIM>;
  constexpr int KP = N::KP, KS = N::KS, PB = TS::PB;
  extern __shared__ __align__(16) unsigned char smraw[];
  TS& S = *reinterpret_cast<TS*>(smraw);
  load_weights<NDIM>(S.w, a.prm);
  __syncthreads();
  const int lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;
  const int warp = threadIdx.x >> 5;
  const float* E = a.prm + N::oE;
  // per-warp slices of the weight-gradient tiles: dW2 has 4 x 8 tiles of 16 x 8
  // (4 per warp), dW1 has 4 x (KP/8) tiles (KP/16 per warp... distributed round-robin)
  constexpr int T2 = 4 * 8 / WARPS;        // 4
  constexpr int NT1 = KP / 8;              // n-tiles of dW1
  constexpr int T1 = (4 * NT1 + WARPS - 1) / WARPS;
  float acc2[T2][4], acc1[T1][4];
#pragma unroll
  for (int i = 0; i < T2; ++i)
#pragma unroll
    for (int e = 0; e < 4; ++e) acc2[i][e] = 0.f;
#pragma unroll
  for (int i = 0; i < T1; ++i)
#pragma unroll
    for (int e = 0; e < 4; ++e) acc1[i][e] = 0.f;
  float gw3[8][2], gb2[8][2], gb1[8][2], gb3 = 0.f, lsum = 0.f;
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
#pragma unroll
    for (int e = 0; e < 2; ++e) gw3[nt][e] = gb2[nt][e] = gb1[nt][e] = 0.f;
  const float inv_n = 1.f / (float)a.n;
  const int ntiles = a.n / ROWS;

  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int r0 = tile * ROWS + warp * 16;
    // sample indices are clamped to subbands 1..R-1 so that a bad index cannot read
    // outside the stacks (the API requires valid indices)
    const int64_t qlo = a.geo.N, qhi = (int64_t)a.R * a.geo.N - 1;
    int64_t q[2] = {min(max((int64_t)a.idx[r0 + gid], qlo), qhi),
                    min(max((int64_t)a.idx[r0 + gid + 8], qlo), qhi)};
    int j[2] = {(int)(q[0] / a.geo.N), (int)(q[1] / a.geo.N)};
    float is[2] = {a.inv_s[j[0]], a.inv_s[j[1]]};
    Fwd<NDIM, true> f;
    mlp_forward<NDIM, true>(S.w, f, a.geo, a.C, q, j, is, E);
    // loss and dz3 (per row; the four threads of a row group hold the same values)
    float dz3[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const float c = a.C[q[r]], cc = a.Cc[q[r]];
      const float res = (f.g[r] * c - cc) * is[r];
      if (tig == 0) lsum += res * res;
      const float dg = 2.f * res * c * is[r] * inv_n;
      dz3[r] = dg * f.g[r] * (1.f - f.g[r]);
    }
    if (tig == 0) gb3 += dz3[0] + dz3[1];
    // dz2 = dz3 w3 [z2 > 0]; w3, b2 gradients; A fragments of dz2
    uint32_t D2[4][4];
    float dz2[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const int n0 = 8 * nt + 2 * tig;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int r = e >> 1, n = n0 + (e & 1);
        const float z = f.z2[nt][e];
        gw3[nt][e & 1] += fmaxf(z, 0.f) * dz3[r];
        dz2[nt][e] = z > 0.f ? dz3[r] * S.w.w3[n] : 0.f;
        gb2[nt][e & 1] += dz2[nt][e];
      }
    }
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {
      D2[ks][0] = pack_bf16(dz2[2 * ks][0], dz2[2 * ks][1]);
      D2[ks][1] = pack_bf16(dz2[2 * ks][2], dz2[2 * ks][3]);
      D2[ks][2] = pack_bf16(dz2[2 * ks + 1][0], dz2[2 * ks + 1][1]);
      D2[ks][3] = pack_bf16(dz2[2 * ks + 1][2], dz2[2 * ks + 1][3]);
    }
    // dh1 = dz2 W2 (B[k = o][n = i] = W2[o][i] = W2T[i][o]); dz1 = dh1 [z1 > 0]
    float dz1[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {
        const __nv_bfloat16* w = S.w.W2T + (8 * nt + gid) * SmemW<NDIM>::P2 + 16 * ks + 2 * tig;
        mma16816(d, D2[ks], *reinterpret_cast<const uint32_t*>(w),
                 *reinterpret_cast<const uint32_t*>(w + 8));
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        dz1[nt][e] = f.z1[nt][e] > 0.f ? d[e] : 0.f;
        gb1[nt][e & 1] += dz1[nt][e];
      }
    }
    // dx for the embedding features: dx = dz1 W1 (B[k = o][n = f] = W1T[f][o])
    {
      uint32_t D1[4][4];
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {
        D1[ks][0] = pack_bf16(dz1[2 * ks][0], dz1[2 * ks][1]);
        D1[ks][1] = pack_bf16(dz1[2 * ks][2], dz1[2 * ks][3]);
        D1[ks][2] = pack_bf16(dz1[2 * ks + 1][0], dz1[2 * ks + 1][1]);
        D1[ks][3] = pack_bf16(dz1[2 * ks + 1][2], dz1[2 * ks + 1][3]);
      }
      constexpr int e0 = N::NB + 1;       // first embedding feature
      constexpr int nt0 = e0 / 8, nt1 = (e0 + EMB - 1) / 8;
#pragma unroll
      for (int nt = nt0; nt <= nt1; ++nt) {
        float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
          const __nv_bfloat16* w = S.w.W1T + (8 * nt + gid) * (H + 8) + 16 * ks + 2 * tig;
          mma16816(d, D1[ks], *reinterpret_cast<const uint32_t*>(w),
                   *reinterpret_cast<const uint32_t*>(w + 8));
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int fcol = 8 * nt + 2 * tig + (e & 1);
          if (fcol >= e0 && fcol < e0 + EMB)
            atomicAdd(a.grad + N::oE + j[e >> 1] * EMB + (fcol - e0), d[e]);
        }
      }
    }
    // stage transposed bf16 tiles for the weight-gradient products
    const int b0 = warp * 16 + gid, b1 = b0 + 8;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const int o = 8 * nt + 2 * tig;
      S.dz2T[o * PB + b0] = __float2bfloat16_rn(dz2[nt][0]);
      S.dz2T[(o + 1) * PB + b0] = __float2bfloat16_rn(dz2[nt][1]);
      S.dz2T[o * PB + b1] = __float2bfloat16_rn(dz2[nt][2]);
      S.dz2T[(o + 1) * PB + b1] = __float2bfloat16_rn(dz2[nt][3]);
      S.dz1T[o * PB + b0] = __float2bfloat16_rn(dz1[nt][0]);
      S.dz1T[(o + 1) * PB + b0] = __float2bfloat16_rn(dz1[nt][1]);
      S.dz1T[o * PB + b1] = __float2bfloat16_rn(dz1[nt][2]);
      S.dz1T[(o + 1) * PB + b1] = __float2bfloat16_rn(dz1[nt][3]);
      S.h1T[o * PB + b0] = __float2bfloat16_rn(fmaxf(f.z1[nt][0], 0.f));
      S.h1T[(o + 1) * PB + b0] = __float2bfloat16_rn(fmaxf(f.z1[nt][1], 0.f));
      S.h1T[o * PB + b1] = __float2bfloat16_rn(fmaxf(f.z1[nt][2], 0.f));
      S.h1T[(o + 1) * PB + b1] = __float2bfloat16_rn(fmaxf(f.z1[nt][3], 0.f));
    }
    // features (already bf16 in the A fragments): A1[ks][0] = (row gid, k 16ks+2tig..+1) ...
#pragma unroll
    for (int ks = 0; ks < KS; ++ks) {
      const uint32_t* fr = f.A1[ks];
      const __nv_bfloat16* h0 = reinterpret_cast<const __nv_bfloat16*>(&fr[0]);
      const __nv_bfloat16* h1 = reinterpret_cast<const __nv_bfloat16*>(&fr[1]);
      const __nv_bfloat16* h2 = reinterpret_cast<const __nv_bfloat16*>(&fr[2]);
      const __nv_bfloat16* h3 = reinterpret_cast<const __nv_bfloat16*>(&fr[3]);
      const int k0 = 16 * ks + 2 * tig;
      S.xT[k0 * PB + b0] = h0[0];
      S.xT[(k0 + 1) * PB + b0] = h0[1];
      S.xT[k0 * PB + b1] = h1[0];
      S.xT[(k0 + 1) * PB + b1] = h1[1];
      S.xT[(k0 + 8) * PB + b0] = h2[0];
      S.xT[(k0 + 9) * PB + b0] = h2[1];
      S.xT[(k0 + 8) * PB + b1] = h3[0];
      S.xT[(k0 + 9) * PB + b1] = h3[1];
    }
    __syncthreads();
    // dW2[o][i] += sum_b dz2T[o][b] h1T[i][b]: A = dz2T (row o, col b), B[k=b][n=i] = h1T[i][b]
#pragma unroll
    for (int t = 0; t < T2; ++t) {
      const int id = warp * T2 + t;  // 0..31
      const int mt = id / 8, nt = id % 8;
#pragma unroll
      for (int ks = 0; ks < ROWS / 16; ++ks) {
        const __nv_bfloat16* ar = S.dz2T + (16 * mt + gid) * PB + 16 * ks + 2 * tig;
        uint32_t af[4] = {*reinterpret_cast<const uint32_t*>(ar),
                          *reinterpret_cast<const uint32_t*>(ar + 8 * PB),
                          *reinterpret_cast<const uint32_t*>(ar + 8),
                          *reinterpret_cast<const uint32_t*>(ar + 8 * PB + 8)};
        const __nv_bfloat16* br = S.h1T + (8 * nt + gid) * PB + 16 * ks + 2 * tig;
        mma16816(acc2[t], af, *reinterpret_cast<const uint32_t*>(br),
                 *reinterpret_cast<const uint32_t*>(br + 8));
      }
    }
    // dW1[o][k] += sum_b dz1T[o][b] xT[k][b]
#pragma unroll
    for (int t = 0; t < T1; ++t) {
      const int id = warp + WARPS * t;  // 0 .. 4*NT1-1
      if (id < 4 * NT1) {
        const int mt = id / NT1, nt = id % NT1;
#pragma unroll
        for (int ks = 0; ks < ROWS / 16; ++ks) {
          const __nv_bfloat16* ar = S.dz1T + (16 * mt + gid) * PB + 16 * ks + 2 * tig;
          uint32_t af[4] = {*reinterpret_cast<const uint32_t*>(ar),
                            *reinterpret_cast<const uint32_t*>(ar + 8 * PB),
                            *reinterpret_cast<const uint32_t*>(ar + 8),
                            *reinterpret_cast<const uint32_t*>(ar + 8 * PB + 8)};
          const __nv_bfloat16* br = S.xT + (8 * nt + gid) * PB + 16 * ks + 2 * tig;
          mma16816(acc1[t], af, *reinterpret_cast<const uint32_t*>(br),
                   *reinterpret_cast<const uint32_t*>(br + 8));
        }
      }
    }
    __syncthreads();  // staging reused by the next tile
  }
  // flush this CTA's gradients
  float* gr = a.grad;
#pragma unroll
  for (int t = 0; t < T2; ++t) {
    const int id = warp * T2 + t, mt = id / 8, nt = id % 8;
    const int o = 16 * mt + gid, i = 8 * nt + 2 * tig;
    atomicAdd(gr + N::oW2 + o * H + i, acc2[t][0]);
    atomicAdd(gr + N::oW2 + o * H + i + 1, acc2[t][1]);
    atomicAdd(gr + N::oW2 + (o + 8) * H + i, acc2[t][2]);
    atomicAdd(gr + N::oW2 + (o + 8) * H + i + 1, acc2[t][3]);
  }
#pragma unroll
  for (int t = 0; t < T1; ++t) {
    const int id = warp + WARPS * t;
    if (id < 4 * NT1) {
      const int mt = id / NT1, nt = id % NT1;
      const int o = 16 * mt + gid, k = 8 * nt + 2 * tig;
      if (k < N::F) {
        atomicAdd(gr + N::oW1 + o * N::F + k, acc1[t][0]);
        atomicAdd(gr + N::oW1 + (o + 8) * N::F + k, acc1[t][2]);
      }
      if (k + 1 < N::F) {
        atomicAdd(gr + N::oW1 + o * N::F + k + 1, acc1[t][1]);
        atomicAdd(gr + N::oW1 + (o + 8) * N::F + k + 1, acc1[t][3]);
      }
    }
  }
  // bias and w3 gradients: reduce over the 8 row groups of the warp, then atomics
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      float v1 = gw3[nt][e], v2 = gb2[nt][e], v3 = gb1[nt][e];
#pragma unroll
      for (int sft = 4; sft < 32; sft <<= 1) {
        v1 += __shfl_xor_sync(0xffffffffu, v1, sft);
        v2 += __shfl_xor_sync(0xffffffffu, v2, sft);
        v3 += __shfl_xor_sync(0xffffffffu, v3, sft);
      }
      if (gid == 0) {
        const int n = 8 * nt + 2 * tig + e;
        atomicAdd(gr + N::ow3 + n, v1);
        atomicAdd(gr + N::ob2 + n, v2);
        atomicAdd(gr + N::ob1 + n, v3);
      }
    }
#pragma unroll
  for (int sft = 4; sft < 32; sft <<= 1) {
    gb3 += __shfl_xor_sync(0xffffffffu, gb3, sft);
    lsum += __shfl_xor_sync(0xffffffffu, lsum, sft);
  }
  if (lane == 0) {
    atomicAdd(gr + N::ob3, gb3);
    atomicAdd(a.loss, lsum * inv_n);
  }
}

// Adam (Kingma & Ba) on the flat parameters; t counts from 1.
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int n, float lr, float c1, float c2) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

thread_local std::string g_mlp_err;

sl_status mfail(sl_status s, const std::string& msg) {
  g_mlp_err = msg;
  return s;
}

}  // namespace

struct sl_mlp {
  const sl_bank* bank = nullptr;
  int ndim = 2, R = 0;
  Geom geo{};
  int P = 0;  // parameters
  float* prm = nullptr;
  float* grad = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  float* loss = nullptr;
  float* inv_s = nullptr;  // [R]
  int* tc_err = nullptr;   // set by a tensor-core wait that ran out
  void* tc_pack = nullptr; // BF16 weight tiles of the tcgen05 inference kernel
  bool tc_packed = false;  // tc_pack holds the current parameters (packed on pack_stream)
  cudaStream_t pack_stream = nullptr;
  int engine = SL_MLP_TCGEN05;
  float* parts = nullptr;  // tensor-core training: one partial-sum row per CTA
  int pstride = 0;         // floats per partial row (P gradients, the loss, padding)
  int nparts_max = 0;      // rows (one training CTA per SM)
  float* coeffs = nullptr; // [2][R][N] for sl_mlp_denoise (allocated on first use)
  std::vector<double> norms;
  int t = 0;
  float sigma_set = -1.f;
};

static int lg2(int64_t v) {
  int l = 0;
  while ((int64_t(1) << l) < v) ++l;
  return l;
}

static int n_params(int ndim, int R) {
  const int F = 1 + (ndim == 2 ? 9 : 27) + EMB;
  return H * F + H + H * H + H + H + 1 + R * EMB;
}

template <int NDIM>
static size_t train_smem() { return sizeof(TrainSmem<NDIM>); }
template <int NDIM>
static size_t apply_smem() { return sizeof(SmemW<NDIM>); }

static sl_status set_sigma(sl_mlp* M, float sigma, cudaStream_t st) {
  if (!(sigma > 0.f) || !std::isfinite(sigma)) return mfail(SL_EINVAL, "sigma must be > 0");
  if (M->sigma_set == sigma) return SL_OK;
  std::vector<float> is(M->R);
  for (int j = 0; j < M->R; ++j) is[j] = (float)(1.0 / ((double)sigma * M->norms[j]));
  // pageable source: the copy is staged before the call returns
  if (cudaMemcpyAsync(M->inv_s, is.data(), M->R * sizeof(float), cudaMemcpyHostToDevice, st) !=
      cudaSuccess)
    return mfail(SL_ECUDA, "uploading 1/s");
  M->sigma_set = sigma;
  return SL_OK;
}

// Per-wait limit in SM cycles of the tensor-core kernels: the default (about two
// seconds), or the value of SL_MLP_WAIT_CYCLES, a test hook that makes the waits run
// out on purpose so that the timeout path (flag, drain, free, sl_mlp_check) can be
// exercised.
static long long tc_wait_limit() {
  long long limit = kTcWaitCycles;
  if (const char* e = std::getenv("SL_MLP_WAIT_CYCLES")) limit = std::max(0LL, std::atoll(e));
  return limit;
}

template <int NDIM>
static sl_status train_tc(sl_mlp* M, const MlpArgs& a, int tiles, cudaStream_t st, int* grid) {
  const size_t sm = tc_train_smem_bytes<NDIM>(M->R);
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (sm > (size_t)optin)
    return mfail(SL_ENOTSUP, "too many subbands for the tensor-core trainer's shared memory "
                             "(select SL_MLP_MMA_SYNC)");
  cudaFuncSetAttribute(k_mlp_train_tc<NDIM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  auto* wt = reinterpret_cast<TcTrainWeights<NDIM>*>(M->tc_pack);
  k_mlp_pack_train<NDIM><<<(tc_train_pack_elems<NDIM>() + 255) / 256, 256, 0, st>>>(M->prm, wt);
  M->tc_packed = false;  // the packed inference tiles are overwritten
  *grid = std::min(tiles, M->nparts_max);
  k_mlp_train_tc<NDIM><<<*grid, TT_THREADS, sm, st>>>(a, wt, M->parts, M->pstride, M->tc_err,
                                                      tc_wait_limit());
  return SL_OK;
}

// Gradients (and the loss) of one sample into M->grad / M->loss; with adam, also one
// Adam step of the parameters (M->t counts the steps).
static sl_status train_launch(sl_mlp* M, const float* noisy, const float* clean, float sigma,
                              const int* idx, int n, cudaStream_t st, bool adam, float lr) {
  if (!M || !noisy || !clean || !idx) return mfail(SL_EINVAL, "NULL argument");
  if (n <= 0 || n % ROWS) return mfail(SL_EINVAL, "n must be a positive multiple of 128");
  sl_status s = set_sigma(M, sigma, st);
  if (s != SL_OK) return s;
  MlpArgs a{};
  a.prm = M->prm;
  a.C = noisy;
  a.Cc = clean;
  a.idx = idx;
  a.n = n;
  a.inv_s = M->inv_s;
  a.grad = M->grad;
  a.loss = M->loss;
  a.geo = M->geo;
  a.R = M->R;
  const int tiles = n / ROWS;
  float c1 = 1.f, c2 = 1.f;
  if (adam) {
    M->t += 1;
    c1 = 1.f - std::pow(0.9f, (float)M->t);
    c2 = 1.f - std::pow(0.999f, (float)M->t);
  }
  if (M->engine == SL_MLP_TCGEN05) {
    int grid = 0;
    s = M->ndim == 2 ? train_tc<2>(M, a, tiles, st, &grid) : train_tc<3>(M, a, tiles, st, &grid);
    if (s != SL_OK) return s;
    k_mlp_reduce<<<(M->P + 1 + 31) / 32, 256, 0, st>>>(M->parts, grid, M->pstride, M->P, M->grad,
                                                      M->loss, M->prm, M->m, M->v, lr, c1, c2,
                                                      adam ? 1 : 0);
  } else {
    if (cudaMemsetAsync(M->grad, 0, M->P * sizeof(float), st) != cudaSuccess ||
        cudaMemsetAsync(M->loss, 0, sizeof(float), st) != cudaSuccess)
      return mfail(SL_ECUDA, "memset");
    const int grid = std::min(tiles, 4 * sm_count());
    if (M->ndim == 2) {
      const size_t sm = train_smem<2>();
      cudaFuncSetAttribute(k_mlp_train<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      k_mlp_train<2><<<grid, 32 * WARPS, sm, st>>>(a);
    } else {
      const size_t sm = train_smem<3>();
      cudaFuncSetAttribute(k_mlp_train<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      k_mlp_train<3><<<grid, 32 * WARPS, sm, st>>>(a);
    }
    if (adam) {
      M->tc_packed = false;
      k_adam<<<(M->P + 255) / 256, 256, 0, st>>>(M->prm, M->grad, M->m, M->v, M->P, lr, c1, c2);
    }
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return mfail(SL_ECUDA, std::string("training step: ") + cudaGetErrorString(e));
  return SL_OK;
}

extern "C" {

const char* sl_mlp_last_error(void) { return g_mlp_err.c_str(); }

sl_status sl_mlp_create(const sl_bank* bank, sl_mlp** out) {
  if (!bank || !out) return mfail(SL_EINVAL, "bank or out is NULL");
  *out = nullptr;
  int ndim = 0, R = 0, J = 0;
  int64_t dims[3];
  if (sl_bank_info(bank, &ndim, dims, &R, &J) != SL_OK) return mfail(SL_EINVAL, "bad bank");
  for (int i = 0; i < ndim; ++i)  // neighbourhoods are addressed with shifts and masks
    if (dims[i] & (dims[i] - 1))
      return mfail(SL_ENOTSUP, "the learned shrinkage needs power-of-two grid sides");
  sl_mlp* M = new sl_mlp();
  M->bank = bank;
  M->ndim = ndim;
  M->R = R;
  M->norms.resize(R);
  sl_bank_norms(bank, M->norms.data(), nullptr, nullptr);
  int64_t N = 1;
  for (int i = 0; i < 3; ++i) {
    M->geo.dims[i] = i < ndim ? (int)dims[i] : 1;
    M->geo.lg[i] = lg2(M->geo.dims[i]);
    N *= M->geo.dims[i];
  }
  M->geo.N = N;
  M->P = n_params(ndim, R);
  bool ok = cudaMalloc(&M->prm, M->P * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&M->grad, M->P * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&M->m, M->P * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&M->v, M->P * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&M->loss, sizeof(float)) == cudaSuccess &&
            cudaMalloc(&M->inv_s, R * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&M->tc_err, sizeof(int)) == cudaSuccess &&
            cudaMalloc(&M->tc_pack, std::max(sizeof(TcTrainWeights<2>),
                                             sizeof(TcTrainWeights<3>))) == cudaSuccess;
  M->pstride = (M->P + 1 + 3) / 4 * 4;
  M->nparts_max = sm_count();
  if (ok)
    ok = cudaMalloc(&M->parts, (size_t)M->nparts_max * M->pstride * sizeof(float)) == cudaSuccess;
  if (ok) ok = cudaMemset(M->prm, 0, M->P * sizeof(float)) == cudaSuccess &&
               cudaMemset(M->tc_err, 0, sizeof(int)) == cudaSuccess &&
               cudaMemset(M->m, 0, M->P * sizeof(float)) == cudaSuccess &&
               cudaMemset(M->v, 0, M->P * sizeof(float)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    sl_mlp_free(M);
    return mfail(SL_ENOMEM, "allocating the MLP");
  }
  *out = M;
  return SL_OK;
}

void sl_mlp_free(sl_mlp* M) {
  if (!M) return;
  cudaFree(M->prm);
  cudaFree(M->grad);
  cudaFree(M->m);
  cudaFree(M->v);
  cudaFree(M->loss);
  cudaFree(M->inv_s);
  cudaFree(M->tc_err);
  cudaFree(M->tc_pack);
  cudaFree(M->parts);
  cudaFree(M->coeffs);
  delete M;
}

int sl_mlp_num_params(const sl_mlp* M) { return M ? M->P : 0; }

sl_status sl_mlp_set_params(sl_mlp* M, const float* host) {
  if (!M || !host) return mfail(SL_EINVAL, "NULL argument");
  M->tc_packed = false;
  if (cudaMemcpy(M->prm, host, M->P * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
    return mfail(SL_ECUDA, "cudaMemcpy");
  cudaMemset(M->m, 0, M->P * sizeof(float));
  cudaMemset(M->v, 0, M->P * sizeof(float));
  M->t = 0;
  return SL_OK;
}

sl_status sl_mlp_get_params(const sl_mlp* M, float* host) {
  if (!M || !host) return mfail(SL_EINVAL, "NULL argument");
  if (cudaMemcpy(host, M->prm, M->P * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
    return mfail(SL_ECUDA, "cudaMemcpy");
  return SL_OK;
}

// Checkpoint file: an 8-byte magic, four int32 (ndim, R, P, Adam step t), then the
// parameters, Adam's first and second moments (P float32 each), little endian.
static const char kCkptMagic[8] = {'S', 'L', 'M', 'L', 'P', '0', '0', '1'};

sl_status sl_mlp_save(const sl_mlp* M, const char* path) {
  if (!M || !path) return mfail(SL_EINVAL, "NULL argument");
  std::vector<float> buf((size_t)3 * M->P);
  if (cudaMemcpy(buf.data(), M->prm, M->P * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(buf.data() + M->P, M->m, M->P * sizeof(float), cudaMemcpyDeviceToHost) !=
          cudaSuccess ||
      cudaMemcpy(buf.data() + 2 * (size_t)M->P, M->v, M->P * sizeof(float),
                 cudaMemcpyDeviceToHost) != cudaSuccess)
    return mfail(SL_ECUDA, "cudaMemcpy");
  FILE* f = std::fopen(path, "wb");
  if (!f) return mfail(SL_EINVAL, std::string("cannot open ") + path + " for writing");
  const int32_t hdr[4] = {M->ndim, M->R, M->P, M->t};
  const bool ok = std::fwrite(kCkptMagic, 1, 8, f) == 8 && std::fwrite(hdr, 4, 4, f) == 4 &&
                  std::fwrite(buf.data(), sizeof(float), buf.size(), f) == buf.size();
  if (std::fclose(f) != 0 || !ok) return mfail(SL_EINVAL, std::string("writing ") + path + " failed");
  return SL_OK;
}

sl_status sl_mlp_load(sl_mlp* M, const char* path) {
  if (!M || !path) return mfail(SL_EINVAL, "NULL argument");
  FILE* f = std::fopen(path, "rb");
  if (!f) return mfail(SL_EINVAL, std::string("cannot open ") + path);
  char magic[8];
  int32_t hdr[4];
  std::vector<float> buf((size_t)3 * M->P);
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kCkptMagic, 8) == 0 &&
            std::fread(hdr, 4, 4, f) == 4;
  if (ok && (hdr[0] != M->ndim || hdr[1] != M->R || hdr[2] != M->P || hdr[3] < 0)) {
    std::fclose(f);
    return mfail(SL_EINVAL, "checkpoint was written for another bank shape");
  }
  ok = ok && std::fread(buf.data(), sizeof(float), buf.size(), f) == buf.size();
  std::fclose(f);
  if (!ok) return mfail(SL_EINVAL, std::string(path) + " is not a complete MLP checkpoint");
  M->tc_packed = false;
  if (cudaMemcpy(M->prm, buf.data(), M->P * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(M->m, buf.data() + M->P, M->P * sizeof(float), cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemcpy(M->v, buf.data() + 2 * (size_t)M->P, M->P * sizeof(float),
                 cudaMemcpyHostToDevice) != cudaSuccess)
    return mfail(SL_ECUDA, "cudaMemcpy");
  M->t = hdr[3];
  return SL_OK;
}

sl_status sl_mlp_gradients(sl_mlp* M, const float* noisy, const float* clean, float sigma,
                           const int* idx, int n, float* grad_host, float* loss_host,
                           void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  sl_status s = train_launch(M, noisy, clean, sigma, idx, n, st, false, 0.f);
  if (s != SL_OK) return s;
  if (grad_host && cudaMemcpyAsync(grad_host, M->grad, M->P * sizeof(float),
                                   cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return mfail(SL_ECUDA, "copy gradients");
  if (loss_host &&
      cudaMemcpyAsync(loss_host, M->loss, sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return mfail(SL_ECUDA, "copy loss");
  if (cudaStreamSynchronize(st) != cudaSuccess) return mfail(SL_ECUDA, "synchronize");
  return SL_OK;
}

sl_status sl_mlp_train_step(sl_mlp* M, const float* noisy, const float* clean, float sigma,
                            const int* idx, int n, float lr, float* loss_dev, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  sl_status s = train_launch(M, noisy, clean, sigma, idx, n, st, true, lr);
  if (s != SL_OK) return s;
  if (loss_dev &&
      cudaMemcpyAsync(loss_dev, M->loss, sizeof(float), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return mfail(SL_ECUDA, "copy loss");
  return SL_OK;
}

sl_status sl_mlp_apply(sl_mlp* M, const float* coeffs, float* out, float sigma, void* stream) {
  if (!M || !coeffs || !out) return mfail(SL_EINVAL, "NULL argument");
  if (out == coeffs) return mfail(SL_EINVAL, "out must not alias coeffs (features read neighbours)");
  cudaStream_t st = (cudaStream_t)stream;
  sl_status s = set_sigma(M, sigma, st);
  if (s != SL_OK) return s;
  MlpArgs a{};
  a.prm = M->prm;
  a.C = coeffs;
  a.out = out;
  a.inv_s = M->inv_s;
  a.geo = M->geo;
  a.R = M->R;
  // The BF16 weight tiles are repacked when the parameters changed, on another
  // stream, and always inside a stream capture (a replayed graph must not depend on
  // what was packed when it was captured).
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return mfail(SL_ECUDA, "cudaStreamIsCapturing");
  const bool repack = !M->tc_packed || M->pack_stream != st || cap != cudaStreamCaptureStatusNone;
  if (M->engine == SL_MLP_TCGEN05) {
    const long long limit = tc_wait_limit();
    // the grid keeps every SM's CTAs within its 512 TMEM columns: no allocation waits
    if (M->ndim == 2) {
      const size_t sm = sizeof(TcApplySmem<2>);
      cudaFuncSetAttribute(k_mlp_apply_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      cudaFuncSetAttribute(k_mlp_apply_tc<2>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
      auto* wt = reinterpret_cast<TcWeights<2>*>(M->tc_pack);
      if (repack)
        k_mlp_pack_tc<2><<<(tc_pack_elems<2>() + 255) / 256, 256, 0, st>>>(M->prm, wt);
      k_mlp_apply_tc<2><<<apply_tc_grid<2>(), TC_THREADS, sm, st>>>(a, wt, M->tc_err, limit);
    } else {
      const size_t sm = sizeof(TcApplySmem<3>);
      cudaFuncSetAttribute(k_mlp_apply_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      cudaFuncSetAttribute(k_mlp_apply_tc<3>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
      auto* wt = reinterpret_cast<TcWeights<3>*>(M->tc_pack);
      if (repack)
        k_mlp_pack_tc<3><<<(tc_pack_elems<3>() + 255) / 256, 256, 0, st>>>(M->prm, wt);
      k_mlp_apply_tc<3><<<apply_tc_grid<3>(), TC_THREADS, sm, st>>>(a, wt, M->tc_err, limit);
    }
  } else {
    const int grid = 4 * sm_count();
    if (M->ndim == 2) {
      const size_t sm = apply_smem<2>();
      cudaFuncSetAttribute(k_mlp_apply<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      k_mlp_apply<2><<<grid, 32 * WARPS, sm, st>>>(a);
    } else {
      const size_t sm = apply_smem<3>();
      cudaFuncSetAttribute(k_mlp_apply<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      k_mlp_apply<3><<<grid, 32 * WARPS, sm, st>>>(a);
    }
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return mfail(SL_ECUDA, std::string("k_mlp_apply: ") + cudaGetErrorString(e));
  if (M->engine == SL_MLP_TCGEN05 && repack) {
    M->tc_packed = cap == cudaStreamCaptureStatusNone;  // a capture packs nothing yet
    M->pack_stream = st;
  }
  return SL_OK;
}

sl_status sl_mlp_set_engine(sl_mlp* M, int engine) {
  if (!M) return mfail(SL_EINVAL, "NULL argument");
  if (engine != SL_MLP_TCGEN05 && engine != SL_MLP_MMA_SYNC) return mfail(SL_EINVAL, "unknown engine");
  M->engine = engine;
  return SL_OK;
}

sl_status sl_mlp_check(sl_mlp* M, void* stream) {
  if (!M) return mfail(SL_EINVAL, "NULL argument");
  int h = 0;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess ||
      cudaMemcpy(&h, M->tc_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return mfail(SL_ECUDA, std::string("sl_mlp_check: ") + cudaGetErrorString(cudaGetLastError()));
  if (h) {
    cudaMemset(M->tc_err, 0, sizeof(int));
    return mfail(SL_ECUDA, "a tensor-core wait ran out (the output of sl_mlp_apply, or the "
                           "gradients of a training call, are incomplete)");
  }
  return SL_OK;
}

sl_status sl_mlp_denoise(sl_mlp* M, const float* noisy, float* out, float sigma, void* stream) {
  if (!M || !noisy || !out) return mfail(SL_EINVAL, "NULL argument");
  if (!M->coeffs &&
      cudaMalloc(&M->coeffs, 2 * (size_t)M->R * M->geo.N * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    return mfail(SL_ENOMEM, "coefficient buffer");
  }
  sl_status s = sl_forward(M->bank, noisy, M->coeffs, stream);
  if (s != SL_OK) return mfail(s, std::string("sl_forward: ") + sl_last_error());
  float* shrunk = M->coeffs + (size_t)M->R * M->geo.N;
  s = sl_mlp_apply(M, M->coeffs, shrunk, sigma, stream);
  if (s != SL_OK) return s;
  s = sl_inverse(M->bank, shrunk, out, stream);
  if (s != SL_OK) return mfail(s, std::string("sl_inverse: ") + sl_last_error());
  return SL_OK;
}

}  // extern "C"
