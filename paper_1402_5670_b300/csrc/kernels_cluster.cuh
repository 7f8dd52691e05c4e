// Fused 2D transforms on thread-block clusters. Internal header.
//
// For an n0 x n1 grid whose half spectrum (n0 x (n1/2 + 1) complex) fits in the
// shared memory of one cluster of 8 CTAs, one cluster computes a whole 2D FFT per
// filter without any round trip through global memory: the 8 CTAs split the spectrum
// into column blocks for the transform along axis 0 and into row blocks for the
// transform along axis 1, and the transposition between the two runs through
// distributed shared memory (a CTA reads the other CTAs' blocks directly).
//
//   k_cl_fwd  (forward filter pass, and the last step of the inverse)
//     columns:  IFFT_0( Xhat * psi_j )   (Xhat, psi_j read from global)
//     rows:     C2R along axis 1, scale, optional threshold -> C_j (global, row-major)
//   k_cl_inv  (inverse filter pass, and the spectrum of the signal)
//     rows:     R2C along axis 1 of C_j (global)
//     columns:  FFT_0, then  P_c += psi_j * (.)  into this cluster's partial sum P_c
//               (global, L2-resident, written only by this cluster's CTAs; the whole
//               accumulator would not fit in the registers of 8 SMs next to the
//               FFT working set).
//
// Layout of the spectra this path reads and writes ("cluster-tiled"): the NH = n1/2+1
// columns are cut into 8 blocks of CW = ceil(NH / 8) columns (the last block padded);
// block r is one contiguous [n0][CW] array:  (k0, col) -> (col / CW) * n0 * CW
// + k0 * CW + col % CW. Pad columns are transformed but never read back.
//
// Every CTA of a cluster runs the same filter loop, so all cluster barriers are
// reached by all 8 CTAs the same number of times; after the last barrier of an
// iteration no CTA reads another CTA's shared memory, so CTAs may exit.
#pragma once

#include <cooperative_groups.h>

#include "kernels2d.cuh"

namespace sl {
namespace dev {

namespace cg = cooperative_groups;

constexpr int kCluster = 8;

template <int L0, int L1>
struct ClGeo {
  static constexpr int NH = L1 / 2 + 1;
  static constexpr int CW = (NH + kCluster - 1) / kCluster;  // columns per CTA
  static constexpr int RW = L0 / kCluster;                   // rows per CTA
  static constexpr int PAIRS = RW / 2;                       // row pairs per CTA
  static constexpr int A0 = Split<L0>::A, B0 = Split<L0>::B;
  static constexpr int A1 = Split<L1>::A, B1 = Split<L1>::B;
  static constexpr int NT = CW * B0;                         // one column pass-2 item each
  static constexpr int XCOL = L0 * CW;                       // column exchange / results
  static constexpr int XROW = PAIRS * B1 * (A1 + 1);         // row exchange (padded)
  static constexpr int NROW = PAIRS * L1;                    // row pairs, natural
  static constexpr int S0 = XCOL > XROW ? XCOL : XROW;
  static constexpr int S = S0 > NROW ? S0 : NROW;
  static constexpr int smem = S * (int)sizeof(float2);
  static constexpr int IT_R1 = (PAIRS * A1 + NT - 1) / NT;   // row pass-1 items per thread
  static constexpr int IT_R2 = (PAIRS * B1 + NT - 1) / NT;   // row pass-2 items per thread
  static constexpr int IT_C1 = (CW * A0 + NT - 1) / NT;      // column pass-1 items per thread
  static constexpr int BLOCK = L0 * CW;                      // one column block, elements
  static constexpr int TOTAL = kCluster * BLOCK;             // one cluster-tiled spectrum
  static_assert(L0 % (2 * kCluster) == 0, "row blocks of whole pairs");
  static_assert(NT <= 1024, "block size");
};

// 32-bit shared-window addresses for distributed shared memory: the address of a
// local shared variable, the same offset in the CTA of another rank, and a load.
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint32_t dsmem_map(uint32_t local, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
  return r;
}
__device__ __forceinline__ float2 dsmem_ld(uint32_t addr) {
  float2 v;
  asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr)
               : "memory");
  return v;
}

struct ClArgs {
  const float2* xhat;   // k_cl_fwd: spectrum to filter (cluster-tiled)
  const float* psi;     // cluster-tiled filters [R][TOTAL] (may be null: no filter)
  float* out_real;      // k_cl_fwd: C [R][n0][n1] (or x when R = 1)
  const float* in_real; // k_cl_inv: C [R][n0][n1] (or x)
  float2* out_spec;     // k_cl_inv: partials [ncl][TOTAL] (or the spectrum)
  int R;                // filters in the loop
  float scale;          // k_cl_fwd: factor on the real output
  const float* thr;     // k_cl_fwd: per-filter thresholds (device, may be null)
};

// Forward direction: for j = cluster id, cluster id + #clusters, ...
template <int L0, int L1>
__global__ void __cluster_dims__(kCluster, 1, 1) __launch_bounds__(ClGeo<L0, L1>::NT)
    k_cl_fwd(ClArgs p) {
  using G = ClGeo<L0, L1>;
  constexpr int CW = G::CW, RW = G::RW, PAIRS = G::PAIRS;
  constexpr int A0 = G::A0, B0 = G::B0, A1 = G::A1, B1 = G::B1, NT = G::NT;
  constexpr int H = L1 / 2;
  constexpr int LS = B1 * (A1 + 1);
  extern __shared__ float2 S[];
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int cid = blockIdx.x / kCluster;
  const int ncl = gridDim.x / kCluster;
  const int tid = threadIdx.x;
  const float2* tw0 = g_twiddle + twiddle_offset(L0);
  const float2* tw1 = g_twiddle + twiddle_offset(L1);
  const int64_t blk = (int64_t)rank * G::BLOCK;  // this CTA's column block

  for (int j = cid; j < p.R; j += ncl) {
    // ---- columns: IFFT_0 of (Xhat * psi_j) on this CTA's CW columns ----
    const float* psij = p.psi ? p.psi + (int64_t)j * G::TOTAL + blk : nullptr;
    for (int it = tid; it < CW * A0; it += NT) {
      const int c = it % CW, a = it / CW;
      float2 v[B0];
#pragma unroll
      for (int b = 0; b < B0; ++b) {
        const int n = a + A0 * b;
        const float2 xv = __ldg(p.xhat + blk + n * CW + c);
        v[b] = psij ? cscale(xv, __ldg(psij + n * CW + c)) : xv;
      }
      Dft<B0, 1>::run(v);
#pragma unroll
      for (int kb = 1; kb < B0; ++kb) v[kb] = ctw<1>(v[kb], tw0[kb * A0 + a]);
#pragma unroll
      for (int kb = 0; kb < B0; ++kb) S[(kb * A0 + a) * CW + c] = v[kb];
    }
    __syncthreads();
    {
      const int c = tid % CW, kb = tid / CW;  // NT = CW * B0: one item per thread
      float2 w[A0];
#pragma unroll
      for (int a = 0; a < A0; ++a) w[a] = S[(kb * A0 + a) * CW + c];
      Dft<A0, 1>::run(w);
      __syncthreads();
#pragma unroll
      for (int ka = 0; ka < A0; ++ka) S[(kb + B0 * ka) * CW + c] = w[ka];  // [row][c]
    }
    cluster.sync();  // every CTA's column block is complete

    // ---- rows: C2R along axis 1 on this CTA's RW rows, reading all blocks ----
    float2 v[G::IT_R1][B1];
#pragma unroll
    for (int i = 0; i < G::IT_R1; ++i) {
      const int it = tid + i * NT;
      const int a = it % A1, q = it / A1;
      const int r0 = rank * RW + 2 * q;
#pragma unroll
      for (int b = 0; b < B1; ++b) {
        float2 z = make_float2(0.f, 0.f);
        if (it < PAIRS * A1) {
          const int n = a + A1 * b;
          const int m = n <= H ? n : L1 - n;
          const uint32_t src = dsmem_map(smem_addr(S + r0 * CW + m % CW), m / CW);
          float2 ya = dsmem_ld(src);
          float2 yb = dsmem_ld(src + CW * (uint32_t)sizeof(float2));
          if (n > H) {
            ya = cconj(ya);
            yb = cconj(yb);
          }
          z = make_float2(ya.x - yb.y, ya.y + yb.x);
        }
        v[i][b] = z;
      }
    }
    cluster.sync();  // all remote reads of this iteration are done
#pragma unroll
    for (int i = 0; i < G::IT_R1; ++i) {
      const int it = tid + i * NT;
      if (it < PAIRS * A1) {
        const int a = it % A1, q = it / A1;
        Dft<B1, 1>::run(v[i]);
#pragma unroll
        for (int kb = 1; kb < B1; ++kb) v[i][kb] = ctw<1>(v[i][kb], tw1[kb * A1 + a]);
#pragma unroll
        for (int kb = 0; kb < B1; ++kb) S[q * LS + kb * (A1 + 1) + a] = v[i][kb];
      }
    }
    __syncthreads();
    const float thr = p.thr ? p.thr[j] : 0.f;
    float* outj = p.out_real + (int64_t)j * L0 * L1;
    for (int it = tid; it < PAIRS * B1; it += NT) {
      const int kb = it % B1, q = it / B1;
      float2 w[A1];
#pragma unroll
      for (int a = 0; a < A1; ++a) w[a] = S[q * LS + kb * (A1 + 1) + a];
      Dft<A1, 1>::run(w);
      float* o0 = outj + (int64_t)(rank * RW + 2 * q) * L1;
#pragma unroll
      for (int ka = 0; ka < A1; ++ka) {
        const int k = kb + B1 * ka;
        float c0 = w[ka].x * p.scale, c1 = w[ka].y * p.scale;
        if (p.thr) {
          if (fabsf(c0) < thr) c0 = 0.f;
          if (fabsf(c1) < thr) c1 = 0.f;
        }
        o0[k] = c0;
        o0[L1 + k] = c1;
      }
    }
    __syncthreads();  // S is reused by the next filter
  }
}

// Inverse direction: for j = cluster id, cluster id + #clusters, ...
//   rows R2C of in_real[j], columns FFT_0, out_spec[cluster id] (+)= psi_j * (.)
// (psi == nullptr: out_spec[0] = the spectrum of in_real[0]).
template <int L0, int L1>
__global__ void __cluster_dims__(kCluster, 1, 1) __launch_bounds__(ClGeo<L0, L1>::NT)
    k_cl_inv(ClArgs p) {
  using G = ClGeo<L0, L1>;
  constexpr int NH = G::NH, CW = G::CW, RW = G::RW, PAIRS = G::PAIRS;
  constexpr int A0 = G::A0, B0 = G::B0, A1 = G::A1, B1 = G::B1, NT = G::NT;
  constexpr int H = L1 / 2;
  constexpr int LS = B1 * (A1 + 1);
  extern __shared__ float2 S[];
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int cid = blockIdx.x / kCluster;
  const int ncl = gridDim.x / kCluster;
  const int tid = threadIdx.x;
  const float2* tw0 = g_twiddle + twiddle_offset(L0);
  const float2* tw1 = g_twiddle + twiddle_offset(L1);
  const int64_t blk = (int64_t)rank * G::BLOCK;
  const int c2 = tid % CW, kb2 = tid / CW;  // column pass-2 item of this thread
  float2* part = p.out_spec + (int64_t)cid * G::TOTAL + blk;

  for (int j = cid; j < p.R; j += ncl) {
    // ---- rows: R2C along axis 1 of this CTA's RW rows ----
    const float* inj = p.in_real + (int64_t)j * L0 * L1;
    for (int it = tid; it < PAIRS * A1; it += NT) {
      const int a = it % A1, q = it / A1;
      const float* r0 = inj + (int64_t)(rank * RW + 2 * q) * L1;
      float2 v[B1];
#pragma unroll
      for (int b = 0; b < B1; ++b) {
        const int n = a + A1 * b;
        v[b] = make_float2(__ldg(r0 + n), __ldg(r0 + L1 + n));
      }
      Dft<B1, -1>::run(v);
#pragma unroll
      for (int kb = 1; kb < B1; ++kb) v[kb] = ctw<-1>(v[kb], tw1[kb * A1 + a]);
#pragma unroll
      for (int kb = 0; kb < B1; ++kb) S[q * LS + kb * (A1 + 1) + a] = v[kb];
    }
    __syncthreads();
    {
      float2 w[G::IT_R2][A1];
#pragma unroll
      for (int i = 0; i < G::IT_R2; ++i) {
        const int it = tid + i * NT;
        const int kb = it % B1, q = it / B1;
        if (it < PAIRS * B1) {
#pragma unroll
          for (int a = 0; a < A1; ++a) w[i][a] = S[q * LS + kb * (A1 + 1) + a];
          Dft<A1, -1>::run(w[i]);
        }
      }
      __syncthreads();
#pragma unroll
      for (int i = 0; i < G::IT_R2; ++i) {
        const int it = tid + i * NT;
        const int kb = it % B1, q = it / B1;
        if (it < PAIRS * B1) {
#pragma unroll
          for (int ka = 0; ka < A1; ++ka) S[q * L1 + kb + B1 * ka] = w[i][ka];
        }
      }
    }
    __syncthreads();
    // Split Z = FFT(x0 + i x1) in place. Line q then holds, for rows r0 = 2q, r1 = 2q+1:
    //   slot m (0 < m < H): X0[m];  slot L1 - m: X1[m];
    //   slot 0: (X0[0], X0[H]);     slot H: (X1[0], X1[H])   (those four are real)
    for (int it = tid; it < PAIRS * (H + 1); it += NT) {
      const int q = it / (H + 1), m = it % (H + 1);
      float2* line = S + q * L1;
      if (m == 0) {
        const float2 z0 = line[0], zh = line[H];
        line[0] = make_float2(z0.x, zh.x);
        line[H] = make_float2(z0.y, zh.y);
      } else if (m < H) {
        const float2 z = line[m], w = line[L1 - m];
        line[m] = make_float2(0.5f * (z.x + w.x), 0.5f * (z.y - w.y));
        line[L1 - m] = make_float2(0.5f * (z.y + w.y), 0.5f * (w.x - z.x));
      }
    }
    cluster.sync();  // every CTA's row block is complete

    // ---- columns: FFT_0 on this CTA's CW columns, reading all row blocks ----
    float2 v[G::IT_C1][B0];
#pragma unroll
    for (int i = 0; i < G::IT_C1; ++i) {
      const int it = tid + i * NT;
      const int c = it % CW, a = it / CW;
      const int col = rank * CW + c;
#pragma unroll
      for (int b = 0; b < B0; ++b) {
        float2 z = make_float2(0.f, 0.f);
        if (it < CW * A0 && col < NH) {
          const int n = a + A0 * b;        // row
          const int own = n / RW, lr = n % RW;
          const int q = lr >> 1;
          // slot of (row, col) in the split line q (see the split above)
          const bool even = (lr & 1) == 0;
          const bool edge = col == 0 || col == H;
          const int slot = edge ? (even ? 0 : H) : (even ? col : L1 - col);
          const float2 t = dsmem_ld(dsmem_map(smem_addr(S + q * L1 + slot), own));
          z = edge ? make_float2(col == 0 ? t.x : t.y, 0.f) : t;
        }
        v[i][b] = z;
      }
    }
    cluster.sync();  // all remote reads of this iteration are done
#pragma unroll
    for (int i = 0; i < G::IT_C1; ++i) {
      const int it = tid + i * NT;
      if (it < CW * A0) {
        const int c = it % CW, a = it / CW;
        Dft<B0, -1>::run(v[i]);
#pragma unroll
        for (int kb = 1; kb < B0; ++kb) v[i][kb] = ctw<-1>(v[i][kb], tw0[kb * A0 + a]);
#pragma unroll
        for (int kb = 0; kb < B0; ++kb) S[(kb * A0 + a) * CW + c] = v[i][kb];
      }
    }
    __syncthreads();
    {
      float2 w[A0];
#pragma unroll
      for (int a = 0; a < A0; ++a) w[a] = S[(kb2 * A0 + a) * CW + c2];
      Dft<A0, -1>::run(w);
      const bool first = j == cid;
      if (p.psi) {
        const float* psij = p.psi + (int64_t)j * G::TOTAL + blk;
#pragma unroll
        for (int ka = 0; ka < A0; ++ka) {
          const int e = (kb2 + B0 * ka) * CW + c2;
          const float f = __ldg(psij + e);
          float2 acc = first ? make_float2(0.f, 0.f) : part[e];
          acc.x = fmaf(f, w[ka].x, acc.x);
          acc.y = fmaf(f, w[ka].y, acc.y);
          part[e] = acc;
        }
      } else {
#pragma unroll
        for (int ka = 0; ka < A0; ++ka) {
          const int e = (kb2 + B0 * ka) * CW + c2;
          part[e] = first ? w[ka] : cadd(part[e], w[ka]);
        }
      }
    }
    __syncthreads();  // S is reused by the next filter
  }
}

// out[e] = (sum_q parts[q][e]) * w[e] over n complex elements (FP64 weight).
__global__ void __launch_bounds__(256) k_cl_reduce(const float2* __restrict__ parts, int nparts,
                                                   int64_t n, const double* __restrict__ w,
                                                   float2* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float2 s = parts[i];
    for (int q = 1; q < nparts; ++q) s = cadd(s, parts[q * n + i]);
    if (w) {
      const double wi = w[i];
      s = make_float2((float)((double)s.x * wi), (float)((double)s.y * wi));
    }
    out[i] = s;
  }
}

}  // namespace dev
}  // namespace sl
