// Transform kernels shared by the 2D and 3D paths: the pencil ("column") pass along
// axis 0 and the 2D row passes along the last axis. Internal header.
//
// Spectra are stored as half spectra along the last axis, row-major: element
// (k0, p) of a spectrum lives at k0 * NP + p, where p enumerates the NP points of one
// slab (2D: NP = n1/2 + 1 columns; 3D: NP = n1 * (n2/2 + 1)). A stack of spectra
// (one per filter of a group) is strided by Nh = n0 * NP.
#pragma once

#include "fft_core.cuh"

namespace sl {
namespace dev {

constexpr int kThreads = 256;
constexpr int kMaxGroup = 256;  // filters per launch whose thresholds travel by value

// Concatenated twiddle tables, one per line length L = 8..1024:
// g_twiddle[twiddle_offset(L) + kb * A + a] = exp(-2 pi i a kb / L).
// Filled once per device from FP64 values by the host (this header is compiled in
// exactly one translation unit).
__device__ float2 g_twiddle[kTwiddleTotal];

enum ColMode { COL_SPEC = 0, COL_FWD_FILT = 1, COL_INV_ACC = 2, COL_INV_FIN = 3 };

struct ColArgs {
  const float2* in;
  float2* out;
  const float* psi;      // [R][Nh] real half spectra
  const double* invPsi;  // [Nh]
  int64_t Nh;
  int NP;                // pencils (columns) per spectrum
  int j0;                // first filter of the group
  int nfilt;             // filters in the group
  int fps;               // filters per split (COL_INV_ACC)
  int part0;             // first partial written (COL_INV_ACC)
  int nparts;            // partials summed (COL_INV_FIN)
  int use_invpsi;        // COL_INV_FIN: 1 = divide by Psi (inverse), 0 = adjoint
};

// Pencil pass along axis 0 (length L = n0), TC = 256/B pencils per CTA.
//   COL_SPEC      in-place forward FFT of a stack of 1 spectrum
//   COL_FWD_FILT  slot s = blockIdx.y: out[s] = IFFT_0( in * psi[j0 + s] )
//   COL_INV_ACC   split q = blockIdx.y: out[part0 + q] = sum_{j in split} psi[j] FFT_0(in[j - j0])
//   COL_INV_FIN   out = IFFT_0( (sum_q in[q]) * invPsi )   (adjoint: without invPsi)
template <int L, int MODE>
__global__ void __launch_bounds__(kThreads) k_col(ColArgs p) {
  constexpr int A = Split<L>::A, B = Split<L>::B;
  constexpr int TC = kThreads / B;
  constexpr int IT1 = TC * A / kThreads;
  constexpr int DIR = (MODE == COL_SPEC || MODE == COL_INV_ACC) ? -1 : 1;
  static_assert(TC * B == kThreads, "one pass-2 item per thread");
  extern __shared__ float2 sm[];  // [B][A][TC]
  const int tid = threadIdx.x;
  const int pc0 = blockIdx.x * TC;
  const float2* tw = g_twiddle + twiddle_offset(L);
  const int64_t Nh = p.Nh;
  const int NP = p.NP;

  int jbeg = 0, jend = 1;
  if constexpr (MODE == COL_FWD_FILT) {
    jbeg = p.j0 + blockIdx.y;
    jend = jbeg + 1;
  } else if constexpr (MODE == COL_INV_ACC) {
    jbeg = p.j0 + blockIdx.y * p.fps;
    jend = min(jbeg + p.fps, p.j0 + p.nfilt);
  }

  // pass-2 item of this thread
  const int line2 = tid % TC, kb2 = tid / TC;
  const int pc2 = pc0 + line2;
  float2 acc[A];
#pragma unroll
  for (int i = 0; i < A; ++i) acc[i] = make_float2(0.f, 0.f);

  for (int j = jbeg; j < jend; ++j) {
#pragma unroll
    for (int i = 0; i < IT1; ++i) {
      const int it = tid + i * kThreads;
      const int line = it % TC, a = it / TC;
      const int pc = pc0 + line;
      float2 v[B];
#pragma unroll
      for (int b = 0; b < B; ++b) {
        const int n = a + A * b;
        const int64_t e = (int64_t)n * NP + pc;
        float2 val = make_float2(0.f, 0.f);
        if (pc < NP) {
          if constexpr (MODE == COL_SPEC) {
            val = p.in[e];
          } else if constexpr (MODE == COL_FWD_FILT) {
            const float f = __ldg(p.psi + (int64_t)j * Nh + e);
            val = cscale(__ldg(p.in + e), f);
          } else if constexpr (MODE == COL_INV_ACC) {
            val = p.in[(int64_t)(j - p.j0) * Nh + e];
          } else {
            float2 s = p.in[e];
            for (int q = 1; q < p.nparts; ++q) s = cadd(s, p.in[(int64_t)q * Nh + e]);
            if (p.use_invpsi) {
              const double w = p.invPsi[e];
              s = make_float2((float)((double)s.x * w), (float)((double)s.y * w));
            }
            val = s;
          }
        }
        v[b] = val;
      }
      Dft<B, DIR>::run(v);
#pragma unroll
      for (int kb = 1; kb < B; ++kb) v[kb] = ctw<DIR>(v[kb], tw[kb * A + a]);
#pragma unroll
      for (int kb = 0; kb < B; ++kb) sm[(kb * A + a) * TC + line] = v[kb];
    }
    __syncthreads();
    float2 w[A];
#pragma unroll
    for (int a = 0; a < A; ++a) w[a] = sm[(kb2 * A + a) * TC + line2];
    Dft<A, DIR>::run(w);
    if (pc2 < NP) {
#pragma unroll
      for (int ka = 0; ka < A; ++ka) {
        const int k = kb2 + B * ka;
        const int64_t e = (int64_t)k * NP + pc2;
        if constexpr (MODE == COL_SPEC || MODE == COL_INV_FIN) {
          p.out[e] = w[ka];
        } else if constexpr (MODE == COL_FWD_FILT) {
          p.out[(int64_t)(j - p.j0) * Nh + e] = w[ka];
        } else {
          const float f = __ldg(p.psi + (int64_t)j * Nh + e);
          acc[ka].x = fmaf(f, w[ka].x, acc[ka].x);
          acc[ka].y = fmaf(f, w[ka].y, acc[ka].y);
        }
      }
    }
    __syncthreads();
  }
  if constexpr (MODE == COL_INV_ACC) {
    if (pc2 < NP) {
      float2* o = p.out + (int64_t)(p.part0 + blockIdx.y) * Nh;
#pragma unroll
      for (int ka = 0; ka < A; ++ka) o[(int64_t)(kb2 + B * ka) * NP + pc2] = acc[ka];
    }
  }
}

template <int L>
constexpr int col_smem_bytes() {
  return Split<L>::B * Split<L>::A * (kThreads / Split<L>::B) * (int)sizeof(float2);
}

// ------------------------------------------------------------------- row passes ---

enum RowMode { ROW_R2C = 0, ROW_C2R = 1, ROW_RT = 2 };

struct Thresholds {
  float v[kMaxGroup];
};

struct RowArgs {
  const float* in_real;   // ROW_R2C: real rows, slot stride in_stride
  const float2* in_half;  // ROW_C2R / ROW_RT: half-spectrum rows, slot stride in_stride
  float* out_real;        // ROW_C2R: real rows, slot stride out_stride
  float2* out_half;       // ROW_R2C / ROW_RT: half rows, slot stride out_stride
  int64_t in_stride, out_stride;
  int n_rows;             // rows per slot (even)
  int nh;                 // L/2 + 1
  float scale;            // ROW_C2R / ROW_RT: factor on the real output
  int use_thr;
  Thresholds thr;         // per slot: keep |c| >= thr (ROW_C2R / ROW_RT)
};

// Row passes along the last axis (length L = n1), two real rows per complex line:
//   ROW_R2C  real rows -> half spectra (unnormalised forward DFT)
//   ROW_C2R  half spectra -> real rows (inverse DFT) * scale, optional threshold
//   ROW_RT   half spectra -> real rows * scale -> threshold -> half spectra
// PAIRS = 256/B row pairs per CTA; blockIdx.y is the slot.
template <int L, int MODE>
__global__ void __launch_bounds__(kThreads) k_row(RowArgs p) {
  constexpr int A = Split<L>::A, B = Split<L>::B;
  constexpr int PAIRS = kThreads / B;
  constexpr int IT1 = PAIRS * A / kThreads;
  constexpr int LS = B * (A + 1);  // padded exchange stride per line
  constexpr int H = L / 2;
  static_assert(PAIRS * B == kThreads, "one pass-2 item per thread");
  extern __shared__ float2 sm[];  // PAIRS * LS float2
  const int tid = threadIdx.x;
  const int slot = blockIdx.y;
  const int pair0 = blockIdx.x * PAIRS;
  const int npairs = p.n_rows / 2;
  const float2* tw = g_twiddle + twiddle_offset(L);
  const int nh = p.nh;

  const int kb2 = tid % B, line2 = tid / B;
  const int pr2 = pair0 + line2;
  const bool ok2 = pr2 < npairs;
  float2 res[A];

  // ---------------------------------------------------------- half -> real ---
  if constexpr (MODE == ROW_C2R || MODE == ROW_RT) {
    const float2* in = p.in_half + (int64_t)slot * p.in_stride;
#pragma unroll
    for (int i = 0; i < IT1; ++i) {
      const int it = tid + i * kThreads;
      const int a = it % A, line = it / A;
      const int pr = pair0 + line;
      float2 v[B];
#pragma unroll
      for (int b = 0; b < B; ++b) {
        const int n = a + A * b;
        float2 z = make_float2(0.f, 0.f);
        if (pr < npairs) {
          const float2* r0 = in + (int64_t)(2 * pr) * nh;
          const float2* r1 = r0 + nh;
          float2 ya, yb;
          if (n <= H) {
            ya = r0[n];
            yb = r1[n];
          } else {
            ya = cconj(r0[L - n]);
            yb = cconj(r1[L - n]);
          }
          z = make_float2(ya.x - yb.y, ya.y + yb.x);  // ya + i yb
        }
        v[b] = z;
      }
      Dft<B, 1>::run(v);
#pragma unroll
      for (int kb = 1; kb < B; ++kb) v[kb] = ctw<1>(v[kb], tw[kb * A + a]);
#pragma unroll
      for (int kb = 0; kb < B; ++kb) sm[line * LS + kb * (A + 1) + a] = v[kb];
    }
    __syncthreads();
#pragma unroll
    for (int a = 0; a < A; ++a) res[a] = sm[line2 * LS + kb2 * (A + 1) + a];
    Dft<A, 1>::run(res);
    const float thr = p.use_thr ? p.thr.v[slot] : 0.f;
#pragma unroll
    for (int ka = 0; ka < A; ++ka) {
      float c0 = res[ka].x * p.scale, c1 = res[ka].y * p.scale;
      if (p.use_thr) {
        if (fabsf(c0) < thr) c0 = 0.f;
        if (fabsf(c1) < thr) c1 = 0.f;
      }
      res[ka] = make_float2(c0, c1);
    }
    if constexpr (MODE == ROW_C2R) {
      if (ok2) {
        float* o0 = p.out_real + (int64_t)slot * p.out_stride + (int64_t)(2 * pr2) * L;
        float* o1 = o0 + L;
#pragma unroll
        for (int ka = 0; ka < A; ++ka) {
          const int k = kb2 + B * ka;
          o0[k] = res[ka].x;
          o1[k] = res[ka].y;
        }
      }
      return;
    }
    // ROW_RT: hand the thresholded rows to the forward pass through shared memory
    __syncthreads();
#pragma unroll
    for (int ka = 0; ka < A; ++ka) sm[line2 * L + kb2 + B * ka] = res[ka];
    __syncthreads();
  }

  // ---------------------------------------------------------- real -> half ---
  {
    float2 v[IT1][B];
#pragma unroll
    for (int i = 0; i < IT1; ++i) {
      const int it = tid + i * kThreads;
      const int a = it % A, line = it / A;
      const int pr = pair0 + line;
#pragma unroll
      for (int b = 0; b < B; ++b) {
        const int n = a + A * b;
        if constexpr (MODE == ROW_R2C) {
          float2 z = make_float2(0.f, 0.f);
          if (pr < npairs) {
            const float* r0 = p.in_real + (int64_t)slot * p.in_stride + (int64_t)(2 * pr) * L;
            z = make_float2(r0[n], r0[L + n]);
          }
          v[i][b] = z;
        } else {
          v[i][b] = sm[line * L + n];
        }
      }
    }
    if constexpr (MODE == ROW_RT) __syncthreads();
#pragma unroll
    for (int i = 0; i < IT1; ++i) {
      const int it = tid + i * kThreads;
      const int a = it % A, line = it / A;
      Dft<B, -1>::run(v[i]);
#pragma unroll
      for (int kb = 1; kb < B; ++kb) v[i][kb] = ctw<-1>(v[i][kb], tw[kb * A + a]);
#pragma unroll
      for (int kb = 0; kb < B; ++kb) sm[line * LS + kb * (A + 1) + a] = v[i][kb];
    }
  }
  __syncthreads();
#pragma unroll
  for (int a = 0; a < A; ++a) res[a] = sm[line2 * LS + kb2 * (A + 1) + a];
  Dft<A, -1>::run(res);
  __syncthreads();
#pragma unroll
  for (int ka = 0; ka < A; ++ka) sm[line2 * L + kb2 + B * ka] = res[ka];
  __syncthreads();
  // Split Z = FFT(x0 + i x1) into the half spectra of x0 and x1.
  float2* out = p.out_half + (int64_t)slot * p.out_stride;
  constexpr int HP = H + 1;
  for (int it = tid; it < PAIRS * HP; it += kThreads) {
    const int line = it / HP, k = it % HP;
    const int pr = pair0 + line;
    if (pr >= npairs) continue;
    const float2 z = sm[line * L + k];
    const float2 w = sm[line * L + ((L - k) & (L - 1))];
    float2* o0 = out + (int64_t)(2 * pr) * nh;
    o0[k] = make_float2(0.5f * (z.x + w.x), 0.5f * (z.y - w.y));
    o0[nh + k] = make_float2(0.5f * (z.y + w.y), 0.5f * (w.x - z.x));
  }
}

template <int L>
constexpr int row_smem_bytes() {
  return (kThreads / Split<L>::B) * Split<L>::B * (Split<L>::A + 1) * (int)sizeof(float2);
}

// ------------------------------------------------------------ elementwise ---

// In-place hard threshold of nf consecutive coefficient arrays of n elements each.
__global__ void __launch_bounds__(kThreads) k_threshold(float* c, int64_t n, int nf,
                                                        Thresholds thr) {
  const int f = blockIdx.y;
  if (f >= nf) return;
  const float t = thr.v[f];
  float* base = c + (int64_t)f * n;
  const int64_t n4 = n / 4;
  float4* b4 = reinterpret_cast<float4*>(base);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
       i += (int64_t)gridDim.x * blockDim.x) {
    float4 v = b4[i];
    v.x = fabsf(v.x) < t ? 0.f : v.x;
    v.y = fabsf(v.y) < t ? 0.f : v.y;
    v.z = fabsf(v.z) < t ? 0.f : v.z;
    v.w = fabsf(v.w) < t ? 0.f : v.w;
    b4[i] = v;
  }
  for (int64_t i = n4 * 4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    base[i] = fabsf(base[i]) < t ? 0.f : base[i];
}

}  // namespace dev
}  // namespace sl
