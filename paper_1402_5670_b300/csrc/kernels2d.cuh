// Transform kernels shared by the 2D and 3D paths: the pencil ("column") pass along
// axis 0 and the 2D row passes along the last axis. Internal header.
//
// Spectra (the signal's spectrum, the per-filter intermediates, the partial sums and
// the filter bank itself) are half spectra along the last axis stored TILE-MAJOR: the
// NP pencils of one spectrum (2D: the n1/2 + 1 columns; 3D: the n1 (n2/2 + 1) points of
// a plane) are cut into tiles of TC consecutive pencils, and a tile is one contiguous
// block [n0][TC]:
//     element (k0, p)  ->  ((p / TC) * n0 + k0) * TC + p % TC.
// A pencil-pass CTA therefore reads and writes one contiguous block per spectrum, and
// a row (or plane) pass reads each row as runs of TC contiguous elements. The last
// tile is padded to TC pencils. Pad pencils are transformed along with the others
// but never read by a row or plane pass, so whatever they hold never reaches a
// result (the bank stores zeros there). NPp = ceil(NP / TC) * TC and a spectrum holds
// Nhp = n0 * NPp elements.
#pragma once

#include "fft_core.cuh"

namespace sl {
namespace dev {

constexpr int kMaxGroup = 256;  // filters per launch whose thresholds travel by value

// Minimum resident CTAs per SM requested from the compiler for the persistent
// filter-loop kernels (register caps; the row pipeline's shared memory allows four
// CTAs per SM up to 512-point rows, two for 1024); compile-time tunables.
#ifndef SL_MINB_COLF
#define SL_MINB_COLF 1
#endif
#ifndef SL_MINB_COLI
#define SL_MINB_COLI 1
#endif
#ifndef SL_MINB_ROW
#define SL_MINB_ROW 4
#endif

// Concatenated twiddle tables, one per line length L = 8..1024:
// g_twiddle[twiddle_offset(L) + kb * A + a] = exp(-2 pi i a kb / L).
// Filled once per device from FP64 values by the host (this header is compiled in
// exactly one translation unit).
__device__ float2 g_twiddle[kTwiddleTotal];

// Lines (pencils or row pairs) per CTA. CTAs are kept small (128 threads) so that
// several independent CTAs share an SM and overlap each other's memory latency.
__host__ __device__ constexpr int col_tile_of(int L) {
  return L == 8 ? 32 : L == 16 ? 32 : L == 32 ? 16 : L == 64 ? 16 : L == 128 ? 8 : L == 256 ? 8
       : L == 192 ? 8
       : 4;  // 384, 512, 1024
}

// Line geometry: TC lines per CTA, T = TC * A threads (one pass-1 item per thread;
// TC * B <= T threads take part in pass 2).
template <int L>
struct Geo {
  static constexpr int A = Split<L>::A, B = Split<L>::B;
  static constexpr int TC = col_tile_of(L);
  static constexpr int T = TC * A;
  // column exchange [B][A][TC] with the kb stride padded to XS = A*TC + PADX so that
  // the lanes of a half-warp (16/TC values of kb, TC lines each) hit distinct banks
  static constexpr int PADX = TC >= 16 ? 0 : TC;
  static constexpr int XS = A * TC + PADX;
  static constexpr int smem_col = B * XS * (int)sizeof(float2);
  static constexpr int smem_row = TC * B * (A + 1) * (int)sizeof(float2);
  static_assert(TC * B <= T, "pass 2 needs no more items than threads");
};

// Offset of element (k0, p) in a tile-major spectrum.
struct TileMap {
  int L0;   // pencil length n0
  int lg;   // log2(TC)
  // 32-bit arithmetic: a spectrum holds fewer than 2^31 elements (N <= 2^31 is checked
  // when the bank is built)
  __device__ __forceinline__ int at(int k0, int p) const {
    return (((p >> lg) * L0 + k0) << lg) + (p & ((1 << lg) - 1));
  }
};
__device__ __forceinline__ int tm_tc(const TileMap& t) { return 1 << t.lg; }

enum ColMode { COL_SPEC = 0, COL_FWD_FILT = 1, COL_INV_ACC = 2, COL_IFFT = 3 };

struct ColArgs {
  const float2* in;
  float2* out;
  const float* psi;      // filters: tile-major [R][Nhp], or natural [R][Nh] (psi_natural)
  int64_t Nhp;           // elements of one tile-major spectrum
  int64_t Nh;            // elements of one natural half spectrum (psi_natural)
  int NP;                // pencils per spectrum
  int psi_natural;       // 1: psi is in natural layout [R][n0][NP]
  int j0;                // first filter of the group
  int nfilt;             // filters in the group
  int fps;               // filters per split (COL_INV_ACC)
  int part0;             // first partial written (COL_INV_ACC)
};

// Pencil pass along axis 0 (length L = n0); CTA blockIdx.x owns tile blockIdx.x.
//   COL_SPEC      in-place forward FFT of one spectrum
//   COL_FWD_FILT  slot s = blockIdx.y: out[s] = IFFT_0( in * psi[j0 + s] )
//   COL_INV_ACC   split q = blockIdx.y: out[part0 + q] = sum_{j in split} psi[j] FFT_0(in[j - j0])
//   COL_IFFT      in-place inverse FFT of one spectrum
template <int L, int MODE>
__global__ void __launch_bounds__(Geo<L>::T) k_col(ColArgs p) {
  using G = Geo<L>;
  constexpr int A = G::A, B = G::B, TC = G::TC;
  constexpr int DIR = (MODE == COL_SPEC || MODE == COL_INV_ACC) ? -1 : 1;
  constexpr int XS = G::XS;
  extern __shared__ float2 sm[];  // [B][XS]: (kb, a, line) at kb * XS + a * TC + line
  const int tid = threadIdx.x;
  const int tile = blockIdx.x;
  const float2* tw = g_twiddle + twiddle_offset(L);
  const int64_t tbase = (int64_t)tile * L * TC;  // this CTA's block in a tile-major spectrum

  int jbeg = 0, jend = 1;
  if constexpr (MODE == COL_FWD_FILT) {
    jbeg = p.j0 + blockIdx.y;
    jend = jbeg + 1;
  } else if constexpr (MODE == COL_INV_ACC) {
    jbeg = p.j0 + blockIdx.y * p.fps;
    jend = min(jbeg + p.fps, p.j0 + p.nfilt);
  }

  // pass-1 item: (line, a); pass-2 item (tid < TC * B): (line2, kb2)
  const int line = tid % TC, a = tid / TC;
  const int line2 = tid % TC, kb2 = tid / TC;
  const bool in2 = tid < TC * B;
  const int pc = tile * TC + line;  // global pencil index
  float2 acc[A];
#pragma unroll
  for (int i = 0; i < A; ++i) acc[i] = make_float2(0.f, 0.f);

  for (int j = jbeg; j < jend; ++j) {
    float2 v[B];
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int n = a + A * b;
      const int64_t e = tbase + n * TC + line;
      if constexpr (MODE == COL_SPEC || MODE == COL_IFFT) {
        v[b] = p.in[e];
      } else if constexpr (MODE == COL_FWD_FILT) {
        float f;
        if (p.psi_natural) f = pc < p.NP ? __ldg(p.psi + (int64_t)j * p.Nh + (int64_t)n * p.NP + pc) : 0.f;
        else f = __ldg(p.psi + (int64_t)j * p.Nhp + e);
        v[b] = cscale(__ldg(p.in + e), f);
      } else {
        v[b] = p.in[(int64_t)(j - p.j0) * p.Nhp + e];
      }
    }
    Dft<B, DIR>::run(v);
#pragma unroll
    for (int kb = 1; kb < B; ++kb) v[kb] = ctw<DIR>(v[kb], tw[kb * A + a]);
#pragma unroll
    for (int kb = 0; kb < B; ++kb) sm[kb * XS + a * TC + line] = v[kb];
    __syncthreads();
    if (in2) {
      float2 w[A];
#pragma unroll
      for (int aa = 0; aa < A; ++aa) w[aa] = sm[kb2 * XS + aa * TC + line2];
      Dft<A, DIR>::run(w);
#pragma unroll
      for (int ka = 0; ka < A; ++ka) {
        const int k = kb2 + B * ka;
        const int64_t e = tbase + k * TC + line2;
        if constexpr (MODE == COL_SPEC || MODE == COL_IFFT) {
          p.out[e] = w[ka];
        } else if constexpr (MODE == COL_FWD_FILT) {
          p.out[(int64_t)(j - p.j0) * p.Nhp + e] = w[ka];
        } else {
          const float f = __ldg(p.psi + (int64_t)j * p.Nhp + e);
          acc[ka].x = fmaf(f, w[ka].x, acc[ka].x);
          acc[ka].y = fmaf(f, w[ka].y, acc[ka].y);
        }
      }
    }
    __syncthreads();
  }
  if constexpr (MODE == COL_INV_ACC) {
    if (in2) {
      float2* o = p.out + (int64_t)(p.part0 + blockIdx.y) * p.Nhp;
#pragma unroll
      for (int ka = 0; ka < A; ++ka) o[tbase + (kb2 + B * ka) * TC + line2] = acc[ka];
    }
  }
}

// ------------------------------------------------------ pipelined pencil pass ---

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// ------------------------------------------------ bulk copies (TMA engine) ---
// Stages of the filter-loop kernels are filled by cp.async.bulk copies that complete
// on one mbarrier per stage (transaction bytes); one thread (or the lanes of warp 0)
// issues them, so the transform warps spend no issue slots on copy loops. Every wait
// is bounded: a wait that runs out sets g_sl_wait_error (reported by sl_device_check)
// and the kernel returns after a bounded drain of its copies in flight.

__device__ int g_sl_wait_error;  // 0, or 1 once a bounded wait ran out

constexpr long long kWaitCycles = 4000000000LL;  // about two seconds of SM clock

__device__ __forceinline__ uint32_t smem_u32(const void* ptr) {
  return (uint32_t)__cvta_generic_to_shared(ptr);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Arrive on the barrier (the one expected arrival) and announce `bytes` of copies.
__device__ __forceinline__ void mbar_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile(
      "{\n.reg .b64 st;\nmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}" ::"r"(
          smem_u32(bar)),
      "r"(bytes)
      : "memory");
}
// Order this thread's earlier generic-proxy accesses of shared memory before the
// bulk copies it issues next (the stage being refilled was just read).
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Global -> shared bulk copy of `bytes` (a multiple of 16; both addresses 16-byte
// aligned), completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// Wait for the phase of the given parity; false once kWaitCycles pass without it.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  while (true) {
    uint32_t done = 0;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > kWaitCycles) return false;
  }
}

// Two-stage ring of a persistent kernel: fill i goes to stage i & 1 and completes
// phase (i >> 1) & 1 of that stage's barrier; fills and waits happen in this order,
// and a stage is refilled only after it was waited on and consumed. The counters are
// CTA-uniform (the loops are).
struct BulkRing {
  uint64_t* bar;    // [2] in shared memory
  int issued = 0;   // fills issued
  int waited = 0;   // fills waited for
  // Wait for the next fill; CTA-uniform result (includes a CTA barrier).
  __device__ __forceinline__ bool wait() {
    const int i = waited++;
    const bool ok = mbar_wait_bounded(bar + (i & 1), (uint32_t)((i >> 1) & 1));
    return !__syncthreads_or(!ok);
  }
  // After a wait ran out: flag it, and let the fills still in flight (the one waited
  // for and any later one) land, each wait bounded again, before the CTA exits.
  __device__ __forceinline__ void abandon() {
    if (threadIdx.x == 0) {
      atomicExch(&g_sl_wait_error, 1);
      for (int i = waited - 1; i < issued; ++i)
        mbar_wait_bounded(bar + (i & 1), (uint32_t)((i >> 1) & 1));
    }
    __syncthreads();
  }
};

// Copy `bytes` (a multiple of 16, both addresses 16-byte aligned) from global to
// shared memory with every thread of the CTA issuing 16-byte asynchronous copies.
template <int T>
__device__ __forceinline__ void cp_async_block(void* dst, const void* src, int bytes) {
  char* d = static_cast<char*>(dst);
  const char* s = static_cast<const char*>(src);
  for (int o = threadIdx.x * 16; o < bytes; o += T * 16) cp_async16(d + o, s + o);
}

// Forward filter pass as a persistent, software-pipelined kernel: work item i is
// (tile i / nfilt, filter j0 + i % nfilt); CTA c takes items c, c + gridDim.x, ...
// While item k is transformed, the signal and filter tiles of item k + 1 (two
// contiguous blocks of the tile-major layout) land in the other shared-memory stage
// by bulk copies, so global-memory latency overlaps with the FFT.
// Output as COL_FWD_FILT: out[s] = IFFT_0(in * psi[j0 + s]).
template <int L>
__global__ void __launch_bounds__(Geo<L>::T, SL_MINB_COLF) k_col_fwd_pipe(ColArgs p) {
  using G = Geo<L>;
  constexpr int A = G::A, B = G::B, TC = G::TC, XS = G::XS;
  constexpr int TILE = L * TC;  // elements of one tile
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* xs = reinterpret_cast<float2*>(smraw);                 // [2][TILE]
  float* ps = reinterpret_cast<float*>(xs + 2 * TILE);           // [2][TILE]
  float2* ex = reinterpret_cast<float2*>(ps + 2 * TILE);         // [B][XS]
  uint64_t* bars = reinterpret_cast<uint64_t*>(ex + B * XS);     // [2]
  const int tid = threadIdx.x;
  const float2* tw = g_twiddle + twiddle_offset(L);
  const int nitems = (int)(p.Nhp / TILE) * p.nfilt;  // tiles x filters
  const int line = tid % TC, a = tid / TC;
  const int line2 = tid % TC, kb2 = tid / TC;
  const bool in2 = tid < TC * B;
  if (tid == 0) {
    mbar_init(bars);
    mbar_init(bars + 1);
    mbar_init_fence();
  }
  __syncthreads();
  BulkRing ring{bars};

  auto issue = [&](int item, int stage) {
    if (item < nitems) {
      if (tid == 0) {
        const int tile = item / p.nfilt, j = p.j0 + item % p.nfilt;
        fence_proxy_async();
        mbar_expect(bars + stage, TILE * 12);
        bulk_g2s(xs + stage * TILE, p.in + (int64_t)tile * TILE, TILE * 8, bars + stage);
        bulk_g2s(ps + stage * TILE, p.psi + (int64_t)j * p.Nhp + (int64_t)tile * TILE, TILE * 4,
                 bars + stage);
      }
      ++ring.issued;
    }
  };

  float2 twr[B];  // this thread's inter-pass twiddles, the same for every item
#pragma unroll
  for (int kb = 1; kb < B; ++kb) twr[kb] = tw[kb * A + a];

  int item = blockIdx.x;
  issue(item, 0);
  issue(item + gridDim.x, 1);
  for (int k = 0; item < nitems; ++k, item += gridDim.x) {
    const int stage = k & 1;
    if (!ring.wait()) {  // stage filled; previous item's exchange reads done
      ring.abandon();
      return;
    }
    const int tile = item / p.nfilt, s = item % p.nfilt;
    float2 v[B];
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int e = (a + A * b) * TC + line;
      v[b] = cscale(xs[stage * TILE + e], ps[stage * TILE + e]);
    }
    Dft<B, 1>::run(v);
#pragma unroll
    for (int kb = 1; kb < B; ++kb) v[kb] = ctw<1>(v[kb], twr[kb]);
#pragma unroll
    for (int kb = 0; kb < B; ++kb) ex[kb * XS + a * TC + line] = v[kb];
    __syncthreads();                        // stage and exchange inputs consumed
    issue(item + 2 * gridDim.x, stage);     // prefetch two items ahead
    if (in2) {
      float2 w[A];
#pragma unroll
      for (int aa = 0; aa < A; ++aa) w[aa] = ex[kb2 * XS + aa * TC + line2];
      Dft<A, 1>::run(w);
      float2* o = p.out + (int64_t)s * p.Nhp + (int64_t)tile * TILE;
#pragma unroll
      for (int ka = 0; ka < A; ++ka) o[(kb2 + B * ka) * TC + line2] = w[ka];
    }
  }
}

template <int L>
constexpr int col_pipe_smem_bytes() {  // two stages, the exchange, two mbarriers
  return 2 * L * Geo<L>::TC * (8 + 4) + Geo<L>::B * Geo<L>::XS * 8 + 16;
}

// out[e] = (sum_q parts[q][e]) * w[e] (w in FP64, or 1 when w == nullptr), over one
// tile-major spectrum of n float2 elements, two elements per thread and step.
__global__ void __launch_bounds__(256) k_reduce_parts(const float2* __restrict__ parts, int nparts,
                                                      int64_t stride, const double* __restrict__ w,
                                                      float2* __restrict__ out, int64_t n) {
  const int64_t n2 = n / 2;
  const float4* p4 = reinterpret_cast<const float4*>(parts);
  float4* o4 = reinterpret_cast<float4*>(out);
  const int64_t s4 = stride / 2;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2;
       i += (int64_t)gridDim.x * blockDim.x) {
    float4 s = p4[i];
#pragma unroll 8
    for (int q = 1; q < nparts; ++q) {  // loads independent of the sum: issued ahead
      const float4 t = __ldg(p4 + q * s4 + i);
      s.x += t.x;
      s.y += t.y;
      s.z += t.z;
      s.w += t.w;
    }
    if (w) {
      const double w0 = w[2 * i], w1 = w[2 * i + 1];
      s = make_float4((float)((double)s.x * w0), (float)((double)s.y * w0),
                      (float)((double)s.z * w1), (float)((double)s.w * w1));
    }
    o4[i] = s;
  }
}

// ------------------------------------------------------------------- row passes ---

enum RowMode { ROW_R2C = 0, ROW_C2R = 1, ROW_RT = 2 };

struct Thresholds {
  float v[kMaxGroup];
};

struct RowArgs {
  const float* in_real;   // ROW_R2C: real rows, slot stride in_stride
  const float2* in_half;  // ROW_C2R / ROW_RT: tile-major spectra, slot stride in_stride
  float* out_real;        // ROW_C2R: real rows, slot stride out_stride
  float2* out_half;       // ROW_R2C / ROW_RT: tile-major spectra, slot stride out_stride
  int64_t in_stride, out_stride;
  int n_rows;             // rows per slot (even) = n0
  TileMap tm;             // layout of the spectra (L0 = n0, TC of the pencil pass)
  float scale;            // ROW_C2R / ROW_RT: factor on the real output
  int use_thr;            // 0: none; 1: hard threshold; 2 (ROW_RT): lattice mask
  Thresholds thr;         // per slot: keep |c| >= thr, or (use_thr == 2) keep the
                          // points whose row and column are multiples of thr (a power
                          // of two), the sampling lattice of a subsampled subband
};

// Lattice mask of the subsampled transform: keep (row, col) iff both are multiples of
// the power of two s.
__device__ __forceinline__ bool on_lattice(int row, int col, int s) {
  return ((row | col) & (s - 1)) == 0;
}

// Row passes along the last axis (length L = n1), two real rows per complex line:
//   ROW_R2C  real rows -> half spectra (unnormalised forward DFT)
//   ROW_C2R  half spectra -> real rows (inverse DFT) * scale, optional threshold
//   ROW_RT   half spectra -> real rows * scale -> threshold -> half spectra
// PAIRS row pairs per CTA (T = PAIRS * A threads); blockIdx.y is the slot.
template <int L, int MODE, int PAIRS>
__global__ void __launch_bounds__(PAIRS * Split<L>::A) k_row(RowArgs p) {
  constexpr int A = Split<L>::A, B = Split<L>::B, T = PAIRS * A;
  constexpr int LS = B * (A + 1);  // padded exchange stride per line
  constexpr int H = L / 2;
  extern __shared__ float2 sm[];  // PAIRS * LS float2
  const int tid = threadIdx.x;
  const int slot = blockIdx.y;
  const int pair0 = blockIdx.x * PAIRS;
  const int npairs = p.n_rows / 2;
  const float2* tw = g_twiddle + twiddle_offset(L);
  const TileMap tm = p.tm;

  const int a1 = tid % A, line1 = tid / A;  // pass-1 item
  const int pr1 = pair0 + line1;
  const int kb2 = tid % B, line2 = tid / B;  // pass-2 item (tid < PAIRS * B)
  const bool in2 = tid < PAIRS * B;
  const int pr2 = pair0 + line2;
  float2 res[A];

  // ---------------------------------------------------------- half -> real ---
  if constexpr (MODE == ROW_C2R || MODE == ROW_RT) {
    const float2* in = p.in_half + (int64_t)slot * p.in_stride;
    {
      float2 v[B];
#pragma unroll
      for (int b = 0; b < B; ++b) {
        const int n = a1 + A * b;
        float2 z = make_float2(0.f, 0.f);
        if (pr1 < npairs) {
          const int m = n <= H ? n : L - n;
          float2 ya = in[tm.at(2 * pr1, m)];
          float2 yb = in[tm.at(2 * pr1 + 1, m)];
          if (n > H) {
            ya = cconj(ya);
            yb = cconj(yb);
          }
          z = make_float2(ya.x - yb.y, ya.y + yb.x);  // ya + i yb
        }
        v[b] = z;
      }
      Dft<B, 1>::run(v);
#pragma unroll
      for (int kb = 1; kb < B; ++kb) v[kb] = ctw<1>(v[kb], tw[kb * A + a1]);
#pragma unroll
      for (int kb = 0; kb < B; ++kb) sm[line1 * LS + kb * (A + 1) + a1] = v[kb];
    }
    __syncthreads();
    const float thr = p.use_thr ? p.thr.v[slot] : 0.f;
    if (in2) {
#pragma unroll
      for (int aa = 0; aa < A; ++aa) res[aa] = sm[line2 * LS + kb2 * (A + 1) + aa];
      Dft<A, 1>::run(res);
#pragma unroll
      for (int ka = 0; ka < A; ++ka) {
        float c0 = res[ka].x * p.scale, c1 = res[ka].y * p.scale;
        if (p.use_thr == 2) {  // rows 2 pr2, 2 pr2 + 1, column kb2 + B ka
          const int st = (int)thr, k = kb2 + B * ka;
          if (!on_lattice(2 * pr2, k, st)) c0 = 0.f;
          if (!on_lattice(2 * pr2 + 1, k, st)) c1 = 0.f;
        } else if (p.use_thr) {
          if (fabsf(c0) < thr) c0 = 0.f;
          if (fabsf(c1) < thr) c1 = 0.f;
        }
        res[ka] = make_float2(c0, c1);
      }
    }
    if constexpr (MODE == ROW_C2R) {
      if (in2 && pr2 < npairs) {
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
    if (in2) {
#pragma unroll
      for (int ka = 0; ka < A; ++ka) sm[line2 * L + kb2 + B * ka] = res[ka];
    }
    __syncthreads();
  }

  // ---------------------------------------------------------- real -> half ---
  {
    float2 v[B];
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int n = a1 + A * b;
      if constexpr (MODE == ROW_R2C) {
        float2 z = make_float2(0.f, 0.f);
        if (pr1 < npairs) {
          const float* r0 = p.in_real + (int64_t)slot * p.in_stride + (int64_t)(2 * pr1) * L;
          z = make_float2(r0[n], r0[L + n]);
        }
        v[b] = z;
      } else {
        v[b] = sm[line1 * L + n];
      }
    }
    if constexpr (MODE == ROW_RT) __syncthreads();
    Dft<B, -1>::run(v);
#pragma unroll
    for (int kb = 1; kb < B; ++kb) v[kb] = ctw<-1>(v[kb], tw[kb * A + a1]);
#pragma unroll
    for (int kb = 0; kb < B; ++kb) sm[line1 * LS + kb * (A + 1) + a1] = v[kb];
  }
  __syncthreads();
  if (in2) {
#pragma unroll
    for (int aa = 0; aa < A; ++aa) res[aa] = sm[line2 * LS + kb2 * (A + 1) + aa];
    Dft<A, -1>::run(res);
  }
  __syncthreads();
  if (in2) {
#pragma unroll
    for (int ka = 0; ka < A; ++ka) sm[line2 * L + kb2 + B * ka] = res[ka];
  }
  __syncthreads();
  // Split Z = FFT(x0 + i x1) into the half spectra of x0 and x1.
  float2* out = p.out_half + (int64_t)slot * p.out_stride;
  constexpr int HP = H + 1;
  for (int it = tid; it < PAIRS * HP; it += T) {
    const int line = it / HP, k = it % HP;
    const int pr = pair0 + line;
    if (pr >= npairs) continue;
    const float2 z = sm[line * L + k];
    const float2 w = sm[line * L + (k == 0 ? 0 : L - k)];
    out[tm.at(2 * pr, k)] = make_float2(0.5f * (z.x + w.x), 0.5f * (z.y - w.y));
    out[tm.at(2 * pr + 1, k)] = make_float2(0.5f * (z.y + w.y), 0.5f * (w.x - z.x));
  }
}

// ------------------------------------------------------- pipelined row passes ---

// Row passes over many slots as a persistent, software-pipelined kernel: work item i
// is (slot i / G, row-pair group i % G) with G = n_rows / (2 PAIRS); CTA c takes items
// c, c + gridDim.x, ... and streams the next item's input rows into the other
// shared-memory stage with cp.async while it transforms the current one.
//   ROW_C2R: input tile-major half spectra (whole tile runs of NPp = ntiles*TC0 points
//            per row are copied), output real rows (* scale, optional threshold).
//   ROW_R2C: input real rows (one contiguous block per item), output tile-major half
//            spectra.
//   ROW_RT : C2R, threshold, R2C (input and output tile-major; may be in place).
template <int L, int MODE, int PAIRS>
struct RowPipe {
  static constexpr int A = Split<L>::A, B = Split<L>::B, T = PAIRS * A;
  static constexpr int LS = B * (A + 1);
  static constexpr int XB = PAIRS * LS * 8;  // exchange bytes (>= PAIRS * L * 8)
};

template <int L, int MODE, int PAIRS>
__global__ void __launch_bounds__(PAIRS * Split<L>::A, L >= 1024 ? 2 : SL_MINB_ROW)
    k_row_pipe(RowArgs p, int nslots, int NPp, int stage_bytes) {
  using RP = RowPipe<L, MODE, PAIRS>;
  constexpr int A = RP::A, B = RP::B, T = RP::T, LS = RP::LS;
  constexpr int H = L / 2;
  extern __shared__ __align__(16) unsigned char smraw[];
  unsigned char* stg = smraw;                                        // [2][stage_bytes]
  float2* sm = reinterpret_cast<float2*>(smraw + 2 * stage_bytes);  // exchange
  uint64_t* bars = reinterpret_cast<uint64_t*>(smraw + 2 * stage_bytes + RP::XB);  // [2]
  const int tid = threadIdx.x;
  const float2* tw = g_twiddle + twiddle_offset(L);
  const TileMap tm = p.tm;
  const int groups = p.n_rows / (2 * PAIRS);
  const int nitems = groups * nslots;
  const int a1 = tid % A, line1 = tid / A;
  const int kb2 = tid % B, line2 = tid / B;
  const bool in2 = tid < PAIRS * B;
  const int nrun = NPp / tm_tc(tm);  // tile runs per row

  // Stage layouts. R2C: the item's 2 PAIRS real rows, contiguous: one bulk copy,
  // completing on the stage's mbarrier. C2R / RT: the item's rows gathered from every
  // pencil tile (runs of TC elements) by 16-byte cp.async copies of all threads into
  // [row][NPp] (one bulk copy per run measured slower: 65 copies of 256 bytes per item
  // at 512^2).
  if (MODE == ROW_R2C && tid == 0) {
    mbar_init(bars);
    mbar_init(bars + 1);
    mbar_init_fence();
  }
  __syncthreads();
  BulkRing ring{bars};

  auto issue = [&](int item, int stage) {
    if (item < nitems) {
      const int slot = item / groups, r0 = (item % groups) * 2 * PAIRS;
      unsigned char* dst = stg + stage * stage_bytes;
      if constexpr (MODE == ROW_R2C) {
        if (tid == 0) {
          const float* src = p.in_real + (int64_t)slot * p.in_stride + (int64_t)r0 * L;
          fence_proxy_async();
          mbar_expect(bars + stage, 2 * PAIRS * L * 4);
          bulk_g2s(dst, src, 2 * PAIRS * L * 4, bars + stage);
        }
        ++ring.issued;
      } else {
        const float2* src = p.in_half + (int64_t)slot * p.in_stride;
        // tile run t of row r0 + rr is TC = 2^lg elements at ((t L0 + r0 + rr) << lg):
        // 2^(lg-1) chunks of 16 bytes; no divisions in the copy loop
        const int lgc = tm.lg - 1;
        const int per_row = nrun << lgc;
        for (int rr = 0; rr < 2 * PAIRS; ++rr) {
          const float2* srow = src + ((int64_t)(r0 + rr) << tm.lg);
          unsigned char* drow = dst + (int64_t)rr * NPp * 8;
          for (int c = tid; c < per_row; c += T) {
            const int t = c >> lgc, ch2 = 2 * (c & ((1 << lgc) - 1));
            cp_async16(drow + (((int64_t)t << tm.lg) + ch2) * 8,
                       srow + ((int64_t)t * tm.L0 << tm.lg) + ch2);
          }
        }
      }
    }
    if constexpr (MODE != ROW_R2C) cp_async_commit();
  };
  // wait for item k's stage (CTA-uniform; includes a CTA barrier)
  auto wait_stage = [&]() -> bool {
    if constexpr (MODE == ROW_R2C) {
      return ring.wait();
    } else {
      cp_async_wait<1>();
      __syncthreads();
      return true;
    }
  };

  // this thread's inter-pass twiddles are the same for every item
  float2 twr[B];
#pragma unroll
  for (int kb = 1; kb < B; ++kb) twr[kb] = tw[kb * A + a1];

  int item = blockIdx.x;
  issue(item, 0);
  issue(item + gridDim.x, 1);
  for (int k = 0; item < nitems; ++k, item += gridDim.x) {
    const int stage = k & 1;
    const int slot = item / groups, r0 = (item % groups) * 2 * PAIRS;
    if (!wait_stage()) {  // stage filled; previous item's exchange reads done
      ring.abandon();
      return;
    }
    float2 res[A];
    if constexpr (MODE == ROW_C2R || MODE == ROW_RT) {
      const float2* in = reinterpret_cast<const float2*>(stg + stage * stage_bytes);
      const float2* in0 = in + (2 * line1) * NPp;
      const float2* in1 = in0 + NPp;
      float2 v[B];
#pragma unroll
      for (int b = 0; b < B; ++b) {
        // n = a1 + A b with 0 <= a1 < A: below H for (b + 1) A <= H, above H for
        // b A > H (both known once the loop is unrolled); only one b straddles H
        const int n = a1 + A * b;
        float2 ya, yb;
        if ((b + 1) * A <= H) {
          ya = in0[n];
          yb = in1[n];
        } else if (b * A > H) {
          ya = cconj(in0[L - n]);
          yb = cconj(in1[L - n]);
        } else {
          const int m = n <= H ? n : L - n;
          ya = in0[m];
          yb = in1[m];
          if (n > H) {
            ya = cconj(ya);
            yb = cconj(yb);
          }
        }
        v[b] = make_float2(ya.x - yb.y, ya.y + yb.x);
      }
      Dft<B, 1>::run(v);
#pragma unroll
      for (int kb = 1; kb < B; ++kb) v[kb] = ctw<1>(v[kb], twr[kb]);
#pragma unroll
      for (int kb = 0; kb < B; ++kb) sm[line1 * LS + kb * (A + 1) + a1] = v[kb];
      __syncthreads();
      if constexpr (MODE == ROW_C2R) issue(item + 2 * gridDim.x, stage);
      const float thr = p.use_thr ? p.thr.v[slot] : 0.f;
      if (in2) {
#pragma unroll
        for (int aa = 0; aa < A; ++aa) res[aa] = sm[line2 * LS + kb2 * (A + 1) + aa];
        Dft<A, 1>::run(res);
        if (p.use_thr == 2) {  // lattice mask: rows r0 + 2 line2 (+1), column kb2 + B ka
          const int st = (int)thr, ra = r0 + 2 * line2;
#pragma unroll
          for (int ka = 0; ka < A; ++ka) {
            const int k = kb2 + B * ka;
            float c0 = res[ka].x * p.scale, c1 = res[ka].y * p.scale;
            if (!on_lattice(ra, k, st)) c0 = 0.f;
            if (!on_lattice(ra + 1, k, st)) c1 = 0.f;
            res[ka] = make_float2(c0, c1);
          }
        } else if (p.use_thr) {  // uniform branch: no per-value predication when unused
#pragma unroll
          for (int ka = 0; ka < A; ++ka) {
            float c0 = res[ka].x * p.scale, c1 = res[ka].y * p.scale;
            if (fabsf(c0) < thr) c0 = 0.f;
            if (fabsf(c1) < thr) c1 = 0.f;
            res[ka] = make_float2(c0, c1);
          }
        } else {
#pragma unroll
          for (int ka = 0; ka < A; ++ka) res[ka] = cscale(res[ka], p.scale);
        }
      }
      if constexpr (MODE == ROW_C2R) {
        if (in2) {
          float* o0 = p.out_real + (int64_t)slot * p.out_stride + (int64_t)(r0 + 2 * line2) * L;
#pragma unroll
          for (int ka = 0; ka < A; ++ka) {
            const int kk = kb2 + B * ka;
            o0[kk] = res[ka].x;
            o0[L + kk] = res[ka].y;
          }
        }
        __syncthreads();  // exchange reused by the next item
        continue;
      }
      __syncthreads();
      if (in2) {
#pragma unroll
        for (int ka = 0; ka < A; ++ka) sm[line2 * L + kb2 + B * ka] = res[ka];
      }
      __syncthreads();
    }
    // real rows -> half spectra
    {
      float2 v[B];
#pragma unroll
      for (int b = 0; b < B; ++b) {
        const int n = a1 + A * b;
        if constexpr (MODE == ROW_R2C) {
          const float* in = reinterpret_cast<const float*>(stg + stage * stage_bytes);
          v[b] = make_float2(in[(2 * line1) * L + n], in[(2 * line1 + 1) * L + n]);
        } else {
          v[b] = sm[line1 * L + n];
        }
      }
      __syncthreads();  // stage (R2C) or natural rows (RT) consumed
      issue(item + 2 * gridDim.x, stage);
      Dft<B, -1>::run(v);
#pragma unroll
      for (int kb = 1; kb < B; ++kb) v[kb] = ctw<-1>(v[kb], twr[kb]);
#pragma unroll
      for (int kb = 0; kb < B; ++kb) sm[line1 * LS + kb * (A + 1) + a1] = v[kb];
    }
    __syncthreads();
    if (in2) {
#pragma unroll
      for (int aa = 0; aa < A; ++aa) res[aa] = sm[line2 * LS + kb2 * (A + 1) + aa];
      Dft<A, -1>::run(res);
    }
    float2* out = p.out_half + (int64_t)slot * p.out_stride;
    const int tcs = tm_tc(tm);  // the two rows of a pair sit TC elements apart
    if constexpr (32 % B == 0 && (A & (A - 1)) == 0 && (PAIRS * B) % 32 == 0) {
      // Split Z = FFT(x0 + i x1) into the half spectra of x0 and x1 in registers: this
      // thread holds Z[k] for k = kb2 + B ka, and Z[L - k] sits in lane (B - kb2) mod B
      // of its B-lane group at index A - 1 - ka (or in this thread at (A - ka) mod A when
      // kb2 = 0). The in2 threads fill whole warps, so the shuffles are warp-uniform.
      if (in2) {
        const int lane = tid & 31;
        const int partner = (lane & ~(B - 1)) | ((B - kb2) & (B - 1));
        const int row = r0 + 2 * line2;
#pragma unroll
        for (int ka = 0; ka <= A / 2; ++ka) {
          const float2 far = res[A - 1 - ka];
          const float2 oth = make_float2(__shfl_sync(0xffffffffu, far.x, partner),
                                         __shfl_sync(0xffffffffu, far.y, partner));
          const float2 w = kb2 == 0 ? res[(A - ka) & (A - 1)] : oth;
          const float2 z = res[ka];
          if (ka < A / 2 || kb2 == 0) {  // k <= H
            float2* o = out + tm.at(row, kb2 + B * ka);
            o[0] = make_float2(0.5f * (z.x + w.x), 0.5f * (z.y - w.y));
            o[tcs] = make_float2(0.5f * (z.y + w.y), 0.5f * (w.x - z.x));
          }
        }
      }
      __syncthreads();  // exchange reused by the next item
      continue;
    }
    __syncthreads();
    if (in2) {
#pragma unroll
      for (int ka = 0; ka < A; ++ka) sm[line2 * L + kb2 + B * ka] = res[ka];
    }
    __syncthreads();
    // lines outer, points inner (no divisions)
#pragma unroll
    for (int line = 0; line < PAIRS; ++line) {
      const float2* zl = sm + line * L;
      for (int kk = tid; kk <= H; kk += T) {
        const float2 z = zl[kk];
        const float2 w = zl[kk == 0 ? 0 : L - kk];
        float2* o = out + tm.at(r0 + 2 * line, kk);
        o[0] = make_float2(0.5f * (z.x + w.x), 0.5f * (z.y - w.y));
        o[tcs] = make_float2(0.5f * (z.y + w.y), 0.5f * (w.x - z.x));
      }
    }
    __syncthreads();  // exchange reused by the next item
  }
  if constexpr (MODE != ROW_R2C) cp_async_wait<0>();
}

// Inverse filter pass (COL_INV_ACC) as a persistent pipelined kernel: work item i is
// (tile i % ntiles, split i / ntiles); the CTA streams the (Z_j tile, psi_j tile)
// pairs of its items' filters through two shared-memory stages (bulk copies) and
// accumulates psi_j * FFT_0(Z_j) in registers, writing one partial per item.
template <int L>
__global__ void __launch_bounds__(Geo<L>::T, SL_MINB_COLI) k_col_inv_pipe(ColArgs p) {
  using G = Geo<L>;
  constexpr int A = G::A, B = G::B, TC = G::TC, XS = G::XS;
  constexpr int TILE = L * TC;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* zs = reinterpret_cast<float2*>(smraw);        // [2][TILE]
  float* ps = reinterpret_cast<float*>(zs + 2 * TILE);  // [2][TILE]
  float2* ex = reinterpret_cast<float2*>(ps + 2 * TILE);
  uint64_t* bars = reinterpret_cast<uint64_t*>(ex + B * XS);  // [2]
  const int tid = threadIdx.x;
  const float2* tw = g_twiddle + twiddle_offset(L);
  const int ntiles = (int)(p.Nhp / TILE);
  const int nsplit = (p.nfilt + p.fps - 1) / p.fps;
  const int nitems = ntiles * nsplit;
  const int line = tid % TC, a = tid / TC;
  const int line2 = tid % TC, kb2 = tid / TC;
  const bool in2 = tid < TC * B;
  if (tid == 0) {
    mbar_init(bars);
    mbar_init(bars + 1);
    mbar_init_fence();
  }
  __syncthreads();
  BulkRing ring{bars};

  // the CTA's load sequence: (item, filter) pairs in order
  auto first_filter = [&](int item) { return (item / ntiles) * p.fps; };
  auto last_filter = [&](int item) { return min(first_filter(item) + p.fps, p.nfilt); };
  auto issue = [&](int item, int f, int stage) {
    if (item < nitems) {
      if (tid == 0) {
        const int tile = item % ntiles;
        fence_proxy_async();
        mbar_expect(bars + stage, TILE * 12);
        bulk_g2s(zs + stage * TILE, p.in + (int64_t)f * p.Nhp + (int64_t)tile * TILE, TILE * 8,
                 bars + stage);
        bulk_g2s(ps + stage * TILE, p.psi + (int64_t)(p.j0 + f) * p.Nhp + (int64_t)tile * TILE,
                 TILE * 4, bars + stage);
      }
      ++ring.issued;
    }
  };
  auto advance = [&](int& item, int& f) {
    if (++f >= last_filter(item)) {
      item += gridDim.x;
      f = item < nitems ? first_filter(item) : 0;
    }
  };

  int cur_item = blockIdx.x, cur_f = cur_item < nitems ? first_filter(cur_item) : 0;
  int pre_item = cur_item, pre_f = cur_f;  // next load to issue
  issue(pre_item, pre_f, 0);
  advance(pre_item, pre_f);
  issue(pre_item, pre_f, 1);
  advance(pre_item, pre_f);
  float2 acc[A];
#pragma unroll
  for (int i = 0; i < A; ++i) acc[i] = make_float2(0.f, 0.f);
  for (int k = 0; cur_item < nitems; ++k) {
    const int stage = k & 1;
    if (!ring.wait()) {  // stage filled; previous exchange reads done
      ring.abandon();
      return;
    }
    float2 v[B];
#pragma unroll
    for (int b = 0; b < B; ++b) v[b] = zs[stage * TILE + (a + A * b) * TC + line];
    Dft<B, -1>::run(v);
#pragma unroll
    for (int kb = 1; kb < B; ++kb) v[kb] = ctw<-1>(v[kb], tw[kb * A + a]);
#pragma unroll
    for (int kb = 0; kb < B; ++kb) ex[kb * XS + a * TC + line] = v[kb];
    __syncthreads();
    if (in2) {
      float2 w[A];
#pragma unroll
      for (int aa = 0; aa < A; ++aa) w[aa] = ex[kb2 * XS + aa * TC + line2];
      Dft<A, -1>::run(w);
#pragma unroll
      for (int ka = 0; ka < A; ++ka) {
        const float f = ps[stage * TILE + (kb2 + B * ka) * TC + line2];
        acc[ka].x = fmaf(f, w[ka].x, acc[ka].x);
        acc[ka].y = fmaf(f, w[ka].y, acc[ka].y);
      }
    }
    __syncthreads();  // stage and exchange consumed
    issue(pre_item, pre_f, stage);
    advance(pre_item, pre_f);
    const int done_item = cur_item;
    advance(cur_item, cur_f);
    if (cur_item != done_item) {  // item complete: write its partial
      if (in2) {
        const int tile = done_item % ntiles, split = done_item / ntiles;
        float2* o = p.out + (int64_t)(p.part0 + split) * p.Nhp + (int64_t)tile * TILE;
#pragma unroll
        for (int ka = 0; ka < A; ++ka) {
          o[(kb2 + B * ka) * TC + line2] = acc[ka];
          acc[ka] = make_float2(0.f, 0.f);
        }
      }
    }
  }
}

template <int L>
constexpr int col_inv_pipe_smem_bytes() {  // two stages, the exchange, two mbarriers
  return 2 * L * Geo<L>::TC * (8 + 4) + Geo<L>::B * Geo<L>::XS * 8 + 16;
}

// ------------------------------------------------------------ elementwise ---

// Error statistics of y against ref over n elements, accumulated in FP64:
// acc[0] = max |y - ref|, acc[1] = max |ref|, acc[2] = sum (y - ref)^2, acc[3] = sum ref^2.
// Maxima of non-negative doubles are ordered like their bit patterns.
__global__ void __launch_bounds__(256) k_error_stats(const float* __restrict__ y,
                                                     const float* __restrict__ ref, int64_t n,
                                                     double* __restrict__ acc) {
  double me = 0.0, mr = 0.0, se = 0.0, sr = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double r = ref[i], e = (double)y[i] - r;
    me = fmax(me, fabs(e));
    mr = fmax(mr, fabs(r));
    se += e * e;
    sr += r * r;
  }
  for (int o = 16; o > 0; o >>= 1) {
    me = fmax(me, __shfl_xor_sync(0xffffffffu, me, o));
    mr = fmax(mr, __shfl_xor_sync(0xffffffffu, mr, o));
    se += __shfl_xor_sync(0xffffffffu, se, o);
    sr += __shfl_xor_sync(0xffffffffu, sr, o);
  }
  __shared__ double red[4][8];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    red[0][w] = me;
    red[1][w] = mr;
    red[2][w] = se;
    red[3][w] = sr;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
      me = fmax(me, red[0][k]);
      mr = fmax(mr, red[1][k]);
      se += red[2][k];
      sr += red[3][k];
    }
    atomicMax(reinterpret_cast<unsigned long long*>(acc), (unsigned long long)__double_as_longlong(me));
    atomicMax(reinterpret_cast<unsigned long long*>(acc + 1),
              (unsigned long long)__double_as_longlong(mr));
    atomicAdd(acc + 2, se);
    atomicAdd(acc + 3, sr);
  }
}

// In-place hard threshold of nf consecutive coefficient arrays of n elements each.
__global__ void __launch_bounds__(256) k_threshold(float* c, int64_t n, int nf, Thresholds thr) {
  const int f = blockIdx.y;
  if (f >= nf) return;
  const float t = thr.v[f];
  float* base = c + (int64_t)f * n;
  const int64_t n4 = n / 4;
  float4* b4 = reinterpret_cast<float4*>(base);
  auto thr4 = [t](float4 v) {
    v.x = fabsf(v.x) < t ? 0.f : v.x;
    v.y = fabsf(v.y) < t ? 0.f : v.y;
    v.z = fabsf(v.z) < t ? 0.f : v.z;
    v.w = fabsf(v.w) < t ? 0.f : v.w;
    return v;
  };
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + 3 * stride < n4; i += 4 * stride) {  // four loads in flight per thread
    const float4 v0 = b4[i], v1 = b4[i + stride], v2 = b4[i + 2 * stride], v3 = b4[i + 3 * stride];
    b4[i] = thr4(v0);
    b4[i + stride] = thr4(v1);
    b4[i + 2 * stride] = thr4(v2);
    b4[i + 3 * stride] = thr4(v3);
  }
  for (; i < n4; i += stride) b4[i] = thr4(b4[i]);
  for (int64_t i = n4 * 4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    base[i] = fabsf(base[i]) < t ? 0.f : base[i];
}

// Inpainting step input: u = f + M (f_masked - f) with M = (mask != 0); f = 0 when
// f_cur is null (the first iteration). Four elements per thread and step.
__global__ void __launch_bounds__(256) k_inpaint_mix(const float* __restrict__ fm,
                                                     const uint8_t* __restrict__ mask,
                                                     const float* __restrict__ f_cur,
                                                     float* __restrict__ u, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; 4 * i < n; i += stride) {
    const int64_t e = 4 * i;
    if (e + 3 < n) {
      const float4 a = reinterpret_cast<const float4*>(fm)[i];
      const uchar4 m = reinterpret_cast<const uchar4*>(mask)[i];
      float4 f = make_float4(0.f, 0.f, 0.f, 0.f);
      if (f_cur) f = reinterpret_cast<const float4*>(f_cur)[i];
      reinterpret_cast<float4*>(u)[i] =
          make_float4(m.x ? a.x : f.x, m.y ? a.y : f.y, m.z ? a.z : f.z, m.w ? a.w : f.w);
    } else {
      for (int64_t k = e; k < n; ++k) {
        const float f = f_cur ? f_cur[k] : 0.f;
        u[k] = mask[k] ? fm[k] : f;
      }
    }
  }
}

// out = a - b over n elements (four per thread and step where aligned).
__global__ void __launch_bounds__(256) k_sub(const float* __restrict__ a, const float* __restrict__ b,
                                             float* __restrict__ out, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; 4 * i < n; i += stride) {
    const int64_t e = 4 * i;
    if (e + 3 < n) {
      const float4 u = reinterpret_cast<const float4*>(a)[i];
      const float4 v = reinterpret_cast<const float4*>(b)[i];
      reinterpret_cast<float4*>(out)[i] = make_float4(u.x - v.x, u.y - v.y, u.z - v.z, u.w - v.w);
    } else {
      for (int64_t k = e; k < n; ++k) out[k] = a[k] - b[k];
    }
  }
}

// ------------------------------------------------- subsampled transform ---
// Compact layout of subsampled coefficients: subband j keeps the points of the lattice
// (s_j Z)^2 of its [n0][n1] plane, row-major [n0 / s_j][n1 / s_j], at offset off[j].

struct SubPlan {
  const int* step;       // [R] lattice step s_j (a power of two)
  const int64_t* off;    // [R + 1] offsets into the compact array
};

// compact[off[j] + (i0 / s) (n1 / s) + i1 / s] = planes[j][i0][i1] on the lattice
// (GATHER), or planes[j] = 0 off the lattice and the compact value on it (SCATTER).
// blockIdx.y = j; threads stride over the plane's points.
template <bool GATHER>
__global__ void __launch_bounds__(256) k_sub_move(float* planes, float* compact, SubPlan sp,
                                                  int n0, int n1) {
  const int j = blockIdx.y, s = sp.step[j];
  const int64_t N = (int64_t)n0 * n1;
  float* pl = planes + (int64_t)j * N;
  float* cp = compact + sp.off[j];
  const int m1 = n1 / s;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i0 = (int)(e / n1), i1 = (int)(e % n1);
    const bool on = on_lattice(i0, i1, s);
    if constexpr (GATHER) {
      if (on) cp[(int64_t)(i0 / s) * m1 + i1 / s] = pl[e];
    } else {
      pl[e] = on ? cp[(int64_t)(i0 / s) * m1 + i1 / s] : 0.f;
    }
  }
}

// Deterministic FP64 dot product, stage 1: block b writes the sum of a[i] b[i] over its
// grid-stride indices (fixed order) to part[b].
__global__ void __launch_bounds__(256) k_dot_partial(const float* __restrict__ a,
                                                     const float* __restrict__ b, int64_t n,
                                                     double* __restrict__ part) {
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    acc += (double)a[i] * (double)b[i];
  __shared__ double red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// Stage 2 (one block of 256): out = sum of part[0, nparts) in a fixed order.
__global__ void __launch_bounds__(256) k_dot_final(const double* __restrict__ part, int nparts,
                                                   double* __restrict__ out) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int i = threadIdx.x; i < nparts; i += 256) acc += part[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

// Conjugate-gradient updates with the step sizes read from device scalars (no host
// round trip): alpha = num / den; x += alpha p; r -= alpha q (q = S p).
__global__ void __launch_bounds__(256) k_cg_xr(float* __restrict__ x, float* __restrict__ r,
                                               const float* __restrict__ p,
                                               const float* __restrict__ q,
                                               const double* __restrict__ num,
                                               const double* __restrict__ den, int64_t n) {
  const double d = *den;
  const float alpha = d != 0.0 ? (float)(*num / d) : 0.f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    x[i] = fmaf(alpha, p[i], x[i]);
    r[i] = fmaf(-alpha, q[i], r[i]);
  }
}

// p = z + beta p with beta = num / den (den the previous iteration's num).
__global__ void __launch_bounds__(256) k_cg_p(float* __restrict__ p, const float* __restrict__ z,
                                              const double* __restrict__ num,
                                              const double* __restrict__ den, int64_t n) {
  const double d = *den;
  const float beta = d != 0.0 ? (float)(*num / d) : 0.f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = fmaf(beta, p[i], z[i]);
}

}  // namespace dev
}  // namespace sl
