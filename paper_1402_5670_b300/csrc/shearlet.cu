// libshearlet: C ABI, bank management and launch orchestration.
// The kernels are in kernels2d.cuh (pencil and row passes) and kernels3d.cuh (plane
// passes); the FP64 filter construction is in bank_host.cpp.

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/shearlet.h"
#include "bank_host.h"
#include "kernels3d.cuh"
#include "kernels_cluster.cuh"
#include "kernels_tc.cuh"
#include "kernels_roww.cuh"

using sl::dev::ColArgs;
using sl::dev::RowArgs;
using sl::dev::Thresholds;
using sl::dev::kMaxGroup;
using sl::dev::kPlaneThreads;
using sl::dev::TileMap;

// ------------------------------------------------------------------ errors ---

static thread_local std::string g_last_error;

static sl_status fail(sl_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

static sl_status cuda_fail(cudaError_t e, const char* what) {
  return fail(SL_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define SL_CUDA(call)                                     \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);   \
  } while (0)

// --------------------------------------------------------------- profiling ---

namespace {
struct ProfKind {
  int64_t launches = 0;
  double ms = 0.0;
  double bytes = 0.0;  // algorithmic bytes of the launches read so far
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
  std::vector<double> pending_bytes;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::map<std::string, ProfKind> g_prof;
}  // namespace

// Algorithmic bytes of the next launch (the HBM traffic the transform needs in
// principle: image, coefficients, filters, 1/Psi), set by the orchestration code
// before each launch and recorded with it when profiling is on.
static thread_local double g_next_bytes = 0.0;

// Launch wrapper: records a pair of events around the launch when profiling is on.
template <typename F>
static cudaError_t timed_launch(const char* kind, cudaStream_t st, F&& f) {
  const double bytes = g_next_bytes;
  g_next_bytes = 0.0;
  if (!g_prof_on) {
    f();
    return cudaGetLastError();
  }
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  cudaEventRecord(a, st);
  f();
  cudaError_t e = cudaGetLastError();
  cudaEventRecord(b, st);
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof[kind].pending.emplace_back(a, b);
  g_prof[kind].pending_bytes.push_back(bytes);
  return e;
}

// ----------------------------------------------------- per-device one-time set-up ---

static std::mutex g_init_mu;
static bool g_dev_init[64] = {false};

static sl_status init_device(int dev) {
  std::lock_guard<std::mutex> lk(g_init_mu);
  if (dev < 0 || dev >= 64) return fail(SL_EINVAL, "device ordinal out of range");
  if (g_dev_init[dev]) return SL_OK;
  std::vector<float2> tw(sl::dev::kTwiddleTotal);
  for (int L : {8, 16, 32, 64, 128, 256, 512, 1024, 384, 192}) {
    int A = 0, B = 0;
    switch (L) {
      case 384: A = 24; B = 16; break;
      case 192: A = 16; B = 12; break;
      case 8: A = 4; B = 2; break;
      case 16: A = 4; B = 4; break;
      case 32: A = 8; B = 4; break;
      case 64: A = 8; B = 8; break;
      case 128: A = 16; B = 8; break;
      case 256: A = 16; B = 16; break;
      case 512: A = 32; B = 16; break;
      default: A = 32; B = 32; break;
    }
    for (int kb = 0; kb < B; ++kb)
      for (int a = 0; a < A; ++a) {
        const double ang = -2.0 * 3.14159265358979323846264338327950288 * (double)(a * kb) / L;
        tw[sl::dev::twiddle_offset(L) + kb * A + a] = make_float2((float)std::cos(ang),
                                                                  (float)std::sin(ang));
      }
  }
  SL_CUDA(cudaMemcpyToSymbol(sl::dev::g_twiddle, tw.data(), tw.size() * sizeof(float2)));
  // full tables exp(-2 pi i m / L), m < L, for the tensor-core stages (powers of two)
  std::vector<float2> wf(sl::dev::kTwiddleTotal, make_float2(0.f, 0.f));
  for (int L = 8; L <= 1024; L *= 2)
    for (int m = 0; m < L; ++m) {
      const double ang = -2.0 * 3.14159265358979323846264338327950288 * (double)m / L;
      wf[sl::dev::twiddle_offset(L) + m] = make_float2((float)std::cos(ang), (float)std::sin(ang));
    }
  SL_CUDA(cudaMemcpyToSymbol(sl::dev::g_wfull, wf.data(), wf.size() * sizeof(float2)));
  g_dev_init[dev] = true;
  return SL_OK;
}

// Dynamic shared memory above 48 KB has to be enabled per kernel and device.
template <typename K>
static cudaError_t ensure_smem(K kernel, int bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

// ------------------------------------------------------------ dispatchers ---

template <int L, int MODE>
static cudaError_t launch_col_t(dim3 grid, cudaStream_t st, const ColArgs& a) {
  auto k = sl::dev::k_col<L, MODE>;
  constexpr int smem = sl::dev::Geo<L>::smem_col;
  cudaError_t e = ensure_smem(k, smem);
  if (e != cudaSuccess) return e;
  static const char* names[4] = {"col_spec", "col_fwd_filter", "col_inv_accumulate",
                                 "col_ifft"};
  return timed_launch(names[MODE], st,
                      [&]() { k<<<grid, sl::dev::Geo<L>::T, smem, st>>>(a); });
}

template <int MODE>
static cudaError_t launch_col(int L, dim3 grid, cudaStream_t st, const ColArgs& a) {
  switch (L) {
    case 8: return launch_col_t<8, MODE>(grid, st, a);
    case 16: return launch_col_t<16, MODE>(grid, st, a);
    case 32: return launch_col_t<32, MODE>(grid, st, a);
    case 64: return launch_col_t<64, MODE>(grid, st, a);
    case 128: return launch_col_t<128, MODE>(grid, st, a);
    case 256: return launch_col_t<256, MODE>(grid, st, a);
    case 512: return launch_col_t<512, MODE>(grid, st, a);
    case 1024: return launch_col_t<1024, MODE>(grid, st, a);
    case 384: return launch_col_t<384, MODE>(grid, st, a);
    case 192: return launch_col_t<192, MODE>(grid, st, a);
    default: return cudaErrorInvalidValue;
  }
}

static int col_tile(int L) { return sl::dev::col_tile_of(L); }  // pencils per CTA

// Persistent pipelined forward filter pass: as many CTAs as fit on the device.
template <int L>
static cudaError_t launch_col_fwd_pipe_t(int nitems, cudaStream_t st, const ColArgs& a) {
  auto k = sl::dev::k_col_fwd_pipe<L>;
  constexpr int smem = sl::dev::col_pipe_smem_bytes<L>();
  cudaError_t e = ensure_smem(k, smem);
  if (e != cudaSuccess) return e;
  static int per_sm[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && per_sm[dev] == 0) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, sl::dev::Geo<L>::T, smem) != cudaSuccess)
      n = 1;
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    per_sm[dev] = std::max(1, n) * sms;
  }
  const int grid = std::min(nitems, per_sm[(dev >= 0 && dev < 64) ? dev : 0]);
  return timed_launch("col_fwd_filter", st,
                      [&]() { k<<<grid, sl::dev::Geo<L>::T, smem, st>>>(a); });
}

// CTAs of a persistent kernel: the device's SMs times the CTAs that fit on one.
template <typename K>
static int persistent_grid(K kernel, int threads, int smem, int kernel_id) {
  static std::mutex mu;
  static std::map<std::tuple<int, int, int>, int> cache;  // (device, kernel, smem)
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find({dev, kernel_id, smem});
  if (it != cache.end()) return it->second;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess) {
    cudaGetLastError();
    n = 1;
  }
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int g = std::max(1, n) * sms;
  cache[{dev, kernel_id, smem}] = g;
  return g;
}

template <int L, int MODE>
static cudaError_t launch_row_pipe_t(int slots, int L0, int NPp, cudaStream_t st,
                                     const RowArgs& a) {
  constexpr int PAIRS = sl::dev::col_tile_of(L);
  constexpr int T = PAIRS * sl::dev::Split<L>::A;
  auto k = sl::dev::k_row_pipe<L, MODE, PAIRS>;
  // two stages (the real rows, or the rows' half spectra), the exchange, two mbarriers
  const int stage = MODE == sl::dev::ROW_R2C ? 2 * PAIRS * L * 4 : 2 * PAIRS * NPp * 8;
  const int smem = 2 * stage + sl::dev::RowPipe<L, MODE, PAIRS>::XB + 16;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const int items = slots * (L0 / (2 * PAIRS));
  const int grid = std::min(items, persistent_grid(k, T, smem, 1000 * L + MODE));
  static const char* names[3] = {"row_r2c", "row_c2r", "row_roundtrip"};
  return timed_launch(names[MODE], st,
                      [&]() { k<<<grid, T, smem, st>>>(a, slots, NPp, stage); });
}

// Warp-pipelined row passes (kernels_roww.cuh) for rows of 512 and 1024 points; used
// for the single-signal passes (one warp per CTA: the few row pairs of one image
// spread over many SMs with both FFT passes on all lanes). For the filter loop the
// CTA-wide pipeline (k_row_pipe) measured as fast or faster on B300.
template <int L, int MODE, int W>
static cudaError_t launch_row_warp_t(int slots, int L0, int NPp, cudaStream_t st,
                                     const RowArgs& a) {
  constexpr int T = 32 * W;
  auto k = sl::dev::k_row_warp<L, MODE, W>;
  const int stage = MODE == sl::dev::ROW_R2C ? 2 * L * 4 : 2 * NPp * 8;
  const int smem = W * (2 * stage + sl::dev::roww_exchange_bytes<L>());
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const int items = slots * (L0 / 2);
  const int ctas = (items + W - 1) / W;
  const int grid = std::min(ctas, persistent_grid(k, T, smem, 6000 + 10 * L + 100 * W + MODE));
  static const char* names[3] = {"row_r2c", "row_c2r", "row_roundtrip"};
  static const char* names1[3] = {"row_r2c_signal", "row_c2r_signal", "row_roundtrip"};
  return timed_launch(slots == 1 ? names1[MODE] : names[MODE], st,
                      [&]() { k<<<grid, T, smem, st>>>(a, slots, NPp, stage); });
}

template <int MODE>
static cudaError_t launch_row_pipe(int L, int slots, int L0, int NPp, cudaStream_t st,
                                   const RowArgs& a) {
  switch (L) {
    case 8: return launch_row_pipe_t<8, MODE>(slots, L0, NPp, st, a);
    case 16: return launch_row_pipe_t<16, MODE>(slots, L0, NPp, st, a);
    case 32: return launch_row_pipe_t<32, MODE>(slots, L0, NPp, st, a);
    case 64: return launch_row_pipe_t<64, MODE>(slots, L0, NPp, st, a);
    case 128: return launch_row_pipe_t<128, MODE>(slots, L0, NPp, st, a);
    case 256: return launch_row_pipe_t<256, MODE>(slots, L0, NPp, st, a);
    case 512: return launch_row_pipe_t<512, MODE>(slots, L0, NPp, st, a);
    case 1024: return launch_row_pipe_t<1024, MODE>(slots, L0, NPp, st, a);
    case 384: return launch_row_pipe_t<384, MODE>(slots, L0, NPp, st, a);
    default: return cudaErrorInvalidValue;
  }
}

template <int L>
static cudaError_t launch_col_inv_pipe_t(int nitems, cudaStream_t st, const ColArgs& a) {
  auto k = sl::dev::k_col_inv_pipe<L>;
  constexpr int smem = sl::dev::col_inv_pipe_smem_bytes<L>();
  cudaError_t e = ensure_smem(k, smem);
  if (e != cudaSuccess) return e;
  const int grid = std::min(nitems, persistent_grid(k, sl::dev::Geo<L>::T, smem, 2000 + L));
  return timed_launch("col_inv_accumulate", st,
                      [&]() { k<<<grid, sl::dev::Geo<L>::T, smem, st>>>(a); });
}

static cudaError_t launch_col_inv_pipe(int L, int nitems, cudaStream_t st, const ColArgs& a) {
  switch (L) {
    case 8: return launch_col_inv_pipe_t<8>(nitems, st, a);
    case 16: return launch_col_inv_pipe_t<16>(nitems, st, a);
    case 32: return launch_col_inv_pipe_t<32>(nitems, st, a);
    case 64: return launch_col_inv_pipe_t<64>(nitems, st, a);
    case 128: return launch_col_inv_pipe_t<128>(nitems, st, a);
    case 256: return launch_col_inv_pipe_t<256>(nitems, st, a);
    case 512: return launch_col_inv_pipe_t<512>(nitems, st, a);
    case 1024: return launch_col_inv_pipe_t<1024>(nitems, st, a);
    case 384: return launch_col_inv_pipe_t<384>(nitems, st, a);
    case 192: return launch_col_inv_pipe_t<192>(nitems, st, a);
    default: return cudaErrorInvalidValue;
  }
}

static cudaError_t launch_col_fwd_pipe(int L, int nitems, cudaStream_t st, const ColArgs& a) {
  switch (L) {
    case 8: return launch_col_fwd_pipe_t<8>(nitems, st, a);
    case 16: return launch_col_fwd_pipe_t<16>(nitems, st, a);
    case 32: return launch_col_fwd_pipe_t<32>(nitems, st, a);
    case 64: return launch_col_fwd_pipe_t<64>(nitems, st, a);
    case 128: return launch_col_fwd_pipe_t<128>(nitems, st, a);
    case 256: return launch_col_fwd_pipe_t<256>(nitems, st, a);
    case 512: return launch_col_fwd_pipe_t<512>(nitems, st, a);
    case 1024: return launch_col_fwd_pipe_t<1024>(nitems, st, a);
    case 384: return launch_col_fwd_pipe_t<384>(nitems, st, a);
    case 192: return launch_col_fwd_pipe_t<192>(nitems, st, a);
    default: return cudaErrorInvalidValue;
  }
}

// Tensor-core (split BF16) pencil passes, persistent like the FP32 pipelines.
template <int L, int OP>
static cudaError_t launch_col_tc_t(bool fwd, int nitems, cudaStream_t st, const ColArgs& a) {
  constexpr int smem = sl::dev::tc_col_smem_bytes<L>();
  constexpr int T = sl::dev::kTcThreads;
  constexpr bool f16 = OP == sl::dev::TC_OP_F16;
  if (fwd) {
    auto k = sl::dev::k_col_fwd_tc<L, OP>;
    cudaError_t e = ensure_smem(k, smem);
    if (e != cudaSuccess) return e;
    const int grid = std::min(nitems, persistent_grid(k, T, smem, 3000 + 100 * OP + L));
    return timed_launch(f16 ? "col_fwd_filter_tc_f16" : "col_fwd_filter_tc", st,
                        [&]() { k<<<grid, T, smem, st>>>(a); });
  }
  auto k = sl::dev::k_col_inv_tc<L, OP>;
  cudaError_t e = ensure_smem(k, smem);
  if (e != cudaSuccess) return e;
  const int grid = std::min(nitems, persistent_grid(k, T, smem, 4000 + 100 * OP + L));
  return timed_launch(f16 ? "col_inv_accumulate_tc_f16" : "col_inv_accumulate_tc", st,
                      [&]() { k<<<grid, T, smem, st>>>(a); });
}

template <int OP>
static cudaError_t launch_col_tc_op(int L, bool fwd, int nitems, cudaStream_t st,
                                    const ColArgs& a) {
  switch (L) {
    case 64: return launch_col_tc_t<64, OP>(fwd, nitems, st, a);
    case 128: return launch_col_tc_t<128, OP>(fwd, nitems, st, a);
    case 256: return launch_col_tc_t<256, OP>(fwd, nitems, st, a);
    case 512: return launch_col_tc_t<512, OP>(fwd, nitems, st, a);
    case 1024: return launch_col_tc_t<1024, OP>(fwd, nitems, st, a);
    default: return cudaErrorInvalidValue;
  }
}

// prec: SL_PREC_TC_BF16 or SL_PREC_TC_FP16
static cudaError_t launch_col_tc(int L, int prec, bool fwd, int nitems, cudaStream_t st,
                                 const ColArgs& a) {
  return prec == SL_PREC_TC_FP16
             ? launch_col_tc_op<sl::dev::TC_OP_F16>(L, fwd, nitems, st, a)
             : launch_col_tc_op<sl::dev::TC_OP_BF16>(L, fwd, nitems, st, a);
}

// Row passes: PAIRS row pairs per CTA. Launches over many filters use the wide
// variant (col_tile_of(L) pairs); single-image launches use one pair per CTA so that
// the few rows of one image still spread over many SMs (rows of 512 and 1024 points:
// the one-warp kernel k_row_warp).
template <int L, int MODE, int PAIRS>
static cudaError_t launch_row_p(dim3 grid, cudaStream_t st, const RowArgs& a) {
  auto k = sl::dev::k_row<L, MODE, PAIRS>;
  constexpr int A = sl::dev::Split<L>::A, B = sl::dev::Split<L>::B;
  constexpr int smem = PAIRS * B * (A + 1) * (int)sizeof(float2);
  cudaError_t e = ensure_smem(k, smem);
  if (e != cudaSuccess) return e;
  // single-signal launches (one row pair per CTA) are reported apart from the
  // filter loop's launches
  static const char* names[3] = {"row_r2c", "row_c2r", "row_roundtrip"};
  static const char* names1[3] = {"row_r2c_signal", "row_c2r_signal", "row_roundtrip"};
  return timed_launch(PAIRS == 1 ? names1[MODE] : names[MODE], st,
                      [&]() { k<<<grid, PAIRS * A, smem, st>>>(a); });
}

template <int L, int MODE>
static cudaError_t launch_row_t(int slots, int L0, int NPp, cudaStream_t st, const RowArgs& a) {
  constexpr int W = sl::dev::col_tile_of(L);
  if constexpr (L == 512 || L == 1024) {
    // one row pair per one-warp CTA, both passes on all 32 lanes
    if (slots == 1 && MODE != sl::dev::ROW_RT)
      return launch_row_warp_t<L, MODE, 1>(1, L0, NPp, st, a);
  }
  if (slots == 1) return launch_row_p<L, MODE, 1>(dim3(L0 / 2, 1), st, a);
  return launch_row_p<L, MODE, W>(dim3((L0 / 2 + W - 1) / W, slots), st, a);
}

template <int MODE>
static cudaError_t launch_row(int L, int slots, int L0, int NPp, cudaStream_t st,
                              const RowArgs& a) {
  switch (L) {
    case 8: return launch_row_t<8, MODE>(slots, L0, NPp, st, a);
    case 16: return launch_row_t<16, MODE>(slots, L0, NPp, st, a);
    case 32: return launch_row_t<32, MODE>(slots, L0, NPp, st, a);
    case 64: return launch_row_t<64, MODE>(slots, L0, NPp, st, a);
    case 128: return launch_row_t<128, MODE>(slots, L0, NPp, st, a);
    case 256: return launch_row_t<256, MODE>(slots, L0, NPp, st, a);
    case 512: return launch_row_t<512, MODE>(slots, L0, NPp, st, a);
    case 1024: return launch_row_t<1024, MODE>(slots, L0, NPp, st, a);
    case 384: return launch_row_t<384, MODE>(slots, L0, NPp, st, a);
    default: return cudaErrorInvalidValue;
  }
}

template <int L1, int L2, int MODE>
static cudaError_t launch_plane_t(dim3 grid, cudaStream_t st, const RowArgs& a) {
  auto k = sl::dev::k_plane<L1, L2, MODE>;
  constexpr int smem = sl::dev::PlaneGeom<L1, L2>::bytes;
  cudaError_t e = ensure_smem(k, smem);
  if (e != cudaSuccess) return e;
  // persistent: grid.x planes x grid.y slots of work, as many CTAs as fit
  const int nslots = (int)grid.y, items = (int)grid.x * nslots;
  const int g = std::min(items, persistent_grid(k, kPlaneThreads, smem, 7000 + 1000 * MODE + 10 * L1 + L2 / 8));
  static const char* names[3] = {"plane_r2c", "plane_c2r", "plane_roundtrip"};
  return timed_launch(names[MODE], st,
                      [&]() { k<<<g, kPlaneThreads, smem, st>>>(a, nslots); });
}

template <int L1, int MODE>
static cudaError_t launch_plane_l2(int L2, dim3 grid, cudaStream_t st, const RowArgs& a) {
  switch (L2) {
    case 8: return launch_plane_t<L1, 8, MODE>(grid, st, a);
    case 16: return launch_plane_t<L1, 16, MODE>(grid, st, a);
    case 32: return launch_plane_t<L1, 32, MODE>(grid, st, a);
    case 64: return launch_plane_t<L1, 64, MODE>(grid, st, a);
    case 128: return launch_plane_t<L1, 128, MODE>(grid, st, a);
    default: return cudaErrorInvalidValue;
  }
}

// 192 x 192 planes: one plane per CTA (no double buffering), one CTA per SM.
template <int MODE>
static cudaError_t launch_plane_big(int slots, cudaStream_t st, const RowArgs& a) {
  auto k = sl::dev::k_plane_big<192, MODE>;
  constexpr int smem = sl::dev::BigPlane<192>::bytes;
  cudaError_t e = ensure_smem(k, smem);
  if (e != cudaSuccess) return e;
  const int items = slots * a.n_rows;
  const int grid = std::min(items, persistent_grid(k, sl::dev::kBigThreads, smem, 90000 + MODE));
  static const char* names[3] = {"plane_r2c", "plane_c2r", "plane_roundtrip"};
  return timed_launch(names[MODE], st,
                      [&]() { k<<<grid, sl::dev::kBigThreads, smem, st>>>(a, slots); });
}

template <int MODE>
static cudaError_t launch_plane(int L1, int L2, dim3 grid, cudaStream_t st, const RowArgs& a) {
  if (L1 == 192 && L2 == 192) return launch_plane_big<MODE>((int)grid.y, st, a);
  switch (L1) {
    case 8: return launch_plane_l2<8, MODE>(L2, grid, st, a);
    case 16: return launch_plane_l2<16, MODE>(L2, grid, st, a);
    case 32: return launch_plane_l2<32, MODE>(L2, grid, st, a);
    case 64: return launch_plane_l2<64, MODE>(L2, grid, st, a);
    case 128: return launch_plane_l2<128, MODE>(L2, grid, st, a);
    default: return cudaErrorInvalidValue;
  }
}

// ------------------------------------------------------- cluster-fused 2D ---

using sl::dev::ClArgs;
using sl::dev::ClGeo;

template <int L0, int L1>
static cudaError_t cl_fwd_launch(int ncl, cudaStream_t st, const ClArgs& a) {
  auto k = sl::dev::k_cl_fwd<L0, L1>;
  constexpr int smem = ClGeo<L0, L1>::smem;
  cudaError_t e = ensure_smem(k, smem);
  if (e != cudaSuccess) return e;
  return timed_launch(a.psi ? "cluster_fwd_filters" : "cluster_c2r", st, [&]() {
    k<<<ncl * sl::dev::kCluster, ClGeo<L0, L1>::NT, smem, st>>>(a);
  });
}

template <int L0, int L1>
static cudaError_t cl_inv_launch(int ncl, cudaStream_t st, const ClArgs& a) {
  auto k = sl::dev::k_cl_inv<L0, L1>;
  constexpr int smem = ClGeo<L0, L1>::smem;
  cudaError_t e = ensure_smem(k, smem);
  if (e != cudaSuccess) return e;
  return timed_launch(a.psi ? "cluster_inv_filters" : "cluster_r2c", st, [&]() {
    k<<<ncl * sl::dev::kCluster, ClGeo<L0, L1>::NT, smem, st>>>(a);
  });
}

// How many 8-CTA clusters of this kernel can be resident at once.
template <int L0, int L1>
static int cl_max_clusters() {
  int best = 1 << 30;
  for (int which = 0; which < 2; ++which) {
    const void* k = which ? (const void*)sl::dev::k_cl_inv<L0, L1>
                          : (const void*)sl::dev::k_cl_fwd<L0, L1>;
    constexpr int smem = ClGeo<L0, L1>::smem;
    if (which) ensure_smem(sl::dev::k_cl_inv<L0, L1>, smem);
    else ensure_smem(sl::dev::k_cl_fwd<L0, L1>, smem);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(sl::dev::kCluster * 64, 1, 1);
    cfg.blockDim = dim3(ClGeo<L0, L1>::NT, 1, 1);
    cfg.dynamicSmemBytes = smem;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k, &cfg) != cudaSuccess) {
      cudaGetLastError();
      n = 0;
    }
    best = std::min(best, n);
  }
  return best;
}

struct ClEntry {
  int L0, L1;
  cudaError_t (*fwd)(int, cudaStream_t, const ClArgs&);
  cudaError_t (*inv)(int, cudaStream_t, const ClArgs&);
  int (*max_clusters)();
  int CW, TOTAL;
};

#define SL_CL(a, b) \
  {a, b, &cl_fwd_launch<a, b>, &cl_inv_launch<a, b>, &cl_max_clusters<a, b>, ClGeo<a, b>::CW, ClGeo<a, b>::TOTAL}
static const ClEntry kClTable[] = {
    SL_CL(64, 64),   SL_CL(64, 128),  SL_CL(64, 256),  SL_CL(64, 512),
    SL_CL(128, 64),  SL_CL(128, 128), SL_CL(128, 256), SL_CL(128, 512),
    SL_CL(256, 64),  SL_CL(256, 128), SL_CL(256, 256), SL_CL(256, 512),
    SL_CL(512, 64),  SL_CL(512, 128), SL_CL(512, 256), SL_CL(512, 512),
};
#undef SL_CL

static const ClEntry* cl_entry(const sl::BankSpec& s) {
  if (s.ndim != 2) return nullptr;
  for (const ClEntry& e : kClTable)
    if (e.L0 == s.dims[0] && e.L1 == s.dims[1]) return &e;
  return nullptr;
}

// ------------------------------------------------------------------- bank ---

struct sl_bank {
  sl::BankSpec spec;
  std::vector<sl::FilterDesc> filt;
  std::vector<double> norms;
  double A = 0.0, B = 0.0, scale = 1.0;
  int device = -1;
  int R = 0;
  int64_t N = 0, Nh = 0;
  int NP = 0;       // pencils per spectrum (Nh / n0)
  int TC = 1, lgTC = 0, ntiles = 0;
  int64_t Nhp = 0;  // elements of one tile-major (padded) spectrum
  int G = 1;        // filters per group
  int ngroups = 1;
  int S = 1;        // partials per group
  int fps = 1;      // filters per partial
  int prec = 0;     // SL_PREC_FP32, or SL_PREC_TC_BF16 / _FP16 (pencil passes on tensor cores)
  float* psi = nullptr;       // [R][Nhp] tile-major
  double* invPsi = nullptr;   // [Nhp] tile-major
  float2* xhat = nullptr;     // [Nhp] spectrum of the signal
  float2* scratch = nullptr;  // [G][Nhp]
  float2* partial = nullptr;  // [ngroups * S][Nhp]
  // cluster-fused 2D path (cl != nullptr): cluster-tiled filters and spectra
  const ClEntry* cl = nullptr;
  int ncl = 0;                // clusters of the filter passes
  float* psi_cl = nullptr;    // [R][TOTAL]
  double* invPsi_cl = nullptr;
  float2* xhat_cl = nullptr;  // [TOTAL]
  float2* part_cl = nullptr;  // [ncl][TOTAL]
  float* inp_u = nullptr;     // sl_inpaint's iterate input (allocated on first use)
  // subsampled transform (allocated on first use): lattice steps and compact offsets,
  // a full coefficient stack, the conjugate-gradient vectors and scalars, and the
  // preconditioner 1 / Psi_sub (FP64, tile-major)
  std::vector<int> sub_step;
  std::vector<int64_t> sub_off;
  int* d_sub_step = nullptr;
  int64_t* d_sub_off = nullptr;
  float* sub_C = nullptr;     // [R][N]
  float* cg = nullptr;        // [5][N]: x-free work vectors r, p, q, z, b
  double* cg_dot = nullptr;   // [kDotParts] partial sums, then 8 scalars
  double* invPsi_sub = nullptr;
  float* e2e_x = nullptr;     // sl_fwdinv_host buffers (allocated on first use)
  float* e2e_c = nullptr;
  cudaStream_t e2e_cap = nullptr;         // sl_fwdinv_host: capture stream, graph and the
  cudaGraphExec_t e2e_graph = nullptr;    // host pointers it was captured with
  const void* e2e_key[2] = {nullptr, nullptr};
  std::unique_ptr<sl::BankEvaluator> ev;
};

static bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

static void free_device(sl_bank* b) {
  cudaFree(b->psi);
  cudaFree(b->invPsi);
  cudaFree(b->xhat);
  cudaFree(b->scratch);
  cudaFree(b->partial);
  cudaFree(b->e2e_x);
  cudaFree(b->e2e_c);
  cudaFree(b->inp_u);
  b->inp_u = nullptr;
  cudaFree(b->d_sub_step);
  cudaFree(b->d_sub_off);
  cudaFree(b->sub_C);
  cudaFree(b->cg);
  cudaFree(b->cg_dot);
  cudaFree(b->invPsi_sub);
  b->d_sub_step = nullptr;
  b->d_sub_off = nullptr;
  b->sub_C = b->cg = nullptr;
  b->cg_dot = b->invPsi_sub = nullptr;
  if (b->e2e_graph) cudaGraphExecDestroy(b->e2e_graph);
  if (b->e2e_cap) cudaStreamDestroy(b->e2e_cap);
  b->e2e_graph = nullptr;
  b->e2e_cap = nullptr;
  cudaFree(b->psi_cl);
  cudaFree(b->invPsi_cl);
  cudaFree(b->xhat_cl);
  cudaFree(b->part_cl);
  b->psi_cl = nullptr;
  b->invPsi_cl = nullptr;
  b->xhat_cl = b->part_cl = nullptr;
  b->psi = nullptr;
  b->invPsi = nullptr;
  b->xhat = b->scratch = b->partial = nullptr;
  b->e2e_x = b->e2e_c = nullptr;
}

// Grouping: the per-filter intermediate spectra of one group stay resident in L2
// between the two passes of a transform; a group holds as many filters as fit in
// the scratch budget (environment variable SL_SCRATCH_MB, default 256 MB).
static void plan_groups(sl_bank* b) {
  // Default budget for the per-filter intermediates: 256 MB holds all 49 spectra of
  // a 1024^2 four-scale system, so the filter loop runs as one group (fewer, larger
  // launches; measured fastest on B300 for every 2D size from 256^2 to 1024^2).
  double mb = 256.0;
  if (const char* s = std::getenv("SL_SCRATCH_MB")) mb = std::max(1.0, std::atof(s));
  const double per = (double)b->Nhp * sizeof(float2);
  int gmax = (int)std::max(1.0, std::floor(mb * 1024.0 * 1024.0 / per));
  gmax = std::min(gmax, kMaxGroup);
  b->ngroups = (b->R + gmax - 1) / gmax;
  b->G = (b->R + b->ngroups - 1) / b->ngroups;
  // pencil tiles of the inverse accumulation; split filters so that the grid holds
  // about four small CTAs per SM (148 SMs on B300), with at least 2 filters per split.
  const int tiles = b->ntiles;
  int want = std::max(1, (4 * 148 + tiles - 1) / tiles);
  b->fps = std::max(2, (b->G + want - 1) / want);
  b->S = (b->G + b->fps - 1) / b->fps;
}

// Natural half spectrum [n0][NP] -> tile-major [ntiles][n0][TC] (pads untouched).
template <typename T>
static void tile_major(const sl_bank* b, const T* nat, T* tiled) {
  const int L0 = (int)b->spec.dims[0];
  for (int k0 = 0; k0 < L0; ++k0)
    for (int p = 0; p < b->NP; ++p)
      tiled[(((int64_t)(p >> b->lgTC) * L0 + k0) << b->lgTC) + (p & (b->TC - 1))] =
          nat[(int64_t)k0 * b->NP + p];
}

// Natural half spectrum [n0][NH] -> cluster-tiled [8][n0][CW] (pads untouched).
template <typename T>
static void cluster_tiled(const sl_bank* b, const T* nat, T* ct) {
  const int L0 = (int)b->spec.dims[0];
  const int NH = (int)b->NP, CW = b->cl->CW;
  for (int k0 = 0; k0 < L0; ++k0)
    for (int c = 0; c < NH; ++c)
      ct[(int64_t)(c / CW) * L0 * CW + (int64_t)k0 * CW + c % CW] = nat[(int64_t)k0 * NH + c];
}

extern "C" {

const char* sl_status_str(sl_status s) {
  switch (s) {
    case SL_OK: return "SL_OK";
    case SL_EINVAL: return "SL_EINVAL";
    case SL_ENOMEM: return "SL_ENOMEM";
    case SL_ECUDA: return "SL_ECUDA";
    case SL_ETIMEOUT: return "SL_ETIMEOUT";
    case SL_ENOTSUP: return "SL_ENOTSUP";
    case SL_ENAN: return "SL_ENAN";
  }
  return "SL_UNKNOWN";
}

const char* sl_last_error(void) { return g_last_error.c_str(); }

sl_status sl_build_filters(int ndim, const int64_t* dims, int nScales, const int* shearLevels,
                           int fullSystem, int device, sl_bank** out) {
  return sl_build_filters_ex(ndim, dims, nScales, shearLevels, fullSystem, device, nullptr, out);
}

sl_status sl_build_filters_ex(int ndim, const int64_t* dims, int nScales, const int* shearLevels,
                              int fullSystem, int device, const sl_options* opt, sl_bank** out) {
  return sl_build_filters_user(ndim, dims, nScales, shearLevels, fullSystem, device, opt, nullptr,
                               out);
}

static sl_status build_filters_impl(int kind, int ndim, const int64_t* dims, int nScales,
                                    const int* shearLevels, int fullSystem, int device,
                                    const sl_options* opt, const sl_filters* filters,
                                    sl_bank** out);

sl_status sl_build_filters_user(int ndim, const int64_t* dims, int nScales, const int* shearLevels,
                                int fullSystem, int device, const sl_options* opt,
                                const sl_filters* filters, sl_bank** out) {
  return build_filters_impl(sl::kShearlets, ndim, dims, nScales, shearLevels, fullSystem, device,
                            opt, filters, out);
}

sl_status sl_build_wavelets(int ndim, const int64_t* dims, int nScales, int device,
                            const sl_filters* filters, sl_bank** out) {
  if (ndim != 2) return fail(ndim == 3 ? SL_ENOTSUP : SL_EINVAL, "wavelet banks are 2D");
  if (filters && filters->fan) return fail(SL_EINVAL, "a wavelet bank takes no fan filter");
  const int zeros[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  return build_filters_impl(sl::kWavelets, ndim, dims, nScales, zeros, 0, device, nullptr,
                            filters, out);
}

}  // extern "C"

static sl_status build_filters_impl(int kind, int ndim, const int64_t* dims, int nScales,
                                    const int* shearLevels, int fullSystem, int device,
                                    const sl_options* opt, const sl_filters* filters,
                                    sl_bank** out) {
  if (!out) return fail(SL_EINVAL, "out is NULL");
  *out = nullptr;
  std::shared_ptr<sl::FilterDesign> design;
  if (filters && (filters->qmf || filters->fan)) {
    design = std::make_shared<sl::FilterDesign>();
    if (filters->qmf) {
      if (filters->qmf_len < 1) return fail(SL_EINVAL, "qmf_len must be >= 1");
      design->h.assign(filters->qmf, filters->qmf + filters->qmf_len);
    }
    if (filters->fan) {
      if (filters->fan_rows < 1 || filters->fan_cols < 1)
        return fail(SL_EINVAL, "fan_rows and fan_cols must be >= 1");
      design->pr = filters->fan_rows;
      design->pc = filters->fan_cols;
      design->p.assign(filters->fan, filters->fan + (size_t)design->pr * design->pc);
    }
    const std::string why = sl::check_design(*design);
    if (!why.empty()) return fail(SL_EINVAL, why);
  }
  const int path = opt ? opt->path : SL_PATH_AUTO;
  if (path < SL_PATH_AUTO || path > SL_PATH_CLUSTER) return fail(SL_EINVAL, "unknown path");
  const int prec = opt ? opt->precision : SL_PREC_FP32;
  if (prec != SL_PREC_FP32 && prec != SL_PREC_TC_BF16 && prec != SL_PREC_TC_FP16)
    return fail(SL_EINVAL, "unknown precision");
  if (ndim != 2 && ndim != 3) return fail(SL_EINVAL, "ndim must be 2 or 3");
  if (!dims || !shearLevels) return fail(SL_EINVAL, "dims or shearLevels is NULL");
  if (nScales < 1 || nScales > 8) return fail(SL_EINVAL, "nScales must be in [1, 8]");
  sl::BankSpec spec;
  spec.design = design;
  spec.kind = kind;
  spec.ndim = ndim;
  spec.J = nScales;
  spec.full = fullSystem != 0;
  for (int i = 0; i < ndim; ++i) {
    if (dims[i] < 8) return fail(SL_EINVAL, "every dimension must be >= 8");
    const bool ok = (is_pow2(dims[i]) && dims[i] <= 1024) || (ndim == 2 && dims[i] == 384) ||
                    (ndim == 3 && dims[i] == 192);
    if (!ok)
      return fail(SL_ENOTSUP,
                  "dimensions must be powers of two in [8, 1024] (2D: or 384; 3D: or 192)");
    spec.dims[i] = dims[i];
  }
  for (int j = 0; j < nScales; ++j) {
    if (shearLevels[j] < 0 || shearLevels[j] > 4)
      return fail(SL_EINVAL, "shearLevels entries must be in [0, 4]");
    spec.d[j] = shearLevels[j];
  }
  if (ndim == 3) {
    const bool big = dims[1] == 192 && dims[2] == 192;  // one plane buffer per CTA
    if (!big && (dims[1] > 128 || dims[2] > 128 || dims[1] == 192 || dims[2] == 192))
      return fail(SL_ENOTSUP, "3D: axes 1 and 2 must be powers of two up to 128, or both 192");
  }
  if (prec != SL_PREC_FP32) {
    if (path == SL_PATH_CLUSTER)
      return fail(SL_ENOTSUP, "tensor-core precision runs on the general path only");
    if (!is_pow2(dims[0]) || dims[0] < 64)
      return fail(SL_ENOTSUP, "tensor-core pencil passes need n0 a power of two in [64, 1024]");
  }
  const int64_t N = spec.N(), Nh = spec.Nh();
  if (N > ((int64_t)1 << 31)) return fail(SL_ENOTSUP, "grid too large");
  std::unique_ptr<sl_bank> b(new sl_bank());
  b->prec = prec;
  b->spec = spec;
  b->device = device;
  b->N = N;
  b->Nh = Nh;
  b->NP = (int)(Nh / spec.dims[0]);
  b->TC = col_tile((int)spec.dims[0]);
  while ((1 << b->lgTC) < b->TC) ++b->lgTC;
  b->ntiles = (b->NP + b->TC - 1) / b->TC;
  b->Nhp = spec.dims[0] * (int64_t)b->ntiles * b->TC;

  sl::HostBank hb;
  std::string err;
  if (!sl::build_host_bank(spec, device >= 0, &hb, &err)) return fail(SL_EINVAL, err);
  b->filt = hb.filt;
  b->R = (int)hb.filt.size();
  b->norms = hb.norms;
  b->A = hb.A;
  b->B = hb.B;
  b->scale = hb.scale;
  b->ev.reset(new sl::BankEvaluator(spec));

  if (device >= 0) {
    int ndev = 0;
    SL_CUDA(cudaGetDeviceCount(&ndev));
    if (device >= ndev) return fail(SL_EINVAL, "no such CUDA device");
    SL_CUDA(cudaSetDevice(device));
    sl_status st = init_device(device);
    if (st != SL_OK) return st;
    plan_groups(b.get());
    auto alloc = [&](void** p, size_t bytes) -> bool {
      return cudaMalloc(p, bytes) == cudaSuccess;
    };
    const int64_t Nhp = b->Nhp;
    if (!alloc((void**)&b->psi, (size_t)b->R * Nhp * sizeof(float)) ||
        !alloc((void**)&b->invPsi, (size_t)Nhp * sizeof(double)) ||
        !alloc((void**)&b->xhat, (size_t)Nhp * sizeof(float2)) ||
        !alloc((void**)&b->scratch, (size_t)b->G * Nhp * sizeof(float2)) ||
        !alloc((void**)&b->partial, (size_t)b->ngroups * b->S * Nhp * sizeof(float2))) {
      cudaGetLastError();
      free_device(b.get());
      return fail(SL_ENOMEM, "device allocation failed");
    }
    // the spectra's pad pencils must hold zeros (see kernels2d.cuh)
    cudaError_t e = cudaMemset(b->xhat, 0, (size_t)Nhp * sizeof(float2));
    if (e == cudaSuccess) e = cudaMemset(b->scratch, 0, (size_t)b->G * Nhp * sizeof(float2));
    if (e == cudaSuccess)
      e = cudaMemset(b->partial, 0, (size_t)b->ngroups * b->S * Nhp * sizeof(float2));
    // filters and 1/Psi in the tile-major layout, zeros in the pads
    {
      std::vector<float> tiled((size_t)Nhp, 0.0f);
      for (int j = 0; j < b->R && e == cudaSuccess; ++j) {
        tile_major(b.get(), hb.psi32.data() + (size_t)j * Nh, tiled.data());
        e = cudaMemcpy(b->psi + (size_t)j * Nhp, tiled.data(), (size_t)Nhp * sizeof(float),
                       cudaMemcpyHostToDevice);
      }
      std::vector<double> ip((size_t)Nhp, 0.0);
      tile_major(b.get(), hb.invPsi.data(), ip.data());
      if (e == cudaSuccess)
        e = cudaMemcpy(b->invPsi, ip.data(), (size_t)Nhp * sizeof(double),
                       cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
      free_device(b.get());
      return cuda_fail(e, "uploading the filter bank");
    }
    // cluster-fused 2D path
    const ClEntry* ce = cl_entry(spec);
    if (path == SL_PATH_CLUSTER && !ce) {
      free_device(b.get());
      return fail(SL_ENOTSUP, "the cluster path covers 2D grids with both sides in [64, 512]");
    }
    // SL_PATH_AUTO takes the general path: on B300 it measures faster than the
    // cluster-fused kernels for every size the cluster path covers.
    if (path == SL_PATH_CLUSTER && ce) {
      const int maxcl = ce->max_clusters();
      if (maxcl < 1) {
        if (path == SL_PATH_CLUSTER) {
          free_device(b.get());
          return fail(SL_ENOTSUP, "no 8-CTA cluster of the fused kernels fits on this device");
        }
      } else {
        b->cl = ce;
        b->ncl = std::min(maxcl, b->R);
        const int64_t T = ce->TOTAL;
        if (!alloc((void**)&b->psi_cl, (size_t)b->R * T * sizeof(float)) ||
            !alloc((void**)&b->invPsi_cl, (size_t)T * sizeof(double)) ||
            !alloc((void**)&b->xhat_cl, (size_t)T * sizeof(float2)) ||
            !alloc((void**)&b->part_cl, (size_t)b->ncl * T * sizeof(float2))) {
          cudaGetLastError();
          free_device(b.get());
          return fail(SL_ENOMEM, "device allocation failed (cluster path)");
        }
        std::vector<float> ct((size_t)T, 0.0f);
        for (int j = 0; j < b->R && e == cudaSuccess; ++j) {
          cluster_tiled(b.get(), hb.psi32.data() + (size_t)j * Nh, ct.data());
          e = cudaMemcpy(b->psi_cl + (size_t)j * T, ct.data(), (size_t)T * sizeof(float),
                         cudaMemcpyHostToDevice);
        }
        std::vector<double> ip((size_t)T, 0.0);
        cluster_tiled(b.get(), hb.invPsi.data(), ip.data());
        if (e == cudaSuccess)
          e = cudaMemcpy(b->invPsi_cl, ip.data(), (size_t)T * sizeof(double),
                         cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemset(b->xhat_cl, 0, (size_t)T * sizeof(float2));
        if (e != cudaSuccess) {
          free_device(b.get());
          return cuda_fail(e, "uploading the cluster-tiled filter bank");
        }
      }
    }
  }
  *out = b.release();
  return SL_OK;
}

extern "C" {

void sl_free_filters(sl_bank* bank) {
  if (!bank) return;
  if (bank->device >= 0) {
    int cur = -1;
    cudaGetDevice(&cur);
    cudaSetDevice(bank->device);
    free_device(bank);
    if (cur >= 0) cudaSetDevice(cur);
  }
  delete bank;
}

sl_status sl_bank_info(const sl_bank* b, int* ndim, int64_t* dims, int* R, int* nScales) {
  if (!b) return fail(SL_EINVAL, "bank is NULL");
  if (ndim) *ndim = b->spec.ndim;
  if (dims)
    for (int i = 0; i < 3; ++i) dims[i] = i < b->spec.ndim ? b->spec.dims[i] : 1;
  if (R) *R = b->R;
  if (nScales) *nScales = b->spec.J;
  return SL_OK;
}

sl_status sl_bank_filter_meta(const sl_bank* b, int* scale_of, int* cone_of, int* k_of) {
  if (!b) return fail(SL_EINVAL, "bank is NULL");
  for (int j = 0; j < b->R; ++j) {
    if (scale_of) scale_of[j] = b->filt[j].scale;
    if (cone_of) cone_of[j] = b->filt[j].cone;
    if (k_of) {
      k_of[2 * j] = b->filt[j].k1;
      k_of[2 * j + 1] = b->filt[j].k2;
    }
  }
  return SL_OK;
}

sl_status sl_bank_norms(const sl_bank* b, double* norms, double* A, double* B) {
  if (!b) return fail(SL_EINVAL, "bank is NULL");
  if (norms) std::memcpy(norms, b->norms.data(), b->R * sizeof(double));
  if (A) *A = b->A;
  if (B) *B = b->B;
  return SL_OK;
}

sl_status sl_bank_path(const sl_bank* b, int* path) {
  if (!b || !path) return fail(SL_EINVAL, "bank or path is NULL");
  *path = b->cl ? SL_PATH_CLUSTER : SL_PATH_GENERAL;
  return SL_OK;
}

sl_status sl_bank_precision(const sl_bank* b, int* precision) {
  if (!b || !precision) return fail(SL_EINVAL, "NULL argument");
  *precision = b->prec;
  return SL_OK;
}

sl_status sl_bank_sizes(const sl_bank* b, int64_t* N, int64_t* Nh) {
  if (!b) return fail(SL_EINVAL, "bank is NULL");
  if (N) *N = b->N;
  if (Nh) *Nh = b->Nh;
  return SL_OK;
}

sl_status sl_bank_eval_f64(const sl_bank* b, int j, double* out) {
  if (!b || !out) return fail(SL_EINVAL, "bank or out is NULL");
  if (j < -1 || j >= b->R) return fail(SL_EINVAL, "filter index out of range");
  if (j >= 0) {
    b->ev->eval(j, out);
    for (int64_t i = 0; i < b->Nh; ++i) out[i] *= b->scale;
    return SL_OK;
  }
  std::vector<double> v(b->Nh);
  std::fill(out, out + b->Nh, 0.0);
  for (int f = 0; f < b->R; ++f) {
    b->ev->eval(f, v.data());
    for (int64_t i = 0; i < b->Nh; ++i) out[i] += v[i] * v[i];
  }
  const double s2 = b->scale * b->scale;
  for (int64_t i = 0; i < b->Nh; ++i) out[i] *= s2;
  return SL_OK;
}

sl_status sl_bank_filters_f32(const sl_bank* b, float* out) {
  if (!b || !out) return fail(SL_EINVAL, "bank or out is NULL");
  if (b->device < 0) return fail(SL_EINVAL, "host-only bank has no device filters");
  std::vector<float> tiled((size_t)b->Nhp);
  for (int j = 0; j < b->R; ++j) {
    SL_CUDA(cudaMemcpy(tiled.data(), b->psi + (size_t)j * b->Nhp, (size_t)b->Nhp * sizeof(float),
                       cudaMemcpyDeviceToHost));
    float* dst = out + (size_t)j * b->Nh;
    const int L0 = (int)b->spec.dims[0];
    for (int k0 = 0; k0 < L0; ++k0)
      for (int pp = 0; pp < b->NP; ++pp)
        dst[(int64_t)k0 * b->NP + pp] =
            tiled[(((int64_t)(pp >> b->lgTC) * L0 + k0) << b->lgTC) + (pp & (b->TC - 1))];
  }
  return SL_OK;
}

}  // extern "C"

// --------------------------------------------------------------- transforms ---

// Device arrays are read and written with 16-byte vector and asynchronous copies.
static bool a16(const void* p) { return ((uintptr_t)p & 15u) == 0; }
static sl_status check_aligned(const void* p, const void* q) {
  if (!a16(p) || !a16(q)) return fail(SL_EINVAL, "device arrays must be 16-byte aligned");
  return SL_OK;
}

static sl_status check_call(const sl_bank* b) {
  if (!b) return fail(SL_EINVAL, "bank is NULL");
  if (b->device < 0) return fail(SL_EINVAL, "host-only bank (built with device = -1)");
  int cur = -1;
  SL_CUDA(cudaGetDevice(&cur));
  if (cur != b->device) return fail(SL_EINVAL, "current CUDA device differs from the bank's");
  return SL_OK;
}

static sl_status launched(cudaError_t e, const char* what) {
  if (e != cudaSuccess) return cuda_fail(e, what);
  return SL_OK;
}

#define SL_TRY(expr)                  \
  do {                                \
    sl_status s_ = (expr);            \
    if (s_ != SL_OK) return s_;       \
  } while (0)

// Everything one transform call needs: geometry, filters and the scratch spectra.
// Built from a bank (its own scratch) or for sl_forward_noalloc (static scratch).
struct Plan {
  const sl::BankSpec* spec;
  int64_t N, Nh, Nhp;
  int NP, TC, lgTC, ntiles, R;
  int G, ngroups, S, fps;
  const float* psi;   // tile-major [R][Nhp], or natural [R][Nh] when psi_natural
  int psi_natural;
  int prec;           // != 0: pencil passes of the filter loops on the tensor cores
  const double* invPsi;
  float2* xhat;       // [Nhp]
  float2* scratch;    // [G][Nhp]
  float2* partial;    // [ngroups * S][Nhp]
  const sl_bank* bank;
};

static Plan plan_of(const sl_bank* b) {
  Plan p{};
  p.spec = &b->spec;
  p.N = b->N;
  p.Nh = b->Nh;
  p.Nhp = b->Nhp;
  p.NP = b->NP;
  p.TC = b->TC;
  p.lgTC = b->lgTC;
  p.ntiles = b->ntiles;
  p.R = b->R;
  p.G = b->G;
  p.ngroups = b->ngroups;
  p.S = b->S;
  p.fps = b->fps;
  p.psi = b->psi;
  p.psi_natural = 0;
  p.prec = b->prec;
  p.invPsi = b->invPsi;
  p.xhat = b->xhat;
  p.scratch = b->scratch;
  p.partial = b->partial;
  p.bank = b;
  return p;
}

static TileMap tilemap(const Plan& P) { return TileMap{(int)P.spec->dims[0], P.lgTC}; }

// Last-axes pass (2D rows / 3D planes) over `slots` spectra.
template <int MODE>
static sl_status last_axes(const Plan& P, RowArgs& ra, int slots, cudaStream_t st) {
  const sl::BankSpec& s = *P.spec;
  const int L0 = (int)s.dims[0];
  ra.n_rows = L0;
  ra.tm = tilemap(P);
  if (s.ndim == 2) {
    const int pairs = sl::dev::col_tile_of((int)s.dims[1]);
    if (slots > 1 && L0 / 2 >= pairs && (L0 / 2) % pairs == 0)
      return launched(launch_row_pipe<MODE>((int)s.dims[1], slots, L0, P.ntiles * P.TC, st, ra),
                      "row pass");
    return launched(launch_row<MODE>((int)s.dims[1], slots, L0, P.ntiles * P.TC, st, ra),
                    "row pass");
  }
  return launched(launch_plane<MODE>((int)s.dims[1], (int)s.dims[2], dim3(L0, slots), st, ra),
                  "plane pass");
}

// Real signal x[dims] -> spectrum P.xhat (last axes, then pencils in place).
static sl_status spectrum_of(const Plan& P, const float* x, cudaStream_t st) {
  RowArgs ra{};
  ra.in_real = x;
  ra.out_half = P.xhat;
  ra.scale = 1.f;
  g_next_bytes = 4.0 * P.N;  // the signal is read once
  SL_TRY(last_axes<sl::dev::ROW_R2C>(P, ra, 1, st));
  ColArgs ca{};
  ca.in = P.xhat;
  ca.out = P.xhat;
  ca.Nhp = P.Nhp;
  ca.NP = P.NP;
  return launched(launch_col<sl::dev::COL_SPEC>((int)P.spec->dims[0], dim3(P.ntiles, 1), st, ca),
                  "col_spec");
}

// Per-filter last-axes pass of one group: ROW_C2R (coefficients out), ROW_R2C
// (coefficients in) or ROW_RT (scratch in place, thresholded). creal_in / creal_out
// address the plane of the group's first filter.
template <int MODE>
static sl_status slab_pass(const Plan& P, int nf, const float* creal_in, float* creal_out,
                           const Thresholds* thr, cudaStream_t st, int thr_mode = 1) {
  RowArgs ra{};
  ra.scale = (float)(1.0 / (double)P.N);
  if (thr) {
    ra.use_thr = thr_mode;
    ra.thr = *thr;
  }
  if (MODE == sl::dev::ROW_C2R) {
    ra.in_half = P.scratch;
    ra.in_stride = P.Nhp;
    ra.out_real = creal_out;
    ra.out_stride = P.N;
  } else if (MODE == sl::dev::ROW_R2C) {
    ra.in_real = creal_in;
    ra.in_stride = P.N;
    ra.out_half = P.scratch;
    ra.out_stride = P.Nhp;
  } else {
    ra.in_half = P.scratch;
    ra.in_stride = P.Nhp;
    ra.out_half = P.scratch;
    ra.out_stride = P.Nhp;
  }
  // coefficients written (C2R) or read (R2C); none for the fused round trip
  g_next_bytes = MODE == sl::dev::ROW_RT ? 0.0 : 4.0 * (double)P.N * nf;
  return last_axes<MODE>(P, ra, nf, st);
}

static sl_status fwd_filter_pass(const Plan& P, int j0, int nf, cudaStream_t st) {
  ColArgs ca{};
  ca.in = P.xhat;
  ca.out = P.scratch;
  ca.psi = P.psi;
  ca.psi_natural = P.psi_natural;
  ca.Nhp = P.Nhp;
  ca.Nh = P.Nh;
  ca.NP = P.NP;
  ca.j0 = j0;
  ca.nfilt = nf;
  g_next_bytes = 4.0 * (double)P.Nh * nf;  // filters read
  if (P.prec && !P.psi_natural)
    return launched(launch_col_tc((int)P.spec->dims[0], P.prec, true, P.ntiles * nf, st, ca),
                    "col_fwd_filter_tc");
  if (!P.psi_natural)
    return launched(launch_col_fwd_pipe((int)P.spec->dims[0], P.ntiles * nf, st, ca),
                    "col_fwd_filter");
  return launched(launch_col<sl::dev::COL_FWD_FILT>((int)P.spec->dims[0], dim3(P.ntiles, nf), st,
                                                    ca),
                  "col_fwd_filter");
}

static sl_status inv_acc_pass(const Plan& P, int g_idx, int j0, int nf, cudaStream_t st) {
  ColArgs ca{};
  ca.in = P.scratch;
  ca.out = P.partial;
  ca.psi = P.psi;
  ca.Nhp = P.Nhp;
  ca.NP = P.NP;
  ca.j0 = j0;
  ca.nfilt = nf;
  ca.fps = P.fps;
  ca.part0 = g_idx * P.S;
  const int splits = (nf + P.fps - 1) / P.fps;
  g_next_bytes = 4.0 * (double)P.Nh * nf;  // filters read
  if (P.prec)
    return launched(launch_col_tc((int)P.spec->dims[0], P.prec, false, P.ntiles * splits, st, ca),
                    "col_inv_accumulate_tc");
  return launched(launch_col_inv_pipe((int)P.spec->dims[0], P.ntiles * splits, st, ca),
                  "col_inv_accumulate");
}

// out = (sum of the spectra parts[0, nparts), `stride` elements apart) times 1/Psi in
// FP64 when use_invpsi: one tile-major spectrum.
static sl_status reduce_spectra(const Plan& P, const float2* parts, int nparts, int64_t stride,
                                bool use_invpsi, float2* out, cudaStream_t st) {
  const int64_t n = P.Nhp;
  const int grid = (int)std::min<int64_t>((n / 2 + 255) / 256, 4 * 148);
  const double* w = use_invpsi ? P.invPsi : nullptr;
  g_next_bytes = use_invpsi ? 8.0 * (double)P.Nh : 0.0;  // 1/Psi read
  return launched(timed_launch("reduce_partials", st, [&]() {
                    sl::dev::k_reduce_parts<<<grid, 256, 0, st>>>(parts, nparts, stride, w, out, n);
                  }),
                  "reduce_partials");
}

// Spectrum P.xhat -> inverse FFT along the pencils -> last axes -> real x.
static sl_status spectrum_to_signal(const Plan& P, float* x, cudaStream_t st) {
  ColArgs ca{};
  ca.in = P.xhat;
  ca.out = P.xhat;
  ca.Nhp = P.Nhp;
  ca.NP = P.NP;
  SL_TRY(launched(launch_col<sl::dev::COL_IFFT>((int)P.spec->dims[0], dim3(P.ntiles, 1), st, ca),
                  "col_ifft"));
  RowArgs ra{};
  ra.in_half = P.xhat;
  ra.out_real = x;
  ra.scale = (float)(1.0 / (double)P.N);
  g_next_bytes = 4.0 * (double)P.N;  // the signal is written once
  return last_axes<sl::dev::ROW_C2R>(P, ra, 1, st);
}

// Spectra parts[0, nparts) -> (sum, times 1/Psi in FP64 for the inverse) -> inverse
// FFT along the pencils -> last axes -> real x.
static sl_status parts_to_signal(const Plan& P, const float2* parts, int nparts,
                                 bool use_invpsi, float* x, cudaStream_t st) {
  SL_TRY(reduce_spectra(P, parts, nparts, P.Nhp, use_invpsi, P.xhat, st));
  return spectrum_to_signal(P, x, st);
}

static sl_status inv_final(const Plan& P, int nparts, bool use_invpsi, float* x,
                           cudaStream_t st) {
  return parts_to_signal(P, P.partial, nparts, use_invpsi, x, st);
}

// Partials are written compactly: group g uses parts [g*S, g*S + splits_g). Every
// group but the last holds G filters and so uses all S of its parts; the used parts
// are therefore the contiguous range [0, parts_used).
static int parts_used(const Plan& P, int nfilters) {
  if (nfilters <= 0) return 0;
  const int ng = (nfilters + P.G - 1) / P.G;
  const int last = nfilters - (ng - 1) * P.G;
  return (ng - 1) * P.S + (last + P.fps - 1) / P.fps;
}
static int parts_used(const Plan& P) { return parts_used(P, P.R); }

static void fill_thresholds(const sl_bank* b, int j0, int nf, float sigma, const float* K,
                            Thresholds* t) {
  for (int i = 0; i < nf; ++i) {
    const sl::FilterDesc& f = b->filt[j0 + i];
    t->v[i] = f.scale < 0 ? 0.f : (float)((double)K[f.scale] * (double)sigma * b->norms[j0 + i]);
  }
}

// Filters [j0, j1) from the spectrum P.xhat: coeffs holds their planes [j1 - j0][dims].
static sl_status forward_filters(const Plan& P, int j0, int j1, float* coeffs, cudaStream_t st) {
  for (int j = j0; j < j1; j += P.G) {
    const int nf = std::min(P.G, j1 - j);
    SL_TRY(fwd_filter_pass(P, j, nf, st));
    SL_TRY(slab_pass<sl::dev::ROW_C2R>(P, nf, nullptr, coeffs + (int64_t)(j - j0) * P.N, nullptr, st));
  }
  return SL_OK;
}

static sl_status forward_plan(const Plan& P, const float* x, float* coeffs, cudaStream_t st) {
  SL_TRY(spectrum_of(P, x, st));
  return forward_filters(P, 0, P.R, coeffs, st);
}

// sum_{j in [j0, j1)} psi_hat_j FFT(C_j) as partial spectra [0, parts_used(P, j1 - j0))
// in P.partial; coeffs holds the planes [j1 - j0][dims].
static sl_status backward_filters(const Plan& P, const float* coeffs, int j0, int j1,
                                  cudaStream_t st) {
  for (int j = j0, g = 0; j < j1; j += P.G, ++g) {
    const int nf = std::min(P.G, j1 - j);
    SL_TRY(slab_pass<sl::dev::ROW_R2C>(P, nf, coeffs + (int64_t)(j - j0) * P.N, nullptr, nullptr, st));
    SL_TRY(inv_acc_pass(P, g, j, nf, st));
  }
  return SL_OK;
}

static sl_status backward(const Plan& P, const float* coeffs, float* x, bool use_invpsi,
                          cudaStream_t st) {
  SL_TRY(backward_filters(P, coeffs, 0, P.R, st));
  return inv_final(P, parts_used(P), use_invpsi, x, st);
}

// Fused denoise: per group, filter, C2R + threshold + R2C in shared memory, accumulate.
// lowpass_thr: threshold of the lowpass subband (0 keeps it whole, as the denoising rule
// does; +infinity drops it).
static sl_status denoise_plan(const Plan& P, const float* noisy, float* out, float sigma,
                              const float* K, cudaStream_t st, float lowpass_thr = 0.f) {
  SL_TRY(spectrum_of(P, noisy, st));
  for (int g = 0; g < P.ngroups; ++g) {
    const int j0 = g * P.G;
    const int nf = std::min(P.G, P.R - j0);
    Thresholds t;
    fill_thresholds(P.bank, j0, nf, sigma, K, &t);
    for (int i = 0; i < nf; ++i)
      if (P.bank->filt[j0 + i].scale < 0) t.v[i] = lowpass_thr;
    SL_TRY(fwd_filter_pass(P, j0, nf, st));
    SL_TRY(slab_pass<sl::dev::ROW_RT>(P, nf, nullptr, nullptr, &t, st));
    SL_TRY(inv_acc_pass(P, g, j0, nf, st));
  }
  return inv_final(P, parts_used(P), true, out, st);
}

// ---------------------------------------------------- subsampled transform ---
// The subsampled digital shearlet transform (Def. digitSH_alpha with sampling
// matrices): subband j is kept on the lattice (s_j Z)^2. Reading: s_j = 2^(J-1-j) for
// scale j (coarse to fine, so the finest scale keeps every point) and 2^(J-1) for the
// lowpass: each subband is sampled at the rate its passband allows. Its adjoint
// scatters the lattice values back (zeros elsewhere). The inverse solves
// S x = T_sub* c, S = T_sub* T_sub, by conjugate gradients (Sec. 3.4 and the frame
// algorithms of Sec. 2.1), preconditioned with the diagonal (in frequency) operator
// 1 / Psi_sub, Psi_sub = sum_j |psi_hat_j|^2 / s_j^2: the frame weight with each
// subband's sampling density, which is exactly S when every s_j = 1.

constexpr int kDotParts = 296;  // two blocks per SM of a B300

static void sub_plan_of(const sl_bank* b, std::vector<int>* step, std::vector<int64_t>* off) {
  const int J = b->spec.J;
  step->assign(b->R, 1);
  off->assign(b->R + 1, 0);
  for (int j = 0; j < b->R; ++j) {
    const int sc = b->filt[j].scale;
    (*step)[j] = sc < 0 ? (1 << (J - 1)) : (1 << std::max(0, J - 1 - sc));
    const int64_t sj = (*step)[j];
    (*off)[j + 1] = (*off)[j] + (b->spec.dims[0] / sj) * (b->spec.dims[1] / sj);
  }
}

static sl_status ensure_sub(sl_bank* b) {
  if (b->spec.ndim != 2) return fail(SL_ENOTSUP, "the subsampled transform is 2D only");
  if (b->cg) return SL_OK;
  sub_plan_of(b, &b->sub_step, &b->sub_off);
  for (int j = 0; j < b->R; ++j)
    if (b->spec.dims[0] % b->sub_step[j] || b->spec.dims[1] % b->sub_step[j])
      return fail(SL_ENOTSUP, "grid sides must be multiples of every lattice step 2^(J-1)");
  const int64_t N = b->N, Nh = b->Nh;
  // 1 / Psi_sub on the half spectrum, FP64, from the normalised filters
  std::vector<double> acc((size_t)Nh, 0.0), f((size_t)Nh);
  for (int j = 0; j < b->R; ++j) {
    b->ev->eval(j, f.data());
    const double w = b->scale * b->scale / ((double)b->sub_step[j] * b->sub_step[j]);
    for (int64_t i = 0; i < Nh; ++i) acc[i] += w * f[i] * f[i];
  }
  for (int64_t i = 0; i < Nh; ++i) {
    if (!(acc[i] > 0.0)) return fail(SL_EINVAL, "the subsampled frame weight vanishes");
    acc[i] = 1.0 / acc[i];
  }
  std::vector<double> tiled((size_t)b->Nhp, 0.0);
  tile_major(b, acc.data(), tiled.data());
  auto bail = [&](const char* what) {
    cudaGetLastError();
    cudaFree(b->d_sub_step);
    cudaFree(b->d_sub_off);
    cudaFree(b->sub_C);
    cudaFree(b->cg);
    cudaFree(b->cg_dot);
    cudaFree(b->invPsi_sub);
    b->d_sub_step = nullptr;
    b->d_sub_off = nullptr;
    b->sub_C = b->cg = nullptr;
    b->cg_dot = b->invPsi_sub = nullptr;
    return fail(SL_ENOMEM, what);
  };
  if (cudaMalloc((void**)&b->d_sub_step, b->R * sizeof(int)) != cudaSuccess ||
      cudaMalloc((void**)&b->d_sub_off, (b->R + 1) * sizeof(int64_t)) != cudaSuccess ||
      cudaMalloc((void**)&b->sub_C, (size_t)b->R * N * sizeof(float)) != cudaSuccess ||
      cudaMalloc((void**)&b->cg_dot, (kDotParts + 8) * sizeof(double)) != cudaSuccess ||
      cudaMalloc((void**)&b->invPsi_sub, (size_t)b->Nhp * sizeof(double)) != cudaSuccess ||
      cudaMalloc((void**)&b->cg, 5 * (size_t)N * sizeof(float)) != cudaSuccess)
    return bail("allocating the subsampled transform's buffers");
  if (cudaMemcpy(b->d_sub_step, b->sub_step.data(), b->R * sizeof(int), cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemcpy(b->d_sub_off, b->sub_off.data(), (b->R + 1) * sizeof(int64_t),
                 cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->invPsi_sub, tiled.data(), tiled.size() * sizeof(double),
                 cudaMemcpyHostToDevice) != cudaSuccess)
    return bail("uploading the subsampled transform's tables");
  return SL_OK;
}

static sl_status sub_move(const sl_bank* b, bool gather, float* planes, float* compact,
                          cudaStream_t st) {
  sl::dev::SubPlan sp{b->d_sub_step, b->d_sub_off};
  const int n0 = (int)b->spec.dims[0], n1 = (int)b->spec.dims[1];
  dim3 grid((unsigned)std::min<int64_t>((b->N + 255) / 256, 64), (unsigned)b->R);
  return launched(timed_launch(gather ? "sub_gather" : "sub_scatter", st, [&]() {
                    if (gather)
                      sl::dev::k_sub_move<true><<<grid, 256, 0, st>>>(planes, compact, sp, n0, n1);
                    else
                      sl::dev::k_sub_move<false><<<grid, 256, 0, st>>>(planes, compact, sp, n0, n1);
                  }),
                  "subsample move");
}

// *out = <a, b> over n floats, FP64, deterministic.
static sl_status dot(const sl_bank* b, const float* x, const float* y, double* out,
                     cudaStream_t st) {
  const int64_t n = b->N;
  double* part = b->cg_dot;
  SL_TRY(launched(timed_launch("cg_dot", st, [&]() {
                    sl::dev::k_dot_partial<<<kDotParts, 256, 0, st>>>(x, y, n, part);
                    sl::dev::k_dot_final<<<1, 256, 0, st>>>(part, kDotParts, out);
                  }),
                  "cg_dot"));
  return SL_OK;
}

// q = S p = T_sub* T_sub p: one fused pass (forward, lattice mask, adjoint) with the
// coefficients never leaving the chip.
static sl_status sub_frame_op(const Plan& P, const float* p, float* q, cudaStream_t st) {
  const sl_bank* b = P.bank;
  SL_TRY(spectrum_of(P, p, st));
  for (int g = 0; g < P.ngroups; ++g) {
    const int j0 = g * P.G;
    const int nf = std::min(P.G, P.R - j0);
    Thresholds t;
    for (int i = 0; i < nf; ++i) t.v[i] = (float)b->sub_step[j0 + i];
    SL_TRY(fwd_filter_pass(P, j0, nf, st));
    SL_TRY(slab_pass<sl::dev::ROW_RT>(P, nf, nullptr, nullptr, &t, st, 2));
    SL_TRY(inv_acc_pass(P, g, j0, nf, st));
  }
  return inv_final(P, parts_used(P), false, q, st);
}

// z = IFFT(FFT(r) / Psi_sub): the preconditioner.
static sl_status sub_precondition(const Plan& P, const float* r, float* z, cudaStream_t st) {
  SL_TRY(spectrum_of(P, r, st));
  const int64_t n = P.Nhp;
  const int grid = (int)std::min<int64_t>((n / 2 + 255) / 256, 4 * 148);
  const double* w = P.bank->invPsi_sub;
  float2* xh = P.xhat;
  SL_TRY(launched(timed_launch("cg_precondition", st, [&]() {
                    sl::dev::k_reduce_parts<<<grid, 256, 0, st>>>(xh, 1, n, w, xh, n);
                  }),
                  "cg_precondition"));
  return spectrum_to_signal(P, z, st);
}

// ------------------------------------------------- cluster-fused orchestration ---// ------------------------------------------------- cluster-fused orchestration ---

// x -> spectrum (one cluster) -> per filter C2R (all clusters).
static sl_status cl_forward(const sl_bank* b, const float* x, float* coeffs, cudaStream_t st) {
  ClArgs a{};
  a.in_real = x;
  a.out_spec = b->xhat_cl;
  a.R = 1;
  g_next_bytes = 4.0 * b->N;  // the signal is read once
  SL_TRY(launched(b->cl->inv(1, st, a), "cluster_r2c"));
  ClArgs f{};
  f.xhat = b->xhat_cl;
  f.psi = b->psi_cl;
  f.out_real = coeffs;
  f.R = b->R;
  f.scale = (float)(1.0 / (double)b->N);
  g_next_bytes = 4.0 * (double)b->R * (b->N + b->Nh);  // filters read, coefficients written
  return launched(b->cl->fwd(b->ncl, st, f), "cluster_fwd_filters");
}

// coefficients -> per-cluster partial sums -> (sum, * 1/Psi) -> C2R (one cluster).
static sl_status cl_backward(const sl_bank* b, const float* coeffs, float* x, bool use_invpsi,
                             cudaStream_t st) {
  ClArgs a{};
  a.in_real = coeffs;
  a.psi = b->psi_cl;
  a.out_spec = b->part_cl;
  a.R = b->R;
  g_next_bytes = 4.0 * (double)b->R * (b->N + b->Nh);  // coefficients and filters read
  SL_TRY(launched(b->cl->inv(b->ncl, st, a), "cluster_inv_filters"));
  const int64_t T = b->cl->TOTAL;
  const int grid = (int)std::min<int64_t>((T + 255) / 256, 4 * 148);
  const float2* parts = b->part_cl;
  const int np = b->ncl;
  const double* w = use_invpsi ? b->invPsi_cl : nullptr;
  float2* out = b->xhat_cl;
  g_next_bytes = use_invpsi ? 8.0 * (double)b->Nh : 0.0;  // 1/Psi read
  SL_TRY(launched(timed_launch("reduce_partials", st, [&]() {
                    sl::dev::k_cl_reduce<<<grid, 256, 0, st>>>(parts, np, T, w, out);
                  }),
                  "reduce_partials"));
  ClArgs f{};
  f.xhat = b->xhat_cl;
  f.out_real = x;
  f.R = 1;
  f.scale = (float)(1.0 / (double)b->N);
  g_next_bytes = 4.0 * b->N;  // the signal is written once
  return launched(b->cl->fwd(1, st, f), "cluster_c2r");
}

extern "C" {

sl_status sl_forward(const sl_bank* b, const float* x, float* coeffs, void* stream) {
  SL_TRY(check_call(b));
  if (!x || !coeffs) return fail(SL_EINVAL, "x or coeffs is NULL");
  SL_TRY(check_aligned(x, coeffs));
  if (b->cl) return cl_forward(b, x, coeffs, (cudaStream_t)stream);
  return forward_plan(plan_of(b), x, coeffs, (cudaStream_t)stream);
}

sl_status sl_adjoint(const sl_bank* b, const float* coeffs, float* x, void* stream) {
  SL_TRY(check_call(b));
  if (!x || !coeffs) return fail(SL_EINVAL, "x or coeffs is NULL");
  SL_TRY(check_aligned(x, coeffs));
  if (b->cl) return cl_backward(b, coeffs, x, false, (cudaStream_t)stream);
  return backward(plan_of(b), coeffs, x, false, (cudaStream_t)stream);
}

sl_status sl_inverse(const sl_bank* b, const float* coeffs, float* x, void* stream) {
  SL_TRY(check_call(b));
  if (!x || !coeffs) return fail(SL_EINVAL, "x or coeffs is NULL");
  SL_TRY(check_aligned(x, coeffs));
  if (b->cl) return cl_backward(b, coeffs, x, true, (cudaStream_t)stream);
  return backward(plan_of(b), coeffs, x, true, (cudaStream_t)stream);
}

// ------------------------------------------------ filter-sharded transform ---
// The inverse is a sum over filters (eq. reconstruction, Algorithm 2), so one large
// transform splits over ranks by filter ranges: every rank turns its coefficients
// into a partial spectrum, the partials are summed (one reduction of a spectrum),
// and one rank divides by Psi and transforms back. The forward needs the signal's
// spectrum on every rank (one broadcast) and then produces each range independently.

static sl_status check_range(const sl_bank* b, int j0, int j1) {
  if (j0 < 0 || j1 < j0 || j1 > b->R)
    return fail(SL_EINVAL, "filter range must satisfy 0 <= j0 <= j1 <= R");
  return SL_OK;
}

sl_status sl_spectrum_points(const sl_bank* b, int64_t* n_points) {
  if (!b || !n_points) return fail(SL_EINVAL, "bank or n_points is NULL");
  *n_points = b->Nhp;
  return SL_OK;
}

sl_status sl_spectrum(const sl_bank* b, const float* x, float* xhat, void* stream) {
  SL_TRY(check_call(b));
  if (!x || !xhat) return fail(SL_EINVAL, "x or xhat is NULL");
  SL_TRY(check_aligned(x, xhat));
  Plan P = plan_of(b);
  P.xhat = reinterpret_cast<float2*>(xhat);
  return spectrum_of(P, x, (cudaStream_t)stream);
}

sl_status sl_forward_range(const sl_bank* b, const float* xhat, int j0, int j1, float* coeffs,
                           void* stream) {
  SL_TRY(check_call(b));
  SL_TRY(check_range(b, j0, j1));
  if (!xhat || (!coeffs && j1 > j0)) return fail(SL_EINVAL, "xhat or coeffs is NULL");
  SL_TRY(check_aligned(xhat, coeffs));
  Plan P = plan_of(b);
  P.xhat = reinterpret_cast<float2*>(const_cast<float*>(xhat));  // read only
  return forward_filters(P, j0, j1, coeffs, (cudaStream_t)stream);
}

sl_status sl_inverse_partial(const sl_bank* b, const float* coeffs, int j0, int j1,
                             float* partial, void* stream) {
  SL_TRY(check_call(b));
  SL_TRY(check_range(b, j0, j1));
  if (!partial || (!coeffs && j1 > j0)) return fail(SL_EINVAL, "coeffs or partial is NULL");
  SL_TRY(check_aligned(coeffs, partial));
  Plan P = plan_of(b);
  cudaStream_t st = (cudaStream_t)stream;
  float2* out = reinterpret_cast<float2*>(partial);
  if (j1 == j0)
    return launched(cudaMemsetAsync(out, 0, (size_t)P.Nhp * sizeof(float2), st), "zero partial");
  SL_TRY(backward_filters(P, coeffs, j0, j1, st));
  return reduce_spectra(P, P.partial, parts_used(P, j1 - j0), P.Nhp, false, out, st);
}

sl_status sl_inverse_finish(const sl_bank* b, const float* summed, int dual, float* x,
                            void* stream) {
  SL_TRY(check_call(b));
  if (!summed || !x) return fail(SL_EINVAL, "summed or x is NULL");
  SL_TRY(check_aligned(summed, x));
  Plan P = plan_of(b);
  return parts_to_signal(P, reinterpret_cast<const float2*>(summed), 1, dual != 0, x,
                         (cudaStream_t)stream);
}

sl_status sl_sub_layout(const sl_bank* b, int* step, int64_t* offset) {
  if (!b) return fail(SL_EINVAL, "bank is NULL");
  if (b->spec.ndim != 2) return fail(SL_ENOTSUP, "the subsampled transform is 2D only");
  std::vector<int> st;
  std::vector<int64_t> off;
  sub_plan_of(b, &st, &off);
  if (step) std::copy(st.begin(), st.end(), step);
  if (offset) std::copy(off.begin(), off.end(), offset);
  return SL_OK;
}

sl_status sl_forward_sub(const sl_bank* cb, const float* x, float* coeffs_sub, void* stream) {
  SL_TRY(check_call(cb));
  if (!x || !coeffs_sub) return fail(SL_EINVAL, "x or coeffs_sub is NULL");
  SL_TRY(check_aligned(x, x));
  sl_bank* b = const_cast<sl_bank*>(cb);
  SL_TRY(ensure_sub(b));
  cudaStream_t st = (cudaStream_t)stream;
  SL_TRY(forward_plan(plan_of(b), x, b->sub_C, st));
  return sub_move(b, true, b->sub_C, coeffs_sub, st);
}

sl_status sl_adjoint_sub(const sl_bank* cb, const float* coeffs_sub, float* x, void* stream) {
  SL_TRY(check_call(cb));
  if (!x || !coeffs_sub) return fail(SL_EINVAL, "x or coeffs_sub is NULL");
  SL_TRY(check_aligned(x, x));
  sl_bank* b = const_cast<sl_bank*>(cb);
  SL_TRY(ensure_sub(b));
  cudaStream_t st = (cudaStream_t)stream;
  SL_TRY(sub_move(b, false, b->sub_C, const_cast<float*>(coeffs_sub), st));
  return backward(plan_of(b), b->sub_C, x, false, st);
}

sl_status sl_inverse_sub(const sl_bank* cb, const float* coeffs_sub, float* x, int iterations,
                         int precondition, double* rel_residual, void* stream) {
  SL_TRY(check_call(cb));
  if (!x || !coeffs_sub) return fail(SL_EINVAL, "x or coeffs_sub is NULL");
  SL_TRY(check_aligned(x, x));
  if (iterations < 0) return fail(SL_EINVAL, "iterations must be >= 0");
  sl_bank* b = const_cast<sl_bank*>(cb);
  SL_TRY(ensure_sub(b));
  cudaStream_t st = (cudaStream_t)stream;
  const Plan P = plan_of(b);
  const int64_t N = b->N;
  float* r = b->cg;
  float* p = b->cg + N;
  float* q = b->cg + 2 * N;
  float* z = precondition ? b->cg + 3 * N : r;
  float* rhs = b->cg + 4 * N;
  double* sc = b->cg_dot + kDotParts;  // [0], [1]: <r, z> of alternate iterations; [2]: <p, q>
  const int grid = (int)std::min<int64_t>((N + 255) / 256, 4 * 148);
  // rhs = T_sub* c; x = 0, r = rhs, z = P^-1 r, p = z
  SL_TRY(sl_adjoint_sub(b, coeffs_sub, rhs, stream));
  SL_CUDA(cudaMemsetAsync(x, 0, (size_t)N * sizeof(float), st));
  SL_CUDA(cudaMemcpyAsync(r, rhs, (size_t)N * sizeof(float), cudaMemcpyDeviceToDevice, st));
  if (precondition) SL_TRY(sub_precondition(P, r, z, st));
  SL_CUDA(cudaMemcpyAsync(p, z, (size_t)N * sizeof(float), cudaMemcpyDeviceToDevice, st));
  SL_TRY(dot(b, r, z, sc + 0, st));
  for (int it = 0; it < iterations; ++it) {
    double* rz_old = sc + (it & 1);
    double* rz_new = sc + ((it + 1) & 1);
    SL_TRY(sub_frame_op(P, p, q, st));
    SL_TRY(dot(b, p, q, sc + 2, st));
    SL_TRY(launched(timed_launch("cg_update", st, [&]() {
                      sl::dev::k_cg_xr<<<grid, 256, 0, st>>>(x, r, p, q, rz_old, sc + 2, N);
                    }),
                    "cg_update"));
    if (precondition) SL_TRY(sub_precondition(P, r, z, st));
    SL_TRY(dot(b, r, z, rz_new, st));
    SL_TRY(launched(timed_launch("cg_update", st, [&]() {
                      sl::dev::k_cg_p<<<grid, 256, 0, st>>>(p, z, rz_new, rz_old, N);
                    }),
                    "cg_update"));
  }
  if (rel_residual) {
    SL_TRY(dot(b, r, r, sc + 3, st));
    SL_TRY(dot(b, rhs, rhs, sc + 4, st));
    double h[2] = {0.0, 0.0};
    SL_CUDA(cudaMemcpyAsync(h, sc + 3, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    SL_CUDA(cudaStreamSynchronize(st));
    *rel_residual = h[1] > 0.0 ? std::sqrt(h[0] / h[1]) : 0.0;
  }
  return SL_OK;
}

sl_status sl_device_check(void* stream) {
  int dev = -1;
  SL_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64 || !g_dev_init[dev]) return SL_OK;  // nothing ran here yet
  SL_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  int h = 0;
  SL_CUDA(cudaMemcpyFromSymbol(&h, sl::dev::g_sl_wait_error, sizeof(int)));
  if (h) {
    const int zero = 0;
    SL_CUDA(cudaMemcpyToSymbol(sl::dev::g_sl_wait_error, &zero, sizeof(int)));
    return fail(SL_ETIMEOUT, "a bounded wait for a bulk copy ran out in a transform kernel "
                             "(its results are incomplete)");
  }
  return SL_OK;
}

sl_status sl_threshold(const sl_bank* b, float* coeffs, float sigma, const float* K,
                       void* stream) {
  SL_TRY(check_call(b));
  if (!coeffs || !K) return fail(SL_EINVAL, "coeffs or K is NULL");
  SL_TRY(check_aligned(coeffs, coeffs));
  if (!(sigma >= 0.f) || !std::isfinite(sigma)) return fail(SL_EINVAL, "sigma must be >= 0");
  for (int j = 0; j < b->spec.J; ++j)
    if (!std::isfinite(K[j])) return fail(SL_EINVAL, "K must be finite");
  cudaStream_t st = (cudaStream_t)stream;
  for (int j0 = 1; j0 < b->R; j0 += kMaxGroup) {
    const int nf = std::min(kMaxGroup, b->R - j0);
    Thresholds t;
    fill_thresholds(b, j0, nf, sigma, K, &t);
    const int64_t n4 = b->N / 4;
    int gx = (int)std::min<int64_t>((n4 + 255) / 256, 64);
    dim3 g(std::max(gx, 1), nf);
    float* base = coeffs + (int64_t)j0 * b->N;
    const int64_t n = b->N;
    g_next_bytes = 8.0 * (double)n * nf;  // read and write
    SL_TRY(launched(timed_launch("threshold", st, [&]() {
                      sl::dev::k_threshold<<<g, 256, 0, st>>>(base, n, nf, t);
                    }),
                    "threshold"));
  }
  return SL_OK;
}

sl_status sl_denoise(const sl_bank* b, const float* noisy, float* out, float sigma,
                     const float* K, void* stream) {
  SL_TRY(check_call(b));
  if (!noisy || !out || !K) return fail(SL_EINVAL, "noisy, out or K is NULL");
  SL_TRY(check_aligned(noisy, out));
  if (!(sigma >= 0.f) || !std::isfinite(sigma)) return fail(SL_EINVAL, "sigma must be >= 0");
  return denoise_plan(plan_of(b), noisy, out, sigma, K, (cudaStream_t)stream);
}

sl_status sl_inpaint(const sl_bank* cb, const float* f_masked, const uint8_t* mask, float* out,
                     float delta_init, float delta_min, int iterations, void* stream) {
  SL_TRY(check_call(cb));
  if (!f_masked || !mask || !out) return fail(SL_EINVAL, "f_masked, mask or out is NULL");
  if ((const void*)out == (const void*)f_masked) return fail(SL_EINVAL, "out must not alias f_masked");
  SL_TRY(check_aligned(f_masked, out));
  if (!a16(mask)) return fail(SL_EINVAL, "device arrays must be 16-byte aligned");
  if (iterations < 1) return fail(SL_EINVAL, "iterations must be >= 1");
  if (!(delta_init > 0.f) || !(delta_min > 0.f) || !std::isfinite(delta_init) ||
      !std::isfinite(delta_min))
    return fail(SL_EINVAL, "delta_init and delta_min must be finite and > 0");
  sl_bank* b = const_cast<sl_bank*>(cb);
  cudaStream_t st = (cudaStream_t)stream;
  if (!b->inp_u && cudaMalloc((void**)&b->inp_u, (size_t)b->N * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    b->inp_u = nullptr;
    return fail(SL_ENOMEM, "allocating the inpainting buffer");
  }
  // delta_k = delta_init lambda^k with delta_init lambda^(iterations - 1) = delta_min
  const double lam = iterations > 1 ? std::pow((double)delta_min / (double)delta_init,
                                               1.0 / (double)(iterations - 1))
                                    : 1.0;
  std::vector<float> ones((size_t)b->spec.J, 1.0f);
  const Plan P = plan_of(b);
  const int64_t n = b->N;
  const int grid = (int)std::min<int64_t>((n / 4 + 255) / 256, 4 * 148);
  double delta = delta_init;
  for (int it = 0; it < iterations; ++it) {
    const float* fcur = it == 0 ? nullptr : out;
    float* u = b->inp_u;
    SL_TRY(launched(timed_launch("inpaint_mix", st, [&]() {
                      sl::dev::k_inpaint_mix<<<grid, 256, 0, st>>>(f_masked, mask, fcur, u, n);
                    }),
                    "inpaint_mix"));
    SL_TRY(denoise_plan(P, u, out, (float)delta, ones.data(), st));
    delta *= lam;
  }
  return SL_OK;
}

sl_status sl_decompose(const sl_bank* ccurv, const sl_bank* iso, const float* f, float* f0,
                       float* f1, float delta_init, float delta_min, int iterations,
                       void* stream) {
  SL_TRY(check_call(ccurv));
  SL_TRY(check_call(iso));
  if (!f || !f0 || !f1) return fail(SL_EINVAL, "f, f0 or f1 is NULL");
  if (ccurv->spec.ndim != iso->spec.ndim || ccurv->N != iso->N ||
      ccurv->spec.dims[0] != iso->spec.dims[0] || ccurv->spec.dims[1] != iso->spec.dims[1] ||
      ccurv->spec.dims[2] != iso->spec.dims[2] || ccurv->device != iso->device)
    return fail(SL_EINVAL, "the two banks must share grid and device");
  if (f0 == f1 || (const float*)f0 == f || (const float*)f1 == f)
    return fail(SL_EINVAL, "f, f0 and f1 must be distinct arrays");
  SL_TRY(check_aligned(f, f0));
  SL_TRY(check_aligned(f1, f1));
  if (iterations < 1) return fail(SL_EINVAL, "iterations must be >= 1");
  if (!(delta_init > 0.f) || !(delta_min > 0.f) || !std::isfinite(delta_init) ||
      !std::isfinite(delta_min))
    return fail(SL_EINVAL, "delta_init and delta_min must be finite and > 0");
  sl_bank* b = const_cast<sl_bank*>(ccurv);
  cudaStream_t st = (cudaStream_t)stream;
  if (!b->inp_u && cudaMalloc((void**)&b->inp_u, (size_t)b->N * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    b->inp_u = nullptr;
    return fail(SL_ENOMEM, "allocating the decomposition buffer");
  }
  const double lam = iterations > 1 ? std::pow((double)delta_min / (double)delta_init,
                                               1.0 / (double)(iterations - 1))
                                    : 1.0;
  std::vector<float> ones0((size_t)b->spec.J, 1.0f), ones1((size_t)iso->spec.J, 1.0f);
  const Plan P0 = plan_of(b), P1 = plan_of(iso);
  const int64_t n = b->N;
  const int grid = (int)std::min<int64_t>((n / 4 + 255) / 256, 4 * 148);
  float* u = b->inp_u;
  SL_CUDA(cudaMemsetAsync(f1, 0, (size_t)n * sizeof(float), st));
  double delta = delta_init;
  for (int it = 0; it < iterations; ++it) {
    const float* other[2] = {f1, f0};
    for (int part = 0; part < 2; ++part) {
      const float* g = other[part];
      SL_TRY(launched(timed_launch("decompose_residual", st, [&]() {
                        sl::dev::k_sub<<<grid, 256, 0, st>>>(f, g, u, n);
                      }),
                      "decompose_residual"));
      if (part == 0)
        SL_TRY(denoise_plan(P0, u, f0, (float)delta, ones0.data(), st, INFINITY));
      else
        SL_TRY(denoise_plan(P1, u, f1, (float)delta, ones1.data(), st));
    }
    delta *= lam;
  }
  return SL_OK;
}

sl_status sl_fwdinv_host(const sl_bank* cb, const float* x_host, float* y_host, void* stream) {
  SL_TRY(check_call(cb));
  if (!x_host || !y_host) return fail(SL_EINVAL, "x_host or y_host is NULL");
  sl_bank* b = const_cast<sl_bank*>(cb);
  cudaStream_t st = (cudaStream_t)stream;
  if (!b->e2e_x) {
    if (cudaMalloc((void**)&b->e2e_x, (size_t)b->N * sizeof(float)) != cudaSuccess ||
        cudaMalloc((void**)&b->e2e_c, (size_t)b->R * b->N * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(b->e2e_x);
      b->e2e_x = nullptr;
      return fail(SL_ENOMEM, "allocating round-trip buffers");
    }
  }
  auto issue = [&](cudaStream_t s) -> sl_status {
    SL_CUDA(cudaMemcpyAsync(b->e2e_x, x_host, (size_t)b->N * sizeof(float),
                            cudaMemcpyHostToDevice, s));
    SL_TRY(sl_forward(b, b->e2e_x, b->e2e_c, s));
    SL_TRY(sl_inverse(b, b->e2e_c, b->e2e_x, s));
    SL_CUDA(cudaMemcpyAsync(y_host, b->e2e_x, (size_t)b->N * sizeof(float),
                            cudaMemcpyDeviceToHost, s));
    return SL_OK;
  };
  // Pinned host buffers: the copies and kernels are captured once into a CUDA graph
  // (per pair of host pointers) and replayed with one launch. Pageable buffers (or
  // a profiling run) take the direct route.
  cudaPointerAttributes ax{}, ay{};
  const bool pinned = cudaPointerGetAttributes(&ax, x_host) == cudaSuccess &&
                      cudaPointerGetAttributes(&ay, y_host) == cudaSuccess &&
                      ax.type == cudaMemoryTypeHost && ay.type == cudaMemoryTypeHost;
  cudaGetLastError();
  if (!pinned || g_prof_on) return issue(st);
  // Pinned buffers that the device can address (mapped; 16-byte aligned) are read
  // and written by the first and last kernels themselves over the host link,
  // without a separate copy (general path only).
  const float* xd = static_cast<const float*>(ax.devicePointer);
  float* yd = static_cast<float*>(ay.devicePointer);
  const bool mapped = !b->cl && xd && yd && a16(xd) && a16(yd);
  auto issue_mapped = [&](cudaStream_t s) -> sl_status {
    SL_TRY(sl_forward(b, xd, b->e2e_c, s));
    return sl_inverse(b, b->e2e_c, yd, s);
  };
  if (!b->e2e_graph || b->e2e_key[0] != x_host || b->e2e_key[1] != y_host) {
    if (!b->e2e_cap) SL_CUDA(cudaStreamCreateWithFlags(&b->e2e_cap, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    SL_CUDA(cudaStreamBeginCapture(b->e2e_cap, cudaStreamCaptureModeRelaxed));
    const sl_status s = mapped ? issue_mapped(b->e2e_cap) : issue(b->e2e_cap);
    cudaError_t e = cudaStreamEndCapture(b->e2e_cap, &g);
    if (s != SL_OK) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return s;
    }
    if (e != cudaSuccess) return cuda_fail(e, "capturing the round trip");
    if (b->e2e_graph) cudaGraphExecDestroy(b->e2e_graph);
    b->e2e_graph = nullptr;
    e = cudaGraphInstantiate(&b->e2e_graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      b->e2e_graph = nullptr;
      return cuda_fail(e, "instantiating the round trip graph");
    }
    b->e2e_key[0] = x_host;
    b->e2e_key[1] = y_host;
  }
  SL_CUDA(cudaGraphLaunch(b->e2e_graph, st));
  return SL_OK;
}

sl_status sl_error_stats(const float* y, const float* ref, int64_t n, double* stats,
                         void* stream) {
  if (!y || !ref || !stats || n <= 0) return fail(SL_EINVAL, "NULL argument or n <= 0");
  cudaStream_t st = (cudaStream_t)stream;
  double* acc = nullptr;
  SL_CUDA(cudaMallocAsync((void**)&acc, 4 * sizeof(double), st));
  SL_CUDA(cudaMemsetAsync(acc, 0, 4 * sizeof(double), st));
  const int grid = (int)std::min<int64_t>((n + 255) / 256, 4 * 148);
  sl::dev::k_error_stats<<<grid, 256, 0, st>>>(y, ref, n, acc);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(stats, acc, 4 * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFreeAsync(acc, st);
  if (e != cudaSuccess) return cuda_fail(e, "sl_error_stats");
  return SL_OK;
}

sl_status sl_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_on = on != 0;
  return SL_OK;
}

sl_status sl_profile_reset(void) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  for (auto& kv : g_prof)
    for (auto& pr : kv.second.pending) {
      cudaEventSynchronize(pr.second);
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
  g_prof.clear();
  return SL_OK;
}

sl_status sl_profile_read(const char** names, int64_t* launches, double* ms, double* bytes,
                          int cap, int* count) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  int i = 0;
  for (auto& kv : g_prof) {
    ProfKind& k = kv.second;
    for (double by : k.pending_bytes) k.bytes += by;
    k.pending_bytes.clear();
    for (auto& pr : k.pending) {
      cudaError_t e = cudaEventSynchronize(pr.second);
      if (e != cudaSuccess) return cuda_fail(e, "profile event");
      float t = 0.f;
      cudaEventElapsedTime(&t, pr.first, pr.second);
      k.ms += t;
      k.launches += 1;
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
    k.pending.clear();
    if (i < cap) {
      if (names) names[i] = kv.first.c_str();
      if (launches) launches[i] = k.launches;
      if (ms) ms[i] = k.ms;
      if (bytes) bytes[i] = k.bytes;
    }
    ++i;
  }
  if (count) *count = std::min(i, cap);
  return SL_OK;
}

}  // extern "C"

// ------------------------------------------------------------ batched runs ---
// A batch holds n transforms: image i on bank banks[i], any mix of shapes. Images are
// spread over K branches, longest estimated cost first onto the least loaded branch.
// Each branch owns a workspace (spectrum, group slab, partials) and a stream and runs
// its images one after another, so the single-image stages of one image (row and
// pencil FFTs of the signal, the final reduction) overlap the filter stages of others.
// The fork/join is captured into a CUDA graph once and then replayed by one
// cudaGraphLaunch per call; it is captured again when the data pointers (or the
// denoise thresholds) differ from the captured ones. Per distinct bank the batch also
// keeps its own filters-per-group cap (the slab width), which the autotuner sets.

namespace {

enum BatchOp { BOP_FWD = 0, BOP_INV = 1, BOP_FWDINV = 2, BOP_DENOISE = 3, BOP_COUNT = 4 };

struct BatchIO {
  const float* const* x = nullptr;   // forward / fwdinv / denoise input
  float* const* c = nullptr;         // coefficients (forward output, inverse input)
  float* const* y = nullptr;         // inverse / fwdinv / denoise output
  float sigma = 0.f;
  const float* const* K = nullptr;   // denoise: per image, nScales of its bank
};

struct BatchGraph {
  cudaGraphExec_t exec = nullptr;
  std::vector<uint64_t> key;
};

}  // namespace

struct sl_batch {
  int device = -1;
  int n = 0;
  std::vector<const sl_bank*> banks;
  std::vector<const sl_bank*> distinct;  // distinct banks, in first-use order
  std::vector<int> shape_of;             // image -> index into distinct
  std::vector<int> gmax;                 // per distinct bank: filters-per-group cap
  int K = 1;                             // branches
  int use_graph = 1;
  std::vector<std::vector<int>> order;   // branch -> its images, in issue order
  std::vector<float2*> ws;               // branch workspaces
  std::vector<int64_t> ws_elems;
  std::vector<cudaStream_t> streams;     // [K]
  std::vector<cudaEvent_t> ev;           // [K + 1]: fork, then one join per branch
  cudaStream_t cap = nullptr;            // capture origin
  BatchGraph graph[BOP_COUNT];
};

// Group layout of bank b with at most gmax filters per group (as plan_groups).
static void group_plan(const sl_bank* b, int gmax, Plan& p) {
  gmax = std::max(1, std::min(gmax, kMaxGroup));
  p.ngroups = (b->R + gmax - 1) / gmax;
  p.G = (b->R + p.ngroups - 1) / p.ngroups;
  const int want = std::max(1, (4 * 148 + b->ntiles - 1) / b->ntiles);
  p.fps = std::max(2, (p.G + want - 1) / want);
  p.S = (p.G + p.fps - 1) / p.fps;
}

static int64_t plan_ws_elems(const Plan& p) {
  return p.Nhp * (1 + (int64_t)p.G + (int64_t)p.ngroups * p.S);
}

static Plan batch_plan(const sl_batch* B, int i, float2* ws) {
  const sl_bank* b = B->banks[i];
  Plan p = plan_of(b);
  group_plan(b, B->gmax[B->shape_of[i]], p);
  p.xhat = ws;
  p.scratch = ws + p.Nhp;
  p.partial = ws + p.Nhp * (1 + (int64_t)p.G);
  return p;
}

static double image_cost(const sl_bank* b) {
  return (double)(b->R + 2) * (double)b->N * std::log2((double)b->N);
}

static void batch_release_graphs(sl_batch* B) {
  for (BatchGraph& g : B->graph) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
    g.key.clear();
  }
}

static void batch_release_branches(sl_batch* B) {
  batch_release_graphs(B);
  for (float2* w : B->ws) cudaFree(w);
  for (cudaStream_t s : B->streams)
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t e : B->ev)
    if (e) cudaEventDestroy(e);
  B->ws.clear();
  B->ws_elems.clear();
  B->streams.clear();
  B->ev.clear();
  B->order.clear();
}

// Schedule the images over K branches and size each branch's workspace. Images of a
// cluster-path bank share the bank's own buffers, so they form one job.
static sl_status batch_schedule(sl_batch* B, int K) {
  batch_release_branches(B);
  struct Job { double cost; std::vector<int> imgs; };
  std::vector<Job> jobs;
  std::map<const sl_bank*, int> cl_job;
  for (int i = 0; i < B->n; ++i) {
    const sl_bank* b = B->banks[i];
    if (b->cl) {
      auto it = cl_job.find(b);
      if (it == cl_job.end()) {
        cl_job[b] = (int)jobs.size();
        jobs.push_back(Job{0.0, {}});
        it = cl_job.find(b);
      }
      jobs[it->second].cost += image_cost(b);
      jobs[it->second].imgs.push_back(i);
    } else {
      jobs.push_back(Job{image_cost(b), {i}});
    }
  }
  K = std::max(1, std::min<int>(K, (int)jobs.size()));
  std::stable_sort(jobs.begin(), jobs.end(),
                   [](const Job& a, const Job& b) { return a.cost > b.cost; });
  std::vector<double> load(K, 0.0);
  B->order.assign(K, {});
  for (const Job& j : jobs) {
    const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    load[k] += j.cost;
    for (int i : j.imgs) B->order[k].push_back(i);
  }
  B->K = K;
  B->ws.assign(K, nullptr);
  B->ws_elems.assign(K, 0);
  B->streams.assign(K, nullptr);
  B->ev.assign(K + 1, nullptr);
  for (int k = 0; k < K; ++k) {
    int64_t need = 0;
    for (int i : B->order[k])
      if (!B->banks[i]->cl) need = std::max(need, plan_ws_elems(batch_plan(B, i, nullptr)));
    B->ws_elems[k] = need;
    if (need > 0 && cudaMalloc((void**)&B->ws[k], (size_t)need * sizeof(float2)) != cudaSuccess) {
      cudaGetLastError();
      B->ws[k] = nullptr;
      batch_release_branches(B);
      return fail(SL_ENOMEM, "allocating batch workspaces");
    }
    // pad pencils hold zeros, as in a bank's own scratch
    if (need > 0) SL_CUDA(cudaMemset(B->ws[k], 0, (size_t)need * sizeof(float2)));
    SL_CUDA(cudaStreamCreateWithFlags(&B->streams[k], cudaStreamNonBlocking));
  }
  for (int k = 0; k <= K; ++k) SL_CUDA(cudaEventCreateWithFlags(&B->ev[k], cudaEventDisableTiming));
  return SL_OK;
}

static sl_status batch_image(const sl_batch* B, int i, int op, const BatchIO& io, int k,
                             cudaStream_t st) {
  const sl_bank* b = B->banks[i];
  if (b->cl) {
    if (op == BOP_FWD || op == BOP_FWDINV) SL_TRY(cl_forward(b, io.x[i], io.c[i], st));
    if (op == BOP_INV || op == BOP_FWDINV) SL_TRY(cl_backward(b, io.c[i], io.y[i], true, st));
    if (op == BOP_DENOISE) return fail(SL_ENOTSUP, "batched denoise needs general-path banks");
    return SL_OK;
  }
  const Plan P = batch_plan(B, i, B->ws[k]);
  if (op == BOP_FWD || op == BOP_FWDINV) SL_TRY(forward_plan(P, io.x[i], io.c[i], st));
  if (op == BOP_INV || op == BOP_FWDINV) SL_TRY(backward(P, io.c[i], io.y[i], true, st));
  if (op == BOP_DENOISE) SL_TRY(denoise_plan(P, io.x[i], io.y[i], io.sigma, io.K[i], st));
  return SL_OK;
}

// Fork from `origin` into the branch streams, run every branch, join back.
static sl_status batch_issue(const sl_batch* B, int op, const BatchIO& io, cudaStream_t origin) {
  SL_CUDA(cudaEventRecord(B->ev[0], origin));
  for (int k = 0; k < B->K; ++k) {
    if (B->order[k].empty()) continue;
    cudaStream_t st = B->streams[k];
    SL_CUDA(cudaStreamWaitEvent(st, B->ev[0], 0));
    for (int i : B->order[k]) SL_TRY(batch_image(B, i, op, io, k, st));
    SL_CUDA(cudaEventRecord(B->ev[k + 1], st));
    SL_CUDA(cudaStreamWaitEvent(origin, B->ev[k + 1], 0));
  }
  return SL_OK;
}

static std::vector<uint64_t> batch_key(const sl_batch* B, int op, const BatchIO& io) {
  std::vector<uint64_t> key;
  for (int i = 0; i < B->n; ++i) {
    key.push_back(io.x ? (uint64_t)(uintptr_t)io.x[i] : 0);
    key.push_back(io.c ? (uint64_t)(uintptr_t)io.c[i] : 0);
    key.push_back(io.y ? (uint64_t)(uintptr_t)io.y[i] : 0);
  }
  if (op == BOP_DENOISE) {
    uint32_t u;
    std::memcpy(&u, &io.sigma, 4);
    key.push_back(u);
    for (int i = 0; i < B->n; ++i)
      for (int j = 0; j < B->banks[i]->spec.J; ++j) {
        std::memcpy(&u, &io.K[i][j], 4);
        key.push_back(u);
      }
  }
  return key;
}

static sl_status batch_check_io(const sl_batch* B, int op, const BatchIO& io) {
  if (!B) return fail(SL_EINVAL, "batch is NULL");
  int cur = -1;
  SL_CUDA(cudaGetDevice(&cur));
  if (cur != B->device) return fail(SL_EINVAL, "current CUDA device differs from the batch's");
  const bool need_x = op != BOP_INV, need_c = op != BOP_DENOISE, need_y = op != BOP_FWD;
  if ((need_x && !io.x) || (need_c && !io.c) || (need_y && !io.y))
    return fail(SL_EINVAL, "a pointer array is NULL");
  for (int i = 0; i < B->n; ++i) {
    if ((need_x && !io.x[i]) || (need_c && !io.c[i]) || (need_y && !io.y[i]))
      return fail(SL_EINVAL, "image " + std::to_string(i) + ": NULL data pointer");
    if ((need_x && !a16(io.x[i])) || (need_c && !a16(io.c[i])) || (need_y && !a16(io.y[i])))
      return fail(SL_EINVAL, "image " + std::to_string(i) + ": data not 16-byte aligned");
  }
  if (op == BOP_DENOISE) {
    if (!io.K) return fail(SL_EINVAL, "K is NULL");
    if (!(io.sigma >= 0.f) || !std::isfinite(io.sigma)) return fail(SL_EINVAL, "sigma must be >= 0");
    for (int i = 0; i < B->n; ++i) {
      if (!io.K[i]) return fail(SL_EINVAL, "image " + std::to_string(i) + ": K is NULL");
      for (int j = 0; j < B->banks[i]->spec.J; ++j)
        if (!std::isfinite(io.K[i][j])) return fail(SL_EINVAL, "K must be finite");
    }
  }
  return SL_OK;
}

static sl_status batch_run(sl_batch* B, int op, const BatchIO& io, cudaStream_t st) {
  SL_TRY(batch_check_io(B, op, io));
  if (!B->use_graph || g_prof_on) return batch_issue(B, op, io, st);
  BatchGraph& G = B->graph[op];
  std::vector<uint64_t> key = batch_key(B, op, io);
  if (!G.exec || G.key != key) {
    cudaGraph_t g = nullptr;
    SL_CUDA(cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeRelaxed));
    const sl_status s = batch_issue(B, op, io, B->cap);
    cudaError_t e = cudaStreamEndCapture(B->cap, &g);
    if (s != SL_OK) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return s;
    }
    if (e != cudaSuccess) return cuda_fail(e, "capturing the batch");
    if (G.exec) {
      cudaGraphExecUpdateResultInfo info;
      if (cudaGraphExecUpdate(G.exec, g, &info) != cudaSuccess) {
        cudaGetLastError();
        cudaGraphExecDestroy(G.exec);
        G.exec = nullptr;
      }
    }
    if (!G.exec) e = cudaGraphInstantiate(&G.exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      G.exec = nullptr;
      return cuda_fail(e, "instantiating the batch graph");
    }
    G.key = std::move(key);
  }
  SL_CUDA(cudaGraphLaunch(G.exec, st));
  return SL_OK;
}

// Device time of `reps` calls of fn on st (minimum over calls), in ms.
template <typename F>
static sl_status time_min(cudaStream_t st, int reps, F&& fn, double* best) {
  cudaEvent_t a, b;
  SL_CUDA(cudaEventCreate(&a));
  SL_CUDA(cudaEventCreate(&b));
  *best = 1e300;
  sl_status s = SL_OK;
  for (int r = 0; r < reps && s == SL_OK; ++r) {
    cudaEventRecord(a, st);
    s = fn();
    cudaEventRecord(b, st);
    cudaError_t e = cudaEventSynchronize(b);
    if (s == SL_OK && e != cudaSuccess) s = cuda_fail(e, "autotune timing");
    float ms = 0.f;
    if (s == SL_OK) cudaEventElapsedTime(&ms, a, b);
    if (s == SL_OK && r > 0) *best = std::min(*best, (double)ms);  // first call warms up
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return s;
}

extern "C" {

sl_status sl_batch_create(const sl_bank* const* banks, int n, const sl_batch_options* opt,
                          sl_batch** out) {
  if (!out) return fail(SL_EINVAL, "out is NULL");
  *out = nullptr;
  if (!banks || n <= 0) return fail(SL_EINVAL, "banks is NULL or n <= 0");
  std::unique_ptr<sl_batch> B(new sl_batch());
  B->n = n;
  for (int i = 0; i < n; ++i) {
    SL_TRY(check_call(banks[i]));
    B->banks.push_back(banks[i]);
    auto it = std::find(B->distinct.begin(), B->distinct.end(), banks[i]);
    if (it == B->distinct.end()) {
      B->shape_of.push_back((int)B->distinct.size());
      B->distinct.push_back(banks[i]);
      B->gmax.push_back(banks[i]->G);
    } else {
      B->shape_of.push_back((int)(it - B->distinct.begin()));
    }
  }
  B->device = banks[0]->device;
  int K = 0;
  if (opt) {
    if (opt->branches < 0) return fail(SL_EINVAL, "branches must be >= 0");
    K = opt->branches;
    B->use_graph = opt->no_graph ? 0 : 1;
  }
  if (K == 0) K = 4;
  SL_CUDA(cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking));
  sl_status s = batch_schedule(B.get(), K);
  if (s != SL_OK) {
    cudaStreamDestroy(B->cap);
    return s;
  }
  *out = B.release();
  return SL_OK;
}

void sl_batch_free(sl_batch* B) {
  if (!B) return;
  int cur = -1;
  cudaGetDevice(&cur);
  if (B->device >= 0) cudaSetDevice(B->device);
  batch_release_branches(B);
  if (B->cap) cudaStreamDestroy(B->cap);
  if (cur >= 0) cudaSetDevice(cur);
  delete B;
}

sl_status sl_batch_info(const sl_batch* B, int* branches, int* branch_of, int* group_cap) {
  if (!B) return fail(SL_EINVAL, "batch is NULL");
  if (branches) *branches = B->K;
  for (int k = 0; k < B->K; ++k)
    for (int i : B->order[k]) {
      if (branch_of) branch_of[i] = k;
      if (group_cap) group_cap[i] = B->banks[i]->cl ? B->banks[i]->R : B->gmax[B->shape_of[i]];
    }
  return SL_OK;
}

sl_status sl_batch_forward(sl_batch* B, const float* const* x, float* const* coeffs, void* stream) {
  BatchIO io;
  io.x = x;
  io.c = coeffs;
  return batch_run(B, BOP_FWD, io, (cudaStream_t)stream);
}

sl_status sl_batch_inverse(sl_batch* B, const float* const* coeffs, float* const* x, void* stream) {
  BatchIO io;
  io.c = const_cast<float* const*>(coeffs);
  io.y = x;
  return batch_run(B, BOP_INV, io, (cudaStream_t)stream);
}

sl_status sl_batch_fwdinv(sl_batch* B, const float* const* x, float* const* coeffs, float* const* y,
                          void* stream) {
  BatchIO io;
  io.x = x;
  io.c = coeffs;
  io.y = y;
  return batch_run(B, BOP_FWDINV, io, (cudaStream_t)stream);
}

sl_status sl_batch_denoise(sl_batch* B, const float* const* noisy, float* const* out, float sigma,
                           const float* const* K, void* stream) {
  BatchIO io;
  io.x = noisy;
  io.y = out;
  io.sigma = sigma;
  io.K = K;
  return batch_run(B, BOP_DENOISE, io, (cudaStream_t)stream);
}

sl_status sl_batch_autotune(sl_batch* B, const float* const* x, float* const* coeffs,
                            float* const* y, int reps, void* stream, double* best_ms) {
  BatchIO io;
  io.x = x;
  io.c = coeffs;
  io.y = y;
  SL_TRY(batch_check_io(B, BOP_FWDINV, io));
  if (reps < 2) return fail(SL_EINVAL, "reps must be >= 2");
  cudaStream_t st = (cudaStream_t)stream;
  SL_CUDA(cudaStreamSynchronize(st));
  // 1. per distinct bank, the filters-per-group cap: one image of that shape, alone
  for (size_t d = 0; d < B->distinct.size(); ++d) {
    const sl_bank* b = B->distinct[d];
    if (b->cl) continue;
    int img = 0;
    while (B->shape_of[img] != (int)d) ++img;
    std::vector<int> cand = {b->G, b->R, (b->R + 1) / 2, (b->R + 3) / 4, (b->R + 7) / 8};
    std::sort(cand.begin(), cand.end());
    cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
    double best = 1e300;
    int best_g = B->gmax[d];
    for (int g : cand) {
      if (g < 2 || g > kMaxGroup) continue;
      Plan p = plan_of(b);
      group_plan(b, g, p);
      const int64_t need = plan_ws_elems(p);
      if ((double)need * sizeof(float2) > 1024.0 * 1024.0 * 1024.0) continue;  // 1 GiB cap
      float2* ws = nullptr;
      if (cudaMalloc((void**)&ws, (size_t)need * sizeof(float2)) != cudaSuccess) {
        cudaGetLastError();
        continue;
      }
      p.xhat = ws;
      p.scratch = ws + p.Nhp;
      p.partial = ws + p.Nhp * (1 + (int64_t)p.G);
      double ms = 0.0;
      sl_status s = time_min(st, reps, [&]() -> sl_status {
        SL_TRY(forward_plan(p, x[img], coeffs[img], st));
        return backward(p, coeffs[img], y[img], true, st);
      }, &ms);
      cudaFree(ws);
      SL_TRY(s);
      if (ms < best) {
        best = ms;
        best_g = g;
      }
    }
    B->gmax[d] = best_g;
  }
  // 2. branch count: the whole batch, captured as it will run
  double best = 1e300;
  int best_k = B->K;
  for (int k : {1, 2, 3, 4, 6, 8, 12, 16}) {
    if (k > B->n) break;
    SL_TRY(batch_schedule(B, k));
    double ms = 0.0;
    SL_TRY(time_min(st, reps, [&]() { return batch_run(B, BOP_FWDINV, io, st); }, &ms));
    if (ms < best * 0.99) {  // prefer fewer branches unless clearly faster
      best = ms;
      best_k = k;
    }
  }
  SL_TRY(batch_schedule(B, best_k));
  if (best_ms) *best_ms = best;
  return SL_OK;
}

// One-shot forms: build a batch (no graph), run it, wait for it, free it.
sl_status sl_forward_batch(const sl_bank* const* banks, int n, const float* const* x,
                           float* const* coeffs, void* stream) {
  sl_batch_options o{};
  o.no_graph = 1;
  sl_batch* B = nullptr;
  SL_TRY(sl_batch_create(banks, n, &o, &B));
  sl_status s = sl_batch_forward(B, x, coeffs, stream);
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  sl_batch_free(B);
  if (s == SL_OK && e != cudaSuccess) s = cuda_fail(e, "sl_forward_batch");
  return s;
}

sl_status sl_inverse_batch(const sl_bank* const* banks, int n, const float* const* coeffs,
                           float* const* x, void* stream) {
  sl_batch_options o{};
  o.no_graph = 1;
  sl_batch* B = nullptr;
  SL_TRY(sl_batch_create(banks, n, &o, &B));
  sl_status s = sl_batch_inverse(B, coeffs, x, stream);
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  sl_batch_free(B);
  if (s == SL_OK && e != cudaSuccess) s = cuda_fail(e, "sl_inverse_batch");
  return s;
}

}  // extern "C"

// ------------------------------------------------- allocation-free forward ---
// Scratch for sl_forward_noalloc: a file-scope device array instead of memory from
// cudaMalloc. Host code must not use the symbol as an address; it asks the runtime
// for the array's device address once per device (noalloc_scratch_ptr).

static __device__ __align__(256) float2 g_noalloc_scratch[SL_NOALLOC_SCRATCH_BYTES / sizeof(float2)];

static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[64] = {nullptr};

static sl_status noalloc_scratch_ptr(int dev, float2** out) {
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (dev < 0 || dev >= 64) return fail(SL_EINVAL, "device ordinal out of range");
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_noalloc_addr[dev] = p;
  }
  *out = static_cast<float2*>(g_noalloc_addr[dev]);
  return SL_OK;
}

extern "C" sl_status sl_forward_noalloc(const sl_bank* b, const float* psi, const float* x,
                                        float* coeffs, void* stream) {
  if (!b) return fail(SL_EINVAL, "bank is NULL");
  if (!psi || !x || !coeffs) return fail(SL_EINVAL, "psi, x or coeffs is NULL");
  SL_TRY(check_aligned(x, coeffs));
  SL_TRY(check_aligned(psi, psi));
  const int64_t cap = (int64_t)(SL_NOALLOC_SCRATCH_BYTES / sizeof(float2));
  if (2 * b->Nhp > cap)
    return fail(SL_ENOTSUP, "sl_forward_noalloc: the signal's spectrum plus one filter's "
                            "spectrum need " + std::to_string(2 * b->Nhp * 8) +
                            " bytes, more than SL_NOALLOC_SCRATCH_BYTES (16 MiB)");
  int dev = -1;
  SL_CUDA(cudaGetDevice(&dev));
  SL_TRY(init_device(dev));
  float2* base = nullptr;
  SL_TRY(noalloc_scratch_ptr(dev, &base));
  // scratch layout: the spectrum of x, then G filter slots. Pad pencils may hold stale
  // values from earlier calls; they never reach a result, because pencils are
  // transformed independently and the last-axes passes read valid pencils only.
  Plan P{};
  P.spec = &b->spec;
  P.N = b->N;
  P.Nh = b->Nh;
  P.Nhp = b->Nhp;
  P.NP = b->NP;
  P.TC = b->TC;
  P.lgTC = b->lgTC;
  P.ntiles = b->ntiles;
  P.R = b->R;
  P.G = (int)std::min<int64_t>({(cap - b->Nhp) / b->Nhp, (int64_t)kMaxGroup, (int64_t)b->R});
  P.ngroups = (P.R + P.G - 1) / P.G;
  P.psi = psi;
  P.psi_natural = 1;
  P.xhat = base;
  P.scratch = base + b->Nhp;
  P.bank = b;
  return forward_plan(P, x, coeffs, (cudaStream_t)stream);
}
