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
#include <vector>

#include "../../include/shearlet.h"
#include "bank_host.h"
#include "kernels3d.cuh"

using sl::dev::ColArgs;
using sl::dev::RowArgs;
using sl::dev::Thresholds;
using sl::dev::kMaxGroup;
using sl::dev::kThreads;
using sl::dev::kPlaneThreads;

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
  for (int L = 8; L <= 1024; L *= 2) {
    int A = 0, B = 0;
    switch (L) {
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
  constexpr int smem = sl::dev::col_smem_bytes<L>();
  cudaError_t e = ensure_smem(k, smem);
  if (e != cudaSuccess) return e;
  static const char* names[4] = {"col_spec", "col_fwd_filter", "col_inv_accumulate",
                                 "col_inv_final"};
  return timed_launch(names[MODE], st, [&]() { k<<<grid, kThreads, smem, st>>>(a); });
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
    default: return cudaErrorInvalidValue;
  }
}

static int col_tile(int L) {  // pencils per CTA = 256 / B
  switch (L) {
    case 8: return 128;
    case 16: return 64;
    case 32: return 64;
    case 64: return 32;
    case 128: return 32;
    case 256: return 16;
    case 512: return 16;
    default: return 8;
  }
}

template <int L, int MODE>
static cudaError_t launch_row_t(dim3 grid, cudaStream_t st, const RowArgs& a) {
  auto k = sl::dev::k_row<L, MODE>;
  constexpr int smem = sl::dev::row_smem_bytes<L>();
  cudaError_t e = ensure_smem(k, smem);
  if (e != cudaSuccess) return e;
  static const char* names[3] = {"row_r2c", "row_c2r", "row_roundtrip"};
  return timed_launch(names[MODE], st, [&]() { k<<<grid, kThreads, smem, st>>>(a); });
}

template <int MODE>
static cudaError_t launch_row(int L, dim3 grid, cudaStream_t st, const RowArgs& a) {
  switch (L) {
    case 8: return launch_row_t<8, MODE>(grid, st, a);
    case 16: return launch_row_t<16, MODE>(grid, st, a);
    case 32: return launch_row_t<32, MODE>(grid, st, a);
    case 64: return launch_row_t<64, MODE>(grid, st, a);
    case 128: return launch_row_t<128, MODE>(grid, st, a);
    case 256: return launch_row_t<256, MODE>(grid, st, a);
    case 512: return launch_row_t<512, MODE>(grid, st, a);
    case 1024: return launch_row_t<1024, MODE>(grid, st, a);
    default: return cudaErrorInvalidValue;
  }
}

static int row_pairs_per_cta(int L) {  // 256 / B
  return col_tile(L);
}

template <int L1, int L2, int MODE>
static cudaError_t launch_plane_t(dim3 grid, cudaStream_t st, const RowArgs& a) {
  auto k = sl::dev::k_plane<L1, L2, MODE>;
  constexpr int smem = sl::dev::PlaneGeom<L1, L2>::bytes;
  cudaError_t e = ensure_smem(k, smem);
  if (e != cudaSuccess) return e;
  static const char* names[3] = {"plane_r2c", "plane_c2r", "plane_roundtrip"};
  return timed_launch(names[MODE], st, [&]() { k<<<grid, kPlaneThreads, smem, st>>>(a); });
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

template <int MODE>
static cudaError_t launch_plane(int L1, int L2, dim3 grid, cudaStream_t st, const RowArgs& a) {
  switch (L1) {
    case 8: return launch_plane_l2<8, MODE>(L2, grid, st, a);
    case 16: return launch_plane_l2<16, MODE>(L2, grid, st, a);
    case 32: return launch_plane_l2<32, MODE>(L2, grid, st, a);
    case 64: return launch_plane_l2<64, MODE>(L2, grid, st, a);
    case 128: return launch_plane_l2<128, MODE>(L2, grid, st, a);
    default: return cudaErrorInvalidValue;
  }
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
  int G = 1;        // filters per group
  int ngroups = 1;
  int S = 1;        // partials per group
  int fps = 1;      // filters per partial
  float* psi = nullptr;       // [R][Nh]
  double* invPsi = nullptr;   // [Nh]
  float2* xhat = nullptr;     // [Nh] spectrum of the signal
  float2* scratch = nullptr;  // [G][Nh]
  float2* partial = nullptr;  // [ngroups * S][Nh]
  float* e2e_x = nullptr;     // sl_fwdinv_host buffers (allocated on first use)
  float* e2e_c = nullptr;
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
  b->psi = nullptr;
  b->invPsi = nullptr;
  b->xhat = b->scratch = b->partial = nullptr;
  b->e2e_x = b->e2e_c = nullptr;
}

// Grouping: the per-filter intermediate spectra of one group stay resident in L2
// between the two passes of a transform; a group holds as many filters as fit in
// the scratch budget (SL_SCRATCH_MB, default 48 MB).
static void plan_groups(sl_bank* b) {
  double mb = 48.0;
  if (const char* s = std::getenv("SL_SCRATCH_MB")) mb = std::max(1.0, std::atof(s));
  const double per = (double)b->Nh * sizeof(float2);
  int gmax = (int)std::max(1.0, std::floor(mb * 1024.0 * 1024.0 / per));
  gmax = std::min(gmax, kMaxGroup);
  b->ngroups = (b->R + gmax - 1) / gmax;
  b->G = (b->R + b->ngroups - 1) / b->ngroups;
  // pencil tiles of the inverse accumulation; split filters so that the grid covers
  // the GPU about twice (148 SMs on B300), with at least 2 filters per split.
  const int L0 = (int)b->spec.dims[0];
  const int NP = (int)(b->Nh / L0);
  const int tiles = (NP + col_tile(L0) - 1) / col_tile(L0);
  int want = std::max(1, (2 * 148 + tiles - 1) / tiles);
  b->fps = std::max(2, (b->G + want - 1) / want);
  b->S = (b->G + b->fps - 1) / b->fps;
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
  if (!out) return fail(SL_EINVAL, "out is NULL");
  *out = nullptr;
  if (ndim != 2 && ndim != 3) return fail(SL_EINVAL, "ndim must be 2 or 3");
  if (!dims || !shearLevels) return fail(SL_EINVAL, "dims or shearLevels is NULL");
  if (nScales < 1 || nScales > 8) return fail(SL_EINVAL, "nScales must be in [1, 8]");
  sl::BankSpec spec;
  spec.ndim = ndim;
  spec.J = nScales;
  spec.full = fullSystem != 0;
  for (int i = 0; i < ndim; ++i) {
    if (dims[i] < 8) return fail(SL_EINVAL, "every dimension must be >= 8");
    if (!is_pow2(dims[i]) || dims[i] > 1024)
      return fail(SL_ENOTSUP, "dimensions must be powers of two in [8, 1024]");
    spec.dims[i] = dims[i];
  }
  for (int j = 0; j < nScales; ++j) {
    if (shearLevels[j] < 0 || shearLevels[j] > 4)
      return fail(SL_EINVAL, "shearLevels entries must be in [0, 4]");
    spec.d[j] = shearLevels[j];
  }
  if (ndim == 3) {
    if (dims[1] > 128 || dims[2] > 128)
      return fail(SL_ENOTSUP, "3D: axes 1 and 2 must be at most 128 (one plane per CTA)");
  }
  const int64_t N = spec.N(), Nh = spec.Nh();
  if (N > ((int64_t)1 << 31)) return fail(SL_ENOTSUP, "grid too large");
  std::unique_ptr<sl_bank> b(new sl_bank());
  b->spec = spec;
  b->device = device;
  b->N = N;
  b->Nh = Nh;

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
    if (!alloc((void**)&b->psi, (size_t)b->R * Nh * sizeof(float)) ||
        !alloc((void**)&b->invPsi, (size_t)Nh * sizeof(double)) ||
        !alloc((void**)&b->xhat, (size_t)Nh * sizeof(float2)) ||
        !alloc((void**)&b->scratch, (size_t)b->G * Nh * sizeof(float2)) ||
        !alloc((void**)&b->partial, (size_t)b->ngroups * b->S * Nh * sizeof(float2))) {
      cudaGetLastError();
      free_device(b.get());
      return fail(SL_ENOMEM, "device allocation failed");
    }
    cudaError_t e = cudaMemcpy(b->psi, hb.psi32.data(), (size_t)b->R * Nh * sizeof(float),
                               cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(b->invPsi, hb.invPsi.data(), (size_t)Nh * sizeof(double),
                     cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      free_device(b.get());
      return cuda_fail(e, "uploading the filter bank");
    }
  }
  *out = b.release();
  return SL_OK;
}

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
  SL_CUDA(cudaMemcpy(out, b->psi, (size_t)b->R * b->Nh * sizeof(float), cudaMemcpyDeviceToHost));
  return SL_OK;
}

}  // extern "C"

// --------------------------------------------------------------- transforms ---

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

// Real signal x[dims] -> half spectrum b->xhat (rows/planes, then pencils).
static sl_status spectrum_of(const sl_bank* b, const float* x, cudaStream_t st) {
  const sl::BankSpec& s = b->spec;
  const int L0 = (int)s.dims[0];
  RowArgs ra{};
  ra.in_real = x;
  ra.out_half = b->xhat;
  ra.in_stride = 0;
  ra.out_stride = 0;
  ra.scale = 1.f;
  g_next_bytes = 4.0 * b->N;  // the signal is read once
  if (s.ndim == 2) {
    const int L1 = (int)s.dims[1];
    ra.n_rows = L0;
    ra.nh = (int)s.nh();
    dim3 g((L0 / 2 + row_pairs_per_cta(L1) - 1) / row_pairs_per_cta(L1), 1);
    SL_TRY(launched(launch_row<sl::dev::ROW_R2C>(L1, g, st, ra), "row_r2c"));
  } else {
    dim3 g(L0, 1);
    g_next_bytes = 4.0 * b->N;
    SL_TRY(launched(launch_plane<sl::dev::ROW_R2C>((int)s.dims[1], (int)s.dims[2], g, st, ra),
                    "plane_r2c"));
  }
  ColArgs ca{};
  ca.in = b->xhat;
  ca.out = b->xhat;
  ca.Nh = b->Nh;
  ca.NP = (int)(b->Nh / L0);
  dim3 g((ca.NP + col_tile(L0) - 1) / col_tile(L0), 1);
  return launched(launch_col<sl::dev::COL_SPEC>(L0, g, st, ca), "col_spec");
}

// Per-filter "last axes" pass of one group: ROW_C2R (coeffs out), ROW_R2C (coeffs in)
// or ROW_RT (scratch in place).
template <int MODE>
static sl_status slab_pass(const sl_bank* b, int j0, int nf, const float* creal_in,
                           float* creal_out, const Thresholds* thr, cudaStream_t st) {
  const sl::BankSpec& s = b->spec;
  const int L0 = (int)s.dims[0];
  RowArgs ra{};
  ra.scale = (float)(1.0 / (double)b->N);
  ra.nh = (int)s.nh();
  ra.n_rows = L0;
  if (thr) {
    ra.use_thr = 1;
    ra.thr = *thr;
  }
  if (MODE == sl::dev::ROW_C2R) {
    ra.in_half = b->scratch;
    ra.in_stride = b->Nh;
    ra.out_real = creal_out + (int64_t)j0 * b->N;
    ra.out_stride = b->N;
  } else if (MODE == sl::dev::ROW_R2C) {
    ra.in_real = creal_in + (int64_t)j0 * b->N;
    ra.in_stride = b->N;
    ra.out_half = b->scratch;
    ra.out_stride = b->Nh;
  } else {
    ra.in_half = b->scratch;
    ra.in_stride = b->Nh;
    ra.out_half = b->scratch;
    ra.out_stride = b->Nh;
  }
  // coefficients written (C2R) or read (R2C); none for the fused round trip
  g_next_bytes = MODE == sl::dev::ROW_RT ? 0.0 : 4.0 * (double)b->N * nf;
  if (s.ndim == 2) {
    const int L1 = (int)s.dims[1];
    dim3 g((L0 / 2 + row_pairs_per_cta(L1) - 1) / row_pairs_per_cta(L1), nf);
    return launched(launch_row<MODE>(L1, g, st, ra), "row pass");
  }
  g_next_bytes = MODE == sl::dev::ROW_RT ? 0.0 : 4.0 * (double)b->N * nf;
  dim3 g(L0, nf);
  return launched(launch_plane<MODE>((int)s.dims[1], (int)s.dims[2], g, st, ra), "plane pass");
}

static sl_status fwd_filter_pass(const sl_bank* b, int j0, int nf, cudaStream_t st) {
  const int L0 = (int)b->spec.dims[0];
  ColArgs ca{};
  ca.in = b->xhat;
  ca.out = b->scratch;
  ca.psi = b->psi;
  ca.Nh = b->Nh;
  ca.NP = (int)(b->Nh / L0);
  ca.j0 = j0;
  ca.nfilt = nf;
  dim3 g((ca.NP + col_tile(L0) - 1) / col_tile(L0), nf);
  g_next_bytes = 4.0 * (double)b->Nh * nf;  // filters read
  return launched(launch_col<sl::dev::COL_FWD_FILT>(L0, g, st, ca), "col_fwd_filter");
}

static sl_status inv_acc_pass(const sl_bank* b, int g_idx, int j0, int nf, cudaStream_t st) {
  const int L0 = (int)b->spec.dims[0];
  ColArgs ca{};
  ca.in = b->scratch;
  ca.out = b->partial;
  ca.psi = b->psi;
  ca.Nh = b->Nh;
  ca.NP = (int)(b->Nh / L0);
  ca.j0 = j0;
  ca.nfilt = nf;
  ca.fps = b->fps;
  ca.part0 = g_idx * b->S;
  const int splits = (nf + b->fps - 1) / b->fps;
  dim3 g((ca.NP + col_tile(L0) - 1) / col_tile(L0), splits);
  g_next_bytes = 4.0 * (double)b->Nh * nf;  // filters read
  return launched(launch_col<sl::dev::COL_INV_ACC>(L0, g, st, ca), "col_inv_accumulate");
}

// Partials -> spectrum (times 1/Psi for the inverse) -> real x.
static sl_status inv_final(const sl_bank* b, int nparts_used, bool use_invpsi, float* x,
                           cudaStream_t st) {
  const sl::BankSpec& s = b->spec;
  const int L0 = (int)s.dims[0];
  ColArgs ca{};
  ca.in = b->partial;
  ca.out = b->xhat;
  ca.invPsi = b->invPsi;
  ca.Nh = b->Nh;
  ca.NP = (int)(b->Nh / L0);
  ca.nparts = nparts_used;
  ca.use_invpsi = use_invpsi ? 1 : 0;
  dim3 g((ca.NP + col_tile(L0) - 1) / col_tile(L0), 1);
  g_next_bytes = use_invpsi ? 8.0 * (double)b->Nh : 0.0;  // 1/Psi read
  SL_TRY(launched(launch_col<sl::dev::COL_INV_FIN>(L0, g, st, ca), "col_inv_final"));
  RowArgs ra{};
  ra.in_half = b->xhat;
  ra.out_real = x;
  ra.scale = (float)(1.0 / (double)b->N);
  ra.nh = (int)s.nh();
  ra.n_rows = L0;
  g_next_bytes = 4.0 * (double)b->N;  // the signal is written once
  if (s.ndim == 2) {
    const int L1 = (int)s.dims[1];
    dim3 gr((L0 / 2 + row_pairs_per_cta(L1) - 1) / row_pairs_per_cta(L1), 1);
    return launched(launch_row<sl::dev::ROW_C2R>(L1, gr, st, ra), "row_c2r");
  }
  g_next_bytes = 4.0 * (double)b->N;
  dim3 gp(L0, 1);
  return launched(launch_plane<sl::dev::ROW_C2R>((int)s.dims[1], (int)s.dims[2], gp, st, ra),
                  "plane_c2r");
}

// Partials are written compactly: group g uses parts [g*S, g*S + splits_g). Every
// group but the last holds G filters and so uses all S of its parts; the used parts
// are therefore the contiguous range [0, parts_used).
static int parts_used(const sl_bank* b) {
  const int last = b->R - (b->ngroups - 1) * b->G;
  return (b->ngroups - 1) * b->S + (last + b->fps - 1) / b->fps;
}

static void fill_thresholds(const sl_bank* b, int j0, int nf, float sigma, const float* K,
                            Thresholds* t) {
  for (int i = 0; i < nf; ++i) {
    const sl::FilterDesc& f = b->filt[j0 + i];
    t->v[i] = f.scale < 0 ? 0.f : (float)((double)K[f.scale] * (double)sigma * b->norms[j0 + i]);
  }
}

static sl_status backward(const sl_bank* b, const float* coeffs, float* x, bool use_invpsi,
                          cudaStream_t st) {
  for (int g = 0; g < b->ngroups; ++g) {
    const int j0 = g * b->G;
    const int nf = std::min(b->G, b->R - j0);
    SL_TRY(slab_pass<sl::dev::ROW_R2C>(b, j0, nf, coeffs, nullptr, nullptr, st));
    SL_TRY(inv_acc_pass(b, g, j0, nf, st));
  }
  return inv_final(b, parts_used(b), use_invpsi, x, st);
}

extern "C" {

sl_status sl_forward(const sl_bank* b, const float* x, float* coeffs, void* stream) {
  SL_TRY(check_call(b));
  if (!x || !coeffs) return fail(SL_EINVAL, "x or coeffs is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  SL_TRY(spectrum_of(b, x, st));
  for (int g = 0; g < b->ngroups; ++g) {
    const int j0 = g * b->G;
    const int nf = std::min(b->G, b->R - j0);
    SL_TRY(fwd_filter_pass(b, j0, nf, st));
    SL_TRY(slab_pass<sl::dev::ROW_C2R>(b, j0, nf, nullptr, coeffs, nullptr, st));
  }
  return SL_OK;
}

sl_status sl_adjoint(const sl_bank* b, const float* coeffs, float* x, void* stream) {
  SL_TRY(check_call(b));
  if (!x || !coeffs) return fail(SL_EINVAL, "x or coeffs is NULL");
  return backward(b, coeffs, x, false, (cudaStream_t)stream);
}

sl_status sl_inverse(const sl_bank* b, const float* coeffs, float* x, void* stream) {
  SL_TRY(check_call(b));
  if (!x || !coeffs) return fail(SL_EINVAL, "x or coeffs is NULL");
  return backward(b, coeffs, x, true, (cudaStream_t)stream);
}

sl_status sl_threshold(const sl_bank* b, float* coeffs, float sigma, const float* K,
                       void* stream) {
  SL_TRY(check_call(b));
  if (!coeffs || !K) return fail(SL_EINVAL, "coeffs or K is NULL");
  if (!(sigma >= 0.f) || !std::isfinite(sigma)) return fail(SL_EINVAL, "sigma must be >= 0");
  for (int j = 0; j < b->spec.J; ++j)
    if (!std::isfinite(K[j])) return fail(SL_EINVAL, "K must be finite");
  cudaStream_t st = (cudaStream_t)stream;
  for (int j0 = 1; j0 < b->R; j0 += kMaxGroup) {
    const int nf = std::min(kMaxGroup, b->R - j0);
    Thresholds t;
    fill_thresholds(b, j0, nf, sigma, K, &t);
    const int64_t n4 = b->N / 4;
    int gx = (int)std::min<int64_t>((n4 + kThreads - 1) / kThreads, 64);
    dim3 g(std::max(gx, 1), nf);
    float* base = coeffs + (int64_t)j0 * b->N;
    const int64_t n = b->N;
    g_next_bytes = 8.0 * (double)n * nf;  // read and write
    SL_TRY(launched(timed_launch("threshold", st, [&]() {
                      sl::dev::k_threshold<<<g, kThreads, 0, st>>>(base, n, nf, t);
                    }),
                    "threshold"));
  }
  return SL_OK;
}

sl_status sl_denoise(const sl_bank* b, const float* noisy, float* out, float sigma,
                     const float* K, void* stream) {
  SL_TRY(check_call(b));
  if (!noisy || !out || !K) return fail(SL_EINVAL, "noisy, out or K is NULL");
  if (!(sigma >= 0.f) || !std::isfinite(sigma)) return fail(SL_EINVAL, "sigma must be >= 0");
  cudaStream_t st = (cudaStream_t)stream;
  SL_TRY(spectrum_of(b, noisy, st));
  for (int g = 0; g < b->ngroups; ++g) {
    const int j0 = g * b->G;
    const int nf = std::min(b->G, b->R - j0);
    Thresholds t;
    fill_thresholds(b, j0, nf, sigma, K, &t);
    SL_TRY(fwd_filter_pass(b, j0, nf, st));
    SL_TRY(slab_pass<sl::dev::ROW_RT>(b, j0, nf, nullptr, nullptr, &t, st));
    SL_TRY(inv_acc_pass(b, g, j0, nf, st));
  }
  return inv_final(b, parts_used(b), true, out, st);
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
  SL_CUDA(cudaMemcpyAsync(b->e2e_x, x_host, (size_t)b->N * sizeof(float),
                          cudaMemcpyHostToDevice, st));
  SL_TRY(sl_forward(b, b->e2e_x, b->e2e_c, stream));
  SL_TRY(sl_inverse(b, b->e2e_c, b->e2e_x, stream));
  SL_CUDA(cudaMemcpyAsync(y_host, b->e2e_x, (size_t)b->N * sizeof(float),
                          cudaMemcpyDeviceToHost, st));
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
  const int64_t cap = (int64_t)(SL_NOALLOC_SCRATCH_BYTES / sizeof(float2));
  if (2 * b->Nh > cap)
    return fail(SL_ENOTSUP, "sl_forward_noalloc: the signal's spectrum plus one filter's "
                            "spectrum need " + std::to_string(2 * b->Nh * 8) +
                            " bytes, more than SL_NOALLOC_SCRATCH_BYTES (16 MiB)");
  int dev = -1;
  SL_CUDA(cudaGetDevice(&dev));
  SL_TRY(init_device(dev));
  float2* xhat = nullptr;
  SL_TRY(noalloc_scratch_ptr(dev, &xhat));
  float2* slots = xhat + b->Nh;
  const int G = (int)std::min<int64_t>({(cap - b->Nh) / b->Nh, (int64_t)kMaxGroup, (int64_t)b->R});
  cudaStream_t st = (cudaStream_t)stream;
  const sl::BankSpec& s = b->spec;
  const int L0 = (int)s.dims[0];
  const int NP = (int)(b->Nh / L0);
  const int ctiles = (NP + col_tile(L0) - 1) / col_tile(L0);

  // spectrum of x: last axes (rows or planes), then pencils along axis 0, in place
  RowArgs ra{};
  ra.in_real = x;
  ra.out_half = xhat;
  ra.scale = 1.f;
  ra.nh = (int)s.nh();
  ra.n_rows = L0;
  if (s.ndim == 2) {
    const int L1 = (int)s.dims[1];
    dim3 g((L0 / 2 + row_pairs_per_cta(L1) - 1) / row_pairs_per_cta(L1), 1);
    SL_TRY(launched(launch_row<sl::dev::ROW_R2C>(L1, g, st, ra), "row_r2c"));
  } else {
    SL_TRY(launched(launch_plane<sl::dev::ROW_R2C>((int)s.dims[1], (int)s.dims[2], dim3(L0, 1),
                                                   st, ra), "plane_r2c"));
  }
  ColArgs ca{};
  ca.in = xhat;
  ca.out = xhat;
  ca.Nh = b->Nh;
  ca.NP = NP;
  SL_TRY(launched(launch_col<sl::dev::COL_SPEC>(L0, dim3(ctiles, 1), st, ca), "col_spec"));

  // per group of G filters: pencils (x psi, inverse FFT) into the slots, then the
  // last axes into the caller's coefficient planes
  for (int j0 = 0; j0 < b->R; j0 += G) {
    const int nf = std::min(G, b->R - j0);
    ColArgs cf{};
    cf.in = xhat;
    cf.out = slots;
    cf.psi = psi;
    cf.Nh = b->Nh;
    cf.NP = NP;
    cf.j0 = j0;
    cf.nfilt = nf;
    SL_TRY(launched(launch_col<sl::dev::COL_FWD_FILT>(L0, dim3(ctiles, nf), st, cf),
                    "col_fwd_filter"));
    RowArgs rc{};
    rc.in_half = slots;
    rc.in_stride = b->Nh;
    rc.out_real = coeffs + (int64_t)j0 * b->N;
    rc.out_stride = b->N;
    rc.scale = (float)(1.0 / (double)b->N);
    rc.nh = (int)s.nh();
    rc.n_rows = L0;
    if (s.ndim == 2) {
      const int L1 = (int)s.dims[1];
      dim3 g((L0 / 2 + row_pairs_per_cta(L1) - 1) / row_pairs_per_cta(L1), nf);
      SL_TRY(launched(launch_row<sl::dev::ROW_C2R>(L1, g, st, rc), "row_c2r"));
    } else {
      SL_TRY(launched(launch_plane<sl::dev::ROW_C2R>((int)s.dims[1], (int)s.dims[2],
                                                     dim3(L0, nf), st, rc), "plane_c2r"));
    }
  }
  return SL_OK;
}
