/*
 * libshearlet: B300-native (sm_103a) non-subsampled digital shearlet transform.
 *
 * The transform of ShearLab 3D (Kutyniok, Lim, Reisenhofer, arXiv 1402.5670) in the
 * shift-invariant form of Sec. 3.4 (eq. convolution): for a real signal x on an
 * n0 x n1 (2D) or n0 x n1 x n2 (3D) grid and a bank of R real, even filters psi_j,
 *
 *   forward   C_j = Re IFFT( FFT(x) * conj(psi_hat_j) )                j = 0..R-1
 *   adjoint   x   = Re IFFT( sum_j FFT(C_j) * psi_hat_j )
 *   inverse   x   = Re IFFT( sum_j FFT(C_j) * psi_hat_j / Psi )       (eq. reconstruction)
 *             Psi = sum_j |psi_hat_j|^2                                (eq. frame_filter)
 *   threshold C_j(m) kept iff |C_j(m)| >= K[s(j)] sigma ||psi_j||_2    (eq. hard_tresholding)
 *
 * Conventions for every call below.
 *   Layout:    signals are contiguous row-major float32 arrays, last axis fastest
 *              (x[i0][i1] or x[i0][i1][i2]). Coefficients are the stack C[R][dims]:
 *              one contiguous plane/volume per filter, filter 0 (the lowpass) first.
 *   Memory:    unless a name ends in _host, data pointers are DEVICE pointers on the
 *              bank's device, owned by the caller; the library never frees them.
 *              Signal and coefficient arrays must be 16-byte aligned (cudaMalloc and
 *              torch allocations are); SL_EINVAL otherwise.
 *              The library owns the bank, its filters and its scratch memory.
 *   Streams:   `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *              stream). Calls are asynchronous on that stream; the caller
 *              synchronises before reading results on the host.
 *   Threading: calls on the same bank share its scratch memory: issue them on one
 *              stream (or serialise them). Distinct banks are independent.
 *   Errors:    every call returns an sl_status; nothing aborts the process and no
 *              exception crosses this boundary. sl_last_error() describes the last
 *              failure on the calling thread.
 * Filter order (index j): 0 is the lowpass; then scales coarse to fine; within a
 * scale cone 1 then cone 2 (2D) or pyramid 1, 2, 3 (3D), shears ascending
 * (3D: k1 outer, k2 inner).
 */
#ifndef SHEARLET_H
#define SHEARLET_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SL_OK = 0,
  SL_EINVAL = 1,    /* invalid argument: sizes, levels, null pointers, wrong device */
  SL_ENOMEM = 2,    /* device or host allocation failed */
  SL_ECUDA = 3,     /* a CUDA runtime call or kernel launch failed */
  SL_ETIMEOUT = 4,  /* a bounded device-side wait gave up */
  SL_ENOTSUP = 5,   /* valid request this build does not implement (e.g. a size) */
  SL_ENAN = 6       /* non-finite values where finite ones are required */
} sl_status;

typedef struct sl_bank sl_bank; /* opaque; owned by the library */

/* Human-readable name of a status code (static storage). */
const char* sl_status_str(sl_status s);

/* Text of the last error raised on the calling thread (static per-thread storage). */
const char* sl_last_error(void);

/*
 * Build the digital shearlet filter bank on an N-grid, once (Algorithm 1 prologue;
 * Sec. 4.3 "SLgetShearletSystem2D").
 *   ndim         2 or 3.
 *   dims         ndim sizes (host array), each a power of two in [8, 1024]; in 2D a
 *                side may also be 384 = 3 * 2^7 (mixed radix-3/radix-2 line FFTs).
 *   nScales      number of scales J >= 1 (Sec. 4.1 'nScales').
 *   shearLevels  J entries d_j in [0, 4] (host array), coarse to fine (Sec. 4.1
 *                'shearLevels'); scale j then has 2^(d_j+2) filters in 2D and
 *                3(2 2^d+1)^2 - 6(2 2^d+1) + 4 in 3D (Sec. 4.4).
 *   fullSystem   0: omit the boundary shearlets on the seams (Sec. 4.4); 1: keep them.
 *   device       CUDA device ordinal that will run the transforms; -1 builds a
 *                host-only bank (filters evaluable with sl_bank_eval_f64, no transforms).
 *   out          receives the bank; free it with sl_free_filters.
 * The filters are evaluated in FP64 on the host from their closed-form frequency
 * responses (eqs. lowhigh, nonsep, dshear*_alpha, Defs. digitSH_alpha and
 * 3DdigitSH_alpha), normalised so that max Psi = 1, and uploaded once: psi_hat as a
 * real FP32 half spectrum, 1/Psi in FP64. Scratch memory for the transforms is
 * allocated here. The calling thread's current device is set to `device`.
 * Errors: SL_EINVAL (arguments), SL_ENOTSUP (sizes), SL_ENOMEM, SL_ECUDA.
 */
sl_status sl_build_filters(int ndim, const int64_t* dims, int nScales,
                           const int* shearLevels, int fullSystem, int device,
                           sl_bank** out);

/* Options of sl_build_filters_ex. Zero-initialise, then set what you need. */
enum { SL_PATH_AUTO = 0, SL_PATH_GENERAL = 1, SL_PATH_CLUSTER = 2 };
typedef struct {
  /* Kernel path of sl_forward / sl_adjoint / sl_inverse:
   *   SL_PATH_AUTO     the path measured faster on B300 (currently the general
   *                    path everywhere);
   *   SL_PATH_GENERAL  pencil pass along axis 0 and row/plane passes, with the
   *                    per-filter intermediates in library scratch memory;
   *   SL_PATH_CLUSTER  2D grids with both sides in [64, 512] only: one cluster of
   *                    8 CTAs transforms a whole filter's spectrum in distributed
   *                    shared memory (SL_ENOTSUP elsewhere).
   * Both paths compute the same result. */
  int path;
  /* Arithmetic of the pencil passes (axis 0) inside the per-filter loops of
   * sl_forward, sl_adjoint, sl_inverse and sl_denoise:
   *   SL_PREC_FP32     FP32 register FFTs (error vs FP64 about 1e-6 relative);
   *   SL_PREC_TC_BF16  radix-8 DFT stages as BF16 tensor-core matrix products with
   *                    split operands (hi + lo) and FP32 accumulation; error vs FP64
   *                    about 1e-5 relative. Needs the general path and n0 a power
   *                    of two in [64, 1024] (SL_ENOTSUP otherwise).
   *   SL_PREC_TC_FP16  the same stages with FP16 operands (hi + lo, about 22 bits);
   *                    each warp's operand block is scaled by a power of two into
   *                    FP16's range first; error vs FP64 about 1e-6 relative. Same
   *                    requirements as SL_PREC_TC_BF16.
   * The last-axis passes, the single-signal FFTs and the FP64 division by Psi are
   * the same in every mode. */
  int precision;
  int reserved[6];
} sl_options;
enum { SL_PREC_FP32 = 0, SL_PREC_TC_BF16 = 1, SL_PREC_TC_FP16 = 2 };

/* sl_build_filters with options (opt may be NULL: defaults). */
sl_status sl_build_filters_ex(int ndim, const int64_t* dims, int nScales,
                              const int* shearLevels, int fullSystem, int device,
                              const sl_options* opt, sl_bank** out);

/* User-supplied filters of the construction (Sec. 4.1: the quadrature mirror
 * filter's lowpass, h_1 of eq. lowhigh, and the 2D directional filter, P of eq.
 * nonsep). NULL pointers keep the built-in designs (the symmetric maximally flat
 * 9-tap lowpass of Sec. 5.1 and a maximally flat fan filter).
 *   qmf:  qmf_len taps h(-m..m) (qmf_len = 2m + 1), symmetric: h(-n) = h(n);
 *         the highpass is g(n) = (-1)^n h(n).
 *   fan:  fan_rows x fan_cols taps P(n1, n2), row-major, centred (both sizes odd),
 *         point-symmetric: P(-n) = P(n); rows pair with xi_1 (the principal axis of
 *         the first cone), columns with xi_2.
 * Symmetry (to 1e-12 relative) keeps every filter's spectrum real and even, which
 * the transforms rely on; asymmetric taps, even sizes, more than 129 qmf taps or
 * more than 65 x 65 fan taps are SL_EINVAL, and so is a system whose frame weight
 * Psi vanishes somewhere on the grid. Taps are copied. */
typedef struct {
  const double* qmf;
  int qmf_len;
  const double* fan;
  int fan_rows;
  int fan_cols;
} sl_filters;

/* sl_build_filters_ex with user filters (filters may be NULL: built-in designs). */
sl_status sl_build_filters_user(int ndim, const int64_t* dims, int nScales,
                                const int* shearLevels, int fullSystem, int device,
                                const sl_options* opt, const sl_filters* filters,
                                sl_bank** out);

/*
 * The separable stationary wavelet system on the same grid (the isotropic dictionary
 * of the image decomposition, Sec. 5.5: "the stationary wavelet transform"), as a
 * bank that every transform call of this header accepts. Filters, in this order:
 * the lowpass h_J(xi_1) h_J(xi_2) (the shearlet system's lowpass), then for each scale
 * j = 0..J-1 coarse to fine, with a = J - j and h_a, g_a the a trous filters of eq.
 * lowhigh: g_a(xi_1) h_a(xi_2), h_a(xi_1) g_a(xi_2), g_a(xi_1) g_a(xi_2)
 * (sl_bank_filter_meta: scale j, cone 1, 2, 3). R = 1 + 3 J. Normalised like a shearlet
 * bank (max Psi = 1, 1/Psi in FP64), so sl_inverse is the dual-frame inverse.
 *   ndim 2 only (SL_ENOTSUP for 3); dims and nScales as sl_build_filters; filters
 *   may be NULL or give a user QMF lowpass (its fan member must be NULL).
 */
sl_status sl_build_wavelets(int ndim, const int64_t* dims, int nScales, int device,
                            const sl_filters* filters, sl_bank** out);

/* Release a bank and all library memory it holds. NULL is ignored. Call it with no
 * transform of this bank still running on the GPU. */
void sl_free_filters(sl_bank* bank);

/* Shape of a bank: ndim, dims[0..ndim-1] (host array of 3), R (number of filters,
 * the redundancy of Sec. 4.3's table: 1 + sum over scales of the filters per scale of
 * Secs. 4.1 and 4.4), nScales. Any output pointer may be NULL. */
sl_status sl_bank_info(const sl_bank* bank, int* ndim, int64_t* dims, int* R,
                       int* nScales);

/* Per-filter metadata (host arrays of R entries; any may be NULL): scale_of[j] in
 * 0..J-1 (-1 for the lowpass), cone_of[j] (2D cone 1/2 of Def. digitSH_alpha and eq.
 * convolution01, 3D pyramid 1..3 of Def. 3DdigitSH_alpha, 0 for the lowpass),
 * k_of[2j], k_of[2j+1] the shear parameter(s) k of the digital shear S^d_{k/2^d}
 * (eqs. dshear1_alpha, dshear2_alpha; 2D: k and 0). */
sl_status sl_bank_filter_meta(const sl_bank* bank, int* scale_of, int* cone_of,
                              int* k_of);

/* norms[j] = ||psi_j||_2 (host array of R, may be NULL; the factor of the threshold of
 * eq. hard_tresholding) and the frame bounds A = min Psi, B = max Psi of the frame
 * weight of eq. frame_filter (= 1 after normalisation; the quantities of Sec. 4.3's
 * table of frame bounds), FP64. */
sl_status sl_bank_norms(const sl_bank* bank, double* norms, double* A, double* B);

/* The kernel path the bank's transforms take: SL_PATH_GENERAL or SL_PATH_CLUSTER
 * (sl_denoise and sl_forward_noalloc always take the general path). */
sl_status sl_bank_path(const sl_bank* bank, int* path);

/* The bank's precision mode (SL_PREC_FP32, SL_PREC_TC_BF16 or SL_PREC_TC_FP16). */
sl_status sl_bank_precision(const sl_bank* bank, int* precision);

/* Number of half-spectrum points Nh = N / n_last * (n_last/2 + 1), and N. */
sl_status sl_bank_sizes(const sl_bank* bank, int64_t* N, int64_t* Nh);

/* Evaluate filter j in FP64 on the host (normalised psi_hat_j on the half spectrum,
 * layout [n0][..][n_last/2+1]) into the host array out[Nh]. j = -1 writes Psi. */
sl_status sl_bank_eval_f64(const sl_bank* bank, int j, double* out);

/* Copy the device FP32 filter bank [R][Nh] into the host array out. */
sl_status sl_bank_filters_f32(const sl_bank* bank, float* out);

/*
 * Forward transform (Algorithm 1 with the conjugation of eq. convolution):
 * x[dims] -> coeffs[R][dims]. Device pointers. coeffs must not alias x.
 */
sl_status sl_forward(const sl_bank* bank, const float* x, float* coeffs, void* stream);

/* Adjoint of sl_forward: coeffs[R][dims] -> x[dims] (Algorithm 2 with the filters
 * psi_hat_j in place of the duals). */
sl_status sl_adjoint(const sl_bank* bank, const float* coeffs, float* x, void* stream);

/* Dual-frame inverse (eq. reconstruction, Algorithm 2): coeffs[R][dims] -> x[dims].
 * The division by Psi is done in FP64. sl_inverse(sl_forward(x)) = x up to rounding. */
sl_status sl_inverse(const sl_bank* bank, const float* coeffs, float* x, void* stream);

/* ------------------------------------------------------ filter ranges ---
 * One transform split by filters, for running it on several GPUs (one rank each).
 * The inverse of eq. reconstruction is a sum over j of FFT(C_j) psi_hat_j / Psi
 * (Algorithm 2), so a rank that holds the coefficients of filters [j0, j1) turns them
 * into one partial spectrum; the ranks add their partials (one reduction, e.g.
 * ncclAllReduce or ncclReduce of 2 * n_points floats, sum), and one rank finishes
 * with the division by Psi and the inverse FFT. The forward transform (Algorithm 1)
 * needs X_hat = FFT(x) on every rank (one broadcast of 2 * n_points floats), after
 * which each rank produces its own range. Every call here takes the general kernel
 * path (whatever the bank's path) and the bank's precision mode; sharded and
 * unsharded results agree to rounding (partials summed in another order).
 * Spectrum buffers are DEVICE float arrays of 2 * n_points floats (complex
 * interleaved) in the library's internal layout (a half spectrum cut into pencil
 * tiles, padded); adding two of them elementwise adds the spectra, and nothing else
 * about the layout may be assumed. 16-byte aligned like every other array.
 */

/* n_points: complex points in one spectrum buffer of this bank. */
sl_status sl_spectrum_points(const sl_bank* bank, int64_t* n_points);

/* X_hat = FFT(x), the first step of Algorithm 1: x DEVICE [dims] -> xhat (spectrum
 * buffer). Errors as sl_forward. */
sl_status sl_spectrum(const sl_bank* bank, const float* x, float* xhat, void* stream);

/* C_j = Re IFFT(X_hat conj(psi_hat_j)) for j in [j0, j1) (Algorithm 1's loop over a
 * filter range; eq. convolution): xhat a spectrum buffer from sl_spectrum (read only),
 * coeffs DEVICE [j1 - j0][dims] (plane i holds filter j0 + i). Concatenating the
 * ranges of all ranks gives exactly sl_forward's coefficients (same kernels).
 * SL_EINVAL unless 0 <= j0 <= j1 <= R; an empty range does nothing (coeffs may then
 * be NULL). */
sl_status sl_forward_range(const sl_bank* bank, const float* xhat, int j0, int j1,
                           float* coeffs, void* stream);

/* partial = sum_{j in [j0, j1)} FFT(C_j) psi_hat_j (the inner sum of eq. reconstruction
 * over one filter range): coeffs DEVICE [j1 - j0][dims] as sl_forward_range writes
 * them (NULL allowed for an empty range); partial a spectrum buffer, overwritten
 * (zeros for an empty range). */
sl_status sl_inverse_partial(const sl_bank* bank, const float* coeffs, int j0, int j1,
                             float* partial, void* stream);

/* x = Re IFFT(summed / Psi) (dual = 1: the dual-frame inverse of eq. reconstruction,
 * division in FP64) or Re IFFT(summed) (dual = 0: the adjoint), where summed is the
 * sum of every range's partial (a spectrum buffer, read only); x DEVICE [dims]. */
sl_status sl_inverse_finish(const sl_bank* bank, const float* summed, int dual, float* x,
                            void* stream);

/* -------------------------------------------------- subsampled transform ---
 * The digital shearlet transform with sampling (Defs. digitSH, digitSH_alpha: the
 * coefficients of scale j are taken on a lattice given by the sampling matrix
 * M_{c_j}), 2D banks only. Reading of the sampling: subband j of scale s(j) keeps
 * the points of (step_j Z)^2 with step_j = 2^(J-1-s(j)) (the finest scale keeps every
 * point), and the lowpass those of (2^(J-1) Z)^2. Grid sides must be multiples of
 * 2^(J-1) (SL_ENOTSUP otherwise). Coefficients are stored compactly: subband j as a
 * row-major [n0 / step_j][n1 / step_j] block at offset_j of one float array of
 * offset_R floats (sl_sub_layout). With sampling there is no direct inverse
 * (Sec. 3.4): sl_inverse_sub solves the frame equation by conjugate gradients.
 * The first call of sl_forward_sub, sl_adjoint_sub or sl_inverse_sub on a bank
 * allocates its working memory there: a full coefficient stack (R N floats), five
 * [dims] vectors and the FP64 preconditioner table.
 */

/* step[R] (lattice step of each subband) and offset[R + 1] (compact offsets; offset[R]
 * is the total count); host arrays, either may be NULL. Host-only banks work too. */
sl_status sl_sub_layout(const sl_bank* bank, int* step, int64_t* offset);

/* Subsampled forward transform: x DEVICE [dims] -> coeffs_sub DEVICE [offset_R]. */
sl_status sl_forward_sub(const sl_bank* bank, const float* x, float* coeffs_sub, void* stream);

/* Its adjoint: coeffs_sub -> x = sum_j psi_j * (coefficients of subband j on its
 * lattice, zero elsewhere) (DEVICE arrays). */
sl_status sl_adjoint_sub(const sl_bank* bank, const float* coeffs_sub, float* x, void* stream);

/* Inverse of the subsampled transform by conjugate gradients (the frame algorithms of
 * Sec. 2.1 and the CG inversion of Sec. 3.4): solves S x = T_sub* c with
 * S = T_sub* T_sub, starting from x = 0, for exactly `iterations` steps. Each step is
 * one fused pass for S p (forward, lattice mask and adjoint with the coefficients kept
 * on chip), FP64 inner products and, if `precondition` is nonzero, the preconditioner
 * z = IFFT(FFT(r) / Psi_sub), Psi_sub = sum_j |psi_hat_j|^2 / step_j^2 (FP64): the
 * frame weight of eq. frame_filter with each subband's sampling density, which equals
 * S when nothing is subsampled. Measured on a 256^2 four-scale bank: preconditioned,
 * about ten steps reach the FP32 limit; plain CG needs several times more.
 * rel_residual (host, may be NULL) receives ||T_sub* c - S x|| / ||T_sub* c|| after the
 * last step; passing it synchronises the stream. Step sizes stay on the device (no
 * host round trip per step). */
sl_status sl_inverse_sub(const sl_bank* bank, const float* coeffs_sub, float* x, int iterations,
                         int precondition, double* rel_residual, void* stream);

/* Synchronises `stream` and reports whether a bounded wait of a transform kernel on
 * the current device ran out since the last check: the filter-loop kernels stage
 * their tiles with bulk copies that complete on shared-memory barriers, and every
 * wait on those gives up after about two seconds, sets a device flag and returns
 * with that CTA's work undone. SL_ETIMEOUT (and the flag cleared) if so, SL_OK
 * otherwise. */
sl_status sl_device_check(void* stream);

/*
 * Hard thresholding in place (eq. hard_tresholding, Sec. 5.3): for every filter
 * j >= 1, C_j(m) = 0 unless |C_j(m)| >= K[scale(j)] * sigma * ||psi_j||_2. The lowpass
 * is left as is. K is a host array of nScales entries, coarse to fine. The threshold
 * is rounded to FP32 and compared in FP32 (a tie is kept).
 */
sl_status sl_threshold(const sl_bank* bank, float* coeffs, float sigma, const float* K,
                       void* stream);

/*
 * Denoising x_out = T^-1 T_delta T x_noisy (Sec. 5.3) in one fused pass: the
 * coefficients are thresholded as they are produced and never written to memory.
 * noisy and out are device arrays [dims] (they may alias); K as in sl_threshold.
 */
sl_status sl_denoise(const sl_bank* bank, const float* noisy, float* out, float sigma,
                     const float* K, void* stream);

/*
 * Image inpainting by iterative thresholding (Sec. 5.4, algorithm image_inpainting).
 * f_masked: DEVICE [dims] image with the occluded pixels set to anything; mask: DEVICE
 * uint8 [dims], nonzero = known pixel; out: DEVICE [dims] result (must not alias
 * f_masked). Starting from 0, each of the `iterations` steps sets the known pixels
 * of the current estimate to f_masked and replaces the estimate by the fused
 * denoising of it (as sl_denoise with K = 1 for every scale and sigma = delta, i.e.
 * subband j >= 1 thresholded at delta ||psi_j||_2, the lowpass kept); delta starts
 * at delta_init and shrinks geometrically to delta_min at the last step. The bank
 * keeps one [dims] float buffer for the iterate (allocated on first use). Work per
 * step: one elementwise pass and one fused denoise.
 */
sl_status sl_inpaint(const sl_bank* bank, const float* f_masked, const uint8_t* mask, float* out,
                     float delta_init, float delta_min, int iterations, void* stream);

/*
 * Image decomposition by iterative thresholding (Sec. 5.5, algorithm
 * image_decomposition): f = f0 + f1 with f0 the curvilinear part, sparse in the
 * shearlet bank `curv`, and f1 the isotropic part, sparse in the wavelet bank `iso`
 * (sl_build_wavelets; same grid and device). f, f0, f1: DEVICE [dims]; f0 and f1 are
 * outputs and must not alias f or each other. Starting from f0 = f1 = 0, each of the
 * `iterations` steps does
 *     f0 = T0^-1 Thr_delta T0 (f - f1)        (= the algorithm's f_res + f0)
 *     f1 = T1^-1 Thr_delta T1 (f - f0)        (f0 already updated: see below)
 * and then shrinks delta geometrically from delta_init to delta_min (as sl_inpaint).
 * Thr_delta keeps coefficient C_j(m) of subband j >= 1 iff |C_j(m)| >= delta ||psi_j||_2
 * (the denoising rule with K = 1, sigma = delta). The curvilinear part gets no lowpass
 * (the shearlet lowpass subband is dropped) and the wavelet lowpass is kept, so the
 * smooth content goes to f1. The residual is recomputed between the two updates (the
 * block-coordinate order of the morphological component analysis the paper cites);
 * the algorithm as printed computes it once per step, which makes content that both
 * dictionaries represent enter both parts at once. Work per step: two elementwise
 * passes and two fused denoising passes (one per bank). The bank `curv` keeps one
 * [dims] float buffer (allocated on first use, shared with sl_inpaint).
 * Errors: SL_EINVAL (banks of different grids or devices, aliasing, iterations < 1,
 * non-positive or non-finite deltas), SL_ENOMEM, SL_ECUDA.
 */
sl_status sl_decompose(const sl_bank* curv, const sl_bank* iso, const float* f, float* f0,
                       float* f1, float delta_init, float delta_min, int iterations,
                       void* stream);

/*
 * End-to-end round trip from HOST memory: copies x_host[dims] to the device,
 * runs sl_forward into library-owned coefficient memory, then sl_inverse, and
 * copies the reconstruction back to y_host[dims]. Host arrays should be pinned
 * (cudaHostAlloc) for asynchronous copies; with pinned buffers the work is captured
 * into a CUDA graph on the first call with a given pair of host pointers and
 * replayed by one graph launch afterwards (the bank's round-trip state is shared:
 * do not run two round trips of one bank at once). Pinned buffers that the device
 * can address (mapped, as cudaHostAlloc memory is under unified addressing) and
 * that are 16-byte aligned are read by the first kernel and written by the last one
 * directly over the host link, with no separate copy (general kernel path); other
 * pinned buffers go through cudaMemcpyAsync. Returns after queuing; synchronise the
 * stream before reading y_host.
 */
sl_status sl_fwdinv_host(const sl_bank* bank, const float* x_host, float* y_host,
                         void* stream);

/* ---------------------------------------------------------------- batches ---
 * A batch transforms n images at once, image i with bank banks[i]; the banks may
 * have different shapes (e.g. sides 256, 384, 512 and 1024 in one batch), and
 * images that share a shape share one bank. The paper transforms one signal per
 * call (Algorithms 1 and 2); a batch runs the same per-image computation, with
 * results identical bit for bit to one sl_forward / sl_inverse / sl_denoise per
 * image.
 * Execution: the images are spread over K branches (largest estimated cost first,
 * onto the least loaded branch); every branch owns a workspace and a stream, and
 * runs its images in turn. The fork and join are captured into one CUDA graph the
 * first time a call is made with a given set of data pointers (and, for denoise,
 * thresholds); later calls with the same pointers replay it with one graph launch.
 * New pointers trigger a new capture (about a millisecond of host time).
 * Arrays of pointers (x, coeffs, y, K) are HOST arrays of n entries; the pointers
 * in them are device pointers (K[i]: host array of nScales floats) on the batch's
 * device. A batch is not reentrant: issue its calls on one stream or serialise
 * them. Its memory: one workspace per branch, sized for the largest image of that
 * branch (spectrum, one filter group, partial sums; tens of MB for 1024^2).
 */
typedef struct sl_batch sl_batch; /* opaque; owned by the library */

typedef struct {
  int branches;   /* concurrent branches K; 0 = default (4), clamped to n */
  int no_graph;   /* 1: issue kernels directly instead of capturing a graph */
  int reserved[6];
} sl_batch_options;

/* Create a batch over banks[0..n) (all built on the current device, any path).
 * opt may be NULL. SL_EINVAL for NULL/invalid arguments or a host-only bank,
 * SL_ENOMEM if the workspaces do not fit. */
sl_status sl_batch_create(const sl_bank* const* banks, int n, const sl_batch_options* opt,
                          sl_batch** out);

/* Release the batch (synchronises the device when workspaces are freed). NULL is a no-op. */
void sl_batch_free(sl_batch* batch);

/* Schedule of the batch: the number of branches, and for every image (arrays of n,
 * each may be NULL) its branch and the filters-per-group cap its plan uses. */
sl_status sl_batch_info(const sl_batch* batch, int* branches, int* branch_of, int* group_cap);

/* Forward transform of every image: x[i][dims_i] -> coeffs[i][R_i][dims_i]. */
sl_status sl_batch_forward(sl_batch* batch, const float* const* x, float* const* coeffs,
                           void* stream);

/* Dual-frame inverse of every image: coeffs[i] -> x[i]. */
sl_status sl_batch_inverse(sl_batch* batch, const float* const* coeffs, float* const* x,
                           void* stream);

/* Forward then inverse of every image (coeffs[i] is written and read back):
 * x[i] -> coeffs[i] -> y[i]. */
sl_status sl_batch_fwdinv(sl_batch* batch, const float* const* x, float* const* coeffs,
                          float* const* y, void* stream);

/* Fused denoise (as sl_denoise) of every image: noisy[i] -> out[i] with thresholds
 * K[i][s] * sigma * ||psi_j||_2. Needs general-path banks (SL_ENOTSUP otherwise). */
sl_status sl_batch_denoise(sl_batch* batch, const float* const* noisy, float* const* out,
                           float sigma, const float* const* K, void* stream);

/* Autotuner. Runs sl_batch_fwdinv-shaped work on the caller's buffers (their
 * contents are overwritten) and keeps the fastest settings: first, per distinct
 * bank, the filters-per-group cap (candidates: the bank's default, R, R/2, R/4,
 * R/8; one image of that shape timed alone); then the number of branches K in
 * {1, 2, 3, 4, 6, 8, 12, 16} (<= n) for the whole batch, captured as it will run.
 * Each candidate is timed `reps` times (>= 2; the first call is a warm-up) with CUDA
 * events on `stream`, keeping the minimum. Synchronous. best_ms (may be NULL)
 * receives the best batch time. */
sl_status sl_batch_autotune(sl_batch* batch, const float* const* x, float* const* coeffs,
                            float* const* y, int reps, void* stream, double* best_ms);

/* One-shot forms: create a batch (no graph, default branches), run it on `stream`,
 * wait for the stream, free the batch. For repeated calls keep a batch instead. */
sl_status sl_forward_batch(const sl_bank* const* banks, int n, const float* const* x,
                           float* const* coeffs, void* stream);
sl_status sl_inverse_batch(const sl_bank* const* banks, int n, const float* const* coeffs,
                           float* const* x, void* stream);

/*
 * Allocation-free forward transform. The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory when they transform, e.g.
 * code running inside a fixed memory budget, a host callback, or an arena that some
 * other component owns. It computes the forward transform with sl_forward's FP32
 * general-path kernels whatever the bank's path or precision mode (so it matches
 * sl_forward within the parity tolerance, 1e-5 relative), but calls no cudaMalloc,
 * cudaFree or other allocating routine: its scratch (the signal's
 * spectrum and the per-filter intermediate spectra) lives in one static device array
 * of SL_NOALLOC_SCRATCH_BYTES (16 MiB) that every GPU which loads the library holds
 * until the process exits.
 *   bank    geometry and filter order; may be host-only (built with device = -1,
 *           which allocates no device memory). Its own device memory, if any, is
 *           not used.
 *   psi     DEVICE array [R][Nh] of the normalised FP32 filter half spectra, owned by
 *           the caller (e.g. sl_bank_filters_f32 or sl_bank_eval_f64, copied into
 *           memory the caller already has).
 *   x       DEVICE input [dims]; coeffs DEVICE output [R][dims] (must not alias x).
 * Runs on the calling thread's current device. The first call on a device does a
 * one-time set-up (looks up the static array's device address and uploads the FFT
 * twiddle tables); make that first call before any stream capture. Every call
 * shares the one array and leaves its contents behind; nothing in it has to start
 * at zero (each call overwrites what it reads), but calls whose kernels overlap on
 * the GPU (other streams, other threads) race on it: serialise them. Keep profiling
 * (sl_profile_enable) off, since it creates events per launch.
 * Errors: SL_EINVAL (NULL pointers); SL_ENOTSUP when two spectra (the half spectrum
 * padded to whole pencil tiles, 8 bytes per point) exceed SL_NOALLOC_SCRATCH_BYTES
 * (e.g. 3D 128^3); SL_ECUDA.
 */
#define SL_NOALLOC_SCRATCH_BYTES (16u << 20)
sl_status sl_forward_noalloc(const sl_bank* bank, const float* psi, const float* x,
                             float* coeffs, void* stream);

/*
 * Learned shrinkage (no counterpart in the paper's method; it replaces the hard
 * threshold of Sec. 5.3, which stays available as sl_threshold / sl_denoise). A small
 * MLP predicts a gain g in [0, 1] per coefficient of subband j >= 1 from
 *   x = [c/s, |c(m+d)|/s for d in {-1,0,1}^ndim (row-major, periodic), E_j]
 * with s = sigma ||psi_j||_2 and E_j a learned 8-vector per subband:
 *   h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), g = sigmoid(w3 . h2 + b3),
 * and the coefficient becomes g c. Width 64; products on the tensor cores in BF16
 * with FP32 accumulation; FP32 master parameters trained with Adam on the GPU.
 * Flat FP32 parameter layout (host arrays of sl_mlp_num_params floats), F = 1 + 3^ndim + 8:
 *   W1[64][F], b1[64], W2[64][64], b2[64], w3[64], b3[1], E[R][8].
 * Training loss on a sample of coefficients: mean(((g c - c_clean) / s)^2).
 */
typedef struct sl_mlp sl_mlp;

/* Create an MLP for a device bank (parameters start at zero; set them with
 * sl_mlp_set_params). The bank must outlive the MLP. */
sl_status sl_mlp_create(const sl_bank* bank, sl_mlp** out);
void sl_mlp_free(sl_mlp* mlp);
int sl_mlp_num_params(const sl_mlp* mlp);
/* Host <-> device copies of the flat parameters; set also resets Adam's state. */
sl_status sl_mlp_set_params(sl_mlp* mlp, const float* host);
sl_status sl_mlp_get_params(const sl_mlp* mlp, float* host);
/* Checkpoint and resume: write the parameters and Adam's state (moments and step
 * count) to a file, or read them back into an MLP of the same bank shape (ndim, R;
 * SL_EINVAL for another shape, a missing file or a truncated one). Training that
 * resumes from a checkpoint takes exactly the steps it would have taken. */
sl_status sl_mlp_save(const sl_mlp* mlp, const char* path);
sl_status sl_mlp_load(sl_mlp* mlp, const char* path);
/* Gradients of the loss over the n samples idx (DEVICE int32 flat indices
 * q = j * N + m with j >= 1; n a positive multiple of 128) of the DEVICE coefficient
 * stacks noisy and clean [R][dims], copied to grad_host[num_params] and *loss_host
 * (either may be NULL). Synchronises the stream. */
sl_status sl_mlp_gradients(sl_mlp* mlp, const float* noisy, const float* clean, float sigma,
                           const int* idx, int n, float* grad_host, float* loss_host,
                           void* stream);
/* One training step: gradients as above, then an Adam update (beta1 0.9, beta2 0.999,
 * eps 1e-8, learning rate lr). The sample's loss (before the update) is written to
 * the DEVICE float loss_dev if not NULL. Asynchronous. */
sl_status sl_mlp_train_step(sl_mlp* mlp, const float* noisy, const float* clean, float sigma,
                            const int* idx, int n, float lr, float* loss_dev, void* stream);
/* out[j] = g * coeffs[j] for every subband j >= 1 and out[0] = coeffs[0] (DEVICE
 * [R][dims]; out must not alias coeffs, whose neighbourhoods the features read). */
sl_status sl_mlp_apply(sl_mlp* mlp, const float* coeffs, float* out, float sigma, void* stream);
/* Engine of sl_mlp_apply, sl_mlp_gradients and sl_mlp_train_step. SL_MLP_TCGEN05
 * (default): tcgen05.mma on tiles of 128 samples with the accumulators in tensor
 * memory; training runs the forward and backward products and the weight-gradient
 * sums over each CTA's tiles there, and adds the CTAs' partial gradients in a fixed
 * order (SL_ENOTSUP from training when R * 32 bytes of embedding gradients do not fit
 * the CTA's shared memory beside its tiles, R above about 2900). SL_MLP_MMA_SYNC:
 * warp-level mma.sync on tiles of 16, gradients summed with atomics. Same BF16 operands
 * and FP32 accumulation; sums may round in another order. SL_EINVAL for another
 * value. */
#define SL_MLP_TCGEN05 0
#define SL_MLP_MMA_SYNC 1
sl_status sl_mlp_set_engine(sl_mlp* mlp, int engine);
/* Synchronises the stream and reports whether a tensor-core wait of an earlier
 * sl_mlp_apply or training call ran out (each wait gives up after about two seconds,
 * sets a device flag and the kernel returns: apply with that tile's output unwritten,
 * training with that CTA's gradient share dropped): SL_ECUDA and the flag cleared if
 * so, SL_OK otherwise. */
sl_status sl_mlp_check(sl_mlp* mlp, void* stream);
/* Learned denoising: sl_forward, sl_mlp_apply, sl_inverse (DEVICE [dims] arrays; the
 * first call allocates 2 R N floats of coefficient memory kept by the MLP). */
sl_status sl_mlp_denoise(sl_mlp* mlp, const float* noisy, float* out, float sigma, void* stream);
/* Text of the last MLP error on the calling thread. */
const char* sl_mlp_last_error(void);

/*
 * Error statistics of y against ref (DEVICE float arrays of n elements), accumulated
 * in FP64 on the GPU: stats[0] = max |y - ref|, stats[1] = max |ref|,
 * stats[2] = sum (y - ref)^2, stats[3] = sum ref^2 (host array of 4 doubles).
 * PSNR (eq. PSNR, Sec. 5.3) = 20 log10(255 sqrt(n) / sqrt(stats[2])); the relative
 * errors of the parity tests are stats[0] / stats[1] and sqrt(stats[2] / stats[3]).
 * Synchronises the stream.
 */
sl_status sl_error_stats(const float* y, const float* ref, int64_t n, double* stats,
                         void* stream);

/*
 * Kernel timing for profiling. When enabled, every kernel launch of the library is
 * bracketed by CUDA events recorded on the launch stream; sl_profile_read returns,
 * per kernel kind, the number of launches, their summed device time (ms) and their
 * summed algorithmic bytes (the DRAM traffic the transform needs in principle: the
 * signal, the coefficients, the filters and 1/Psi, each counted once where it is
 * read or written), after synchronising those events. Disabled by default; enabling
 * it adds two event records per launch. Not for use inside stream capture.
 */
sl_status sl_profile_enable(int on);
sl_status sl_profile_reset(void);
/* Up to `cap` kinds: names[i] (valid until the next sl_profile_reset), launches[i],
 * ms[i], bytes[i]; any array may be NULL. *count receives the number of kinds. */
sl_status sl_profile_read(const char** names, int64_t* launches, double* ms, double* bytes,
                          int cap, int* count);

#ifdef __cplusplus
}
#endif

#endif /* SHEARLET_H */
