"""ctypes binding of libshearlet (include/shearlet.h): argument marshalling only.

Every function here forwards to the C ABI function of the same name; the transform
itself runs in the library's CUDA kernels. Device buffers are torch CUDA tensors
(float32, contiguous); the stream is torch's current stream unless one is given.
There is no fallback: if libshearlet.so is missing or fails to load, the import of
this module's functions raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libshearlet.so")

SL_OK = 0
STATUS = {0: "SL_OK", 1: "SL_EINVAL", 2: "SL_ENOMEM", 3: "SL_ECUDA", 4: "SL_ETIMEOUT",
          5: "SL_ENOTSUP", 6: "SL_ENAN"}

_c_int64_p = ctypes.POINTER(ctypes.c_int64)
_c_int_p = ctypes.POINTER(ctypes.c_int)
_c_double_p = ctypes.POINTER(ctypes.c_double)
_c_float_p = ctypes.POINTER(ctypes.c_float)
_vp = ctypes.c_void_p

# name -> (restype, argtypes); the declarations of include/shearlet.h
SIGNATURES = {
    "sl_status_str": (ctypes.c_char_p, [ctypes.c_int]),
    "sl_last_error": (ctypes.c_char_p, []),
    "sl_build_filters": (ctypes.c_int, [ctypes.c_int, _c_int64_p, ctypes.c_int, _c_int_p,
                                        ctypes.c_int, ctypes.c_int, ctypes.POINTER(_vp)]),
    "sl_build_filters_user": (ctypes.c_int, [ctypes.c_int, _c_int64_p, ctypes.c_int, _c_int_p,
                                             ctypes.c_int, ctypes.c_int, _vp, _vp,
                                             ctypes.POINTER(_vp)]),
    "sl_build_filters_ex": (ctypes.c_int, [ctypes.c_int, _c_int64_p, ctypes.c_int, _c_int_p,
                                           ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                           ctypes.POINTER(_vp)]),
    "sl_build_wavelets": (ctypes.c_int, [ctypes.c_int, _c_int64_p, ctypes.c_int, ctypes.c_int, _vp,
                                         ctypes.POINTER(_vp)]),
    "sl_decompose": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, ctypes.c_float, ctypes.c_float,
                                    ctypes.c_int, _vp]),
    "sl_free_filters": (None, [_vp]),
    "sl_bank_info": (ctypes.c_int, [_vp, _c_int_p, _c_int64_p, _c_int_p, _c_int_p]),
    "sl_bank_filter_meta": (ctypes.c_int, [_vp, _c_int_p, _c_int_p, _c_int_p]),
    "sl_bank_norms": (ctypes.c_int, [_vp, _c_double_p, _c_double_p, _c_double_p]),
    "sl_bank_sizes": (ctypes.c_int, [_vp, _c_int64_p, _c_int64_p]),
    "sl_bank_path": (ctypes.c_int, [_vp, _c_int_p]),
    "sl_bank_precision": (ctypes.c_int, [_vp, _c_int_p]),
    "sl_bank_eval_f64": (ctypes.c_int, [_vp, ctypes.c_int, _c_double_p]),
    "sl_bank_filters_f32": (ctypes.c_int, [_vp, _c_float_p]),
    "sl_forward": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "sl_adjoint": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "sl_inverse": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "sl_threshold": (ctypes.c_int, [_vp, _vp, ctypes.c_float, _c_float_p, _vp]),
    "sl_denoise": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_float, _c_float_p, _vp]),
    "sl_fwdinv_host": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "sl_forward_noalloc": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "sl_spectrum_points": (ctypes.c_int, [_vp, _c_int64_p]),
    "sl_sub_layout": (ctypes.c_int, [_vp, _c_int_p, _c_int64_p]),
    "sl_forward_sub": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "sl_adjoint_sub": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "sl_inverse_sub": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int, _c_double_p, _vp]),
    "sl_spectrum": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "sl_forward_range": (ctypes.c_int, [_vp, _vp, ctypes.c_int, ctypes.c_int, _vp, _vp]),
    "sl_inverse_partial": (ctypes.c_int, [_vp, _vp, ctypes.c_int, ctypes.c_int, _vp, _vp]),
    "sl_inverse_finish": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp, _vp]),
    "sl_inpaint": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_float, ctypes.c_float, ctypes.c_int,
                                  _vp]),
    "sl_batch_create": (ctypes.c_int, [_vp, ctypes.c_int, _vp, ctypes.POINTER(_vp)]),
    "sl_batch_free": (None, [_vp]),
    "sl_batch_info": (ctypes.c_int, [_vp, _c_int_p, _c_int_p, _c_int_p]),
    "sl_batch_forward": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "sl_batch_inverse": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "sl_batch_fwdinv": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "sl_batch_denoise": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_float, _vp, _vp]),
    "sl_batch_autotune": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_int, _vp, _c_double_p]),
    "sl_forward_batch": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _vp]),
    "sl_inverse_batch": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _vp]),
    "sl_mlp_create": (ctypes.c_int, [_vp, ctypes.POINTER(_vp)]),
    "sl_mlp_free": (None, [_vp]),
    "sl_mlp_num_params": (ctypes.c_int, [_vp]),
    "sl_mlp_set_params": (ctypes.c_int, [_vp, _c_float_p]),
    "sl_mlp_get_params": (ctypes.c_int, [_vp, _c_float_p]),
    "sl_mlp_gradients": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_float, _vp, ctypes.c_int,
                                        _c_float_p, _c_float_p, _vp]),
    "sl_mlp_train_step": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_float, _vp, ctypes.c_int,
                                         ctypes.c_float, _vp, _vp]),
    "sl_mlp_apply": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_float, _vp]),
    "sl_mlp_denoise": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_float, _vp]),
    "sl_mlp_last_error": (ctypes.c_char_p, []),
    "sl_mlp_save": (ctypes.c_int, [_vp, ctypes.c_char_p]),
    "sl_mlp_load": (ctypes.c_int, [_vp, ctypes.c_char_p]),
    "sl_mlp_set_engine": (ctypes.c_int, [_vp, ctypes.c_int]),
    "sl_mlp_check": (ctypes.c_int, [_vp, _vp]),
    "sl_error_stats": (ctypes.c_int, [_vp, _vp, ctypes.c_int64, _c_double_p, _vp]),
    "sl_device_check": (ctypes.c_int, [_vp]),
    "sl_profile_enable": (ctypes.c_int, [ctypes.c_int]),
    "sl_profile_reset": (ctypes.c_int, []),
    "sl_profile_read": (ctypes.c_int, [ctypes.POINTER(ctypes.c_char_p), _c_int64_p,
                                       _c_double_p, _c_double_p, ctypes.c_int, _c_int_p]),
}

_LIB: Optional[ctypes.CDLL] = None


class ShearletError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}" + (f" ({detail})" if detail else ""))


def lib() -> ctypes.CDLL:
    """Load libshearlet.so (built in-tree by paper_1402_5670_b300.build)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -m paper_1402_5670_b300.build`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


def _check(status: int, where: str) -> None:
    if status != SL_OK:
        raise ShearletError(status, where, lib().sl_last_error().decode(errors="replace"))


def _stream_ptr(stream) -> Optional[int]:
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream


def _dev_ptr(t, name: str, numel: int) -> int:
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float32 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous float32 tensor")
    if t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements, expected {numel}")
    return t.data_ptr()


# ------------------------------------------------------- C ABI, same names ---

PATHS = {"auto": 0, "general": 1, "cluster": 2}


class sl_options(ctypes.Structure):
    _fields_ = [("path", ctypes.c_int), ("precision", ctypes.c_int),
                ("reserved", ctypes.c_int * 6)]


PRECISIONS = {"fp32": 0, "tc_bf16": 1, "tc_fp16": 2}


class sl_filters(ctypes.Structure):
    _fields_ = [("qmf", _c_double_p), ("qmf_len", ctypes.c_int), ("fan", _c_double_p),
                ("fan_rows", ctypes.c_int), ("fan_cols", ctypes.c_int)]


def sl_build_filters(dims: Sequence[int], n_scales: int, shear_levels: Sequence[int],
                     full_system: bool = False, device: int = 0) -> int:
    nd = len(dims)
    d = (ctypes.c_int64 * nd)(*[int(v) for v in dims])
    sl = (ctypes.c_int * len(shear_levels))(*[int(v) for v in shear_levels])
    out = _vp()
    _check(lib().sl_build_filters(nd, d, int(n_scales), sl, int(bool(full_system)), int(device),
                                  ctypes.byref(out)), "sl_build_filters")
    return out.value


def sl_build_filters_ex(dims: Sequence[int], n_scales: int, shear_levels: Sequence[int],
                        full_system: bool = False, device: int = 0, path: str = "auto",
                        precision: str = "fp32", qmf=None, fan=None) -> int:
    """sl_build_filters_ex, or sl_build_filters_user when qmf (1D taps) or fan (2D
    taps) is given."""
    nd = len(dims)
    d = (ctypes.c_int64 * nd)(*[int(v) for v in dims])
    sl = (ctypes.c_int * len(shear_levels))(*[int(v) for v in shear_levels])
    opt = sl_options()
    opt.path = PATHS[path]
    opt.precision = PRECISIONS[precision]
    out = _vp()
    if qmf is None and fan is None:
        _check(lib().sl_build_filters_ex(nd, d, int(n_scales), sl, int(bool(full_system)),
                                         int(device), ctypes.byref(opt), ctypes.byref(out)),
               "sl_build_filters_ex")
        return out.value
    f = sl_filters()
    keep = []
    if qmf is not None:
        h = np.ascontiguousarray(qmf, dtype=np.float64).ravel()
        keep.append(h)
        f.qmf, f.qmf_len = h.ctypes.data_as(_c_double_p), h.size
    if fan is not None:
        P = np.ascontiguousarray(fan, dtype=np.float64)
        if P.ndim != 2:
            raise ValueError("fan taps must be a 2D array")
        keep.append(P)
        f.fan, f.fan_rows, f.fan_cols = P.ctypes.data_as(_c_double_p), P.shape[0], P.shape[1]
    _check(lib().sl_build_filters_user(nd, d, int(n_scales), sl, int(bool(full_system)),
                                       int(device), ctypes.byref(opt), ctypes.byref(f),
                                       ctypes.byref(out)), "sl_build_filters_user")
    return out.value


def sl_build_wavelets(dims: Sequence[int], n_scales: int, device: int = 0, qmf=None) -> int:
    """The separable stationary wavelet bank (sl_build_wavelets), optionally on a user QMF."""
    nd = len(dims)
    d = (ctypes.c_int64 * nd)(*[int(v) for v in dims])
    out = _vp()
    f = None
    if qmf is not None:
        h = np.ascontiguousarray(qmf, dtype=np.float64).ravel()
        f = sl_filters()
        f.qmf, f.qmf_len = h.ctypes.data_as(_c_double_p), h.size
    _check(lib().sl_build_wavelets(nd, d, int(n_scales), int(device),
                                   ctypes.byref(f) if f is not None else None, ctypes.byref(out)),
           "sl_build_wavelets")
    return out.value


def sl_free_filters(bank: int) -> None:
    lib().sl_free_filters(bank)


def sl_forward(bank: int, x, coeffs, stream=None) -> None:
    _check(lib().sl_forward(bank, x, coeffs, stream), "sl_forward")


def sl_adjoint(bank: int, coeffs, x, stream=None) -> None:
    _check(lib().sl_adjoint(bank, coeffs, x, stream), "sl_adjoint")


def sl_inverse(bank: int, coeffs, x, stream=None) -> None:
    _check(lib().sl_inverse(bank, coeffs, x, stream), "sl_inverse")


def sl_threshold(bank: int, coeffs, sigma: float, K: Sequence[float], stream=None) -> None:
    k = (ctypes.c_float * len(K))(*[float(v) for v in K])
    _check(lib().sl_threshold(bank, coeffs, float(sigma), k, stream), "sl_threshold")


def sl_denoise(bank: int, noisy, out, sigma: float, K: Sequence[float], stream=None) -> None:
    k = (ctypes.c_float * len(K))(*[float(v) for v in K])
    _check(lib().sl_denoise(bank, noisy, out, float(sigma), k, stream), "sl_denoise")


def sl_fwdinv_host(bank: int, x_host, y_host, stream=None) -> None:
    _check(lib().sl_fwdinv_host(bank, x_host, y_host, stream), "sl_fwdinv_host")


def sl_forward_noalloc(bank: int, psi, x, coeffs, stream=None) -> None:
    """Forward transform that allocates nothing (static device scratch); psi, x and
    coeffs are device pointers owned by the caller."""
    _check(lib().sl_forward_noalloc(bank, psi, x, coeffs, stream), "sl_forward_noalloc")


def sl_spectrum_points(bank: int) -> int:
    n = ctypes.c_int64()
    _check(lib().sl_spectrum_points(bank, ctypes.byref(n)), "sl_spectrum_points")
    return n.value


def sl_spectrum(bank: int, x, xhat, stream=None) -> None:
    _check(lib().sl_spectrum(bank, x, xhat, stream), "sl_spectrum")


def sl_forward_range(bank: int, xhat, j0: int, j1: int, coeffs, stream=None) -> None:
    _check(lib().sl_forward_range(bank, xhat, int(j0), int(j1), coeffs, stream), "sl_forward_range")


def sl_inverse_partial(bank: int, coeffs, j0: int, j1: int, partial, stream=None) -> None:
    _check(lib().sl_inverse_partial(bank, coeffs, int(j0), int(j1), partial, stream),
           "sl_inverse_partial")


def sl_inverse_finish(bank: int, summed, dual: bool, x, stream=None) -> None:
    _check(lib().sl_inverse_finish(bank, summed, int(bool(dual)), x, stream), "sl_inverse_finish")


def sl_error_stats(y, ref, stream=None) -> dict:
    """GPU error statistics (FP64 accumulation) of device tensors y against ref:
    max_abs_err, max_abs_ref, sum_sq_err, sum_sq_ref, and the derived rel_max, rel_l2
    and psnr (peak 255, eq. PSNR)."""
    n = ref.numel()
    out = np.zeros(4)
    _check(lib().sl_error_stats(_dev_ptr(y, "y", n), _dev_ptr(ref, "ref", n), n,
                                out.ctypes.data_as(_c_double_p), _stream_ptr(stream)),
           "sl_error_stats")
    import math
    return {"max_abs_err": out[0], "max_abs_ref": out[1], "sum_sq_err": out[2],
            "sum_sq_ref": out[3], "rel_max": out[0] / max(out[1], 1e-300),
            "rel_l2": math.sqrt(out[2] / max(out[3], 1e-300)),
            "psnr": 20 * math.log10(255 * math.sqrt(n) / math.sqrt(max(out[2], 1e-300)))}


def sl_device_check(stream=None) -> None:
    """Synchronise and raise if a bounded wait of a transform kernel ran out."""
    _check(lib().sl_device_check(_stream_ptr(stream)), "sl_device_check")


def sl_profile_enable(on: bool) -> None:
    _check(lib().sl_profile_enable(int(bool(on))), "sl_profile_enable")


def sl_profile_reset() -> None:
    _check(lib().sl_profile_reset(), "sl_profile_reset")


def sl_profile_read(cap: int = 64) -> dict:
    """{kernel kind: (launches, total ms, total algorithmic bytes)}"""
    names = (ctypes.c_char_p * cap)()
    launches = (ctypes.c_int64 * cap)()
    ms = (ctypes.c_double * cap)()
    by = (ctypes.c_double * cap)()
    cnt = ctypes.c_int()
    _check(lib().sl_profile_read(names, launches, ms, by, cap, ctypes.byref(cnt)),
           "sl_profile_read")
    return {names[i].decode(): (int(launches[i]), float(ms[i]), float(by[i]))
            for i in range(cnt.value)}


# ------------------------------------------------------------ Bank object ---

class Bank:
    """A filter bank on one device (sl_build_filters) with the transforms bound to it.

    device=-1 builds a host-only bank: its filters can be evaluated (eval_f64) but it
    runs no transforms.
    """

    def __init__(self, dims: Sequence[int], n_scales: int, shear_levels: Sequence[int],
                 full_system: bool = False, device: int = 0, path: str = "auto",
                 precision: str = "fp32", qmf=None, fan=None):
        if device >= 0:
            import torch
            torch.cuda.set_device(device)
        self.path = path
        self.handle = sl_build_filters_ex(dims, n_scales, shear_levels, full_system, device, path,
                                          precision, qmf, fan)
        self._describe(device)

    @classmethod
    def wavelets(cls, dims: Sequence[int], n_scales: int, device: int = 0, qmf=None) -> "Bank":
        """The separable stationary wavelet bank on the same grid (sl_build_wavelets):
        lowpass, then per scale coarse to fine g(x)h, h(x)g, g(x)g; R = 1 + 3 n_scales."""
        if device >= 0:
            import torch
            torch.cuda.set_device(device)
        b = cls.__new__(cls)
        b.path = "auto"
        b.handle = sl_build_wavelets(dims, n_scales, device, qmf)
        b._describe(device)
        return b

    def _describe(self, device: int) -> None:
        L = lib()
        nd, R, J = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        dd = (ctypes.c_int64 * 3)()
        _check(L.sl_bank_info(self.handle, ctypes.byref(nd), dd, ctypes.byref(R), ctypes.byref(J)),
               "sl_bank_info")
        self.ndim = nd.value
        self.dims = tuple(int(dd[i]) for i in range(self.ndim))
        self.R = R.value
        self.n_scales = J.value
        self.device = device
        N, Nh = ctypes.c_int64(), ctypes.c_int64()
        _check(L.sl_bank_sizes(self.handle, ctypes.byref(N), ctypes.byref(Nh)), "sl_bank_sizes")
        self.N, self.Nh = N.value, Nh.value
        self.norms = np.zeros(self.R)
        A, B = ctypes.c_double(), ctypes.c_double()
        _check(L.sl_bank_norms(self.handle, self.norms.ctypes.data_as(_c_double_p),
                               ctypes.byref(A), ctypes.byref(B)), "sl_bank_norms")
        self.A, self.B = A.value, B.value
        pth = ctypes.c_int()
        _check(L.sl_bank_path(self.handle, ctypes.byref(pth)), "sl_bank_path")
        self.kernel_path = {1: "general", 2: "cluster"}[pth.value]
        pr = ctypes.c_int()
        _check(L.sl_bank_precision(self.handle, ctypes.byref(pr)), "sl_bank_precision")
        self.precision = {v: k for k, v in PRECISIONS.items()}[pr.value]
        self.scale_of = np.zeros(self.R, dtype=np.int32)
        self.cone_of = np.zeros(self.R, dtype=np.int32)
        self.k_of = np.zeros((self.R, 2), dtype=np.int32)
        _check(L.sl_bank_filter_meta(self.handle, self.scale_of.ctypes.data_as(_c_int_p),
                                     self.cone_of.ctypes.data_as(_c_int_p),
                                     self.k_of.ctypes.data_as(_c_int_p)), "sl_bank_filter_meta")

    @property
    def half_shape(self):
        return self.dims[:-1] + (self.dims[-1] // 2 + 1,)

    def eval_f64(self, j: int) -> np.ndarray:
        """Normalised psi_hat_j on the half spectrum (j = -1: Psi), FP64, on the host."""
        out = np.zeros(self.Nh)
        _check(lib().sl_bank_eval_f64(self.handle, int(j), out.ctypes.data_as(_c_double_p)),
               "sl_bank_eval_f64")
        return out.reshape(self.half_shape)

    def filters_f32(self) -> np.ndarray:
        out = np.zeros((self.R,) + self.half_shape, dtype=np.float32)
        _check(lib().sl_bank_filters_f32(self.handle, out.ctypes.data_as(_c_float_p)),
               "sl_bank_filters_f32")
        return out

    # -------- transforms (device tensors) --------

    def _empty(self, shape):
        import torch
        return torch.empty(shape, dtype=torch.float32, device=f"cuda:{self.device}")

    def forward(self, x, out=None, stream=None):
        out = self._empty((self.R,) + self.dims) if out is None else out
        sl_forward(self.handle, _dev_ptr(x, "x", self.N), _dev_ptr(out, "coeffs", self.R * self.N),
                   _stream_ptr(stream))
        return out

    def adjoint(self, coeffs, out=None, stream=None):
        out = self._empty(self.dims) if out is None else out
        sl_adjoint(self.handle, _dev_ptr(coeffs, "coeffs", self.R * self.N),
                   _dev_ptr(out, "x", self.N), _stream_ptr(stream))
        return out

    def inverse(self, coeffs, out=None, stream=None):
        out = self._empty(self.dims) if out is None else out
        sl_inverse(self.handle, _dev_ptr(coeffs, "coeffs", self.R * self.N),
                   _dev_ptr(out, "x", self.N), _stream_ptr(stream))
        return out

    # -------- filter ranges (one transform sharded over ranks) --------

    @property
    def spectrum_points(self) -> int:
        """Complex points of one spectrum buffer (library layout)."""
        return sl_spectrum_points(self.handle)

    def spectrum(self, x, out=None, stream=None):
        """X_hat = FFT(x) as a float32 tensor of 2 * spectrum_points (sl_spectrum)."""
        n = 2 * self.spectrum_points
        out = self._empty((n,)) if out is None else out
        sl_spectrum(self.handle, _dev_ptr(x, "x", self.N), _dev_ptr(out, "xhat", n),
                    _stream_ptr(stream))
        return out

    def forward_range(self, xhat, j0: int, j1: int, out=None, stream=None):
        """Coefficients of filters [j0, j1) from a spectrum (sl_forward_range)."""
        out = self._empty((j1 - j0,) + self.dims) if out is None else out
        sl_forward_range(self.handle, _dev_ptr(xhat, "xhat", 2 * self.spectrum_points), j0, j1,
                         _dev_ptr(out, "coeffs", (j1 - j0) * self.N), _stream_ptr(stream))
        return out

    def inverse_partial(self, coeffs, j0: int, j1: int, out=None, stream=None):
        """sum_{j in [j0, j1)} FFT(C_j) psi_hat_j as a spectrum (sl_inverse_partial)."""
        n = 2 * self.spectrum_points
        out = self._empty((n,)) if out is None else out
        sl_inverse_partial(self.handle, _dev_ptr(coeffs, "coeffs", (j1 - j0) * self.N), j0, j1,
                           _dev_ptr(out, "partial", n), _stream_ptr(stream))
        return out

    def inverse_finish(self, summed, dual: bool = True, out=None, stream=None):
        """x from the sum of all partials: / Psi (dual) or not (adjoint) (sl_inverse_finish)."""
        out = self._empty(self.dims) if out is None else out
        sl_inverse_finish(self.handle, _dev_ptr(summed, "summed", 2 * self.spectrum_points), dual,
                          _dev_ptr(out, "x", self.N), _stream_ptr(stream))
        return out

    # -------- subsampled transform (2D) --------

    def sub_layout(self):
        """(steps [R], offsets [R + 1]) of the subsampled transform's compact layout."""
        st = np.zeros(self.R, dtype=np.int32)
        off = np.zeros(self.R + 1, dtype=np.int64)
        _check(lib().sl_sub_layout(self.handle, st.ctypes.data_as(_c_int_p),
                                   off.ctypes.data_as(_c_int64_p)), "sl_sub_layout")
        return st, off

    def forward_sub(self, x, out=None, stream=None):
        n = int(self.sub_layout()[1][-1])
        out = self._empty((n,)) if out is None else out
        _check(lib().sl_forward_sub(self.handle, _dev_ptr(x, "x", self.N),
                                    _dev_ptr(out, "coeffs_sub", n), _stream_ptr(stream)),
               "sl_forward_sub")
        return out

    def adjoint_sub(self, coeffs_sub, out=None, stream=None):
        n = int(self.sub_layout()[1][-1])
        out = self._empty(self.dims) if out is None else out
        _check(lib().sl_adjoint_sub(self.handle, _dev_ptr(coeffs_sub, "coeffs_sub", n),
                                    _dev_ptr(out, "x", self.N), _stream_ptr(stream)),
               "sl_adjoint_sub")
        return out

    def inverse_sub(self, coeffs_sub, iterations: int, precondition: bool = True, out=None,
                    stream=None):
        """(x, relative residual) after `iterations` conjugate-gradient steps."""
        n = int(self.sub_layout()[1][-1])
        out = self._empty(self.dims) if out is None else out
        res = ctypes.c_double()
        _check(lib().sl_inverse_sub(self.handle, _dev_ptr(coeffs_sub, "coeffs_sub", n),
                                    _dev_ptr(out, "x", self.N), int(iterations),
                                    int(bool(precondition)), ctypes.byref(res),
                                    _stream_ptr(stream)), "sl_inverse_sub")
        return out, res.value

    def threshold_(self, coeffs, sigma: float, K: Sequence[float], stream=None):
        self._check_K(K)
        sl_threshold(self.handle, _dev_ptr(coeffs, "coeffs", self.R * self.N), sigma, K,
                     _stream_ptr(stream))
        return coeffs

    def denoise(self, noisy, sigma: float, K: Sequence[float], out=None, stream=None):
        self._check_K(K)
        out = self._empty(self.dims) if out is None else out
        sl_denoise(self.handle, _dev_ptr(noisy, "noisy", self.N), _dev_ptr(out, "out", self.N),
                   sigma, K, _stream_ptr(stream))
        return out

    def inpaint(self, f_masked, mask, delta_init: float, delta_min: float, iterations: int,
                out=None, stream=None):
        """Iterative-thresholding inpainting (sl_inpaint); mask: uint8 CUDA tensor."""
        import torch
        if not (isinstance(mask, torch.Tensor) and mask.is_cuda and mask.dtype == torch.uint8
                and mask.is_contiguous() and mask.numel() == self.N):
            raise TypeError("mask must be a contiguous uint8 CUDA tensor of the image size")
        out = self._empty(self.dims) if out is None else out
        _check(lib().sl_inpaint(self.handle, _dev_ptr(f_masked, "f_masked", self.N), mask.data_ptr(),
                                _dev_ptr(out, "out", self.N), float(delta_init), float(delta_min),
                                int(iterations), _stream_ptr(stream)), "sl_inpaint")
        return out

    def decompose(self, iso: "Bank", f, delta_init: float, delta_min: float, iterations: int,
                  out0=None, out1=None, stream=None):
        """Image decomposition (sl_decompose) of f into the curvilinear part (this
        shearlet bank) and the isotropic part (iso, a wavelet bank): returns (f0, f1)."""
        out0 = self._empty(self.dims) if out0 is None else out0
        out1 = self._empty(self.dims) if out1 is None else out1
        _check(lib().sl_decompose(self.handle, iso.handle, _dev_ptr(f, "f", self.N),
                                  _dev_ptr(out0, "f0", self.N), _dev_ptr(out1, "f1", self.N),
                                  float(delta_init), float(delta_min), int(iterations),
                                  _stream_ptr(stream)), "sl_decompose")
        return out0, out1

    def fwdinv_host(self, x_host, y_host, stream=None):
        """Round trip from host memory (x_host, y_host: pinned CPU float32 tensors)."""
        for t, n in ((x_host, "x_host"), (y_host, "y_host")):
            if t.is_cuda or t.numel() != self.N or not t.is_contiguous():
                raise ValueError(f"{n} must be a contiguous CPU tensor of {self.N} floats")
        sl_fwdinv_host(self.handle, x_host.data_ptr(), y_host.data_ptr(), _stream_ptr(stream))
        return y_host

    def _check_K(self, K):
        if len(K) != self.n_scales:
            raise ValueError(f"K needs {self.n_scales} entries (one per scale)")

    def close(self):
        if getattr(self, "handle", None):
            sl_free_filters(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# ------------------------------------------------------- learned shrinkage ---

def _mcheck(status: int, where: str) -> None:
    if status != SL_OK:
        raise ShearletError(status, where, lib().sl_mlp_last_error().decode(errors="replace"))


MLP_ENGINES = {"tcgen05": 0, "mma_sync": 1}


class MLP:
    """Learned shrinkage bound to a device Bank (sl_mlp_*)."""

    def __init__(self, bank: "Bank"):
        self.bank = bank
        h = _vp()
        _mcheck(lib().sl_mlp_create(bank.handle, ctypes.byref(h)), "sl_mlp_create")
        self.handle = h.value
        self.num_params = lib().sl_mlp_num_params(self.handle)

    def set_params(self, flat: np.ndarray) -> None:
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        assert flat.size == self.num_params
        _mcheck(lib().sl_mlp_set_params(self.handle, flat.ctypes.data_as(_c_float_p)),
                "sl_mlp_set_params")

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.num_params, dtype=np.float32)
        _mcheck(lib().sl_mlp_get_params(self.handle, out.ctypes.data_as(_c_float_p)),
                "sl_mlp_get_params")
        return out

    def save(self, path: str) -> None:
        """Checkpoint: parameters and Adam's state."""
        _mcheck(lib().sl_mlp_save(self.handle, os.fsencode(path)), "sl_mlp_save")

    def load(self, path: str) -> None:
        _mcheck(lib().sl_mlp_load(self.handle, os.fsencode(path)), "sl_mlp_load")

    def _sample(self, idx):
        import torch
        if idx.dtype != torch.int32 or not idx.is_cuda or not idx.is_contiguous():
            raise TypeError("idx must be a contiguous int32 CUDA tensor")
        return idx.data_ptr(), idx.numel()

    def gradients(self, noisy, clean, sigma: float, idx, stream=None):
        n_all = self.bank.R * self.bank.N
        ip, n = self._sample(idx)
        g = np.zeros(self.num_params, dtype=np.float32)
        loss = ctypes.c_float()
        _mcheck(lib().sl_mlp_gradients(self.handle, _dev_ptr(noisy, "noisy", n_all),
                                       _dev_ptr(clean, "clean", n_all), float(sigma), ip, n,
                                       g.ctypes.data_as(_c_float_p), ctypes.byref(loss),
                                       _stream_ptr(stream)), "sl_mlp_gradients")
        return float(loss.value), g

    def train_step(self, noisy, clean, sigma: float, idx, lr: float, loss_out=None, stream=None):
        n_all = self.bank.R * self.bank.N
        ip, n = self._sample(idx)
        lp = None if loss_out is None else loss_out.data_ptr()
        _mcheck(lib().sl_mlp_train_step(self.handle, _dev_ptr(noisy, "noisy", n_all),
                                        _dev_ptr(clean, "clean", n_all), float(sigma), ip, n,
                                        float(lr), lp, _stream_ptr(stream)), "sl_mlp_train_step")

    def apply(self, coeffs, sigma: float, out=None, stream=None):
        n_all = self.bank.R * self.bank.N
        out = self.bank._empty((self.bank.R,) + self.bank.dims) if out is None else out
        _mcheck(lib().sl_mlp_apply(self.handle, _dev_ptr(coeffs, "coeffs", n_all),
                                   _dev_ptr(out, "out", n_all), float(sigma),
                                   _stream_ptr(stream)), "sl_mlp_apply")
        return out

    def set_engine(self, engine: str):
        """'tcgen05' (default) or 'mma_sync': the tensor-core path of apply, gradients and
        train_step."""
        if engine not in MLP_ENGINES:
            raise ValueError(f"engine must be one of {sorted(MLP_ENGINES)}")
        _mcheck(lib().sl_mlp_set_engine(self.handle, MLP_ENGINES[engine]), "sl_mlp_set_engine")

    def check(self, stream=None):
        """Synchronise and raise if a tensor-core wait of an earlier apply ran out."""
        _mcheck(lib().sl_mlp_check(self.handle, _stream_ptr(stream)), "sl_mlp_check")

    def denoise(self, noisy, sigma: float, out=None, stream=None):
        out = self.bank._empty(self.bank.dims) if out is None else out
        _mcheck(lib().sl_mlp_denoise(self.handle, _dev_ptr(noisy, "noisy", self.bank.N),
                                     _dev_ptr(out, "out", self.bank.N), float(sigma),
                                     _stream_ptr(stream)), "sl_mlp_denoise")
        return out

    def close(self):
        if getattr(self, "handle", None):
            lib().sl_mlp_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ batches ---

class _BatchOptions(ctypes.Structure):
    _fields_ = [("branches", ctypes.c_int), ("no_graph", ctypes.c_int),
                ("reserved", ctypes.c_int * 6)]


def _ptr_array(tensors, what, sizes):
    arr = (_vp * len(tensors))()
    for i, (t, n) in enumerate(zip(tensors, sizes)):
        arr[i] = _dev_ptr(t, f"{what}[{i}]", n)
    return arr


class Batch:
    """Many images of (possibly) different shapes transformed together (sl_batch_*):
    image i uses banks[i]. Inputs and outputs are lists of device tensors; the
    pointer arrays are built here, the work runs in the library."""

    def __init__(self, banks: Sequence["Bank"], branches: int = 0, graph: bool = True):
        self.banks = list(banks)
        n = len(self.banks)
        self._handles = (_vp * n)(*[b.handle for b in self.banks])
        opt = _BatchOptions(int(branches), 0 if graph else 1)
        h = _vp()
        _check(lib().sl_batch_create(self._handles, n, ctypes.byref(opt), ctypes.byref(h)),
               "sl_batch_create")
        self.handle = h.value

    def _sizes(self, coeffs=False):
        return [b.R * b.N if coeffs else b.N for b in self.banks]

    def info(self):
        n = len(self.banks)
        K = ctypes.c_int()
        br = (ctypes.c_int * n)()
        gc = (ctypes.c_int * n)()
        _check(lib().sl_batch_info(self.handle, ctypes.byref(K), br, gc), "sl_batch_info")
        return {"branches": K.value, "branch_of": list(br), "group_cap": list(gc)}

    def forward(self, xs, cs, stream=None):
        _check(lib().sl_batch_forward(self.handle, _ptr_array(xs, "x", self._sizes()),
                                      _ptr_array(cs, "coeffs", self._sizes(True)),
                                      _stream_ptr(stream)), "sl_batch_forward")
        return cs

    def inverse(self, cs, ys, stream=None):
        _check(lib().sl_batch_inverse(self.handle, _ptr_array(cs, "coeffs", self._sizes(True)),
                                      _ptr_array(ys, "x", self._sizes()),
                                      _stream_ptr(stream)), "sl_batch_inverse")
        return ys

    def fwdinv(self, xs, cs, ys, stream=None):
        _check(lib().sl_batch_fwdinv(self.handle, _ptr_array(xs, "x", self._sizes()),
                                     _ptr_array(cs, "coeffs", self._sizes(True)),
                                     _ptr_array(ys, "y", self._sizes()),
                                     _stream_ptr(stream)), "sl_batch_fwdinv")
        return ys

    def denoise(self, xs, ys, sigma: float, K, stream=None):
        """K: one list of nScales values per image (or one list for all)."""
        Ks = K if (len(K) and isinstance(K[0], (list, tuple, np.ndarray))) else [K] * len(xs)
        self._Kbufs = [(ctypes.c_float * len(k))(*[float(v) for v in k]) for k in Ks]
        for b, k in zip(self.banks, Ks):
            b._check_K(k)
        kp = (_vp * len(Ks))(*[ctypes.cast(k, _vp).value for k in self._Kbufs])
        _check(lib().sl_batch_denoise(self.handle, _ptr_array(xs, "noisy", self._sizes()),
                                      _ptr_array(ys, "out", self._sizes()), float(sigma), kp,
                                      _stream_ptr(stream)), "sl_batch_denoise")
        return ys

    def autotune(self, xs, cs, ys, reps: int = 3, stream=None) -> float:
        best = ctypes.c_double()
        _check(lib().sl_batch_autotune(self.handle, _ptr_array(xs, "x", self._sizes()),
                                       _ptr_array(cs, "coeffs", self._sizes(True)),
                                       _ptr_array(ys, "y", self._sizes()), int(reps),
                                       _stream_ptr(stream), ctypes.byref(best)),
               "sl_batch_autotune")
        return best.value

    def close(self):
        if getattr(self, "handle", None):
            lib().sl_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sl_forward_batch(banks: Sequence["Bank"], xs, cs, stream=None) -> None:
    h = (_vp * len(banks))(*[b.handle for b in banks])
    _check(lib().sl_forward_batch(h, len(banks), _ptr_array(xs, "x", [b.N for b in banks]),
                                  _ptr_array(cs, "coeffs", [b.R * b.N for b in banks]),
                                  _stream_ptr(stream)), "sl_forward_batch")


def sl_inverse_batch(banks: Sequence["Bank"], cs, ys, stream=None) -> None:
    h = (_vp * len(banks))(*[b.handle for b in banks])
    _check(lib().sl_inverse_batch(h, len(banks), _ptr_array(cs, "coeffs", [b.R * b.N for b in banks]),
                                  _ptr_array(ys, "x", [b.N for b in banks]),
                                  _stream_ptr(stream)), "sl_inverse_batch")
