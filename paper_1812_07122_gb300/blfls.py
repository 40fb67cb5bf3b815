"""Thin ctypes binding of ``libblfls.so`` with the C ABI's names (see ``include/blfls.h``).

Argument marshalling only: every step of the smoother runs in the library's CUDA kernels.
Image arguments accept a CUDA ``torch.Tensor`` (its ``data_ptr()``) or a raw integer address;
streams accept a ``torch.cuda.Stream``, a raw ``cudaStream_t`` integer or ``None`` (the legacy
default stream).  A non-zero status raises :class:`BlflsError` carrying the code and the
library's message.  If the library has not been built, loading raises instead of falling back
to anything else.
"""
from __future__ import annotations

import ctypes
import os

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "libblfls.so")
# BLFLS_LIBRARY names another build of the same library to load instead (for example the debug
# build with device range checks, see build.py); it must exist like the default one.
LIB_ENV = "BLFLS_LIBRARY"

BLFLS_OK = 0
BLFLS_EINVAL = -1
BLFLS_ENOMEM = -2
BLFLS_ECUDA = -3
BLFLS_ETIMEOUT = -4
BLFLS_EBUSY = -5

BLFLS_FP32 = 0
BLFLS_FP16W = 1
BLFLS_BF16W = 2

BLFLS_DETAIL_ENHANCE = 0
BLFLS_LOG_TONE = 1
BLFLS_LOG_FLOOR = 1e-6
BLFLS_MAX_GAUSS_SIGMA = 32.0

BLFLS_MAX_DIM = 8192
BLFLS_MAX_CHANNELS = 4
BLFLS_MAX_ITERS = 64

_PREC_NAMES = {"fp32": BLFLS_FP32, "fp16": BLFLS_FP16W, "fp16w": BLFLS_FP16W,
               "bf16": BLFLS_BF16W, "bf16w": BLFLS_BF16W}


class BlflsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"blfls error {code}: {msg}")
        self.code = code


class blfls_job(ctypes.Structure):
    _fields_ = [("img", ctypes.c_void_p), ("out", ctypes.c_void_p),
                ("H", ctypes.c_int), ("W", ctypes.c_int), ("C", ctypes.c_int),
                ("lambda_", ctypes.c_float), ("sigma_s", ctypes.c_float),
                ("sigma_r", ctypes.c_float), ("radius", ctypes.c_int), ("iters", ctypes.c_int),
                ("prec", ctypes.c_int)]


class blfls_request(ctypes.Structure):
    _fields_ = [("img_host", ctypes.c_void_p), ("out_host", ctypes.c_void_p),
                ("H", ctypes.c_int), ("W", ctypes.c_int), ("C", ctypes.c_int),
                ("lambda_", ctypes.c_float), ("sigma_s", ctypes.c_float),
                ("sigma_r", ctypes.c_float), ("radius", ctypes.c_int), ("iters", ctypes.c_int),
                ("prec", ctypes.c_int)]


class blfls_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("failed", ctypes.c_uint64), ("cancelled", ctypes.c_uint64),
                ("rejected", ctypes.c_uint64), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("megapixels", ctypes.c_double),
                ("busy_s", ctypes.c_double), ("mp_per_s", ctypes.c_double),
                ("device_bytes_peak", ctypes.c_size_t), ("device_bytes_budget", ctypes.c_size_t),
                ("max_batch_seen", ctypes.c_int)]


_LIB = None

_c_int, _c_float, _vp, _sz = ctypes.c_int, ctypes.c_float, ctypes.c_void_p, ctypes.c_size_t

# name -> (restype, argtypes); the exported C symbols
_SIGNATURES = {
    "blfls_create": (_c_int, [ctypes.POINTER(_vp), _c_int, _sz, ctypes.c_char_p]),
    "blfls_destroy": (None, [_vp]),
    "blfls_last_error": (ctypes.c_char_p, [_vp]),
    "blfls_smooth": (_c_int, [_vp, _vp, _vp, _c_int, _c_int, _c_int, _c_float, _c_float,
                              _c_float, _c_int, _c_int, _c_int, _vp]),
    "blfls_smooth_host": (_c_int, [_vp, _vp, _vp, _c_int, _c_int, _c_int, _c_float, _c_float,
                                   _c_float, _c_int, _c_int, _c_int, _vp]),
    "blfls_blf_residual": (_c_int, [_vp, _vp, _vp, _vp, _c_int, _c_int, _c_int, _c_float,
                                    _c_float, _c_int, _c_int, _vp]),
    "blfls_solve_residual": (_c_int, [_vp, _vp, _vp, _vp, _vp, _c_int, _c_int, _c_int,
                                      _c_float, _vp]),
    "blfls_smooth_batch": (_c_int, [_vp, ctypes.POINTER(blfls_job), _c_int, _vp]),
    "blfls_profile_begin": (_c_int, [_vp, _c_int]),
    "blfls_submit": (_c_int, [_vp, ctypes.POINTER(blfls_job), ctypes.POINTER(ctypes.c_uint64)]),
    "blfls_poll": (_c_int, [_vp, ctypes.c_uint64, ctypes.POINTER(_c_int)]),
    "blfls_server_create": (_c_int, [ctypes.POINTER(_vp), _c_int, _sz, _c_int, _c_int,
                                     ctypes.c_char_p]),
    "blfls_server_destroy": (None, [_vp]),
    "blfls_server_submit": (_c_int, [_vp, ctypes.POINTER(blfls_request),
                                     ctypes.POINTER(ctypes.c_uint64)]),
    "blfls_server_poll": (_c_int, [_vp, ctypes.c_uint64, ctypes.POINTER(_c_int)]),
    "blfls_server_wait": (_c_int, [_vp, ctypes.c_uint64, _c_int]),
    "blfls_server_cancel": (_c_int, [_vp, ctypes.c_uint64]),
    "blfls_server_release": (_c_int, [_vp, ctypes.c_uint64]),
    "blfls_server_get_stats": (_c_int, [_vp, ctypes.POINTER(blfls_server_stats)]),
    "blfls_autotune": (_c_int, [_vp, _c_int, _c_int, _c_int, _c_int, _c_int, ctypes.c_char_p]),
    "blfls_pipe_rates": (_c_int, [_c_int, ctypes.POINTER(ctypes.c_double), _c_int]),
    "blfls_device_checks": (_c_int, [_c_int, ctypes.POINTER(ctypes.c_uint)]),
    "blfls_solve_residual_noalloc": (_c_int, [_vp, _vp, _vp, _vp, _c_int, _c_int, _c_int,
                                              _c_float, _vp]),
    "blfls_profile_end": (_c_int, [_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_c_int)]),
    "blfls_smooth_ls": (_c_int, [_vp, _vp, _vp, _c_int, _c_int, _c_int, _c_float, _c_int, _vp]),
    "blfls_layers": (_c_int, [_vp, _vp, _vp, _c_int, _c_int, _c_int, _c_int, _c_float, _c_float,
                              _c_float, _c_float, _c_int, _c_int, _c_int, _vp]),
    "blfls_smooth_guided": (_c_int, [_vp, _vp, _vp, _vp, _c_int, _c_int, _c_int, _c_int, _c_float,
                                     _c_float, _c_float, _c_int, _c_int, _c_int, _vp]),
    "blfls_smooth_rolling": (_c_int, [_vp, _vp, _vp, _c_int, _c_int, _c_int, _c_float, _c_float,
                                      _c_float, _c_int, _c_int, _c_float, _c_int, _vp]),
    "blfls_gaussian": (_c_int, [_vp, _vp, _vp, _c_int, _c_int, _c_int, _c_float, _vp]),
    "blfls_smooth_grid": (_c_int, [_vp, _vp, _vp, _c_int, _c_int, _c_int, _c_float, _c_float,
                                   _c_float, _c_int, _vp]),
    "blfls_smooth_nc": (_c_int, [_vp, _vp, _vp, _c_int, _c_int, _c_int, _c_float, _c_float,
                                 _c_float, _c_int, _c_int, _vp]),
    "blfls_smooth_normalized": (_c_int, [_vp, _vp, _vp, _c_int, _c_int, _c_int, _c_float,
                                         _c_float, _c_float, _c_int, _c_int, _c_int, _vp]),
}


def load():
    """Load the library (once).  Raises if it has not been built."""
    global _LIB
    if _LIB is None:
        path = os.environ.get(LIB_ENV) or LIB_PATH
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with "
                               "`python -m paper_1812_07122_gb300.build` (needs nvcc)")
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = lib
    return _LIB


def exported_symbols() -> list[str]:
    return list(_SIGNATURES)


def _ptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    if hasattr(x, "ctypes"):          # numpy array (host memory)
        return int(x.ctypes.data)
    raise TypeError(f"cannot take an address of {type(x)!r}")


def _stream(s) -> int:
    if s is None:
        return 0
    if isinstance(s, int):
        return s
    return int(s.cuda_stream)


def _prec(p) -> int:
    if isinstance(p, str):
        return _PREC_NAMES[p.lower()]
    return int(p)


def _check(rc: int, h=None):
    if rc != BLFLS_OK:
        msg = load().blfls_last_error(h)
        raise BlflsError(rc, msg.decode() if msg else "")


def blfls_create(device: int = 0, mem_budget_bytes: int = 0, tune_table_path: str | None = None):
    h = _vp()
    path = tune_table_path.encode() if tune_table_path else None
    _check(load().blfls_create(ctypes.byref(h), int(device), int(mem_budget_bytes), path))
    return h


def blfls_destroy(h) -> None:
    if h is not None:
        load().blfls_destroy(h)


def blfls_last_error(h=None) -> str:
    msg = load().blfls_last_error(h)
    return msg.decode() if msg else ""


def blfls_smooth(h, img, out, H, W, C, lam, sigma_s, sigma_r, radius, iters=1, prec=BLFLS_FP32,
                 stream=None) -> None:
    _check(load().blfls_smooth(h, _ptr(img), _ptr(out), int(H), int(W), int(C), float(lam),
                               float(sigma_s), float(sigma_r), int(radius), int(iters),
                               _prec(prec), _stream(stream)), h)


def blfls_smooth_host(h, img_host, out_host, H, W, C, lam, sigma_s, sigma_r, radius, iters=1,
                      prec=BLFLS_FP32, stream=None) -> None:
    _check(load().blfls_smooth_host(h, _ptr(img_host), _ptr(out_host), int(H), int(W), int(C),
                                    float(lam), float(sigma_s), float(sigma_r), int(radius),
                                    int(iters), _prec(prec), _stream(stream)), h)


def blfls_smooth_ls(h, img, out, H, W, C, lam, iters=1, stream=None) -> None:
    """The LS model (Eqs. 5-6) on device buffers."""
    _check(load().blfls_smooth_ls(h, _ptr(img), _ptr(out), int(H), int(W), int(C), float(lam),
                                  int(iters), _stream(stream)), h)


def blfls_layers(h, img, out, H, W, C, mode, strength, lam, sigma_s, sigma_r, radius, iters=1,
                 prec=BLFLS_FP32, stream=None) -> None:
    """Detail enhancement (mode BLFLS_DETAIL_ENHANCE) or log-domain tone mapping
    (BLFLS_LOG_TONE) on top of the smoother, device buffers."""
    _check(load().blfls_layers(h, _ptr(img), _ptr(out), int(H), int(W), int(C), int(mode),
                               float(strength), float(lam), float(sigma_s), float(sigma_r),
                               int(radius), int(iters), _prec(prec), _stream(stream)), h)


def blfls_smooth_guided(h, img, guide, out, H, W, C, Cg, lam, sigma_s, sigma_r, radius, iters=1,
                        prec=BLFLS_FP32, stream=None) -> None:
    """Joint BLF-LS: range weights from the guidance image's gradients (Section III-D)."""
    _check(load().blfls_smooth_guided(h, _ptr(img), _ptr(guide), _ptr(out), int(H), int(W),
                                      int(C), int(Cg), float(lam), float(sigma_s),
                                      float(sigma_r), int(radius), int(iters), _prec(prec),
                                      _stream(stream)), h)


def blfls_smooth_rolling(h, img, out, H, W, C, lam, sigma_s, sigma_r, radius, iters, sigma_g,
                         prec=BLFLS_FP32, stream=None) -> None:
    """Rolling guidance (Section III-D): first guidance = Gaussian(img, sigma_g)."""
    _check(load().blfls_smooth_rolling(h, _ptr(img), _ptr(out), int(H), int(W), int(C),
                                       float(lam), float(sigma_s), float(sigma_r), int(radius),
                                       int(iters), float(sigma_g), _prec(prec), _stream(stream)), h)


def blfls_gaussian(h, img, out, H, W, C, sigma, stream=None) -> None:
    """Periodic separable Gaussian blur (the rolling guidance's first guidance)."""
    _check(load().blfls_gaussian(h, _ptr(img), _ptr(out), int(H), int(W), int(C), float(sigma),
                                 _stream(stream)), h)


def blfls_smooth_grid(h, img, out, H, W, C, lam, sigma_s, sigma_r, iters=1, stream=None) -> None:
    """BLF-LS with the bilateral-grid approximation of the BLF (synchronises once per pass)."""
    _check(load().blfls_smooth_grid(h, _ptr(img), _ptr(out), int(H), int(W), int(C), float(lam),
                                    float(sigma_s), float(sigma_r), int(iters), _stream(stream)), h)


def blfls_smooth_normalized(h, img, out, H, W, C, lam, sigma_s, sigma_r, radius, iters=1,
                            prec=BLFLS_FP32, stream=None) -> None:
    """BLF-LS with every gradient field normalised to [0, 1] per channel (synchronises once per
    pass)."""
    _check(load().blfls_smooth_normalized(h, _ptr(img), _ptr(out), int(H), int(W), int(C),
                                          float(lam), float(sigma_s), float(sigma_r), int(radius),
                                          int(iters), _prec(prec), _stream(stream)), h)


def blfls_smooth_nc(h, img, out, H, W, C, lam, sigma_s, sigma_r, iters=1, nc_iters=3,
                    stream=None) -> None:
    """NC-LS: the domain-transform normalised convolution in place of the BLF."""
    _check(load().blfls_smooth_nc(h, _ptr(img), _ptr(out), int(H), int(W), int(C), float(lam),
                                  float(sigma_s), float(sigma_r), int(iters), int(nc_iters),
                                  _stream(stream)), h)


def blfls_blf_residual(h, img, ex, ey, H, W, C, sigma_s, sigma_r, radius, prec=BLFLS_FP32,
                       stream=None) -> None:
    _check(load().blfls_blf_residual(h, _ptr(img), _ptr(ex), _ptr(ey), int(H), int(W), int(C),
                                     float(sigma_s), float(sigma_r), int(radius), _prec(prec),
                                     _stream(stream)), h)


def blfls_solve_residual(h, img, ex, ey, out, H, W, C, lam, stream=None) -> None:
    _check(load().blfls_solve_residual(h, _ptr(img), _ptr(ex), _ptr(ey), _ptr(out), int(H),
                                       int(W), int(C), float(lam), _stream(stream)), h)


def blfls_solve_residual_noalloc(img, ex, ey, out, H, W, C, lam, stream=None) -> None:
    """The solve step without device allocation; scratch is the library's static array."""
    _check(load().blfls_solve_residual_noalloc(_ptr(img), _ptr(ex), _ptr(ey), _ptr(out), int(H),
                                               int(W), int(C), float(lam), _stream(stream)))


def make_job(img, out, H, W, C, lam, sigma_s, sigma_r, radius, iters=1, prec=BLFLS_FP32):
    return blfls_job(_ptr(img), _ptr(out), int(H), int(W), int(C), float(lam), float(sigma_s),
                     float(sigma_r), int(radius), int(iters), _prec(prec))


def blfls_smooth_batch(h, jobs, stream=None) -> None:
    arr = (blfls_job * len(jobs))(*jobs)
    _check(load().blfls_smooth_batch(h, arr, len(jobs), _stream(stream)), h)


def blfls_submit(h, job) -> int:
    """Queue one device-pointer job (see make_job) on the handle's queue; returns its ticket."""
    t = ctypes.c_uint64()
    _check(load().blfls_submit(h, ctypes.byref(job), ctypes.byref(t)), h)
    return t.value


def blfls_poll(h, ticket) -> bool:
    """True once the job has finished (the ticket is then forgotten); raises if it failed."""
    d = ctypes.c_int()
    _check(load().blfls_poll(h, ctypes.c_uint64(ticket), ctypes.byref(d)), h)
    return bool(d.value)


def blfls_autotune(h, H, W, C, radius, prec=BLFLS_FP32, table_path: str | None = None) -> None:
    path = table_path.encode() if table_path else None
    _check(load().blfls_autotune(h, int(H), int(W), int(C), int(radius), _prec(prec), path), h)


def blfls_profile_begin(h, max_events: int) -> None:
    _check(load().blfls_profile_begin(h, int(max_events)), h)


def blfls_profile_end(h):
    """Returns (ms[4], launches[4]) for stages K1, K2, K3, K4."""
    ms = (ctypes.c_double * 4)()
    n = (ctypes.c_int * 4)()
    _check(load().blfls_profile_end(h, ms, n), h)
    return list(ms), list(n)


PIPE_RATE_NAMES = ["ffma_f32", "ffma2_f32", "ex2_f32", "ex2_f16x2", "ex2_bf16x2", "hfma2_f16",
                   "hmma_m16n8k16_mac"]


def blfls_pipe_rates(device: int = 0) -> dict:
    """Results per clock per SM of each arithmetic pipe, measured on the device."""
    r = (ctypes.c_double * len(PIPE_RATE_NAMES))()
    _check(load().blfls_pipe_rates(int(device), r, len(PIPE_RATE_NAMES)))
    return dict(zip(PIPE_RATE_NAMES, list(r)))


def blfls_server_create(device=0, mem_budget_bytes=80 << 30, slots=4, max_batch=16,
                        tune_table_path=None):
    srv = _vp()
    path = tune_table_path.encode() if tune_table_path else None
    _check(load().blfls_server_create(ctypes.byref(srv), int(device), int(mem_budget_bytes),
                                      int(slots), int(max_batch), path))
    return srv


def blfls_server_destroy(srv) -> None:
    if srv is not None:
        load().blfls_server_destroy(srv)


def make_request(img_host, out_host, H, W, C, lam, sigma_s, sigma_r, radius, iters=1,
                 prec=BLFLS_FP32):
    return blfls_request(_ptr(img_host), _ptr(out_host), int(H), int(W), int(C), float(lam),
                         float(sigma_s), float(sigma_r), int(radius), int(iters), _prec(prec))


def blfls_server_submit(srv, req) -> int:
    t = ctypes.c_uint64()
    _check(load().blfls_server_submit(srv, ctypes.byref(req), ctypes.byref(t)))
    return t.value


def blfls_server_poll(srv, ticket) -> int:
    st = ctypes.c_int()
    _check(load().blfls_server_poll(srv, ctypes.c_uint64(ticket), ctypes.byref(st)))
    return st.value


def blfls_server_wait(srv, ticket, timeout_ms=60000) -> None:
    _check(load().blfls_server_wait(srv, ctypes.c_uint64(ticket), int(timeout_ms)))


def blfls_server_cancel(srv, ticket) -> None:
    _check(load().blfls_server_cancel(srv, ctypes.c_uint64(ticket)))


def blfls_server_release(srv, ticket) -> None:
    _check(load().blfls_server_release(srv, ctypes.c_uint64(ticket)))


def blfls_server_get_stats(srv) -> dict:
    st = blfls_server_stats()
    _check(load().blfls_server_get_stats(srv, ctypes.byref(st)))
    return {name: getattr(st, name) for name, _ in st._fields_}


class Smoother:
    """Owns a handle; ``smooth(img, ...)`` smooths a CUDA tensor [C, H, W] (or [H, W]) into a new
    tensor (or into ``out``) on the current torch stream."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0, tune_table_path=None):
        self.h = blfls_create(device, mem_budget_bytes, tune_table_path)

    def close(self):
        if self.h is not None:
            blfls_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def smooth(self, img, lam, sigma_s, sigma_r, radius, iters=1, prec=BLFLS_FP32, out=None,
               stream=None):
        import torch
        if img.dtype != torch.float32 or not img.is_cuda or not img.is_contiguous():
            raise ValueError("img must be a contiguous float32 CUDA tensor")
        shape = img.shape
        C, H, W = (1, *shape) if img.dim() == 2 else shape
        if out is None:
            out = torch.empty_like(img)
        if stream is None:
            stream = torch.cuda.current_stream(img.device)
        blfls_smooth(self.h, img, out, H, W, C, lam, sigma_s, sigma_r, radius, iters, prec,
                     stream)
        return out


def blfls_device_checks(device: int = 0) -> int:
    """OR of the device range-check words since the last call (0 in a release build)."""
    w = ctypes.c_uint()
    _check(load().blfls_device_checks(int(device), ctypes.byref(w)))
    return int(w.value)
