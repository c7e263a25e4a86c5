"""Python binding of the C-ABI in include/fuse.h (ctypes; argument marshalling only).

One Python function per C entry point, with the same name.  Device buffers are passed as
integer device addresses (e.g. torch.Tensor.data_ptr()), streams as integer cudaStream_t
handles (torch.cuda.current_stream().cuda_stream).  Every step of the solve runs inside
libfuse.so; if the library is missing this module raises instead of computing anything.

`Fusion` wraps a context for torch tensors: it checks device, dtype and contiguity and
forwards pointers and the current stream.
"""
from __future__ import annotations

import ctypes
import pathlib

import numpy as np

LIB_PATH = pathlib.Path(__file__).resolve().parent / "_build" / "libfuse.so"

FUSE_OK, FUSE_EINVAL, FUSE_ENOMEM, FUSE_ECUDA = 0, 1, 2, 3
FUSE_ETIMEOUT, FUSE_ENONFINITE, FUSE_ESTATE, FUSE_EUNSUPPORTED = 4, 5, 6, 7
FUSE_F32, FUSE_F64, FUSE_BF16 = 0, 1, 2
FUSE_OPT_PROFILE, FUSE_OPT_GRAPH = 1, 2
FUSE_OPT_LATENT_IMPL, FUSE_OPT_LATENT_THREADS, FUSE_OPT_LATENT_STAGES, FUSE_OPT_WAIT_LIMIT = 3, 4, 5, 6
FUSE_OPT_HALF_WINDOW, FUSE_OPT_LATENT_BANDS, FUSE_OPT_FFT_ROWS, FUSE_OPT_FFT_COLS = 7, 8, 9, 10
FUSE_OPT_GRAD_SEGMENT, FUSE_OPT_GRAD_WEIGHTS, FUSE_OPT_STATE_FORMAT = 11, 12, 13
FUSE_OPT_X_UPDATE, FUSE_OPT_RESIDUALS, FUSE_OPT_SEPARABLE_BLUR, FUSE_OPT_FFT_IMPL = 14, 15, 16, 17
FUSE_K_ALL, FUSE_K_LATENT = 0, 1

DTYPES = {"f32": FUSE_F32, "f64": FUSE_F64, "bf16": FUSE_BF16}


class fuse_geometry(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int), ("W", ctypes.c_int), ("L_l", ctypes.c_int),
                ("L_h", ctypes.c_int), ("L_s", ctypes.c_int), ("L_guide", ctypes.c_int)]


class FuseError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_status_name(status)}: {msg}")
        self.status = status


_lib = None
_D = ctypes.POINTER(ctypes.c_double)
_VP = ctypes.c_void_p
_I = ctypes.c_int
_ST = ctypes.c_int


def load(path: str | pathlib.Path | None = None):
    """Load libfuse.so (built by paper_2210_04184_gb300.build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    p = pathlib.Path(path) if path else LIB_PATH
    if not p.exists():
        raise RuntimeError(f"{p} is missing: the CUDA library must be built (build.build()) "
                           "before the solver can run")
    lib = ctypes.CDLL(str(p))
    sig = {
        "fuse_workspace_bytes": (_ST, [ctypes.POINTER(fuse_geometry), _I, _I, _I, _I, _I,
                                       ctypes.POINTER(ctypes.c_size_t)]),
        "fuse_init": (_ST, [ctypes.POINTER(_VP), ctypes.POINTER(fuse_geometry), _D, _I, _I, _I, _D, _D,
                            _I, _I, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                            _I, _I, _VP]),
        "fuse_destroy": (_ST, [_VP]),
        "fuse_set_stream": (_ST, [_VP, _VP]),
        "fuse_weights": (_ST, [_VP, _VP]),
        "fuse_set_weights": (_ST, [_VP, _VP]),
        "fuse_get_weights": (_ST, [_VP, _VP]),
        "fuse_solve": (_ST, [_VP, _VP, _VP, _I, _I, _VP, _VP]),
        "fuse_run_host": (_ST, [_VP, _VP, _VP, _VP, _I, _VP, _VP]),
        "fuse_objective": (_ST, [_VP, _VP, _VP, _D]),
        "fuse_residuals": (_ST, [_VP, _D]),
        "fuse_state_bytes": (_ST, [_VP, ctypes.POINTER(ctypes.c_size_t)]),
        "fuse_get_state": (_ST, [_VP, _VP]),
        "fuse_set_state": (_ST, [_VP, _VP]),
        "fuse_set_option": (_ST, [_VP, _I, ctypes.c_longlong]),
        "fuse_profile": (_ST, [_VP, _I, _D, ctypes.POINTER(ctypes.c_longlong), _I]),
        "fuse_sync": (_ST, [_VP]),
        "fuse_get_option": (_ST, [_VP, _I, ctypes.POINTER(ctypes.c_longlong)]),
        "fuse_autotune": (_ST, [_VP, _VP, _VP, _I]),
        "fuse_batch_autotune": (_ST, [_VP, ctypes.POINTER(_VP), ctypes.POINTER(_VP), _I]),
        "fuse_selftest": (_ST, [_VP, _I]),
        "fuse_grad_bytes": (_ST, [_VP, _I, ctypes.POINTER(ctypes.c_size_t)]),
        "fuse_conditioning": (_ST, [_VP, _D]),
        "fuse_set_mask": (_ST, [_VP, _VP]),
        "fuse_grad_forward": (_ST, [_VP, _VP, _VP, _I, _VP]),
        "fuse_grad_backward": (_ST, [_VP, _VP, _VP, _VP, _VP, _D]),
        "fuse_grad": (_ST, [_VP, _VP, _VP, _I, _VP, _VP, _VP, _VP, _VP, _D]),
        "fuse_grad_weights": (_ST, [_VP, _VP, _VP, _VP]),
        "fuse_phi_static": (_ST, [_VP, _VP, _I, _I, _I, _I, _I, _I, _I, _VP, _VP]),
        "fuse_batch_create": (_ST, [ctypes.POINTER(_VP), ctypes.POINTER(_VP), _I, _VP]),
        "fuse_batch_solve": (_ST, [_VP, ctypes.POINTER(_VP), ctypes.POINTER(_VP), _I, ctypes.POINTER(_VP),
                                   ctypes.POINTER(_VP)]),
        "fuse_batch_run_host": (_ST, [_VP, ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.POINTER(_VP), _I,
                                      ctypes.POINTER(_VP), ctypes.POINTER(_VP)]),
        "fuse_batch_set_option": (_ST, [_VP, _I, ctypes.c_longlong]),
        "fuse_batch_get_option": (_ST, [_VP, _I, ctypes.POINTER(ctypes.c_longlong)]),
        "fuse_batch_profile": (_ST, [_VP, _I, _D, ctypes.POINTER(ctypes.c_longlong), _I]),
        "fuse_batch_sync": (_ST, [_VP]),
        "fuse_batch_destroy": (_ST, [_VP]),
        "fuse_batch_last_error": (ctypes.c_char_p, [_VP]),
        "fuse_last_error": (ctypes.c_char_p, [_VP]),
        "fuse_reset_error": (_ST, [_VP]),
        "fuse_status_string": (ctypes.c_char_p, [_I]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _status_name(s: int) -> str:
    names = ["FUSE_OK", "FUSE_EINVAL", "FUSE_ENOMEM", "FUSE_ECUDA", "FUSE_ETIMEOUT",
             "FUSE_ENONFINITE", "FUSE_ESTATE", "FUSE_EUNSUPPORTED"]
    return names[s] if 0 <= s < len(names) else f"status {s}"


def _check(st: int, ctx=None):
    if st != FUSE_OK:
        msg = ""
        if ctx is not None and _lib is not None:
            raw = _lib.fuse_last_error(ctx)
            msg = raw.decode() if raw else ""
        raise FuseError(st, msg)


def _dptr(a: np.ndarray | None):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a.ctypes.data_as(_D), a          # keep `a` alive alongside the pointer


# ----- one function per entry point --------------------------------------------------------

def fuse_workspace_bytes(geom: fuse_geometry, K: int, S: int, ratio: int, dtype: int, wdtype: int) -> int:
    out = ctypes.c_size_t(0)
    _check(load().fuse_workspace_bytes(ctypes.byref(geom), K, S, ratio, dtype, wdtype, ctypes.byref(out)))
    return out.value


def fuse_init(geom: fuse_geometry, blur: np.ndarray, ratio: int, R: np.ndarray, E: np.ndarray | None,
              K: int, S: int, lambda1: float, lambda2: float, rho: float, h: float,
              dtype: int, wdtype: int, stream: int = 0):
    blur = np.ascontiguousarray(blur, dtype=np.float64)
    pb, kb = _dptr(blur)
    pr, kr = _dptr(R)
    pe, ke = _dptr(E) if E is not None else (None, None)
    ctx = _VP()
    st = load().fuse_init(ctypes.byref(ctx), ctypes.byref(geom), pb, blur.shape[0], blur.shape[1], ratio,
                          pr, pe, K, S, lambda1, lambda2, rho, h, dtype, wdtype, _VP(stream or None))
    _check(st)
    return ctx


def fuse_destroy(ctx):
    _check(load().fuse_destroy(ctx))


def fuse_set_stream(ctx, stream: int):
    _check(load().fuse_set_stream(ctx, _VP(stream or None)), ctx)


def fuse_weights(ctx, guide_dev: int):
    _check(load().fuse_weights(ctx, _VP(guide_dev)), ctx)


def fuse_set_weights(ctx, w_dev: int):
    _check(load().fuse_set_weights(ctx, _VP(w_dev)), ctx)


def fuse_get_weights(ctx, w_dev: int):
    _check(load().fuse_get_weights(ctx, _VP(w_dev)), ctx)


def fuse_solve(ctx, Yl_dev: int, Yh_dev: int, iters: int, warm: int, X_out: int | None, Z_out: int | None):
    _check(load().fuse_solve(ctx, _VP(Yl_dev), _VP(Yh_dev), iters, warm, _VP(X_out or None),
                             _VP(Z_out or None)), ctx)


def fuse_run_host(ctx, Yl_host: int, Yh_host: int, guide_host: int | None, iters: int,
                  X_host: int | None, Z_host: int | None):
    _check(load().fuse_run_host(ctx, _VP(Yl_host), _VP(Yh_host), _VP(guide_host or None), iters,
                                _VP(X_host or None), _VP(Z_host or None)), ctx)


def fuse_objective(ctx, Yl_dev: int, Yh_dev: int) -> np.ndarray:
    out = np.zeros(4)
    _check(load().fuse_objective(ctx, _VP(Yl_dev), _VP(Yh_dev), out.ctypes.data_as(_D)), ctx)
    return out


def fuse_residuals(ctx) -> tuple[float, float]:
    out = np.zeros(2)
    _check(load().fuse_residuals(ctx, out.ctypes.data_as(_D)), ctx)
    return float(out[0]), float(out[1])


def fuse_state_bytes(ctx) -> int:
    out = ctypes.c_size_t(0)
    _check(load().fuse_state_bytes(ctx, ctypes.byref(out)), ctx)
    return out.value


def fuse_get_state(ctx, dst: int):
    _check(load().fuse_get_state(ctx, _VP(dst)), ctx)


def fuse_set_state(ctx, src: int):
    _check(load().fuse_set_state(ctx, _VP(src)), ctx)


def fuse_set_option(ctx, option: int, value: int):
    _check(load().fuse_set_option(ctx, option, value), ctx)


def fuse_profile(ctx, which: int, reset: bool = False) -> tuple[float, int]:
    ms = ctypes.c_double(0.0)
    n = ctypes.c_longlong(0)
    _check(load().fuse_profile(ctx, which, ctypes.byref(ms), ctypes.byref(n), int(reset)), ctx)
    return ms.value, n.value


def fuse_get_option(ctx, option: int) -> int:
    v = ctypes.c_longlong(0)
    _check(load().fuse_get_option(ctx, option, ctypes.byref(v)), ctx)
    return v.value


def fuse_autotune(ctx, Yl_dev: int, Yh_dev: int, iters: int = 2):
    _check(load().fuse_autotune(ctx, _VP(Yl_dev), _VP(Yh_dev), iters), ctx)


def fuse_batch_autotune(b, Yl_devs, Yh_devs, iters: int = 2):
    _bcheck(load().fuse_batch_autotune(b, _ptrs(Yl_devs), _ptrs(Yh_devs), iters), b)


def fuse_sync(ctx):
    _check(load().fuse_sync(ctx), ctx)


def fuse_selftest(ctx, which: int):
    _check(load().fuse_selftest(ctx, which), ctx)


def fuse_phi_static(X_dev: int, omega_dev: int, H: int, W: int, L_s: int, K: int, S: int,
                    dtype: int, wdtype: int, phi_dev: int, stream: int = 0):
    _check(load().fuse_phi_static(_VP(X_dev), _VP(omega_dev), H, W, L_s, K, S, dtype, wdtype,
                                  _VP(phi_dev), _VP(stream or None)))


def fuse_set_mask(ctx, mask_ptr: int | None):
    _check(load().fuse_set_mask(ctx, _VP(mask_ptr or None)), ctx)


def fuse_conditioning(ctx) -> tuple[float, float, float]:
    out = (ctypes.c_double * 3)()
    _check(load().fuse_conditioning(ctx, out), ctx)
    return out[0], out[1], out[2]


def fuse_grad_bytes(ctx, iters: int) -> int:
    out = ctypes.c_size_t(0)
    _check(load().fuse_grad_bytes(ctx, iters, ctypes.byref(out)), ctx)
    return int(out.value)


def fuse_grad_forward(ctx, Yl_dev: int, Yh_dev: int, iters: int, X_out: int | None):
    _check(load().fuse_grad_forward(ctx, _VP(Yl_dev), _VP(Yh_dev), iters, _VP(X_out or None)), ctx)


def fuse_grad_backward(ctx, Xbar_dev: int | None, Zbar_dev: int | None, Yl_bar: int | None,
                       Yh_bar: int | None, want_params: bool = True):
    """Returns (dL/dlambda1, dL/dlambda2, dL/drho) when want_params, else None."""
    pb = (ctypes.c_double * 3)()
    _check(load().fuse_grad_backward(ctx, _VP(Xbar_dev or None), _VP(Zbar_dev or None), _VP(Yl_bar or None),
                                     _VP(Yh_bar or None), pb if want_params else None), ctx)
    return (pb[0], pb[1], pb[2]) if want_params else None


def fuse_grad_weights(ctx, omega_bar: int | None, guide_dev: int | None, guide_bar: int | None):
    _check(load().fuse_grad_weights(ctx, _VP(omega_bar or None), _VP(guide_dev or None), _VP(guide_bar or None)),
           ctx)


def fuse_grad(ctx, Yl_dev: int, Yh_dev: int, iters: int, Xbar_dev: int | None, Zbar_dev: int | None,
              X_out: int | None, Yl_bar: int | None, Yh_bar: int | None, want_params: bool = True):
    pb = (ctypes.c_double * 3)()
    _check(load().fuse_grad(ctx, _VP(Yl_dev), _VP(Yh_dev), iters, _VP(Xbar_dev or None), _VP(Zbar_dev or None),
                            _VP(X_out or None), _VP(Yl_bar or None), _VP(Yh_bar or None),
                            pb if want_params else None), ctx)
    return (pb[0], pb[1], pb[2]) if want_params else None


def _bcheck(st: int, b=None):
    if st != FUSE_OK:
        msg = ""
        if b is not None and _lib is not None:
            raw = _lib.fuse_batch_last_error(b)
            msg = raw.decode() if raw else ""
        raise FuseError(st, msg)


def _ptrs(vals):
    arr = (_VP * len(vals))()
    for i, v in enumerate(vals):
        arr[i] = v or None
    return arr


def fuse_batch_create(ctxs, stream: int = 0):
    out = _VP()
    arr = (_VP * len(ctxs))(*[c.value if isinstance(c, _VP) else c for c in ctxs])
    _bcheck(load().fuse_batch_create(ctypes.byref(out), arr, len(ctxs), _VP(stream or None)))
    return out


def fuse_batch_solve(b, Yl_devs, Yh_devs, iters: int, X_outs=None, Z_outs=None):
    n = len(Yl_devs)
    xo = _ptrs(X_outs) if X_outs is not None else None
    zo = _ptrs(Z_outs) if Z_outs is not None else None
    _bcheck(load().fuse_batch_solve(b, _ptrs(Yl_devs), _ptrs(Yh_devs), iters, xo, zo), b)


def fuse_batch_run_host(b, Yl_hosts, Yh_hosts, guide_hosts, iters: int, X_hosts=None, Z_hosts=None):
    go = _ptrs(guide_hosts) if guide_hosts is not None else None
    xo = _ptrs(X_hosts) if X_hosts is not None else None
    zo = _ptrs(Z_hosts) if Z_hosts is not None else None
    _bcheck(load().fuse_batch_run_host(b, _ptrs(Yl_hosts), _ptrs(Yh_hosts), go, iters, xo, zo), b)


def fuse_batch_set_option(b, option: int, value: int):
    _bcheck(load().fuse_batch_set_option(b, option, value), b)


def fuse_batch_get_option(b, option: int) -> int:
    v = ctypes.c_longlong(0)
    _bcheck(load().fuse_batch_get_option(b, option, ctypes.byref(v)), b)
    return v.value


def fuse_batch_profile(b, which: int, reset: bool = False):
    ms = ctypes.c_double(0.0)
    n = ctypes.c_longlong(0)
    _bcheck(load().fuse_batch_profile(b, which, ctypes.byref(ms), ctypes.byref(n), int(reset)), b)
    return ms.value, n.value


def fuse_batch_sync(b):
    _bcheck(load().fuse_batch_sync(b), b)


def fuse_batch_destroy(b):
    _bcheck(load().fuse_batch_destroy(b))


def fuse_batch_last_error(b) -> str:
    raw = load().fuse_batch_last_error(b)
    return raw.decode() if raw else ""


def fuse_last_error(ctx) -> str:
    raw = load().fuse_last_error(ctx)
    return raw.decode() if raw else ""


def fuse_reset_error(ctx):
    _check(load().fuse_reset_error(ctx))


def fuse_status_string(status: int) -> str:
    return load().fuse_status_string(status).decode()


# ----- torch convenience wrapper (marshalling only) ----------------------------------------

class Fusion:
    """One solver context bound to the current CUDA device and stream.

    Arrays: images planar (L, H, W); blur (bh, bw); R (L_l, L_h); E (L_s, L_l) or None."""

    def __init__(self, *, H, W, L_l, L_h, L_s, blur, ratio, R, E, K, S, lam1, lam2, rho, h,
                 dtype="f32", wdtype="bf16", L_guide=None, stream=None):
        import torch
        self.torch = torch
        self.geom = fuse_geometry(H, W, L_l, L_h, L_s, L_guide or L_h)
        self.H, self.W, self.L_l, self.L_h, self.L_s, self.ratio = H, W, L_l, L_h, L_s, ratio
        self.K, self.S = K, S
        self.nW = (2 * S + 1) ** 2 - 1
        self.dtype = dtype
        self.wdtype = wdtype
        self.tdtype = torch.float64 if dtype == "f64" else torch.float32
        self.wtdtype = {"bf16": torch.bfloat16, "f32": torch.float32, "f64": torch.float64}[wdtype]
        self._lam1, self._lam2, self._rho = float(lam1), float(lam2), float(rho)
        s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        self.ctx = fuse_init(self.geom, blur, ratio, R, E, K, S, lam1, lam2, rho, h,
                             DTYPES[dtype], DTYPES[wdtype], s)

    @classmethod
    def from_problem(cls, p, dtype="f32", wdtype="bf16", **kw):
        return cls(H=p.H, W=p.W, L_l=p.L_l, L_h=p.L_h, L_s=p.L_s, blur=p.blur, ratio=p.d, R=p.R, E=p.E,
                   K=p.K, S=p.S, lam1=p.lam1, lam2=p.lam2, rho=p.rho, h=p.h, dtype=dtype, wdtype=wdtype, **kw)

    def _t(self, a, shape=None, dtype=None):
        t = self.torch
        dtype = dtype or self.tdtype
        if not isinstance(a, t.Tensor):
            a = t.as_tensor(np.asarray(a), dtype=dtype, device="cuda")
        if a.device.type != "cuda" or a.dtype != dtype or not a.is_contiguous():
            raise ValueError(f"expected a contiguous CUDA tensor of {dtype}")
        if shape is not None and tuple(a.shape) != tuple(shape):
            raise ValueError(f"expected shape {shape}, got {tuple(a.shape)}")
        return a

    def _sync_stream(self):
        fuse_set_stream(self.ctx, self.torch.cuda.current_stream().cuda_stream)

    def weights(self, guide):
        g = self._t(guide, (self.geom.L_guide, self.H, self.W))
        self._sync_stream()
        fuse_weights(self.ctx, g.data_ptr())
        return g

    def set_weights(self, w):
        w = self._t(w, (self.nW, self.H, self.W), self.wtdtype)
        self._sync_stream()
        fuse_set_weights(self.ctx, w.data_ptr())

    def get_weights(self):
        w = self.torch.empty((self.nW, self.H, self.W), dtype=self.wtdtype, device="cuda")
        self._sync_stream()
        fuse_get_weights(self.ctx, w.data_ptr())
        return w

    def solve(self, Yl, Yh, iters, warm=False, want_X=True, want_Z=False):
        d = self.ratio
        yl = self._t(Yl, (self.L_l, self.H // d, self.W // d))
        yh = self._t(Yh, (self.L_h, self.H, self.W))
        X = self.torch.empty((self.L_s, self.H, self.W), dtype=self.tdtype, device="cuda") if want_X else None
        Z = self.torch.empty((self.L_l, self.H, self.W), dtype=self.tdtype, device="cuda") if want_Z else None
        self._sync_stream()
        fuse_solve(self.ctx, yl.data_ptr(), yh.data_ptr(), iters, int(warm),
                   X.data_ptr() if X is not None else None, Z.data_ptr() if Z is not None else None)
        self._keep = (yl, yh)
        return X, Z

    def objective(self, Yl, Yh):
        d = self.ratio
        yl = self._t(Yl, (self.L_l, self.H // d, self.W // d))
        yh = self._t(Yh, (self.L_h, self.H, self.W))
        self._sync_stream()
        return fuse_objective(self.ctx, yl.data_ptr(), yh.data_ptr())

    def residuals(self):
        """(primal, dual) ADMM residual norms of the last iteration of the last solve (run with
        FUSE_OPT_RESIDUALS = 1)."""
        self._sync_stream()
        return fuse_residuals(self.ctx)

    def get_state(self):
        nb = fuse_state_bytes(self.ctx)
        buf = self.torch.empty(nb, dtype=self.torch.uint8, device="cuda")
        self._sync_stream()
        fuse_get_state(self.ctx, buf.data_ptr())
        return buf

    def set_state(self, buf):
        self._sync_stream()
        fuse_set_state(self.ctx, buf.data_ptr())

    def profile(self, which=FUSE_K_LATENT, reset=False):
        return fuse_profile(self.ctx, which, reset)

    def set_option(self, option, value):
        fuse_set_option(self.ctx, option, value)

    def get_option(self, option):
        return fuse_get_option(self.ctx, option)

    def sync(self):
        fuse_sync(self.ctx)

    def autotune(self, Yl, Yh, iters=2):
        d = self.ratio
        yl = self._t(Yl, (self.L_l, self.H // d, self.W // d))
        yh = self._t(Yh, (self.L_h, self.H, self.W))
        self._sync_stream()
        fuse_autotune(self.ctx, yl.data_ptr(), yh.data_ptr(), iters)
        return {k: fuse_get_option(self.ctx, v) for k, v in
                (("latent_threads", FUSE_OPT_LATENT_THREADS), ("latent_stages", FUSE_OPT_LATENT_STAGES),
                 ("latent_bands", FUSE_OPT_LATENT_BANDS), ("fft_rows", FUSE_OPT_FFT_ROWS),
                 ("fft_cols", FUSE_OPT_FFT_COLS))}

    # ---- reverse pass ----
    def grad_forward(self, Yl, Yh, iters):
        """`iters` iterations from zero state with checkpoints; returns X of the last one."""
        d = self.ratio
        yl = self._t(Yl, (self.L_l, self.H // d, self.W // d))
        yh = self._t(Yh, (self.L_h, self.H, self.W))
        X = self.torch.empty((self.L_s, self.H, self.W), dtype=self.tdtype, device="cuda")
        self._sync_stream()
        fuse_grad_forward(self.ctx, yl.data_ptr(), yh.data_ptr(), iters, X.data_ptr())
        self._keep = (yl, yh)
        return X

    def grad_backward(self, Xbar=None, Zbar=None):
        """Reverse pass of the last grad_forward for dL/dX (and/or dL/dZ) of the last iterate.
        Returns (dL/dY_l, dL/dY_h, {"lam1", "lam2", "rho"})."""
        t = self.torch
        xb = self._t(Xbar, (self.L_s, self.H, self.W)) if Xbar is not None else None
        zb = self._t(Zbar, (self.L_l, self.H, self.W)) if Zbar is not None else None
        d = self.ratio
        gl = t.empty((self.L_l, self.H // d, self.W // d), dtype=self.tdtype, device="cuda")
        gh = t.empty((self.L_h, self.H, self.W), dtype=self.tdtype, device="cuda")
        self._sync_stream()
        p = fuse_grad_backward(self.ctx, xb.data_ptr() if xb is not None else None,
                               zb.data_ptr() if zb is not None else None, gl.data_ptr(), gh.data_ptr())
        return gl, gh, dict(lam1=p[0], lam2=p[1], rho=p[2])

    def grad_weights(self, guide=None):
        """dL/domega of the last grad_backward (run with FUSE_OPT_GRAD_WEIGHTS = 1) and, when the
        guide that produced the weights is given, dL/dguide through eq. wts."""
        t = self.torch
        ob = t.empty((self.nW, self.H, self.W), dtype=self.tdtype, device="cuda")
        g = self._t(guide, (self.geom.L_guide, self.H, self.W)) if guide is not None else None
        gb = t.empty((self.geom.L_guide, self.H, self.W), dtype=self.tdtype, device="cuda") if g is not None else None
        self._sync_stream()
        fuse_grad_weights(self.ctx, ob.data_ptr(), g.data_ptr() if g is not None else None,
                          gb.data_ptr() if gb is not None else None)
        return ob, gb

    def set_mask(self, mask):
        """Sampling mask (H, W) of 0/1 (any integer or bool array or tensor; ratio 1), or None for
        the regular lattice; Y_l is then given at full resolution."""
        if mask is None:
            fuse_set_mask(self.ctx, None)
            return
        t = self.torch
        m = t.as_tensor(np.asarray(mask.cpu() if isinstance(mask, t.Tensor) else mask) != 0,
                        dtype=t.uint8).contiguous()
        if tuple(m.shape) != (self.H, self.W):
            raise ValueError(f"expected a mask of shape {(self.H, self.W)}")
        self._sync_stream()
        fuse_set_mask(self.ctx, m.data_ptr())
        self.sync()                     # the host copy is read by the asynchronous copy

    def params(self):
        """(lambda1, lambda2, rho) of the context as a float64 CPU tensor, for unrolled()."""
        return self.torch.tensor([self._lam1, self._lam2, self._rho], dtype=self.torch.float64)

    def unrolled(self, Yl, Yh, iters, params=None, guide=None):
        """X after `iters` iterations from zero state as a differentiable function of Y_l, Y_h,
        params = (lambda1, lambda2, rho) (a tensor equal to the context's values, see params())
        and, when given, the guide: the weights are then computed from it (fuse_weights) and
        differentiated through; without a guide the context's current weights are constants.
        Passing Y_h itself as the guide gives it both gradient paths (torch adds them)."""
        if params is None:
            params = self.params()
        return UnrolledADMM.apply(Yl, Yh, params, guide, self, iters)

    def close(self):
        if getattr(self, "ctx", None):
            fuse_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class FusionBatch:
    """Several Fusion contexts solved together (one launch per ADMM phase over all problems)."""

    def __init__(self, fusions, stream=None):
        import torch
        self.torch = torch
        self.fusions = list(fusions)
        s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        self.b = fuse_batch_create([f.ctx for f in self.fusions], s)

    def solve(self, Yls, Yhs, iters, want_X=True, want_Z=False):
        t = self.torch
        yl = [f._t(y, (f.L_l, f.H // f.ratio, f.W // f.ratio)) for f, y in zip(self.fusions, Yls)]
        yh = [f._t(y, (f.L_h, f.H, f.W)) for f, y in zip(self.fusions, Yhs)]
        Xs = [t.empty((f.L_s, f.H, f.W), dtype=f.tdtype, device="cuda") for f in self.fusions] if want_X else None
        Zs = [t.empty((f.L_l, f.H, f.W), dtype=f.tdtype, device="cuda") for f in self.fusions] if want_Z else None
        fuse_batch_solve(self.b, [y.data_ptr() for y in yl], [y.data_ptr() for y in yh], iters,
                         [x.data_ptr() for x in Xs] if Xs else None, [z.data_ptr() for z in Zs] if Zs else None)
        self._keep = (yl, yh)
        return Xs, Zs

    def run_host(self, Yls, Yhs, iters, want_X=False, want_Z=True, guides=None):
        """End to end on host tensors (pinned CPU tensors of the contexts' dtype): inputs copied
        in, weights, batched solve from zero, X and/or Z copied back (fuse_batch_run_host)."""
        t = self.torch
        for f, a, b in zip(self.fusions, Yls, Yhs):
            if a.device.type != "cpu" or b.device.type != "cpu" or a.dtype != f.tdtype or b.dtype != f.tdtype:
                raise ValueError(f"expected CPU tensors of {f.tdtype}")
            if not (a.is_contiguous() and b.is_contiguous()):
                raise ValueError("expected contiguous tensors")
            if tuple(a.shape) != (f.L_l, f.H // f.ratio, f.W // f.ratio) or tuple(b.shape) != (f.L_h, f.H, f.W):
                raise ValueError("input shape does not match its context")
        Xs = [t.empty((f.L_s, f.H, f.W), dtype=f.tdtype).pin_memory() for f in self.fusions] if want_X else None
        Zs = [t.empty((f.L_l, f.H, f.W), dtype=f.tdtype).pin_memory() for f in self.fusions] if want_Z else None
        gp = [g.data_ptr() for g in guides] if guides is not None else None
        fuse_batch_run_host(self.b, [a.data_ptr() for a in Yls], [b.data_ptr() for b in Yhs], gp, iters,
                            [x.data_ptr() for x in Xs] if Xs else None, [z.data_ptr() for z in Zs] if Zs else None)
        return Xs, Zs

    def set_option(self, option, value):
        fuse_batch_set_option(self.b, option, value)

    def latent_shape(self):
        """The batch's latent launch shape (consumer threads, ring slots, bands per block)."""
        return {k: fuse_batch_get_option(self.b, v) for k, v in
                (("latent_threads", FUSE_OPT_LATENT_THREADS), ("latent_stages", FUSE_OPT_LATENT_STAGES),
                 ("latent_bands", FUSE_OPT_LATENT_BANDS))}

    def profile(self, which=FUSE_K_LATENT, reset=False):
        return fuse_batch_profile(self.b, which, reset)

    def autotune(self, Yls, Yhs, iters=2):
        fuse_batch_autotune(self.b, [y.data_ptr() for y in Yls], [y.data_ptr() for y in Yhs], iters)

    def sync(self):
        fuse_batch_sync(self.b)

    def close(self):
        if getattr(self, "b", None):
            fuse_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _unrolled_function():
    import torch

    class _Unrolled(torch.autograd.Function):
        """X_K of K unrolled ADMM iterations (fuse_grad_forward) with its reverse pass
        (fuse_grad_backward).  The weights omega are constants of the map."""

        @staticmethod
        def forward(ctx, Yl, Yh, params, guide, fusion, iters):
            p = [float(v) for v in params.detach().cpu().tolist()]
            ref = (fusion._lam1, fusion._lam2, fusion._rho)
            if any(abs(a - b) > 1e-12 * max(1.0, abs(b)) for a, b in zip(p, ref)):
                raise ValueError(f"params {p} differ from the context's (lambda1, lambda2, rho) = {ref}")
            ctx.fusion = fusion
            ctx.pdev = params.device
            ctx.pdtype = params.dtype
            ctx.guide = guide.detach() if guide is not None else None
            if guide is not None:
                fusion.weights(ctx.guide)
            fusion.set_option(FUSE_OPT_GRAD_WEIGHTS, int(guide is not None and guide.requires_grad))
            return fusion.grad_forward(Yl.detach(), Yh.detach(), iters)

        @staticmethod
        def backward(ctx, Xbar):
            f = ctx.fusion
            gl, gh, p = f.grad_backward(Xbar=Xbar.contiguous())
            gp = torch.tensor([p["lam1"], p["lam2"], p["rho"]], dtype=ctx.pdtype, device=ctx.pdev)
            gg = None
            if ctx.guide is not None and ctx.needs_input_grad[3]:
                _, gg = f.grad_weights(ctx.guide)
            return gl, gh, gp, gg, None, None

    return _Unrolled


class _LazyFunction:
    _fn = None

    def apply(self, *args):
        if _LazyFunction._fn is None:
            _LazyFunction._fn = _unrolled_function()
        return _LazyFunction._fn.apply(*args)


UnrolledADMM = _LazyFunction()
