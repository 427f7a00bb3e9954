"""ctypes binding of the SCSC C ABI (include/scsc.h).

Argument marshalling only: every step runs in the CUDA library.  Functions
carry the names of the C entry points; :class:`Context` and :class:`Batch`
hold the handle and the host descriptor arrays.  Tensors are torch CUDA
float32 tensors (contiguous); torch supplies device memory and streams.
The library is loaded on first use; if it is missing and cannot be built,
the call raises -- there is no other implementation to fall back to.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

c_int, c_double, c_u32, c_u64, c_i64, c_void_p, c_size_t = (
    ctypes.c_int, ctypes.c_double, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int64,
    ctypes.c_void_p, ctypes.c_size_t)

SCSC_OK, SCSC_EINVAL, SCSC_ENOMEM, SCSC_ECUDA, SCSC_ETIMEOUT, SCSC_ENONFINITE, SCSC_EUNSUPPORTED = range(7)
STATUS_NAMES = ["SCSC_OK", "SCSC_EINVAL", "SCSC_ENOMEM", "SCSC_ECUDA", "SCSC_ETIMEOUT",
                "SCSC_ENONFINITE", "SCSC_EUNSUPPORTED"]
SCSC_FP32, SCSC_BF16, SCSC_TF32 = 0, 1, 2
SCSC_DICT_BATCH, SCSC_DICT_ONLINE, SCSC_DICT_BATCH_GS = 0, 1, 2
(SCSC_FLAG_PER_IMAGE, SCSC_FLAG_NO_GRAPH, SCSC_FLAG_NO_AUTOTUNE, SCSC_FLAG_UNSAMPLED_KEEP,
 SCSC_FLAG_TWO_KERNEL) = 1, 2, 4, 8, 16


class scsc_config(ctypes.Structure):
    _fields_ = [("K", c_int), ("s", c_int), ("lambda_", c_double), ("p_num", c_u32),
                ("p_den", c_u32), ("seed", c_u64), ("prec", c_int), ("step", c_double),
                ("flags", c_u32)]


class scsc_batch(ctypes.Structure):
    _fields_ = [("n_images", c_int), ("offsets", ctypes.POINTER(c_i64)),
                ("H", ctypes.POINTER(c_int)), ("W", ctypes.POINTER(c_int)),
                ("image_ids", ctypes.POINTER(c_i64))]


class ScscError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {msg}")


_lock = threading.Lock()
_lib = None

_SIGNATURES = {
    "scsc_create": [ctypes.POINTER(scsc_config), c_void_p, ctypes.POINTER(c_void_p)],
    "scsc_destroy": [c_void_p],
    "scsc_mask": [c_void_p, ctypes.POINTER(scsc_batch), c_u64, c_void_p],
    "scsc_code_step": [c_void_p, ctypes.POINTER(scsc_batch), c_void_p, c_void_p, c_void_p, c_u64,
                       c_int],
    "scsc_code_step_observed": [c_void_p, ctypes.POINTER(scsc_batch), c_void_p, c_void_p,
                                c_void_p, c_void_p, c_u64, c_int],
    "scsc_code_step_host": [c_void_p, ctypes.POINTER(scsc_batch), c_void_p, c_void_p, c_void_p,
                            c_u64, c_int],
    "scsc_code_step_admm": [c_void_p, ctypes.POINTER(scsc_batch), c_void_p, c_void_p, c_void_p,
                            c_u64, c_int, c_int, c_double, c_double],
    "scsc_screen": [c_void_p, ctypes.POINTER(scsc_batch), c_void_p, c_void_p, c_void_p, c_void_p,
                    c_void_p, c_void_p],
    "scsc_code_step_screened": [c_void_p, ctypes.POINTER(scsc_batch), c_void_p, c_void_p,
                                c_void_p, c_u64, c_int, c_int, c_void_p, c_void_p],
    "scsc_dict_step": [c_void_p, ctypes.POINTER(scsc_batch), c_void_p, c_void_p, c_void_p, c_int,
                       c_u64],
    "scsc_objective_observed": [c_void_p, ctypes.POINTER(scsc_batch), c_void_p, c_void_p,
                                c_void_p, c_void_p, ctypes.POINTER(c_double)],
    "scsc_objective": [c_void_p, ctypes.POINTER(scsc_batch), c_void_p, c_void_p, c_void_p,
                       ctypes.POINTER(c_double)],
    "scsc_lipschitz_codes": [c_void_p, ctypes.POINTER(scsc_batch), c_void_p,
                             ctypes.POINTER(c_double)],
    "scsc_synth": [c_void_p, ctypes.POINTER(scsc_batch), c_void_p, c_void_p, c_u64, c_int,
                   c_void_p],
    "scsc_synth_backward": [c_void_p, ctypes.POINTER(scsc_batch), c_void_p, c_void_p, c_void_p,
                            c_u64, c_int, c_void_p, c_void_p],
    "scsc_sync": [c_void_p],
    "scsc_online_reset": [c_void_p],
    "scsc_online_state_size": [c_void_p, ctypes.POINTER(c_size_t)],
    "scsc_online_save": [c_void_p, c_void_p, c_size_t],
    "scsc_online_load": [c_void_p, c_void_p, c_size_t],
    "scsc_diag_tc_gemm": [c_int, c_void_p, c_void_p, c_void_p],
    "scsc_diag_tc_gemm_mn": [c_int, c_void_p, c_void_p, c_void_p, c_int],
    "scsc_diag_wait_timeout": [c_double],
    "scsc_diag_ffma_peak": [ctypes.POINTER(c_double), ctypes.POINTER(c_double)],
    "scsc_diag_mma_rate": [c_int, c_int, ctypes.POINTER(c_double), ctypes.POINTER(c_double)],
    "scsc_objective_noalloc": [ctypes.POINTER(scsc_config), c_int, c_int, c_int, c_void_p,
                               c_void_p, c_void_p, c_void_p, c_void_p],
    "scsc_diag_profile": [c_void_p, c_int],
    "scsc_diag_kernel_time": [c_void_p, ctypes.c_char_p, ctypes.POINTER(c_double),
                              ctypes.POINTER(c_int)],
}


def lib() -> ctypes.CDLL:
    """Load the in-tree CUDA library, building it first if it is stale."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ctypes.CDLL(path)
            for name, args in _SIGNATURES.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = c_int
            L.scsc_last_error.argtypes = [c_void_p]
            L.scsc_last_error.restype = ctypes.c_char_p
            _lib = L
    return _lib


def library_path() -> str:
    return _build.LIB


def _check(status: int, handle=None, what: str = "") -> None:
    if status != SCSC_OK:
        msg = what
        if handle:
            m = lib().scsc_last_error(handle)
            if m:
                msg = f"{what}: {m.decode()}" if what else m.decode()
        raise ScscError(status, msg)


def _ptr(t) -> int:
    """Device pointer of a contiguous CUDA float32/uint32 tensor (0 for None)."""
    if t is None:
        return 0
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _need(t, n: int, esize: int, name: str) -> None:
    """The C entry points take raw pointers: check here that a tensor holds at
    least n elements of esize bytes, so that no kernel runs past its end."""
    if t is None:
        return
    if t.element_size() != esize:
        raise ValueError(f"{name}: expected {esize}-byte elements, got {t.element_size()}")
    if t.numel() < n:
        raise ValueError(f"{name}: {t.numel()} elements, the batch needs {n}")


def _need_step(ctx, batch, x=None, d=None, z=None, observed=None, bits=None) -> None:
    """Sizes of the batch-level arguments: x and observed one per pixel, z K
    per pixel, d K s s, bits ceil(K/32) words per pixel."""
    P, K = batch.total_pixels, ctx.K
    _need(x, P, 4, "x")
    _need(d, K * ctx.s * ctx.s, 4, "d")
    _need(z, P * K, 4, "z")
    _need(observed, P, 1, "observed")
    _need(bits, P * ((K + 31) // 32), 4, "bits")


class Batch:
    """Host descriptor of images packed back to back (scsc_batch)."""

    def __init__(self, H, W, ids=None):
        self.H = np.ascontiguousarray(np.atleast_1d(H), dtype=np.int32)
        self.W = np.ascontiguousarray(np.atleast_1d(W), dtype=np.int32)
        if self.H.shape != self.W.shape:
            raise ValueError("H and W must have the same length")
        n = len(self.H)
        self.ids = np.ascontiguousarray(np.arange(n) if ids is None else ids, dtype=np.int64)
        sizes = self.H.astype(np.int64) * self.W.astype(np.int64)
        self.offsets = np.ascontiguousarray(
            np.concatenate([[0], np.cumsum(sizes)[:-1]]), dtype=np.int64)
        self.total_pixels = int(sizes.sum())
        self.c = scsc_batch(n, self.offsets.ctypes.data_as(ctypes.POINTER(c_i64)),
                            self.H.ctypes.data_as(ctypes.POINTER(c_int)),
                            self.W.ctypes.data_as(ctypes.POINTER(c_int)),
                            self.ids.ctypes.data_as(ctypes.POINTER(c_i64)))

    @property
    def n(self) -> int:
        return len(self.H)


def _stream_handle(stream) -> int:
    import torch
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


class Context:
    """An scsc_ctx bound to the current device and a CUDA stream."""

    def __init__(self, K: int, s: int = 11, lam: float = 1.0, p=(1, 1), seed: int = 0,
                 prec: str = "fp32", step: float = 0.0, stream=None, flags: int = 0):
        self.K, self.s, self.lam = int(K), int(s), float(lam)
        self.p = (int(p[0]), int(p[1]))
        self.seed = int(seed)
        self.prec = {"fp32": SCSC_FP32, "bf16": SCSC_BF16, "tf32": SCSC_TF32}[prec]
        self.cfg = scsc_config(self.K, self.s, self.lam, self.p[0], self.p[1], self.seed,
                               self.prec, float(step), int(flags))
        self.stream = stream
        self.handle = c_void_p()
        _check(lib().scsc_create(ctypes.byref(self.cfg), c_void_p(_stream_handle(stream)),
                                 ctypes.byref(self.handle)), None, "scsc_create")

    def close(self) -> None:
        if self.handle:
            lib().scsc_destroy(self.handle)
            self.handle = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # methods mirror the C entry points
    def code_step(self, batch, x, d, z, t, n_iters):
        return scsc_code_step(self, batch, x, d, z, t, n_iters)

    def code_step_observed(self, batch, x, d, z, observed, t, n_iters):
        return scsc_code_step_observed(self, batch, x, d, z, observed, t, n_iters)

    def code_step_host(self, batch, x, d, z, t, n_iters):
        return scsc_code_step_host(self, batch, x, d, z, t, n_iters)

    def code_step_admm(self, batch, x, d, z, t, n_iters, cg_iters, rho=0.0, alpha=0.0):
        return scsc_code_step_admm(self, batch, x, d, z, t, n_iters, cg_iters, rho, alpha)

    def screen(self, batch, x, d, z, bits):
        return scsc_screen(self, batch, x, d, z, bits)

    def code_step_screened(self, batch, x, d, z, t, n_iters, screen_every):
        return scsc_code_step_screened(self, batch, x, d, z, t, n_iters, screen_every)

    def objective_observed(self, batch, x, z, d, observed) -> float:
        return scsc_objective_observed(self, batch, x, z, d, observed)

    def dict_step(self, batch, x, z, d, mode=SCSC_DICT_BATCH, t=1):
        return scsc_dict_step(self, batch, x, z, d, mode, t)

    def objective(self, batch, x, z, d) -> float:
        return scsc_objective(self, batch, x, z, d)

    def mask(self, batch, t):
        return scsc_mask(self, batch, t)

    def lipschitz_codes(self, batch, d) -> float:
        return scsc_lipschitz_codes(self, batch, d)

    def synth(self, batch, z, d, t=0, masked=False, out=None):
        return scsc_synth(self, batch, z, d, t, masked, out)

    def synth_backward(self, batch, grad, z, d, t=0, masked=False, need_z=True, need_d=True):
        return scsc_synth_backward(self, batch, grad, z, d, t, masked, need_z, need_d)

    def sync(self):
        return scsc_sync(self)


# ------------------------------------------------------------------ entry points

def scsc_create(K, s=11, lam=1.0, p=(1, 1), seed=0, prec="fp32", step=0.0, stream=None, flags=0):
    return Context(K, s, lam, p, seed, prec, step, stream, flags)


def scsc_destroy(ctx: Context) -> None:
    ctx.close()


def scsc_last_error(ctx: Context) -> str:
    return lib().scsc_last_error(ctx.handle).decode()


def scsc_mask(ctx: Context, batch: Batch, t: int):
    import torch
    kw = (ctx.K + 31) // 32
    bits = torch.empty(batch.total_pixels * kw, dtype=torch.int32, device="cuda")
    _check(lib().scsc_mask(ctx.handle, ctypes.byref(batch.c), t, _ptr(bits)), ctx.handle,
           "scsc_mask")
    return bits


def scsc_code_step(ctx: Context, batch: Batch, x, d, z, t: int, n_iters: int) -> None:
    _need_step(ctx, batch, x=x, d=d, z=z)
    _check(lib().scsc_code_step(ctx.handle, ctypes.byref(batch.c), _ptr(x), _ptr(d), _ptr(z), t,
                                n_iters), ctx.handle, "scsc_code_step")


def scsc_dict_step(ctx: Context, batch: Batch, x, z, d, mode: int = SCSC_DICT_BATCH,
                   t: int = 1) -> None:
    _need_step(ctx, batch, x=x, d=d, z=z)
    _check(lib().scsc_dict_step(ctx.handle, ctypes.byref(batch.c), _ptr(x), _ptr(z), _ptr(d),
                                mode, t), ctx.handle, "scsc_dict_step")


def scsc_objective(ctx: Context, batch: Batch, x, z, d) -> float:
    _need_step(ctx, batch, x=x, d=d, z=z)
    out = c_double()
    _check(lib().scsc_objective(ctx.handle, ctypes.byref(batch.c), _ptr(x), _ptr(z), _ptr(d),
                                ctypes.byref(out)), ctx.handle, "scsc_objective")
    return out.value


def scsc_code_step_observed(ctx: Context, batch: Batch, x, d, z, observed, t: int,
                            n_iters: int) -> None:
    """Inpainting code update: observed is a uint8 device tensor, one byte per
    pixel (nonzero = observed), or None for every pixel."""
    _need_step(ctx, batch, x=x, d=d, z=z, observed=observed)
    _check(lib().scsc_code_step_observed(ctx.handle, ctypes.byref(batch.c), _ptr(x), _ptr(d),
                                         _ptr(z), _ptr(observed) if observed is not None else None,
                                         t, n_iters), ctx.handle, "scsc_code_step_observed")


def _host_ptr(t) -> int:
    """Address of a contiguous CPU float32 tensor (pinned for copy overlap)."""
    if t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CPU tensor")
    return t.data_ptr()


def scsc_code_step_host(ctx: Context, batch: Batch, x, d, z, t: int, n_iters: int) -> None:
    """scsc_code_step on host (CPU) tensors; z is updated in place."""
    _need_step(ctx, batch, x=x, d=d, z=z)
    _check(lib().scsc_code_step_host(ctx.handle, ctypes.byref(batch.c), _host_ptr(x),
                                     _host_ptr(d), _host_ptr(z), t, n_iters), ctx.handle,
           "scsc_code_step_host")


def scsc_code_step_admm(ctx: Context, batch: Batch, x, d, z, t: int, n_iters: int,
                        cg_iters: int, rho: float = 0.0, alpha: float = 0.0) -> None:
    """ADMM code update (rho, alpha <= 0: the paper's 10 lambda and 1.8)."""
    _need_step(ctx, batch, x=x, d=d, z=z)
    _check(lib().scsc_code_step_admm(ctx.handle, ctypes.byref(batch.c), _ptr(x), _ptr(d), _ptr(z),
                                     t, n_iters, cg_iters, float(rho), float(alpha)), ctx.handle,
           "scsc_code_step_admm")


def scsc_screen(ctx: Context, batch: Batch, x, d, z, bits):
    """Safe screening test on the active set `bits` (int32 device tensor in
    the scsc_mask layout; updated in place, as are the codes z).  Returns
    (per-image duality gaps, per-image active counts) as numpy arrays."""
    import numpy as np
    _need_step(ctx, batch, x=x, d=d, z=z, bits=bits)
    gaps = np.zeros(batch.n, dtype=np.float64)
    kept = np.zeros(batch.n, dtype=np.int64)
    _check(lib().scsc_screen(ctx.handle, ctypes.byref(batch.c), _ptr(x), _ptr(d), _ptr(z),
                             _ptr(bits), gaps.ctypes.data, kept.ctypes.data), ctx.handle,
           "scsc_screen")
    return gaps, kept


def scsc_code_step_screened(ctx: Context, batch: Batch, x, d, z, t: int, n_iters: int,
                            screen_every: int):
    """Code step with the screening test every `screen_every` iterations.
    Returns (per-image gaps, per-image active counts) of the last test."""
    import numpy as np
    _need_step(ctx, batch, x=x, d=d, z=z)
    gaps = np.zeros(batch.n, dtype=np.float64)
    kept = np.zeros(batch.n, dtype=np.int64)
    _check(lib().scsc_code_step_screened(ctx.handle, ctypes.byref(batch.c), _ptr(x), _ptr(d),
                                         _ptr(z), t, n_iters, screen_every,
                                         gaps.ctypes.data if n_iters > 0 else None,
                                         kept.ctypes.data if n_iters > 0 else None), ctx.handle,
           "scsc_code_step_screened")
    return gaps, kept


def scsc_objective_observed(ctx: Context, batch: Batch, x, z, d, observed) -> float:
    _need_step(ctx, batch, x=x, d=d, z=z, observed=observed)
    out = c_double()
    _check(lib().scsc_objective_observed(ctx.handle, ctypes.byref(batch.c), _ptr(x), _ptr(z),
                                         _ptr(d),
                                         _ptr(observed) if observed is not None else None,
                                         ctypes.byref(out)), ctx.handle, "scsc_objective_observed")
    return out.value


def scsc_lipschitz_codes(ctx: Context, batch: Batch, d) -> float:
    _need_step(ctx, batch, d=d)
    out = c_double()
    _check(lib().scsc_lipschitz_codes(ctx.handle, ctypes.byref(batch.c), _ptr(d),
                                      ctypes.byref(out)), ctx.handle, "scsc_lipschitz_codes")
    return out.value


def scsc_synth(ctx: Context, batch: Batch, z, d, t: int = 0, masked: bool = False, out=None):
    import torch
    if out is None:
        out = torch.empty(batch.total_pixels, dtype=torch.float32, device=z.device)
    _need_step(ctx, batch, x=out, d=d, z=z)
    _check(lib().scsc_synth(ctx.handle, ctypes.byref(batch.c), _ptr(z), _ptr(d), t, int(masked),
                            _ptr(out)), ctx.handle, "scsc_synth")
    return out


def scsc_synth_backward(ctx: Context, batch: Batch, grad, z, d, t: int = 0, masked: bool = False,
                        need_z: bool = True, need_d: bool = True):
    import torch
    gz = torch.empty(batch.total_pixels * ctx.K, dtype=torch.float32, device=grad.device) if need_z else None
    gd = torch.empty(ctx.K * ctx.s * ctx.s, dtype=torch.float32, device=grad.device) if need_d else None
    _need_step(ctx, batch, x=grad, d=d, z=z)
    _check(lib().scsc_synth_backward(ctx.handle, ctypes.byref(batch.c), _ptr(grad), _ptr(z),
                                     _ptr(d), t, int(masked), _ptr(gz), _ptr(gd)), ctx.handle,
           "scsc_synth_backward")
    return gz, gd


def scsc_objective_noalloc(K: int, s: int, lam: float, n_images: int, H: int, W: int, x, z, d,
                           out, stream=None) -> None:
    """Eq. 1 for equal-size images into the device double `out`, using only the
    library's built-in scratch (no device allocation).  Buffer sizes and
    element types are checked here, before the library is touched: the C
    entry point takes raw pointers and cannot see a short or wrongly typed
    tensor."""
    P = int(n_images) * int(H) * int(W)
    for name, t, n, fp in (("x", x, P, 4), ("z", z, P * int(K), 4),
                           ("d", d, int(K) * int(s) * int(s), 4), ("out", out, 1, 8)):
        if t is None:
            raise ValueError(f"{name}: a tensor is required")
        if not t.is_floating_point():
            raise ValueError(f"{name}: expected a float{8 * fp} tensor, got {t.dtype}")
        _need(t, n, fp, name)
    cfg = scsc_config(int(K), int(s), float(lam), 1, 1, 0, SCSC_FP32, 0.0, 0)
    _check(lib().scsc_objective_noalloc(ctypes.byref(cfg), n_images, H, W, _ptr(x), _ptr(z),
                                        _ptr(d), _ptr(out), c_void_p(_stream_handle(stream))),
           None, "scsc_objective_noalloc")


def scsc_sync(ctx: Context) -> None:
    _check(lib().scsc_sync(ctx.handle), ctx.handle, "scsc_sync")


def scsc_online_reset(ctx: Context) -> None:
    _check(lib().scsc_online_reset(ctx.handle), ctx.handle, "scsc_online_reset")


def scsc_online_state_size(ctx: Context) -> int:
    n = c_size_t()
    _check(lib().scsc_online_state_size(ctx.handle, ctypes.byref(n)), ctx.handle)
    return n.value


def scsc_online_save(ctx: Context) -> bytearray:
    n = scsc_online_state_size(ctx)
    buf = bytearray(n)
    cbuf = (ctypes.c_char * n).from_buffer(buf)
    _check(lib().scsc_online_save(ctx.handle, ctypes.addressof(cbuf), n), ctx.handle,
           "scsc_online_save")
    return buf


def scsc_online_load(ctx: Context, buf) -> None:
    buf = bytearray(buf)
    cbuf = (ctypes.c_char * len(buf)).from_buffer(buf)
    _check(lib().scsc_online_load(ctx.handle, ctypes.addressof(cbuf), len(buf)), ctx.handle,
           "scsc_online_load")


def scsc_diag_tc_gemm(A, B):
    """tcgen05 self-check: returns D = bf16(A) bf16(B)^T computed on the tensor core."""
    import torch
    N = B.shape[0]
    D = torch.empty((128, N), dtype=torch.float32, device=A.device)
    _check(lib().scsc_diag_tc_gemm(N, _ptr(A), _ptr(B), _ptr(D)), None, "scsc_diag_tc_gemm")
    return D


def scsc_diag_tc_gemm_mn(A, B, swap: int):
    """tcgen05 self-check with B held MN-major: D = bf16(A) bf16(B)^T when the
    descriptor fields carry the strides the way `swap` selects."""
    import torch
    N = B.shape[0]
    D = torch.empty((128, N), dtype=torch.float32, device=A.device)
    _check(lib().scsc_diag_tc_gemm_mn(N, _ptr(A), _ptr(B), _ptr(D), int(swap)), None,
           "scsc_diag_tc_gemm_mn")
    return D


def scsc_diag_wait_timeout(limit_ms: float = 20.0) -> int:
    """Run the kernels' bounded mbarrier wait on a barrier that nothing
    completes; returns the status (SCSC_ETIMEOUT when the wait ran out)."""
    return int(lib().scsc_diag_wait_timeout(float(limit_ms)))


def scsc_diag_ffma_peak():
    """(TFLOP/s, ms): the measured FP32 FMA rate of the current device."""
    tf, ms = c_double(), c_double()
    _check(lib().scsc_diag_ffma_peak(ctypes.byref(tf), ctypes.byref(ms)), None,
           "scsc_diag_ffma_peak")
    return tf.value, ms.value


def scsc_diag_mma_rate(N: int, layout: int = 0):
    """(issue, completion) SM cycles per tcgen05 MMA of 128 x N x 16."""
    iss, comp = c_double(), c_double()
    _check(lib().scsc_diag_mma_rate(int(N), int(layout), ctypes.byref(iss), ctypes.byref(comp)),
           None, "scsc_diag_mma_rate")
    return iss.value, comp.value


def scsc_diag_profile(ctx: Context, enable: bool = True) -> None:
    _check(lib().scsc_diag_profile(ctx.handle, int(enable)), ctx.handle, "scsc_diag_profile")


def scsc_diag_kernel_time(ctx: Context, name: str):
    """(total device ms, launches) of one library kernel since profiling began."""
    ms, n = c_double(), c_int()
    _check(lib().scsc_diag_kernel_time(ctx.handle, name.encode(), ctypes.byref(ms),
                                       ctypes.byref(n)), ctx.handle, "scsc_diag_kernel_time")
    return ms.value, n.value
