"""Thin ctypes binding of libttround (include/ttround.h): argument marshalling only.

Cores are torch CUDA float64 tensors of shape (r_{k-1}, n_k, r_k); PyTorch provides device
memory and the current stream.  Every step of the rounding runs inside the library's CUDA
kernels; there is no CPU path: if the library is missing this module raises on load.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libttround.so")

TTR_PREC_FP64 = 0
TTR_PREC_SLICED = 1
TTR_PREC_TF32_SKETCH = 2
TTR_PREC_BF16_SKETCH = 3
STATUS = {0: "TTR_OK", 1: "TTR_ERR_ARG", 2: "TTR_ERR_OOM", 3: "TTR_ERR_NONFINITE", 4: "TTR_ERR_QR_BREAKDOWN",
          5: "TTR_ERR_TIMEOUT", 6: "TTR_ERR_CUDA", 7: "TTR_ERR_UNSUPPORTED"}


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("slices", ctypes.c_int32), ("adap_r", ctypes.c_int32),
                ("adap_r_tau_scale", ctypes.c_double), ("nrmx", ctypes.c_double), ("f_init", ctypes.c_double),
                ("f_inc", ctypes.c_double), ("width_hint", ctypes.c_int64), ("kernel_timing", ctypes.c_int32),
                ("max_sms", ctypes.c_int32), ("est_min", ctypes.c_int32), ("est_safety", ctypes.c_double),
                ("rl_percore", ctypes.c_int32), ("block_loop_df", ctypes.c_int32),
                ("block_loop_tc", ctypes.c_int32), ("autotune", ctypes.c_int32)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("d", ctypes.c_int32), ("ranks", ctypes.POINTER(ctypes.c_int64)),
                ("cores", ctypes.POINTER(ctypes.c_void_p)), ("arena", ctypes.c_void_p), ("tau", ctypes.c_double),
                ("nrmx", ctypes.c_double), ("width", ctypes.c_int64), ("extensions", ctypes.c_int32),
                ("n_estimates", ctypes.c_int32), ("estimates", ctypes.POINTER(ctypes.c_double)),
                ("est_core", ctypes.POINTER(ctypes.c_int32)), ("ms_sketch_rl", ctypes.c_float),
                ("ms_sweep_lr", ctypes.c_float), ("ms_total", ctypes.c_float), ("kernel_launches", ctypes.c_int64),
                ("ms_block_loop", ctypes.c_double), ("flops_block_loop", ctypes.c_double),
                ("ms_rl_kernel", ctypes.c_double), ("bytes_rl_kernel", ctypes.c_double),
                ("n_block_loop", ctypes.c_int32), ("n_rl_kernel", ctypes.c_int32)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("workers", ctypes.c_int32), ("max_sms", ctypes.c_int32), ("device_budget", ctypes.c_uint64),
                ("device", ctypes.c_int32)]


class ServerResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("d", ctypes.c_int32), ("ranks", ctypes.POINTER(ctypes.c_int64)),
                ("data", ctypes.POINTER(ctypes.c_double)), ("cores", ctypes.POINTER(ctypes.POINTER(ctypes.c_double))),
                ("ms_queue", ctypes.c_double), ("ms_run", ctypes.c_double), ("footprint", ctypes.c_uint64),
                ("bytes_in", ctypes.c_uint64), ("admit_order", ctypes.c_int64), ("message", ctypes.c_char * 256)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("waiting", ctypes.c_int64), ("running", ctypes.c_int64), ("in_use", ctypes.c_uint64),
                ("peak_in_use", ctypes.c_uint64)]


class TTRoundError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def lib():
    """Load libttround.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libttround.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        i32, i64, u64, dbl, vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p
        P64 = ctypes.POINTER(ctypes.c_int64)
        PP = ctypes.POINTER(ctypes.c_void_p)
        L.ttr_default_options.argtypes = [ctypes.POINTER(Options)]
        L.tt_round_fixed.argtypes = [i32, P64, P64, PP, i64, i64, u64, ctypes.POINTER(Options), vp, ctypes.POINTER(Result)]
        L.tt_round_adaptive.argtypes = [i32, P64, P64, PP, dbl, i64, u64, ctypes.POINTER(Options), vp, ctypes.POINTER(Result)]
        L.tt_round_deterministic.argtypes = [i32, P64, P64, PP, dbl, vp, ctypes.POINTER(Result)]
        L.ttr_free.argtypes = [ctypes.POINTER(Result), vp]
        L.ttr_free.restype = None
        L.ttr_strerror.restype = ctypes.c_char_p
        L.ttr_last_error.restype = ctypes.c_char_p
        L.ttr_sketch_omega.argtypes = [u64, i32, i64, i64, i64, vp, vp]
        L.ttr_partial_contractions.argtypes = [i32, P64, P64, PP, u64, i64, i64, i32, i32, i32, PP, vp]
        L.ttr_partial_contractions_noalloc.argtypes = [i32, P64, P64, PP, u64, i64, i64, i32, PP, vp]
        L.ttr_selftest_rsqrt.argtypes = [vp, vp, i64, vp]
        L.ttr_selftest_jacobi_rotation.argtypes = [vp, ctypes.c_double, vp, i64, vp]
        L.ttr_partial_contractions_percore.argtypes = [i32, P64, P64, PP, u64, i64, i64, i32, PP, vp]
        L.tt_round_adaptive_matvec.argtypes = [i32, P64, P64, P64, PP, P64, PP, dbl, i64, u64,
                                               ctypes.POINTER(Options), vp, ctypes.POINTER(Result)]
        L.ttr_partial_contractions_matvec.argtypes = [i32, P64, P64, P64, PP, P64, PP, u64, i64, i64, i32, i32, i32,
                                                      PP, vp]
        L.tt_round_adaptive_sum.argtypes = [i32, i32, P64, ctypes.POINTER(P64), ctypes.POINTER(PP), dbl, i64, u64,
                                            ctypes.POINTER(Options), vp, ctypes.POINTER(Result)]
        L.ttr_server_create.argtypes = [ctypes.POINTER(ServerConfig), ctypes.POINTER(ctypes.c_void_p)]
        L.ttr_server_submit.argtypes = [vp, i32, i32, P64, ctypes.POINTER(P64), ctypes.POINTER(PP), dbl, i64, u64,
                                        ctypes.POINTER(Options), ctypes.POINTER(ctypes.c_int64)]
        L.ttr_server_wait.argtypes = [vp, i64, ctypes.POINTER(ServerResult)]
        L.ttr_server_result_free.argtypes = [ctypes.POINTER(ServerResult)]
        L.ttr_server_result_free.restype = None
        L.ttr_server_get_stats.argtypes = [vp, ctypes.POINTER(ServerStats)]
        L.ttr_server_destroy.argtypes = [vp]
        L.ttr_server_destroy.restype = None
        for f in ("ttr_server_create", "ttr_server_submit", "ttr_server_wait", "ttr_server_get_stats"):
            getattr(L, f).restype = ctypes.c_int
        for f in ("tt_round_fixed", "tt_round_adaptive", "tt_round_adaptive_sum", "tt_round_deterministic", "ttr_sketch_omega",
                  "ttr_partial_contractions", "ttr_partial_contractions_noalloc"):
            getattr(L, f).restype = ctypes.c_int
        _lib = L
    return _lib


def _check(st: int):
    if st != 0:
        raise TTRoundError(st, lib().ttr_last_error().decode(errors="replace"))


def _stream_handle(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _tt_args(cores):
    import torch
    d = len(cores)
    for c in cores:
        if not (isinstance(c, torch.Tensor) and c.is_cuda and c.dtype == torch.float64 and c.dim() == 3
                and c.is_contiguous()):
            raise ValueError("cores must be contiguous CUDA float64 tensors of shape (r0, n, r1)")
    n = (ctypes.c_int64 * d)(*[int(c.shape[1]) for c in cores])
    r = (ctypes.c_int64 * (d + 1))(*([int(cores[0].shape[0])] + [int(c.shape[2]) for c in cores]))
    ptrs = (ctypes.c_void_p * d)(*[c.data_ptr() for c in cores])
    return d, n, r, ptrs


def options(precision: int = TTR_PREC_FP64, slices: int = 0, adap_r: bool = False, adap_r_tau_scale: float = 1.0,
            nrmx: float = 0.0, f_init: float = 0.1, f_inc: float = 0.05, width_hint: int = 0,
            kernel_timing: bool = False, max_sms: int = 0, est_min: int = 0, est_safety: float = 1.0,
            rl_percore: int = 0, block_loop_df: bool = False, block_loop_tc: bool = False,
            autotune: bool = False) -> Options:
    o = Options()
    lib().ttr_default_options(ctypes.byref(o))
    o.precision, o.slices, o.adap_r = precision, slices, int(adap_r)
    o.adap_r_tau_scale, o.nrmx, o.f_init, o.f_inc, o.width_hint = adap_r_tau_scale, nrmx, f_init, f_inc, width_hint
    o.kernel_timing = int(kernel_timing)
    o.max_sms = int(max_sms)
    o.est_min, o.est_safety = int(est_min), float(est_safety)
    o.rl_percore = int(rl_percore)
    o.block_loop_df = int(block_loop_df)
    o.block_loop_tc = int(block_loop_tc)
    o.autotune = int(autotune)
    return o


class Rounded:
    """A rounded TT owned by the library (device arena); call ``free()`` or use as a context manager."""

    def __init__(self, res: Result, stream):
        self._res, self._stream = res, stream

    @property
    def d(self) -> int:
        return self._res.d

    @property
    def result(self) -> Result:
        """The underlying ttr_result (valid until free())."""
        return self._res

    @property
    def ranks(self) -> list:
        return [int(self._res.ranks[i]) for i in range(self._res.d + 1)]

    @property
    def info(self) -> dict:
        r = self._res
        ne = r.n_estimates
        return {"ranks": self.ranks, "tau": r.tau, "nrmx": r.nrmx, "width": int(r.width),
                "extensions": int(r.extensions),
                "estimates": [r.estimates[i] for i in range(ne)] if ne else [],
                "est_core": [int(r.est_core[i]) for i in range(ne)] if ne else [],
                "ms_sketch_rl": r.ms_sketch_rl, "ms_sweep_lr": r.ms_sweep_lr, "ms_total": r.ms_total,
                "kernel_launches": int(r.kernel_launches),
                "ms_block_loop": r.ms_block_loop, "flops_block_loop": r.flops_block_loop, "n_block_loop": r.n_block_loop,
                "ms_rl_kernel": r.ms_rl_kernel, "bytes_rl_kernel": r.bytes_rl_kernel, "n_rl_kernel": r.n_rl_kernel}

    def core_ptr(self, k: int) -> int:
        return int(self._res.cores[k])

    def to_torch(self):
        """Copies of the cores as torch CUDA tensors (ordered before later work on the current stream)."""
        import torch
        out = []
        rk = self.ranks
        s = torch.cuda.ExternalStream(self._stream.value) if self._stream.value else torch.cuda.current_stream()
        with torch.cuda.stream(s):
            for k in range(self.d):
                shape = (rk[k], self._res_n[k], rk[k + 1])
                t = torch.empty(shape, dtype=torch.float64, device="cuda")
                nbytes = t.numel() * 8
                _cuda_memcpy_d2d(t.data_ptr(), self.core_ptr(k), nbytes, self._stream)
                out.append(t)
        torch.cuda.current_stream().wait_stream(s)
        return out

    def to_numpy(self):
        return [t.cpu().numpy() for t in self.to_torch()]

    def free(self):
        if self._res.arena:
            lib().ttr_free(ctypes.byref(self._res), self._stream)

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.free()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _cuda_memcpy_d2d(dst: int, src: int, nbytes: int, stream):
    import torch
    # a byte view copy through torch on the same stream (no host round trip)
    s = torch.cuda.ExternalStream(stream.value) if stream.value else torch.cuda.current_stream()
    with torch.cuda.stream(s):
        src_t = _wrap_device_ptr(src, nbytes)
        dst_t = _wrap_device_ptr(dst, nbytes)
        dst_t.copy_(src_t)


def _wrap_device_ptr(ptr: int, nbytes: int):
    import torch

    class _Holder:
        def __init__(self, p, n):
            self.__cuda_array_interface__ = {"shape": (n,), "typestr": "|u1", "data": (p, False), "version": 3}

    return torch.as_tensor(_Holder(ptr, nbytes), device="cuda")


def _finish(res: Result, st: int, stream, n):
    _check(st)
    out = Rounded(res, stream)
    out._res_n = n
    return out


def round_fixed(cores, ell: int, seed: int, target: int = 0, opts: Options | None = None, stream=None) -> Rounded:
    """Algorithm 4 (fixed rank ell, optional truncation to ``target``); see tt_round_fixed."""
    d, n, r, p = _tt_args(cores)
    res = Result()
    s = _stream_handle(stream)
    st = lib().tt_round_fixed(d, n, r, p, int(ell), int(target), ctypes.c_uint64(seed),
                              ctypes.byref(opts) if opts else None, s, ctypes.byref(res))
    return _finish(res, st, s, list(n))


def round_adaptive(cores, tol: float, block: int, seed: int, opts: Options | None = None, stream=None) -> Rounded:
    """Algorithm 6 (adaptive rank to relative tolerance ``tol``); see tt_round_adaptive."""
    d, n, r, p = _tt_args(cores)
    res = Result()
    s = _stream_handle(stream)
    st = lib().tt_round_adaptive(d, n, r, p, float(tol), int(block), ctypes.c_uint64(seed),
                                 ctypes.byref(opts) if opts else None, s, ctypes.byref(res))
    return _finish(res, st, s, list(n))


def round_adaptive_sum(summands, tol: float, block: int, seed: int, opts: Options | None = None,
                       stream=None) -> Rounded:
    """Adaptive rounding of the sum of the TTs in ``summands`` (a list of core lists sharing d and
    the mode sizes) without forming the formal sum; see tt_round_adaptive_sum."""
    if len(summands) < 1:
        raise ValueError("at least one summand")
    args = [_tt_args(x) for x in summands]
    d, n = args[0][0], args[0][1]
    for a in args[1:]:
        if a[0] != d or list(a[1]) != list(n):
            raise ValueError("summands must share d and the mode sizes")
    P64 = ctypes.POINTER(ctypes.c_int64)
    PP = ctypes.POINTER(ctypes.c_void_p)
    rs = (P64 * len(args))(*[ctypes.cast(a[2], P64) for a in args])
    ps = (PP * len(args))(*[ctypes.cast(a[3], PP) for a in args])
    res = Result()
    s = _stream_handle(stream)
    st = lib().tt_round_adaptive_sum(len(args), d, n, rs, ps, float(tol), int(block), ctypes.c_uint64(seed),
                                     ctypes.byref(opts) if opts else None, s, ctypes.byref(res))
    return _finish(res, st, s, list(n))


def round_deterministic(cores, tol: float, stream=None) -> Rounded:
    """Algorithm 1 (deterministic TT-rounding, FP64); see tt_round_deterministic."""
    d, n, r, p = _tt_args(cores)
    res = Result()
    s = _stream_handle(stream)
    st = lib().tt_round_deterministic(d, n, r, p, float(tol), s, ctypes.byref(res))
    return _finish(res, st, s, list(n))


def sketch_omega(seed: int, k: int, n_k: int, col0: int, col1: int, stream=None):
    import torch
    out = torch.empty((n_k, col1 - col0), dtype=torch.float64, device="cuda")
    _check(lib().ttr_sketch_omega(ctypes.c_uint64(seed), k, n_k, col0, col1, ctypes.c_void_p(out.data_ptr()),
                                  _stream_handle(stream)))
    return out


def partial_contractions(cores, seed: int, col0: int, col1: int, t: int = 2, precision: int = TTR_PREC_FP64,
                         slices: int = 0, stream=None) -> dict:
    """Algorithm 3 on sketch columns [col0, col1): {k: W_k} for k = t..d (1-based)."""
    import torch
    d, n, r, p = _tt_args(cores)
    w = col1 - col0
    bufs = {k: torch.empty((r[k - 1], w), dtype=torch.float64, device="cuda") for k in range(t, d + 1)}
    ptrs = (ctypes.c_void_p * d)(*[bufs[k + 1].data_ptr() if (k + 1) in bufs else 0 for k in range(d)])
    _check(lib().ttr_partial_contractions(d, n, r, p, ctypes.c_uint64(seed), col0, col1, t, precision, slices, ptrs,
                                          _stream_handle(stream)))
    return bufs


def partial_contractions_percore(cores, seed: int, col0: int, col1: int, t: int = 2, stream=None) -> dict:
    """Algorithm 3's W_k in the per-core-parallel form (ttr_partial_contractions_percore), FP64."""
    import torch
    d, n, r, p = _tt_args(cores)
    w = col1 - col0
    bufs = {k: torch.empty((r[k - 1], w), dtype=torch.float64, device=cores[0].device) for k in range(t, d + 1)}
    ptrs = (ctypes.c_void_p * d)(*[bufs[k + 1].data_ptr() if (k + 1) in bufs else 0 for k in range(d)])
    _check(lib().ttr_partial_contractions_percore(d, n, r, p, ctypes.c_uint64(seed), col0, col1, t, ptrs,
                                                  _stream_handle(stream)))
    return bufs


def _op_args(op, x):
    import torch
    d = len(op)
    if len(x) != d:
        raise ValueError("operator and vector must have the same number of cores")
    for a in op:
        if not (isinstance(a, torch.Tensor) and a.is_cuda and a.dtype == torch.float64 and a.dim() == 4
                and a.is_contiguous()):
            raise ValueError("operator cores must be contiguous CUDA float64 tensors of shape (p0, n, m, p1)")
    dx, m, r, px = _tt_args(x)
    # the C side cannot check device buffer sizes: the operator cores must chain and match x's modes
    for k, a in enumerate(op):
        if int(a.shape[2]) != int(m[k]):
            raise ValueError(f"operator core {k} has input size {int(a.shape[2])}, x has mode size {int(m[k])}")
        if k > 0 and int(a.shape[0]) != int(op[k - 1].shape[3]):
            raise ValueError(f"operator ranks do not chain at core {k}")
    n = (ctypes.c_int64 * d)(*[int(a.shape[1]) for a in op])
    p = (ctypes.c_int64 * (d + 1))(*([int(op[0].shape[0])] + [int(a.shape[3]) for a in op]))
    pa = (ctypes.c_void_p * d)(*[a.data_ptr() for a in op])
    return d, n, m, p, pa, r, px


def round_adaptive_matvec(op, x, tol: float, block: int, seed: int, opts: Options | None = None,
                          stream=None) -> Rounded:
    """Algorithm 6 on y = A x without forming y (tt_round_adaptive_matvec); op: cores (p0, n, m, p1)."""
    d, n, m, p, pa, r, px = _op_args(op, x)
    res = Result()
    s = _stream_handle(stream)
    st = lib().tt_round_adaptive_matvec(d, n, m, p, pa, r, px, float(tol), int(block), ctypes.c_uint64(seed),
                                        ctypes.byref(opts) if opts else None, s, ctypes.byref(res))
    return _finish(res, st, s, list(n))


def partial_contractions_matvec(op, x, seed: int, col0: int, col1: int, t: int = 2, precision: int = TTR_PREC_FP64,
                                slices: int = 0, stream=None) -> dict:
    """Algorithm 3 on y = A x without forming y (ttr_partial_contractions_matvec): {k: W_k}."""
    import torch
    d, n, m, p, pa, r, px = _op_args(op, x)
    w = col1 - col0
    bufs = {k: torch.empty((p[k - 1] * r[k - 1], w), dtype=torch.float64, device=x[0].device) for k in range(t, d + 1)}
    ptrs = (ctypes.c_void_p * d)(*[bufs[k + 1].data_ptr() if (k + 1) in bufs else 0 for k in range(d)])
    _check(lib().ttr_partial_contractions_matvec(d, n, m, p, pa, r, px, ctypes.c_uint64(seed), col0, col1, t,
                                                 precision, slices, ptrs, _stream_handle(stream)))
    return bufs


def partial_contractions_noalloc(cores, seed: int, col0: int, col1: int, t: int = 2, out: dict | None = None,
                                 stream=None) -> dict:
    """FP64 Algorithm 3 through ttr_partial_contractions_noalloc: the library allocates no device
    memory (its scratch is a fixed static array); the outputs {k: W_k} are the caller's, given in
    `out` or created here on the cores' device.  Enqueued on `stream` without synchronizing.

    The C side cannot check buffer sizes, so a given `out` must hold, for k = t..d, a contiguous
    float64 tensor of shape (r_{k-1}, col1 - col0) on the cores' device (ValueError otherwise)."""
    import torch
    d, n, r, p = _tt_args(cores)
    w = col1 - col0
    device = cores[0].device
    if out is None:
        bufs = {k: torch.empty((r[k - 1], w), dtype=torch.float64, device=device) for k in range(t, d + 1)}
    else:
        bufs = out
        for k in range(t, d + 1):
            b = bufs.get(k)
            if not isinstance(b, torch.Tensor):
                raise ValueError(f"out[{k}] is missing or not a tensor")
            if b.dtype != torch.float64 or not b.is_contiguous() or b.device != device:
                raise ValueError(f"out[{k}] must be a contiguous float64 tensor on {device}")
            if tuple(b.shape) != (r[k - 1], w):
                raise ValueError(f"out[{k}] has shape {tuple(b.shape)}, expected {(r[k - 1], w)}")
    ptrs = (ctypes.c_void_p * d)(*[bufs[k + 1].data_ptr() if t <= k + 1 <= d else 0 for k in range(d)])
    _check(lib().ttr_partial_contractions_noalloc(d, n, r, p, ctypes.c_uint64(seed), col0, col1, t, ptrs,
                                                  _stream_handle(stream)))
    return bufs


def selftest_jacobi_rotation(abg, tiny=0.0, stream=None):
    """The one-sided Jacobi rotation (cs, sn) for each row (A2, B2, G) of the CUDA float64 tensor abg
    of shape (count, 3); returns a (count, 2) tensor (ttr_selftest_jacobi_rotation)."""
    import torch
    if not (isinstance(abg, torch.Tensor) and abg.is_cuda and abg.dtype == torch.float64 and abg.is_contiguous()
            and abg.dim() == 2 and abg.shape[1] == 3):
        raise ValueError("abg must be a contiguous CUDA float64 tensor of shape (count, 3)")
    out = torch.empty((abg.shape[0], 2), dtype=torch.float64, device=abg.device)
    _check(lib().ttr_selftest_jacobi_rotation(ctypes.c_void_p(abg.data_ptr()), float(tiny),
                                              ctypes.c_void_p(out.data_ptr()), abg.shape[0], _stream_handle(stream)))
    return out


def selftest_rsqrt(x, stream=None):
    """The block loop's reciprocal square root applied to the CUDA float64 tensor x (ttr_selftest_rsqrt)."""
    import torch
    if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float64 and x.is_contiguous()):
        raise ValueError("x must be a contiguous CUDA float64 tensor")
    out = torch.empty_like(x)
    _check(lib().ttr_selftest_rsqrt(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()), x.numel(),
                                    _stream_handle(stream)))
    return out


@dataclass
class HostRounding:
    cores: list
    ranks: list
    info: dict


def round_adaptive_host(cores_np, tol: float, block: int, seed: int, opts: Options | None = None) -> HostRounding:
    """End-to-end call with HOST inputs: upload, round, download (what a CPU-side user calls)."""
    import torch
    dev = [torch.from_numpy(np.ascontiguousarray(c)).pin_memory().to("cuda", non_blocking=True) for c in cores_np]
    with round_adaptive(dev, tol, block, seed, opts) as y:
        out = [t.cpu().numpy() for t in y.to_torch()]
        return HostRounding(out, y.ranks, y.info)


class Server:
    """The library's request server (ttr_server_*): requests are sums of TTs in host memory, admitted
    in arrival order within a device-memory budget and rounded by `workers` threads at once."""

    def __init__(self, workers: int = 3, device_budget: int = 64 << 30, max_sms: int = 0, device: int | None = None):
        if device is None:   # the caller's current CUDA device (one server per rank under torchrun)
            import torch
            device = torch.cuda.current_device() if torch.cuda.is_available() else 0
        cfg = ServerConfig(int(workers), int(max_sms), int(device_budget), int(device))
        h = ctypes.c_void_p()
        _check(lib().ttr_server_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h
        self._keep = {}

    def submit(self, summands, tol: float, block: int, seed: int, opts: Options | None = None) -> int:
        """Queue the rounding of sum(summands); each summand is a list of C-contiguous float64 numpy
        arrays of shape (r0, n, r1) (pinned memory copies fastest).  Returns the request id."""
        import numpy as np
        if len(summands) < 1:
            raise ValueError("at least one summand")
        d = len(summands[0])
        modes = [int(c.shape[1]) for c in summands[0]]
        keep = [summands]
        P64 = ctypes.POINTER(ctypes.c_int64)
        PP = ctypes.POINTER(ctypes.c_void_p)
        rs, ps = [], []
        for x in summands:
            if len(x) != d or [int(c.shape[1]) for c in x] != modes:
                raise ValueError("summands must share d and the mode sizes")
            for c in x:
                if not (isinstance(c, np.ndarray) and c.dtype == np.float64 and c.ndim == 3 and c.flags.c_contiguous):
                    raise ValueError("cores must be C-contiguous float64 arrays of shape (r0, n, r1)")
            r = (ctypes.c_int64 * (d + 1))(*([int(x[0].shape[0])] + [int(c.shape[2]) for c in x]))
            p = (ctypes.c_void_p * d)(*[c.ctypes.data for c in x])
            keep += [r, p]
            rs.append(ctypes.cast(r, P64))
            ps.append(ctypes.cast(p, PP))
        n = (ctypes.c_int64 * d)(*modes)
        ra = (P64 * len(rs))(*rs)
        pa = (PP * len(ps))(*ps)
        keep += [n, ra, pa]
        rid = ctypes.c_int64()
        _check(lib().ttr_server_submit(self._h, len(summands), d, n, ra, pa, float(tol), int(block),
                                       ctypes.c_uint64(seed), ctypes.byref(opts) if opts else None,
                                       ctypes.byref(rid)))
        self._keep[rid.value] = (keep, modes)
        return rid.value

    def wait(self, rid: int, fetch: bool = True):
        """(cores as numpy arrays, info) of request rid; raises TTRoundError if it failed.  The
        result is already in host memory when the request completes; fetch=False skips copying
        it into numpy arrays (cores is then None) and just releases it."""
        import numpy as np
        res = ServerResult()
        st = lib().ttr_server_wait(self._h, int(rid), ctypes.byref(res))
        _, modes = self._keep.pop(rid, (None, None))
        try:
            if st != 0:
                raise TTRoundError(st, f"request {rid}: " + res.message.decode(errors="replace"))
            rk = [int(res.ranks[k]) for k in range(res.d + 1)]
            cores = [] if fetch else None
            nbytes = 0
            for k in range(res.d):
                cnt = rk[k] * modes[k] * rk[k + 1]
                nbytes += 8 * cnt
                if fetch:
                    a = np.ctypeslib.as_array(res.cores[k], shape=(cnt,)).copy()
                    cores.append(a.reshape(rk[k], modes[k], rk[k + 1]))
            info = {"ranks": rk, "ms_queue": res.ms_queue, "ms_run": res.ms_run, "footprint": int(res.footprint),
                    "bytes_in": int(res.bytes_in), "admit_order": int(res.admit_order), "result_bytes": nbytes}
            return cores, info
        finally:
            lib().ttr_server_result_free(ctypes.byref(res))

    def stats(self) -> dict:
        st = ServerStats()
        _check(lib().ttr_server_get_stats(self._h, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

    def close(self):
        if self._h:
            lib().ttr_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
