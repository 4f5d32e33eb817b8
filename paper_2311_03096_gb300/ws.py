"""Thin ctypes binding over libws_prox.so (C ABI in include/ws_prox.h).

Argument marshalling only: every step of the prox runs in the library's
kernels.  PyTorch provides device memory and the current CUDA stream.  There
is no fallback: if the library is missing or no GPU is visible, calls raise.

    out, ids, n = prox(w, lam)                  # one vector, w a CUDA tensor
    plan = Plan(offsets, dtype=torch.float32)   # a batch of segments
    out, ids, nc = plan.forward(values, lambdas)
    y = WSProx.apply(w, lam)                    # differentiable (cluster-mean backward)
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libws_prox.so")

WS_OK, WS_ERR_INVALID, WS_ERR_NONFINITE, WS_ERR_CUDA, WS_ERR_NOMEM, WS_ERR_TIMEOUT, WS_ERR_INTERNAL = range(7)
WS_F32, WS_F64 = 0, 1
PREC = {"fp32comp": 0, "fp64": 1}

_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_lib = None
_lock = threading.Lock()


class WSError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        name = _load().ws_status_string(code).decode() if _lib is not None else str(code)
        super().__init__(f"{what}: {name} (status {code})" if what else f"{name} (status {code})")


def _load():
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libws_prox.so is not built ({LIB_PATH}); run __graft_entry__.build()")
            lib = ctypes.CDLL(LIB_PATH)
            lib.ws_status_string.restype = ctypes.c_char_p
            lib.ws_status_string.argtypes = [ctypes.c_int]
            lib.ws_ctx_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int]
            lib.ws_ctx_destroy.argtypes = [_vp]
            lib.ws_ctx_destroy.restype = None
            lib.ws_plan_create.argtypes = [_vp, ctypes.POINTER(_vp), _vp, _i64, ctypes.c_int]
            lib.ws_plan_destroy.argtypes = [_vp]
            lib.ws_plan_destroy.restype = None
            lib.ws_prox_batched.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_int, _vp]
            lib.ws_prox_batched_warm.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_int, _vp]
            lib.ws_plan_params.argtypes = [_vp, ctypes.POINTER(_i64), ctypes.POINTER(ctypes.c_int)]
            lib.ws_prox.argtypes = [_vp, _vp, _i64, ctypes.c_double, _vp, _vp, _vp, ctypes.c_int, ctypes.c_int, _vp]
            lib.ws_R.argtypes = [_vp, _vp, _i64, ctypes.c_int, _vp, _vp, _vp]
            lib.ws_prox_dlambda_batched.argtypes = [_vp, _vp, _vp, _vp, _vp]
            lib.ws_prox_dlambda.argtypes = [_vp, _vp, _vp, _i64, _vp, ctypes.c_int, _vp]
            lib.ws_plan_autotune.argtypes = [_vp, _vp, _vp, _i64, ctypes.c_int, _vp, _vp, _vp, _vp, ctypes.c_int,
                                             _vp, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp]
            lib.ws_prox_batched_l1.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_int, _vp]
            lib.ws_prox_l1.argtypes = [_vp, _vp, _i64, ctypes.c_double, _vp, _vp, _vp, _vp, ctypes.c_int,
                                       ctypes.c_int, _vp]
            lib.ws_prox_backward_batched.argtypes = [_vp, _vp, _vp, _vp, _vp]
            lib.ws_prox_backward.argtypes = [_vp, _vp, _vp, _i64, _vp, ctypes.c_int, _vp]
            lib.ws_get_status.argtypes = [_vp, _vp]
            lib.ws_get_inexact.argtypes = [_vp, ctypes.POINTER(ctypes.c_int), _vp]
            lib.ws_debug_set_spin_limit.argtypes = [_vp, _i64]
            lib.ws_debug_set_spin_limit.restype = None
            lib.ws_debug_set_small_max.argtypes = [_vp, _i64]
            lib.ws_debug_set_small_max.restype = None
            lib.ws_debug_sort.argtypes = [_vp, _vp, _vp, _vp]
            lib.ws_debug_profile.argtypes = [_vp, ctypes.c_int]
            lib.ws_debug_profile_read.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                                  ctypes.POINTER(_i64)]
            lib.ws_debug_kernel_name.argtypes = [ctypes.c_int]
            lib.ws_debug_kernel_name.restype = ctypes.c_char_p
            lib.ws_debug_launch_count.argtypes = [_vp]
            lib.ws_debug_launch_count.restype = _i64
            for f in ("ws_ctx_create", "ws_plan_create", "ws_prox_batched", "ws_prox", "ws_prox_backward_batched",
                      "ws_prox_backward", "ws_get_status", "ws_debug_sort", "ws_debug_profile",
                      "ws_debug_profile_read"):
                getattr(lib, f).restype = ctypes.c_int
            _lib = lib
    return _lib


def lib():
    return _load()


def _check(rc: int, what: str):
    if rc != WS_OK:
        raise WSError(rc, what)


def _dtype_code(dt: torch.dtype) -> int:
    if dt == torch.float32:
        return WS_F32
    if dt == torch.float64:
        return WS_F64
    raise TypeError(f"unsupported dtype {dt} (float32 or float64)")


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Context:
    """A ws_ctx on one CUDA device (owns the device status word and cached plans)."""

    _per_device = {}

    def __init__(self, device: int = 0):
        if not torch.cuda.is_available():
            raise RuntimeError("ws_prox needs a CUDA device")
        self.device = device
        h = _vp()
        _check(_load().ws_ctx_create(ctypes.byref(h), device), "ws_ctx_create")
        self.handle = h

    @classmethod
    def get(cls, device=None) -> "Context":
        dev = torch.cuda.current_device() if device is None else int(device)
        if dev not in cls._per_device:
            cls._per_device[dev] = Context(dev)
        return cls._per_device[dev]

    def status(self, stream=None) -> int:
        """Synchronise the stream and return (and clear) the device status."""
        return _load().ws_get_status(self.handle, _stream(stream))

    def inexact(self, stream=None) -> bool:
        """ws_get_inexact: did a call since the last query truncate input values in its fixed point?"""
        flag = ctypes.c_int(0)
        _check(_load().ws_get_inexact(self.handle, ctypes.byref(flag), _stream(stream)), "ws_get_inexact")
        return bool(flag.value)

    def check(self, stream=None, what="ws_prox"):
        _check(self.status(stream), what)

    def set_spin_limit(self, limit: int):
        _load().ws_debug_set_spin_limit(self.handle, int(limit))

    def set_small_max(self, n: int):
        _load().ws_debug_set_small_max(self.handle, int(n))

    def set_ic_cap(self, cap: int):
        """Round cap of the in-tile Imminent Collisions rounds (0: tree merges only; < 0: default)."""
        fn = _load().ws_debug_set_ic_cap
        fn.argtypes = [_vp, ctypes.c_int]
        fn.restype = None
        fn(self.handle, int(cap))

    def hull_stats(self, d: int, dtype=torch.float32, n: int = 34):
        """Tiles of the last prox call for (d, dtype): {"general": g, "capped": c, "rounds": [count of tiles
        converged after r rounds for r = 0 ..]} (ws_debug_hull_stats)."""
        fn = _load().ws_debug_hull_stats
        fn.argtypes = [_vp, _i64, ctypes.c_int, _vp, ctypes.c_int]
        fn.restype = ctypes.c_int
        counts = np.zeros(n, np.int64)
        _check(fn(self.handle, int(d), _dtype_code(dtype), counts.ctypes.data_as(_vp), n), "ws_debug_hull_stats")
        return {"general": int(counts[0]), "capped": int(counts[1]), "rounds": [int(x) for x in counts[1:]]}

    def profile(self, enable: bool):
        """Start (and clear) or stop per-kernel event timing."""
        _check(_load().ws_debug_profile(self.handle, 1 if enable else 0), "ws_debug_profile")

    def profile_read(self) -> dict:
        """{kernel kind: (total_ms, launches)} recorded since profile(True)."""
        res = {}
        k = 0
        while True:
            name = _load().ws_debug_kernel_name(k)
            if name is None:
                break
            ms, cnt = ctypes.c_double(0), _i64(0)
            _check(_load().ws_debug_profile_read(self.handle, k, ctypes.byref(ms), ctypes.byref(cnt)), "profile_read")
            if cnt.value:
                res[name.decode()] = (ms.value, cnt.value)
            k += 1
        return res

    def launch_count(self) -> int:
        return int(_load().ws_debug_launch_count(self.handle))

    def __del__(self):
        try:
            if getattr(self, "handle", None) and _lib is not None:
                _lib.ws_ctx_destroy(self.handle)
        except Exception:
            pass


def prox(w: torch.Tensor, lam: float, prec: str = "fp32comp", ids: bool = True, ctx: Context | None = None,
         out: torch.Tensor | None = None, n_clusters: torch.Tensor | None = None, stream=None,
         id_out: torch.Tensor | None = None):
    """prox_{lam R}(w) for one CUDA vector.  Returns (out, ids or None, n_clusters int64 tensor[1])."""
    if not w.is_cuda or w.dim() != 1 or not w.is_contiguous():
        raise ValueError("w must be a contiguous 1-D CUDA tensor")
    ctx = ctx or Context.get(w.device.index)
    out = torch.empty_like(w) if out is None else out
    idt = id_out if id_out is not None else \
        (torch.empty(w.shape[0], dtype=torch.int32, device=w.device) if ids else None)
    nc = torch.zeros(1, dtype=torch.int64, device=w.device) if n_clusters is None else n_clusters
    _check(_load().ws_prox(ctx.handle, _ptr(w), w.shape[0], float(lam), _ptr(out), _ptr(idt), _ptr(nc),
                           _dtype_code(w.dtype), PREC[prec], _stream(stream)), "ws_prox")
    return out, idt, nc


def prox_dlambda(grad_out: torch.Tensor, ids: torch.Tensor, ctx: Context | None = None, stream=None):
    """sum_i grad_out[i] * d prox_i / d lambda (partition held fixed) for one vector, through
    ws_prox_dlambda.  Returns a float64 CUDA tensor of one element."""
    ctx = ctx or Context.get(grad_out.device.index)
    res = torch.empty(1, dtype=torch.float64, device=grad_out.device)
    _check(_load().ws_prox_dlambda(ctx.handle, _ptr(grad_out), _ptr(ids), grad_out.shape[0], _ptr(res),
                                   _dtype_code(grad_out.dtype), _stream(stream)), "ws_prox_dlambda")
    return res


def R(w: torch.Tensor, ctx: Context | None = None, stream=None):
    """R(w) (Eq. (1)) and the weight-sharing measure (#distinct nonzero / #nonzero) of one
    CUDA vector, through ws_R.  Returns two float64 CUDA tensors of one element."""
    if not w.is_cuda or w.dim() != 1 or not w.is_contiguous():
        raise ValueError("w must be a contiguous 1-D CUDA tensor")
    ctx = ctx or Context.get(w.device.index)
    r = torch.empty(1, dtype=torch.float64, device=w.device)
    m = torch.empty(1, dtype=torch.float64, device=w.device)
    _check(_load().ws_R(ctx.handle, _ptr(w), w.shape[0], _dtype_code(w.dtype), _ptr(r), _ptr(m), _stream(stream)),
           "ws_R")
    return r, m


class L1Rewind(ctypes.Structure):
    """ws_l1_rewind: l1 coefficient beta, rewinding rho, displacement scale v_scale."""
    _fields_ = [("beta", ctypes.c_double), ("rho", ctypes.c_double), ("v_scale", ctypes.c_double)]


def prox_l1(w: torch.Tensor, lam: float, beta: float, rho: float = 0.0, v_scale: float = 1.0,
            prec: str = "fp32comp", ids: bool = True, ctx: Context | None = None, out: torch.Tensor | None = None,
            n_clusters: torch.Tensor | None = None, stream=None):
    """Weight sharing + l1 with rewinding (Alg. 2) for one CUDA vector, through ws_prox_l1."""
    if not w.is_cuda or w.dim() != 1 or not w.is_contiguous():
        raise ValueError("w must be a contiguous 1-D CUDA tensor")
    ctx = ctx or Context.get(w.device.index)
    out = torch.empty_like(w) if out is None else out
    idt = torch.empty(w.shape[0], dtype=torch.int32, device=w.device) if ids else None
    nc = torch.zeros(1, dtype=torch.int64, device=w.device) if n_clusters is None else n_clusters
    epi = L1Rewind(float(beta), float(rho), float(v_scale))
    _check(_load().ws_prox_l1(ctx.handle, _ptr(w), w.shape[0], float(lam), ctypes.byref(epi), _ptr(out), _ptr(idt),
                              _ptr(nc), _dtype_code(w.dtype), PREC[prec], _stream(stream)), "ws_prox_l1")
    return out, idt, nc


def prox_backward(grad_out: torch.Tensor, ids: torch.Tensor, ctx: Context | None = None, grad_in=None, stream=None):
    ctx = ctx or Context.get(grad_out.device.index)
    gin = torch.empty_like(grad_out) if grad_in is None else grad_in
    _check(_load().ws_prox_backward(ctx.handle, _ptr(grad_out), _ptr(ids), grad_out.shape[0], _ptr(gin),
                                    _dtype_code(grad_out.dtype), _stream(stream)), "ws_prox_backward")
    return gin


NOALLOC_MAX_ELEMS = 1 << 20


def prox_backward_noalloc(grad_out: torch.Tensor, ids: torch.Tensor, grad_in: torch.Tensor, stream=None):
    """Backward for one vector (d <= 2^20) through ws_prox_backward_noalloc: no
    device allocation inside the call; scratch is the library's fixed device
    array.  For callers that must not allocate where the backward runs.

    grad_out and grad_in: contiguous 1-D CUDA tensors of one float dtype and length d
    (grad_in may be grad_out itself); ids: contiguous int32 CUDA tensor of length d;
    all three on one device, which is made current for the call."""
    for name, t in (("grad_out", grad_out), ("ids", ids), ("grad_in", grad_in)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dim() != 1 or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous 1-D CUDA tensor")
    d = grad_out.shape[0]
    if ids.dtype != torch.int32:
        raise ValueError("ids must be int32")
    if grad_in.dtype != grad_out.dtype:
        raise ValueError("grad_in must have grad_out's dtype")
    if ids.shape[0] != d or grad_in.shape[0] != d:
        raise ValueError("grad_out, ids and grad_in must have the same length")
    if ids.device != grad_out.device or grad_in.device != grad_out.device:
        raise ValueError("grad_out, ids and grad_in must be on one device")
    lib_ = _load()
    fn = lib_.ws_prox_backward_noalloc
    fn.argtypes = [_vp, _vp, _i64, _vp, ctypes.c_int, _vp]
    fn.restype = ctypes.c_int
    with torch.cuda.device(grad_out.device):
        _check(fn(_ptr(grad_out), _ptr(ids), d, _ptr(grad_in), _dtype_code(grad_out.dtype), _stream(stream)),
               "ws_prox_backward_noalloc")
    return grad_in


class Plan:
    """A ws_plan for a fixed batch layout (host offsets, int64, n_seg + 1 entries)."""

    def __init__(self, offsets, dtype=torch.float32, ctx: Context | None = None):
        self.ctx = ctx or Context.get()
        off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        self.offsets = off
        self.n_seg = off.shape[0] - 1
        self.n = int(off[-1]) if off.shape[0] else 0
        self.dtype = dtype
        h = _vp()
        _check(_load().ws_plan_create(self.ctx.handle, ctypes.byref(h), off.ctypes.data_as(_vp), self.n_seg,
                                      _dtype_code(dtype)), "ws_plan_create")
        self.handle = h

    @classmethod
    def autotuned(cls, offsets, values: torch.Tensor, lambdas: torch.Tensor, prec: str = "fp32comp",
                  thresholds=None, reps: int = 3, ctx: Context | None = None, stream=None):
        """Plan whose one-CTA / tiled length threshold is picked by timing (ws_plan_autotune).
        Returns the plan; .threshold and .times_ms hold the choice and every candidate's time."""
        self = cls.__new__(cls)
        self.ctx = ctx or Context.get(values.device.index)
        off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        self.offsets, self.n_seg, self.n, self.dtype = off, off.shape[0] - 1, int(off[-1]), values.dtype
        th = None if thresholds is None else np.ascontiguousarray(np.asarray(thresholds, dtype=np.int64))
        n_cand = 5 if th is None else th.shape[0]
        times = np.zeros(n_cand, np.float64)
        chosen = ctypes.c_int64(-1)
        out = torch.empty_like(values)
        ids = torch.empty(self.n, dtype=torch.int32, device=values.device)
        h = _vp()
        _check(_load().ws_plan_autotune(self.ctx.handle, ctypes.byref(h), off.ctypes.data_as(_vp), self.n_seg,
                                        _dtype_code(values.dtype), _ptr(values), _ptr(lambdas), _ptr(out), _ptr(ids),
                                        PREC[prec], None if th is None else th.ctypes.data_as(_vp), n_cand, reps,
                                        ctypes.byref(chosen), times.ctypes.data_as(_vp), _stream(stream)),
               "ws_plan_autotune")
        self.handle = h
        self.threshold = int(chosen.value)
        self.times_ms = times.tolist()
        sm, cap = ctypes.c_int64(-1), ctypes.c_int(-1)
        _check(_load().ws_plan_params(h, ctypes.byref(sm), ctypes.byref(cap)), "ws_plan_params")
        self.ic_cap = int(cap.value)
        return self

    def forward(self, values: torch.Tensor, lambdas: torch.Tensor, prec: str = "fp32comp", ids: bool = True,
                out=None, id_out=None, n_clusters=None, stream=None, ids_prev=None):
        """ws_prox_batched; with ids_prev (int32, one per element, e.g. the previous
        step's cluster ids, may be id_out itself) ws_prox_batched_warm: same outputs."""
        if values.dtype != self.dtype or values.shape[0] != self.n or not values.is_cuda:
            raise ValueError("values must be a CUDA tensor of the plan's dtype and length")
        if lambdas.dtype != torch.float64 or lambdas.shape[0] != self.n_seg or not lambdas.is_cuda:
            raise ValueError("lambdas must be a float64 CUDA tensor with one entry per segment")
        out = torch.empty_like(values) if out is None else out
        idt = (torch.empty(self.n, dtype=torch.int32, device=values.device) if ids else None) if id_out is None \
            else id_out
        nc = torch.zeros(max(self.n_seg, 1), dtype=torch.int64, device=values.device) if n_clusters is None \
            else n_clusters
        if ids_prev is None:
            _check(_load().ws_prox_batched(self.handle, _ptr(values), _ptr(lambdas), _ptr(out), _ptr(idt), _ptr(nc),
                                           PREC[prec], _stream(stream)), "ws_prox_batched")
        else:
            if (ids_prev.dtype != torch.int32 or ids_prev.dim() != 1 or ids_prev.shape[0] != self.n
                    or not ids_prev.is_cuda or not ids_prev.is_contiguous()):
                raise ValueError("ids_prev must be a contiguous 1-D int32 CUDA tensor of the plan's length")
            _check(_load().ws_prox_batched_warm(self.handle, _ptr(values), _ptr(lambdas), _ptr(ids_prev), _ptr(out),
                                                _ptr(idt), _ptr(nc), PREC[prec], _stream(stream)),
                   "ws_prox_batched_warm")
        return out, idt, nc

    def forward_l1(self, values: torch.Tensor, lambdas: torch.Tensor, beta: float, rho: float = 0.0,
                   v_scale: float = 1.0, prec: str = "fp32comp", out=None, id_out=None, n_clusters=None, stream=None):
        """Weight sharing + l1 with rewinding (Alg. 2) per segment, through ws_prox_batched_l1."""
        if values.dtype != self.dtype or values.shape[0] != self.n or not values.is_cuda:
            raise ValueError("values must be a CUDA tensor of the plan's dtype and length")
        if lambdas.dtype != torch.float64 or lambdas.shape[0] != self.n_seg or not lambdas.is_cuda:
            raise ValueError("lambdas must be a float64 CUDA tensor with one entry per segment")
        out = torch.empty_like(values) if out is None else out
        idt = torch.empty(self.n, dtype=torch.int32, device=values.device) if id_out is None else id_out
        nc = torch.zeros(max(self.n_seg, 1), dtype=torch.int64, device=values.device) if n_clusters is None \
            else n_clusters
        epi = L1Rewind(float(beta), float(rho), float(v_scale))
        _check(_load().ws_prox_batched_l1(self.handle, _ptr(values), _ptr(lambdas), ctypes.byref(epi), _ptr(out),
                                          _ptr(idt), _ptr(nc), PREC[prec], _stream(stream)), "ws_prox_batched_l1")
        return out, idt, nc

    def backward(self, grad_out: torch.Tensor, ids: torch.Tensor, grad_in=None, stream=None):
        gin = torch.empty_like(grad_out) if grad_in is None else grad_in
        _check(_load().ws_prox_backward_batched(self.handle, _ptr(grad_out), _ptr(ids), _ptr(gin), _stream(stream)),
               "ws_prox_backward_batched")
        return gin

    def dlambda(self, grad_out: torch.Tensor, ids: torch.Tensor, stream=None):
        """Per segment: sum_i grad_out[i] * d out_i / d lambda_s (ws_prox_dlambda_batched)."""
        res = torch.empty(max(self.n_seg, 1), dtype=torch.float64, device=grad_out.device)
        _check(_load().ws_prox_dlambda_batched(self.handle, _ptr(grad_out), _ptr(ids), _ptr(res), _stream(stream)),
               "ws_prox_dlambda_batched")
        return res[: self.n_seg]

    def debug_sort(self, values: torch.Tensor, sorted_out: torch.Tensor, stream=None):
        _check(_load().ws_debug_sort(self.handle, _ptr(values), _ptr(sorted_out), _stream(stream)), "ws_debug_sort")
        return sorted_out

    def __del__(self):
        try:
            if getattr(self, "handle", None) and _lib is not None:
                _lib.ws_plan_destroy(self.handle)
        except Exception:
            pass


class WSProx(torch.autograd.Function):
    """y = prox_{lam R}(w) with the cluster-averaging backward (partition held fixed).

    ``w`` may be 1-D (one vector) or 2-D (one segment per row, e.g. the rows of
    a weight matrix, all with the same ``lam``)."""

    @staticmethod
    def forward(ctx, w: torch.Tensor, lam: float, prec: str = "fp32comp"):
        wc = w.contiguous()
        if wc.dim() == 1:
            out, ids, _ = prox(wc, lam, prec)
            ctx.plan = None
        else:
            rows, cols = wc.shape
            plan = _row_plan(rows, cols, wc.dtype)
            lams = torch.full((rows,), float(lam), dtype=torch.float64, device=wc.device)
            out, ids, _ = plan.forward(wc.reshape(-1), lams, prec)
            out = out.reshape(rows, cols)
            ctx.plan = plan
        ctx.save_for_backward(ids)
        return out

    @staticmethod
    def backward(ctx, g):
        (ids,) = ctx.saved_tensors
        gc = g.contiguous()
        if ctx.plan is None:
            gin = prox_backward(gc, ids)
        else:
            gin = ctx.plan.backward(gc.reshape(-1), ids).reshape(gc.shape)
        return gin, None, None


_row_plans = {}


def _row_plan(rows: int, cols: int, dtype) -> Plan:
    key = (rows, cols, dtype, torch.cuda.current_device())
    if key not in _row_plans:
        _row_plans[key] = Plan(np.arange(rows + 1, dtype=np.int64) * cols, dtype)
    return _row_plans[key]
