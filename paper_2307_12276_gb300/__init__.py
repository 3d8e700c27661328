"""Python binding of libanidiff (include/anidiff.h): argument marshalling only.

Every computation runs in the CUDA kernels of the shared library; this module
converts tensors and arrays to pointers, checks shapes and types, and turns
status codes into exceptions.  Function names are those of the C ABI without
the ``ad_`` prefix.  There is no fallback: if the library is missing or does
not load, importing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import Callable, Optional, Sequence

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libanidiff.so")

AD_OK, AD_ERR_INVALID, AD_ERR_CUDA, AD_ERR_NOT_CONVERGED, AD_ERR_TIMEOUT, AD_ERR_NOMEM = range(6)
BC_PERIODIC, BC_DIRICHLET0 = 0, 1
FP64, FP32_STORAGE = 0, 1
BOUND_GERSHGORIN, BOUND_POWER, BOUND_LEARNED = 0, 1, 2
MAX_SOURCES = 16

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: run __graft_entry__.build() (nvcc, sm_103a) first")
_lib = C.CDLL(LIB_PATH)


class _Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("x0", C.c_double), ("x1", C.c_double),
                ("y0", C.c_double), ("y1", C.c_double), ("bc", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("iters", C.c_int), ("matvecs", C.c_int), ("substeps", C.c_int),
                ("converged", C.c_int), ("err_est", C.c_double), ("alpha", C.c_double),
                ("kernel_launches", C.c_int), ("rejected", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_PROFILE = C.CFUNCTYPE(C.c_double, C.c_int, C.c_double, C.c_void_p)


class _Source(C.Structure):
    _fields_ = [("nterms", C.c_int), ("g", C.POINTER(C.c_void_p)), ("h", _PROFILE),
                ("ctx", C.c_void_p)]


class _Momentum(C.Structure):
    _fields_ = [("np", C.c_int), ("P", C.POINTER(C.c_double)), ("beta", C.POINTER(C.c_double)),
                ("dpp", C.POINTER(C.c_double)), ("b", C.POINTER(C.c_double)),
                ("loss", C.POINTER(C.c_double))]


_vp, _dp, _i, _d = C.c_void_p, C.c_double, C.c_int, C.c_double
_sig = {
    "ad_create_operator": (_i, [C.POINTER(_Grid), _vp, _vp, _vp, _vp, _vp, _d, _d, _i, _vp,
                                C.POINTER(_vp)]),
    "ad_destroy_operator": (_i, [_vp]),
    "ad_set_options": (_i, [_vp, _d, _i]),
    "ad_set_substep_control": (_i, [_vp, _i]),
    "ad_spectral_bound": (_i, [_vp, _i, _vp, C.c_ulonglong, _i, _d, C.POINTER(_d)]),
    "ad_set_spectral_bound": (_i, [_vp, _d]),
    "ad_get_spectral_bound": (_i, [_vp, C.POINTER(_d)]),
    "ad_apply": (_i, [_vp, _vp, _vp]),
    "ad_leja_phi1": (_i, [_vp, _vp, _vp, _d, _d, _i, C.POINTER(Stats)]),
    "ad_expquad_step": (_i, [_vp, _vp, _d, _d, _i, C.POINTER(_d), C.POINTER(_Source), _d, _i,
                             C.POINTER(Stats)]),
    "ad_expquad_step_async": (_i, [_vp, _vp, _d, _d, _i, C.POINTER(_d), C.POINTER(_Source),
                                   _d]),
    "ad_async_totals": (_i, [_vp, C.POINTER(Stats)]),
    "ad_cn_step": (_i, [_vp, _vp, _d, _d, C.POINTER(_Source), _d, _i, _i, C.POINTER(Stats)]),
    "ad_reserve_gmres": (_i, [_vp, _i]),
    "ad_penalised_step": (_i, [_vp, _vp, _d, _d, C.POINTER(_Source), _d, _d, _i,
                               C.POINTER(Stats)]),
    "ad_penalty_beta": (_i, [C.POINTER(_Grid), _vp, _vp, _vp, _vp, C.POINTER(_d)]),
    "ad_profile_leja_iteration": (_i, [_vp, _i, _i, C.POINTER(_d)]),
    "ad_leja_phi1_noalloc": (_i, [C.POINTER(_Grid), _vp, _vp, _vp, _d, _d, _d, _vp, _vp, _d, _d,
                                  _i, _vp, C.POINTER(Stats)]),
    "ad_create_batch": (_i, [C.POINTER(_vp), _i, _i, C.POINTER(_vp)]),
    "ad_destroy_batch": (_i, [_vp]),
    "ad_batch_midpoint_step": (_i, [_vp, C.POINTER(_vp), _d, _d, _vp, _d, _i, C.POINTER(Stats)]),
    "ad_batch_iteration_hint": (_i, [_vp, _vp]),
    "ad_batch_bind": (_i, [_vp, _vp, _vp]),
    "ad_batch_step": (_i, [_vp, _d, _d, _d, _i, _vp]),
    "ad_batch_order": (_i, [_vp, _vp]),
    "ad_batch_info": (_i, [_vp, C.POINTER(_i), C.POINTER(_i), C.POINTER(_i), C.POINTER(_d),
                          C.POINTER(_i)]),
    "ad_mlp_create": (_i, [_i, _i, _i, C.c_ulonglong, _vp, C.POINTER(_vp)]),
    "ad_mlp_destroy": (_i, [_vp]),
    "ad_mlp_num_params": (_i, [_vp, C.POINTER(_i)]),
    "ad_mlp_params": (_i, [_vp, _vp, _i, _i]),
    "ad_mlp_normalization": (_i, [_vp, _vp, _vp, _vp, _vp, _i]),
    "ad_mlp_loss_grad": (_i, [_vp, _vp, _vp, _i, C.POINTER(C.c_float), _vp]),
    "ad_mlp_train": (_i, [_vp, _vp, _vp, _i, _i, C.c_float, _i, C.POINTER(C.c_float)]),
    "ad_mlp_predict": (_i, [_vp, _vp, _i, _i, _vp]),
    "ad_field_features": (_i, [C.POINTER(_Grid), _vp, _vp, _vp, _d, _d, _vp, _vp]),
    "ad_learned_bounds": (_i, [_vp, C.POINTER(_vp), _i, C.POINTER(_d), _d, _i, C.POINTER(_d),
                               C.POINTER(_d)]),
    "ad_set_bound_model": (_i, [_vp, _vp, _d, _d]),
    "ad_fp64_fma_rate": (_i, [_i, _i, _vp, C.POINTER(_d)]),
    "ad_bound_training_sample": (_i, [_vp, _d, C.c_ulonglong, _i, _d, _d, C.POINTER(C.c_float),
                                      C.POINTER(C.c_float), C.POINTER(_d)]),
    "ad_create_momentum_operator": (_i, [C.POINTER(_Grid), C.POINTER(_Momentum), _vp, _vp, _vp,
                                         _d, _d, _vp, C.POINTER(_vp)]),
    "ad_destroy_momentum_operator": (_i, [_vp]),
    "ad_momentum_spectral_bound": (_i, [_vp, C.POINTER(_d)]),
    "ad_momentum_set_spectral_bound": (_i, [_vp, _d]),
    "ad_momentum_set_options": (_i, [_vp, _d, _i]),
    "ad_momentum_apply": (_i, [_vp, _vp, _vp]),
    "ad_momentum_leja_phi1": (_i, [_vp, _vp, _vp, _d, _d, _i, C.POINTER(Stats)]),
    "ad_momentum_step": (_i, [_vp, _vp, _d, _vp, _d, _i, C.POINTER(Stats)]),
    "ad_time_series": (_i, [_vp, _i]),
    "ad_series_timing": (_i, [_vp, C.POINTER(_d), C.POINTER(_i), C.POINTER(C.c_longlong),
                              C.POINTER(_i)]),
    "ad_check_wait_timeout": (_i, [_d, _vp]),
    "ad_last_error": (C.c_char_p, []),
    "ad_version": (_i, []),
}
for _name, (_res, _args) in _sig.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_sig)


class AdError(RuntimeError):
    def __init__(self, status: int, msg: str, stats: Optional[dict] = None):
        super().__init__(f"anidiff status {status}: {msg}")
        self.status = status
        self.stats = stats


class NotConverged(AdError):
    pass


def last_error() -> str:
    return _lib.ad_last_error().decode()


def version() -> int:
    return _lib.ad_version()


def _check(status: int, stats: Optional[Stats] = None):
    if status == AD_OK:
        return
    d = stats.as_dict() if stats is not None else None
    cls = NotConverged if status == AD_ERR_NOT_CONVERGED else AdError
    raise cls(status, last_error(), d)


_TORCH = None


def _torch_types():
    """(torch.Tensor, {dtype name: torch dtype}) once torch is importable, else None."""
    global _TORCH
    if _TORCH is None:
        try:
            import torch
            _TORCH = (torch.Tensor, {"float64": torch.float64, "float32": torch.float32})
        except ImportError:
            _TORCH = False
    return _TORCH


def _ptr(x, dtype_name: str, n: int, what: str):
    """Pointer of a contiguous tensor/array with n elements of the given dtype."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    tt = _torch_types()
    if tt and isinstance(x, tt[0]):
        if x.dtype != tt[1][dtype_name]:
            raise TypeError(f"{what}: expected {dtype_name}, got {x.dtype}")
        if not x.is_contiguous():
            raise ValueError(f"{what}: tensor must be contiguous")
        if x.numel() != n:
            raise ValueError(f"{what}: expected {n} elements, got {x.numel()}")
        return x.data_ptr()
    import numpy as np
    if isinstance(x, np.ndarray):
        if x.dtype != np.dtype(dtype_name):
            raise TypeError(f"{what}: expected {dtype_name}, got {x.dtype}")
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError(f"{what}: array must be C-contiguous")
        if x.size != n:
            raise ValueError(f"{what}: expected {n} elements, got {x.size}")
        return x.ctypes.data
    raise TypeError(f"{what}: unsupported type {type(x)}")


@dataclass
class Source:
    """S(x, y, t) = sum_k h_k(t) g_k(x, y); g: device tensors of the storage type,
    h: callables of t (None: time-independent, every h_k = 1)."""
    g: Sequence
    h: Optional[Sequence[Callable[[float], float]]] = None


class Operator:
    """Handle of an ad_operator (see include/anidiff.h for the semantics)."""

    def __init__(self, handle: int, nx: int, ny: int, precision: int, keep=()):
        self.handle = handle
        self.nx, self.ny, self.precision = nx, ny, precision
        self.n = nx * ny
        self.dtype_name = "float64" if precision == FP64 else "float32"
        self._keep = keep

    def close(self):
        if self.handle:
            _lib.ad_destroy_operator(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def vec(self, x, what):
        return _ptr(x, self.dtype_name, self.n, what)


def create_operator(nx: int, ny: int, bc: int, Dxx, Dxy, Dyy, ax=0.0, ay=0.0,
                    precision: int = FP64, stream=None, x0=-1.0, x1=1.0, y0=-1.0,
                    y1=1.0) -> Operator:
    """ad_create_operator.  Dxx/Dxy/Dyy: float64 device tensors [ny][nx];
    ax/ay: float constants or float64 device tensors."""
    g = _Grid(nx, ny, x0, x1, y0, y1, bc)
    n = nx * ny
    pf = [_ptr(f, "float64", n, name) for f, name in ((Dxx, "Dxx"), (Dxy, "Dxy"), (Dyy, "Dyy"))]
    axp = None if isinstance(ax, (int, float)) else _ptr(ax, "float64", n, "ax")
    ayp = None if isinstance(ay, (int, float)) else _ptr(ay, "float64", n, "ay")
    axc = float(ax) if isinstance(ax, (int, float)) else 0.0
    ayc = float(ay) if isinstance(ay, (int, float)) else 0.0
    sptr = _stream_ptr(stream)
    h = _vp()
    _check(_lib.ad_create_operator(C.byref(g), pf[0], pf[1], pf[2], axp, ayp, axc, ayc,
                                   precision, sptr, C.byref(h)))
    return Operator(h.value, nx, ny, precision)


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    return stream if isinstance(stream, int) else stream.cuda_stream


def destroy_operator(op: Operator):
    op.close()


def set_options(op: Operator, rho_max: float = 0.0, max_iters: int = 0):
    _check(_lib.ad_set_options(op.handle, rho_max, max_iters))


def set_substep_control(op: Operator, adaptive: bool = True):
    """ad_set_substep_control: adaptive substeps (True) or the fixed rho_max rule."""
    _check(_lib.ad_set_substep_control(op.handle, 1 if adaptive else 0))


def spectral_bound(op: Operator, method: int = BOUND_GERSHGORIN, x0=None, seed: int = 0,
                   power_iters: int = 30, safety: float = 1.1) -> float:
    a = _d()
    _check(_lib.ad_spectral_bound(op.handle, method, op.vec(x0, "x0"), seed, power_iters,
                                  safety, C.byref(a)))
    return a.value


def set_spectral_bound(op: Operator, alpha: float):
    _check(_lib.ad_set_spectral_bound(op.handle, alpha))


def get_spectral_bound(op: Operator) -> float:
    a = _d()
    _check(_lib.ad_get_spectral_bound(op.handle, C.byref(a)))
    return a.value


def apply(op: Operator, u, out):
    _check(_lib.ad_apply(op.handle, op.vec(u, "u"), op.vec(out, "out")))


def leja_phi1(op: Operator, v, out, dt: float, tol: float = 1e-10, force_iters: int = -1) -> dict:
    st = Stats()
    _check(_lib.ad_leja_phi1(op.handle, op.vec(v, "v"), op.vec(out, "out"), dt, tol,
                             force_iters, C.byref(st)), st)
    return st.as_dict()


def _source_struct(op: Operator, src: Optional[Source]):
    if src is None or len(src.g) == 0:
        return None, ()
    if len(src.g) > MAX_SOURCES:
        raise ValueError("at most 16 source terms")
    arr = (C.c_void_p * len(src.g))(*[op.vec(gk, f"g[{k}]") for k, gk in enumerate(src.g)])
    cb = _PROFILE(0)
    if src.h is not None:
        hs = list(src.h)

        def _h(k, t, ctx):
            return float(hs[k](t))
        cb = _PROFILE(_h)
    s = _Source(len(src.g), C.cast(arr, C.POINTER(C.c_void_p)), cb, None)
    return s, (arr, cb)


def expquad_step(op: Operator, u, t: float, dt: float, s: int = 1, c: Sequence[float] = (0.5,),
                 source: Optional[Source] = None, tol: float = 1e-10,
                 force_iters: int = -1) -> dict:
    st = Stats()
    carr = (C.c_double * max(2, len(c)))(*list(c) + [0.0] * (max(2, len(c)) - len(c)))
    srcs, keep = _source_struct(op, source)
    _check(_lib.ad_expquad_step(op.handle, op.vec(u, "u"), t, dt, s, carr,
                                C.byref(srcs) if srcs is not None else None, tol, force_iters,
                                C.byref(st)), st)
    del keep
    return st.as_dict()


def expquad_step_async(op: Operator, u, t: float, dt: float, s: int = 1,
                       c: Sequence[float] = (0.5,), source: Optional[Source] = None,
                       tol: float = 1e-10) -> None:
    """ad_expquad_step_async: enqueue one step (no synchronisation for a device
    tensor u under the fixed one-substep rule); read the totals with
    async_totals.  u must stay alive until then."""
    carr = (C.c_double * max(2, len(c)))(*list(c) + [0.0] * (max(2, len(c)) - len(c)))
    srcs, keep = _source_struct(op, source)
    _check(_lib.ad_expquad_step_async(op.handle, op.vec(u, "u"), t, dt, s, carr,
                                      C.byref(srcs) if srcs is not None else None, tol))
    del keep


def async_totals(op: Operator) -> dict:
    """ad_async_totals: synchronise and return the totals of the asynchronous
    steps since the last call (raises NotConverged / AdError as the steps'
    worst status says)."""
    st = Stats()
    _check(_lib.ad_async_totals(op.handle, C.byref(st)), st)
    return st.as_dict()


def reserve_gmres(op: Operator, max_restart: int) -> None:
    """ad_reserve_gmres: allocate the GMRES basis for restarts up to max_restart."""
    _check(_lib.ad_reserve_gmres(op.handle, int(max_restart)))


def cn_step(op: Operator, u, t: float, dt: float, source: Optional[Source] = None,
            gmres_tol: float = 1e-10, restart: int = 50, force_iters: int = 0) -> dict:
    st = Stats()
    srcs, keep = _source_struct(op, source)
    _check(_lib.ad_cn_step(op.handle, op.vec(u, "u"), t, dt,
                           C.byref(srcs) if srcs is not None else None, gmres_tol, restart,
                           force_iters, C.byref(st)), st)
    del keep
    return st.as_dict()


def penalised_step(op: Operator, u, t: float, dt: float, source: Optional[Source] = None,
                   beta: float = 1.0, cg_tol: float = 1e-12, max_cg: int = 2000) -> dict:
    """ad_penalised_step: one penalised IMEX Euler step (FP64 operators)."""
    st = Stats()
    srcs, keep = _source_struct(op, source)
    _check(_lib.ad_penalised_step(op.handle, op.vec(u, "u"), t, dt,
                                  C.byref(srcs) if srcs is not None else None, beta, cg_tol,
                                  max_cg, C.byref(st)), st)
    del keep
    return st.as_dict()


def penalty_beta(nx: int, ny: int, Dxx, Dxy, Dyy, stream=None) -> float:
    """ad_penalty_beta: max over cells of lambda_max(D) (float64 device fields)."""
    g = _Grid(nx, ny, -1.0, 1.0, -1.0, 1.0, 0)
    n = nx * ny
    pf = [_ptr(f, "float64", n, name) for f, name in ((Dxx, "Dxx"), (Dxy, "Dxy"), (Dyy, "Dyy"))]
    b = _d()
    _check(_lib.ad_penalty_beta(C.byref(g), pf[0], pf[1], pf[2], _stream_ptr(stream),
                                C.byref(b)))
    return b.value


def profile_leja_iteration(op: Operator, aug: int = 0, reps: int = 200) -> float:
    """Mean duration (ms) of the fused Leja iteration kernel, CUDA events on
    the operator's stream (ad_profile_leja_iteration)."""
    ms = _d()
    _check(_lib.ad_profile_leja_iteration(op.handle, aug, reps, C.byref(ms)))
    return ms.value


def time_series(op: Operator, enable: bool = True) -> None:
    """ad_time_series: start (and reset) or stop recording the device time of
    every Newton series the operator runs."""
    _check(_lib.ad_time_series(op.handle, 1 if enable else 0))


SERIES_KERNELS = {0: None, 1: "leja_persistent_f64_k", 2: "leja_nsync_f64_k",
                  3: "graph loop of per-iteration kernels", 4: "host-driven per-iteration kernels",
                  5: "graph loop of two-iteration kernels", 6: "host-driven two-iteration kernels",
                  7: "leja_tile_f64_k", 8: "graph loop of two-iteration kernels, TMA rows",
                  9: "host-driven two-iteration kernels, TMA rows", 10: "leja_cluster_f64_k"}


def series_timing(op: Operator) -> dict:
    """ad_series_timing: {"ms", "series", "iters", "kernel"} since the last
    enable ("kernel": the path of the last timed series)."""
    ms, ns, it, k = _d(), _i(), C.c_longlong(), _i()
    _check(_lib.ad_series_timing(op.handle, C.byref(ms), C.byref(ns), C.byref(it), C.byref(k)))
    return {"ms": ms.value, "series": ns.value, "iters": it.value,
            "kernel": SERIES_KERNELS.get(k.value)}


NOALLOC_MAX_CELLS = 1 << 16


def leja_phi1_noalloc(nx: int, ny: int, bc: int, Dxx, Dxy, Dyy, v, out, dt: float,
                      ax: float = 0.0, ay: float = 0.0, alpha: float = 0.0, tol: float = 1e-10,
                      force_iters: int = -1, stream=None, x0=-1.0, x1=1.0, y0=-1.0,
                      y1=1.0) -> dict:
    """ad_leja_phi1_noalloc: phi_1(dt A) v with no device allocation (fields,
    v and out are float64 device tensors; see include/anidiff.h for limits)."""
    g = _Grid(nx, ny, x0, x1, y0, y1, bc)
    n = nx * ny
    ptr = lambda x, w: _ptr(x, "float64", n, w)
    st = Stats()
    _check(_lib.ad_leja_phi1_noalloc(C.byref(g), ptr(Dxx, "Dxx"), ptr(Dxy, "Dxy"), ptr(Dyy, "Dyy"),
                                     float(ax), float(ay), alpha, ptr(v, "v"), ptr(out, "out"),
                                     dt, tol, force_iters, _stream_ptr(stream), C.byref(st)), st)
    return st.as_dict()


class Batch:
    """Handle of an ad_batch: FP32-storage operators advanced together."""

    def __init__(self, handle, ops):
        self.handle = handle
        self.ops = list(ops)          # keep the operators alive

    def close(self):
        if self.handle:
            _lib.ad_destroy_batch(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def create_batch(ops, autotune: bool = True) -> Batch:
    """ad_create_batch over a list of FP32_STORAGE operators."""
    arr = (_vp * len(ops))(*[o.handle for o in ops])
    h = _vp()
    _check(_lib.ad_create_batch(arr, len(ops), 1 if autotune else 0, C.byref(h)))
    return Batch(h.value, ops)


def destroy_batch(b: Batch):
    b.close()


def batch_bind(b: Batch, us, sources=None) -> None:
    """ad_batch_bind: the state vectors (float32 device tensors, one per slice)
    and sources that ad_batch_step advances.  The tensors and the callables of
    the sources are kept referenced by the batch."""
    S = len(b.ops)
    if len(us) != S:
        raise ValueError("one state vector per slice")
    uptr = (_vp * S)(*[b.ops[s].vec(us[s], "u") for s in range(S)])
    srcp, keep = None, ()
    if sources is not None:
        if len(sources) != S:
            raise ValueError("one Source (or None) per slice")
        srcp, keep = _batch_sources(b.ops, sources)
    _check(_lib.ad_batch_bind(b.handle, uptr, srcp))
    b._bound = (us, sources, keep)


def batch_step(b: Batch, t: float, dt: float, tol: float = 1e-6, force_iters: int = -1,
               raise_not_converged: bool = True):
    """ad_batch_step: one exponential-midpoint step of the vectors bound by
    batch_bind.  Returns the per-slice stats."""
    S = len(b.ops)
    stats = (Stats * S)()
    status = _lib.ad_batch_step(b.handle, t, dt, tol, force_iters, stats)
    if not (status == AD_ERR_NOT_CONVERGED and not raise_not_converged):
        _check(status, stats[0])
    return [stats[s].as_dict() for s in range(S)]


def batch_iteration_hint(b: Batch, iters=None) -> None:
    """ad_batch_iteration_hint: expected Leja iterations per slice (the longest
    series are queued first in every pass), or None for slice order."""
    import numpy as np
    if iters is None:
        _check(_lib.ad_batch_iteration_hint(b.handle, None))
        return
    arr = np.ascontiguousarray(np.asarray(iters, dtype=np.float64))
    if arr.size != len(b.ops):
        raise ValueError("one iteration hint per slice")
    _check(_lib.ad_batch_iteration_hint(b.handle, arr.ctypes.data))


def batch_order(b: Batch) -> list:
    """ad_batch_order: the slices in the queue order of their warp tiles."""
    import numpy as np
    out = np.zeros(len(b.ops), dtype=np.int32)
    _check(_lib.ad_batch_order(b.handle, out.ctypes.data))
    return out.tolist()


def batch_info(b: Batch) -> dict:
    ty, nb, nt, ms, mr = _i(), _i(), _i(), _d(), _i()
    _check(_lib.ad_batch_info(b.handle, C.byref(ty), C.byref(nb), C.byref(nt), C.byref(ms),
                              C.byref(mr)))
    return {"tile_rows": ty.value, "blocks": nb.value, "tiles": nt.value, "tuned_ms": ms.value,
            "marching": mr.value}


_SOURCE_FIELDS = ("nterms", "g", "h", "ctx")


def _batch_sources(ops, sources):
    """ad_source[S] of a batch built in one buffer: every slice's term pointers
    packed into one void* array, the records written column by column (the
    batched step is called once per time step for every slice, so this avoids
    one ctypes array and callback object per slice).  Returns (pointer, objects
    to keep alive during the call)."""
    import numpy as np
    S = len(ops)
    counts = np.zeros(S, dtype=np.int64)
    ptrs, hcalls = [], []
    for s, src in enumerate(sources):
        if src is None or len(src.g) == 0:
            continue
        if len(src.g) > MAX_SOURCES:
            raise ValueError("at most 16 source terms")
        counts[s] = len(src.g)
        ptrs.extend(ops[s].vec(gk, "source term") for gk in src.g)
        if src.h is not None:
            hs = list(src.h)
            hcalls.append((s, _PROFILE(lambda k, t, ctx, hs=hs: float(hs[k](t)))))
    flat = (C.c_void_p * max(1, len(ptrs)))(*ptrs)
    buf = (C.c_byte * (C.sizeof(_Source) * S))()
    dt = np.dtype({"names": list(_SOURCE_FIELDS), "formats": ["i4", "u8", "u8", "u8"],
                   "offsets": [getattr(_Source, f).offset for f in _SOURCE_FIELDS],
                   "itemsize": C.sizeof(_Source)})
    rec = np.frombuffer(buf, dtype=dt)
    first = np.concatenate(([0], np.cumsum(counts)[:-1]))
    rec["nterms"] = counts
    rec["g"] = np.where(counts > 0, C.addressof(flat) + C.sizeof(C.c_void_p) * first, 0)
    for s, cb in hcalls:
        rec["h"][s] = C.cast(cb, C.c_void_p).value
    return C.cast(buf, _vp), (flat, buf, hcalls)


def batch_midpoint_step(b: Batch, us, t: float, dt: float, sources=None, tol: float = 1e-6,
                        force_iters: int = -1, raise_not_converged: bool = True):
    """ad_batch_midpoint_step: us = list of float32 device tensors (one per slice),
    sources = None or a list of Source (at most 4 terms each).  Returns the
    per-slice stats."""
    S = len(b.ops)
    if len(us) != S:
        raise ValueError("one state vector per slice")
    ops = b.ops
    uptr = (_vp * S)(*[ops[s].vec(us[s], "u") for s in range(S)])
    keep = ()
    srcp = None
    if sources is not None:
        if len(sources) != S:
            raise ValueError("one Source (or None) per slice")
        srcp, keep = _batch_sources(ops, sources)
    stats = (Stats * S)()
    status = _lib.ad_batch_midpoint_step(b.handle, uptr, t, dt, srcp, tol, force_iters, stats)
    if not (status == AD_ERR_NOT_CONVERGED and not raise_not_converged):
        _check(status, stats[0])
    del keep
    return [stats[s].as_dict() for s in range(S)]


class MLP:
    """Handle of an ad_mlp (the learned spectral-bound network)."""

    def __init__(self, n_in=21, n_hidden=64, n_out=2, seed=0, stream=None):
        h = _vp()
        _check(_lib.ad_mlp_create(n_in, n_hidden, n_out, seed, _stream_ptr(stream), C.byref(h)))
        self.handle = h.value
        self.n_in, self.n_hidden, self.n_out = n_in, n_hidden, n_out
        n = _i()
        _check(_lib.ad_mlp_num_params(self.handle, C.byref(n)))
        self.n_params = n.value

    def close(self):
        if self.handle:
            _lib.ad_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _f32(self, x, cols, what):
        return _ptr(x, "float32", x.numel() if hasattr(x, "numel") else x.size, what)

    def get_params(self):
        import numpy as np
        out = np.empty(self.n_params, dtype=np.float32)
        _check(_lib.ad_mlp_params(self.handle, out.ctypes.data, self.n_params, 0))
        return out

    def set_params(self, theta):
        import numpy as np
        t = np.ascontiguousarray(theta, dtype=np.float32)
        _check(_lib.ad_mlp_params(self.handle, t.ctypes.data, self.n_params, 1))

    def normalization(self, x_mean=None, x_std=None, y_mean=None, y_std=None):
        import numpy as np
        if x_mean is None:
            bufs = [np.empty(k, dtype=np.float32) for k in (self.n_in, self.n_in, self.n_out, self.n_out)]
            _check(_lib.ad_mlp_normalization(self.handle, *[b.ctypes.data for b in bufs], 0))
            return bufs
        bufs = [np.ascontiguousarray(b, dtype=np.float32) for b in (x_mean, x_std, y_mean, y_std)]
        _check(_lib.ad_mlp_normalization(self.handle, *[b.ctypes.data for b in bufs], 1))

    def loss_grad(self, X, Y):
        import numpy as np
        B = X.shape[0]
        g = np.empty(self.n_params, dtype=np.float32)
        L = C.c_float()
        _check(_lib.ad_mlp_loss_grad(self.handle, X.data_ptr(), Y.data_ptr(), B, C.byref(L),
                                     g.ctypes.data))
        return L.value, g

    def train(self, X, Y, epochs=2000, lr=3e-3, fit_normalization=True):
        B = X.shape[0]
        L = C.c_float()
        _check(_lib.ad_mlp_train(self.handle, X.data_ptr(), Y.data_ptr(), B, epochs, lr,
                                 1 if fit_normalization else 0, C.byref(L)))
        return L.value

    def predict(self, X, bf16=True):
        import torch
        B = X.shape[0]
        Y = torch.empty((B, self.n_out), dtype=torch.float32, device=X.device)
        _check(_lib.ad_mlp_predict(self.handle, X.data_ptr(), B, 1 if bf16 else 0, Y.data_ptr()))
        return Y


def fp64_fma_rate(blocks_per_sm: int = 2, iters: int = 1 << 16, stream=None) -> float:
    """ad_fp64_fma_rate: the FP64 FMA rate of the device in TFLOP/s."""
    r = _d()
    _check(_lib.ad_fp64_fma_rate(int(blocks_per_sm), int(iters), _stream_ptr(stream), C.byref(r)))
    return r.value


def learned_bounds(model: "MLP", ops: Sequence[Operator], dts, margin: float = 1.1,
                   bf16: bool = True):
    """ad_learned_bounds: set every operator's spectral bound from the model's
    prediction; returns (alphas, predicted iterations) as lists."""
    import numpy as np
    n = len(ops)
    handles = (_vp * n)(*[op.handle for op in ops])
    dt = (_d * n)(*np.broadcast_to(np.asarray(dts, dtype=np.float64), (n,)).tolist())
    a, it = (_d * n)(), (_d * n)()
    _check(_lib.ad_learned_bounds(model.handle, handles, n, dt, float(margin), 1 if bf16 else 0,
                                  a, it))
    return list(a), list(it)


def set_bound_model(op: Operator, model: Optional["MLP"], margin: float = 1.1,
                    dt: float = 1.0) -> None:
    """ad_set_bound_model: the model spectral_bound(op, BOUND_LEARNED) uses."""
    _check(_lib.ad_set_bound_model(op.handle, model.handle if model is not None else None,
                                   float(margin), float(dt)))
    op._bound_model = model               # keep the model alive while attached


def bound_training_sample(op: Operator, dt: float, seed: int, power_iters: int = 60,
                          safety: float = 1.1, tol: float = 1e-6):
    """ad_bound_training_sample: (inputs[21], targets[2], power estimate)."""
    import numpy as np
    x = (C.c_float * 21)()
    t = (C.c_float * 2)()
    est = _d()
    _check(_lib.ad_bound_training_sample(op.handle, float(dt), int(seed), int(power_iters),
                                         float(safety), float(tol), x, t, C.byref(est)))
    return np.array(x, dtype=np.float32), np.array(t, dtype=np.float32), est.value


def field_features(nx, ny, bc, Dxx, Dxy, Dyy, max_a, dt, stream=None, x0=-1.0, x1=1.0, y0=-1.0,
                   y1=1.0):
    """ad_field_features: the 21 network inputs of one field (numpy float32)."""
    import numpy as np
    g = _Grid(nx, ny, x0, x1, y0, y1, bc)
    n = nx * ny
    out = np.empty(21, dtype=np.float32)
    _check(_lib.ad_field_features(C.byref(g), _ptr(Dxx, "float64", n, "Dxx"),
                                  _ptr(Dxy, "float64", n, "Dxy"), _ptr(Dyy, "float64", n, "Dyy"),
                                  float(max_a), float(dt), _stream_ptr(stream), out.ctypes.data))
    return out


def check_wait_timeout(timeout_ms: float = 50.0, stream=None) -> int:
    """ad_check_wait_timeout: returns the status (AD_ERR_TIMEOUT expected)."""
    return _lib.ad_check_wait_timeout(timeout_ms, _stream_ptr(stream))


# ----------------------------------------------------------------------- momentum coupling
class MomentumOperator:
    """Handle of an ad_momentum_operator (Eq. cr_full's momentum terms coupling
    np slices of the spatial operator; FP64, slice-major vectors)."""

    def __init__(self, handle: int, n: int, npm: int):
        self.handle = handle
        self.n, self.np = n, npm
        self.N = n * npm

    def close(self):
        if self.handle:
            _lib.ad_destroy_momentum_operator(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def vec(self, x, what):
        return _ptr(x, "float64", self.N, what)


def create_momentum_operator(nx: int, ny: int, bc: int, Dxx, Dxy, Dyy, P, beta, dpp, b, loss,
                             ax: float = 0.0, ay: float = 0.0, stream=None, x0=-1.0, x1=1.0,
                             y0=-1.0, y1=1.0) -> MomentumOperator:
    """ad_create_momentum_operator.  D fields: float64 device tensors [ny][nx];
    P, dpp, b: np + 1 face values; beta, loss: np cell values (host sequences)."""
    import numpy as np
    g = _Grid(nx, ny, x0, x1, y0, y1, bc)
    n = nx * ny
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (P, beta, dpp, b, loss)]
    npm = len(arrs[1])
    dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
    mom = _Momentum(npm, dp(arrs[0]), dp(arrs[1]), dp(arrs[2]), dp(arrs[3]), dp(arrs[4]))
    pf = [_ptr(f, "float64", n, name) for f, name in ((Dxx, "Dxx"), (Dxy, "Dxy"), (Dyy, "Dyy"))]
    h = _vp()
    _check(_lib.ad_create_momentum_operator(C.byref(g), C.byref(mom), pf[0], pf[1], pf[2],
                                            float(ax), float(ay), _stream_ptr(stream),
                                            C.byref(h)))
    return MomentumOperator(h.value, n, npm)


def momentum_spectral_bound(op: MomentumOperator) -> float:
    a = _d()
    _check(_lib.ad_momentum_spectral_bound(op.handle, C.byref(a)))
    return a.value


def momentum_set_spectral_bound(op: MomentumOperator, alpha: float):
    _check(_lib.ad_momentum_set_spectral_bound(op.handle, alpha))


def momentum_set_options(op: MomentumOperator, rho_max: float = 0.0, max_iters: int = 0):
    _check(_lib.ad_momentum_set_options(op.handle, rho_max, max_iters))


def momentum_apply(op: MomentumOperator, u, out):
    _check(_lib.ad_momentum_apply(op.handle, op.vec(u, "u"), op.vec(out, "out")))


def momentum_leja_phi1(op: MomentumOperator, v, out, dt: float, tol: float = 1e-10,
                       force_iters: int = -1) -> dict:
    st = Stats()
    _check(_lib.ad_momentum_leja_phi1(op.handle, op.vec(v, "v"), op.vec(out, "out"), dt, tol,
                                      force_iters, C.byref(st)), st)
    return st.as_dict()


def momentum_step(op: MomentumOperator, u, dt: float, S=None, tol: float = 1e-10,
                  force_iters: int = -1) -> dict:
    """u += dt phi_1(dt A)(A u + S) for a time-independent source S (or None)."""
    st = Stats()
    _check(_lib.ad_momentum_step(op.handle, op.vec(u, "u"), dt, op.vec(S, "S"), tol,
                                 force_iters, C.byref(st)), st)
    return st.as_dict()
