"""Thin Python binding of the C ABI in include/hq.h (argument marshalling only).

Every function keeps the C name and calls straight into libhq.so; all work runs in
the library's CUDA kernels.  Arrays are numpy arrays (host memory, HQ_HOST) or
torch CUDA tensors (device memory, HQ_DEVICE).  There is no CPU fallback: if the
library cannot be built or loaded, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

HQ_OK, HQ_EINVAL, HQ_ENOMEM, HQ_EUNSTABLE, HQ_ENOTCONVERGED = 0, -1, -2, -3, -4
HQ_EDIVERGED, HQ_ETIMEOUT, HQ_ECUDA, HQ_ESTATE = -5, -6, -7, -8
HQ_LOSS, HQ_FINITE, HQ_INFINITE = 0, 1, 2
HQ_HOST, HQ_DEVICE = 0, 1
HQ_PREC_FP64, HQ_PREC_DF64, HQ_PREC_FP32, HQ_PREC_FP32_DF64, HQ_PREC_FP32_FP64, HQ_PREC_FP32_IR = 0, 1, 2, 3, 4, 5
HQ_TOL_STEP, HQ_TOL_RESIDUAL = 0, 1
HQ_WARM_NONE, HQ_WARM_GIVEN, HQ_WARM_MLP, HQ_WARM_PRODUCT = 0, 1, 2, 3
HQ_ORDER_ASCENDING, HQ_ORDER_REDBLACK = 0, 1
ORDER = {"ascending": HQ_ORDER_ASCENDING, "redblack": HQ_ORDER_REDBLACK}

PRECISION = {"fp64": HQ_PREC_FP64, "df64": HQ_PREC_DF64, "fp32": HQ_PREC_FP32,
             "fp32+df64": HQ_PREC_FP32_DF64, "fp32+fp64": HQ_PREC_FP32_FP64, "fp32+ir": HQ_PREC_FP32_IR}


class hq_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("tol_kind", ctypes.c_int), ("max_sweeps", ctypes.c_int),
                ("precision", ctypes.c_int), ("check_every", ctypes.c_int),
                ("warm_start", ctypes.c_int), ("warm_mem", ctypes.c_int),
                ("warm_p", ctypes.c_void_p), ("fp32_stall", ctypes.c_double),
                ("omega", ctypes.c_double), ("sweep_order", ctypes.c_int),
                ("debug_barrier", ctypes.c_int), ("reserved", ctypes.c_int * 2)]


class hq_stats(ctypes.Structure):
    _fields_ = [("sweeps_fp32", ctypes.c_int), ("sweeps_hi", ctypes.c_int),
                ("residual_checks", ctypes.c_int), ("converged", ctypes.c_int),
                ("final_step", ctypes.c_double), ("final_residual", ctypes.c_double),
                ("ms_total", ctypes.c_double), ("ms_table", ctypes.c_double),
                ("state_updates", ctypes.c_double), ("warm_used", ctypes.c_int),
                ("ir_bases", ctypes.c_int), ("omega", ctypes.c_double),
                ("ms_sweeps_fp32", ctypes.c_double), ("ms_sweeps_hi", ctypes.c_double),
                ("reserved", ctypes.c_int * 2)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class HQError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (status {code})")
        self.code = code


_lib = None
_lock = threading.Lock()
_vp, _i, _d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double

_SIGS = {
    "hq_default_opts": (None, [ctypes.POINTER(hq_opts)]),
    "hq_create": (_i, [_i, _i, _i, _i, _vp, ctypes.POINTER(_vp)]),
    "hq_load": (_i, [_vp, _vp, _vp, _vp, _i]),
    "hq_solve": (_i, [_vp, ctypes.POINTER(hq_opts), ctypes.POINTER(hq_stats)]),
    "hq_get_stationary": (_i, [_vp, _vp, _i]),
    "hq_get_layer_marginals": (_i, [_vp, _vp, _vp, _i]),
    "hq_get_conditional": (_i, [_vp, _vp, _i]),
    "hq_get_utilisation": (_i, [_vp, _vp, _i]),
    "hq_get_response_pattern": (_i, [_vp, _vp, _i]),
    "hq_get_workload": (_i, [_vp, _vp, _i]),
    "hq_get_summary": (_i, [_vp, _vp]),
    "hq_get_table": (_i, [_vp, _vp, _vp, _i]),
    "hq_get_info": (_i, [_vp, _vp]),
    "hq_destroy": (None, [_vp]),
    "hq_strerror": (ctypes.c_char_p, [_i]),
    "hq_last_error": (ctypes.c_char_p, []),
    "hq_launch_count": (ctypes.c_int64, [_i]),
    "hq_profile_sweep": (_i, [_vp, _i, _i, _vp]),
    "hq_sweep_bytes": (_d, [_vp, _i]),
    "hq_dispatch_table_static": (_i, [_i, _i, _vp, _vp, _vp, _vp]),
    "hq_profile_phases": (_i, [_vp, _vp, _i]),
    "hq_batch_create": (_i, [_vp, _i, _vp, ctypes.POINTER(_vp)]),
    "hq_batch_tune": (_i, [_vp, _i, _i, _vp, _vp]),
    "hq_batch_solve": (_i, [_vp, ctypes.POINTER(hq_opts), _vp, _vp]),
    "hq_batch_info": (_i, [_vp, _vp]),
    "hq_batch_set_variant": (_i, [_vp, _i, _i]),
    "hq_batch_destroy": (None, [_vp]),
    "hq_mlp_create": (_i, [_i, ctypes.c_uint64, _vp, ctypes.POINTER(_vp)]),
    "hq_mlp_num_params": (ctypes.c_int64, [_vp]),
    "hq_mlp_set_weights": (_i, [_vp, _vp, ctypes.c_int64, _i]),
    "hq_mlp_get_weights": (_i, [_vp, _vp, ctypes.c_int64, _i]),
    "hq_mlp_forward": (_i, [_vp, _vp, _i, _vp]),
    "hq_mlp_gradients": (_i, [_vp, _vp, _vp, _i, _vp, _vp]),
    "hq_mlp_train_step": (_i, [_vp, _vp, _vp, _i, ctypes.c_float, _vp]),
    "hq_mlp_features": (_i, [_vp, _vp, _i]),
    "hq_mlp_predict": (_i, [_vp, _vp, _vp, _vp, _vp, _i]),
    "hq_attach_mlp": (_i, [_vp, _vp]),
    "hq_mlp_destroy": (None, [_vp]),
    "hq_des_simulate": (_i, [_i, _i, _vp, _vp, _vp, _vp, _i, ctypes.c_int64, ctypes.c_int64,
                             ctypes.c_int64, ctypes.c_uint64, _vp, _vp, _vp, _vp, _vp, _i, _vp]),
}


def load(build: bool = True):
    """Build (if stale) and load libhq.so.  Raises if it cannot."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build() if build else _build.LIB
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def library_path() -> str:
    return _build.LIB


def _check(rc: int, allow=(HQ_OK,)) -> int:
    if rc not in allow:
        lib = load()
        raise HQError(rc, f"{lib.hq_strerror(rc).decode()}: {lib.hq_last_error().decode()}")
    return rc


def _ptr(a, dtype, count: int, name: str):
    """(address, mem) of a numpy array or torch tensor (None: (None, HOST)), after the
    checks the C side cannot make on a bare pointer: the element type (`dtype`, or one of
    a tuple of types of the same width), C-contiguity, at least `count` elements, and for
    a CUDA tensor the current device (the kernels run there)."""
    if a is None:
        return None, HQ_HOST
    wants = [np.dtype(d) for d in (dtype if isinstance(dtype, tuple) else (dtype,))]
    if isinstance(a, np.ndarray):
        if a.dtype not in wants or not a.flags["C_CONTIGUOUS"]:
            raise ValueError(f"{name}: a C-contiguous {wants[0]} array is needed")
        if a.size < count:
            raise ValueError(f"{name}: {a.size} elements, {count} needed")
        return a.ctypes.data, HQ_HOST
    import torch

    if a.dtype not in [_TORCH_DTYPES[w.str] for w in wants] or not a.is_contiguous():
        raise ValueError(f"{name}: a contiguous {wants[0]} tensor is needed")
    if a.numel() < count:
        raise ValueError(f"{name}: {a.numel()} elements, {count} needed")
    if a.is_cuda and a.device.index != torch.cuda.current_device():
        raise ValueError(f"{name}: on {a.device}, not on the current device")
    return a.data_ptr(), (HQ_DEVICE if a.is_cuda else HQ_HOST)


class _TorchDtypes(dict):
    """numpy dtype string -> torch dtype, filled on first use (torch imported lazily)."""

    def __missing__(self, key):
        import torch

        self.update({"<f8": torch.float64, "<f4": torch.float32, "<i4": torch.int32,
                     "<u4": torch.uint32 if hasattr(torch, "uint32") else torch.int32,
                     "<i8": torch.int64})
        return dict.__getitem__(self, key)


_TORCH_DTYPES = _TorchDtypes()


def _sizes(h: int) -> tuple[int, int, int, int]:
    """(N, J, mode, C) of a solver."""
    info = hq_get_info(h)
    return int(info[0]), int(info[1]), int(info[2]), int(info[3])


# ---- the C calls, same names ------------------------------------------------------------

def hq_default_opts() -> hq_opts:
    o = hq_opts()
    load().hq_default_opts(ctypes.byref(o))
    return o


def hq_create(N: int, J: int, mode: int = HQ_LOSS, capacity_C: int = 0, stream=None) -> int:
    h = _vp()
    s = stream if isinstance(stream, int) or stream is None else stream.cuda_stream
    _check(load().hq_create(N, J, mode, capacity_C, s, ctypes.byref(h)))
    return h.value


def hq_load(h: int, lambda_j, nu, pref) -> None:
    N, J, _, _ = _sizes(h)
    pl, ml = _ptr(lambda_j, np.float64, J, "lambda_j")
    pn, mn = _ptr(nu, np.float64, N, "nu")
    pp, mp = _ptr(pref, np.int32, J * N, "pref")
    if not (ml == mn == mp):
        raise ValueError("lambda_j, nu and pref must live in the same memory")
    _check(load().hq_load(h, pl, pn, pp, ml))


def hq_solve(h: int, opts: hq_opts | None = None, allow_notconverged: bool = True) -> tuple[int, hq_stats]:
    st = hq_stats()
    allow = (HQ_OK, HQ_ENOTCONVERGED) if allow_notconverged else (HQ_OK,)
    rc = load().hq_solve(h, ctypes.byref(opts) if opts is not None else None, ctypes.byref(st))
    _check(rc, allow)
    return rc, st


def _get(fn, h, out, count):
    p, m = _ptr(out, np.float64, count, fn)
    _check(getattr(load(), fn)(h, p, m))
    return out


def hq_get_stationary(h, out):
    N, _, _, _ = _sizes(h)
    return _get("hq_get_stationary", h, out, 1 << N)


def hq_get_conditional(h, out):
    N, _, _, _ = _sizes(h)
    return _get("hq_get_conditional", h, out, 1 << N)


def hq_get_layer_marginals(h, out, tail=None):
    N, _, mode, C = _sizes(h)
    p, m = _ptr(out, np.float64, N + 1 + (C if mode == HQ_FINITE else 0), "p_n")
    pt, mt = _ptr(tail, np.float64, 1, "tail")
    if tail is not None and mt != m:
        raise ValueError("p_n and tail must live in the same memory")
    _check(load().hq_get_layer_marginals(h, p, pt, m))
    return out


def hq_get_utilisation(h, out):
    N, _, _, _ = _sizes(h)
    return _get("hq_get_utilisation", h, out, N)


def hq_get_response_pattern(h, out):
    N, J, _, _ = _sizes(h)
    return _get("hq_get_response_pattern", h, out, J * N)


def hq_get_workload(h, out):
    N, J, _, _ = _sizes(h)
    return _get("hq_get_workload", h, out, N * J)


def hq_get_summary(h) -> np.ndarray:
    out = np.zeros(5)
    _check(load().hq_get_summary(h, out.ctypes.data))
    return out


def hq_get_table(h, T=None, masks=None):
    info = hq_get_info(h)
    pt, mt = _ptr(T, np.float64, int(info[5]), "T")
    pm, mm = _ptr(masks, (np.uint32, np.int32), int(info[4]), "masks")
    if T is not None and masks is not None and mt != mm:
        raise ValueError("T and masks must live in the same memory")
    _check(load().hq_get_table(h, pt, pm, mt if T is not None else mm))
    return T, masks


def hq_get_info(h) -> np.ndarray:
    out = np.zeros(8, dtype=np.int64)
    _check(load().hq_get_info(h, out.ctypes.data))
    return out


def hq_profile_sweep(h: int, precision: int, sweeps: int) -> float:
    """Mean milliseconds per sweep of one persistent-kernel launch of `sweeps` sweeps."""
    out = np.zeros(1, dtype=np.float32)
    _check(load().hq_profile_sweep(h, precision, sweeps, out.ctypes.data))
    return float(out[0])


def hq_profile_phases(h: int, max_out: int = 64) -> np.ndarray:
    """Per-phase wall time (us) of the last sweep-kernel launch."""
    out = np.zeros(max_out)
    n = load().hq_profile_phases(h, out.ctypes.data, max_out)
    _check(n if n < 0 else 0)
    return out[:n]


def hq_sweep_bytes(h: int, precision: int) -> float:
    return float(load().hq_sweep_bytes(h, precision))


def hq_dispatch_table_static(N: int, J: int, lambda_j, pref, T, stream=None) -> None:
    """Upward-rate table without any device allocation.  lambda_j (J float64), pref (J x N
    int32) and T (at least N 2^(N-1) float64) are contiguous CUDA tensors on the current
    device; the C side cannot check pointers, so the binding does."""
    import torch

    dev = torch.cuda.current_device()
    for name, t, dt, count in (("lambda_j", lambda_j, torch.float64, J),
                               ("pref", pref, torch.int32, J * N),
                               ("T", T, torch.float64, N << (N - 1) if N >= 1 else 0)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.device.index == dev):
            raise ValueError(f"{name} must be a CUDA tensor on the current device (cuda:{dev})")
        if t.dtype != dt or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous {dt} tensor")
        if t.numel() < count:
            raise ValueError(f"{name} holds {t.numel()} elements, {count} needed")
    s = stream if isinstance(stream, int) or stream is None else stream.cuda_stream
    _check(load().hq_dispatch_table_static(N, J, lambda_j.data_ptr(), pref.data_ptr(),
                                           T.data_ptr(), s))


def hq_destroy(h: int) -> None:
    if h:
        load().hq_destroy(h)


def hq_batch_create(handles, stream=None) -> int:
    arr = (_vp * len(handles))(*handles)
    b = _vp()
    s = stream if isinstance(stream, int) or stream is None else stream.cuda_stream
    _check(load().hq_batch_create(arr, len(handles), s, ctypes.byref(b)))
    return b.value


def hq_batch_tune(b: int, precision: int, sweeps: int = 4) -> tuple[int, np.ndarray]:
    ms = np.zeros(4, dtype=np.float32)
    v = ctypes.c_int(0)
    _check(load().hq_batch_tune(b, precision, sweeps, ctypes.addressof(v), ms.ctypes.data))
    return v.value, ms


def hq_batch_solve(b: int, count: int, opts: hq_opts | None = None,
                   allow_notconverged: bool = True) -> tuple[int, list, float]:
    st = (hq_stats * count)()
    ms = np.zeros(1)
    allow = (HQ_OK, HQ_ENOTCONVERGED) if allow_notconverged else (HQ_OK,)
    rc = load().hq_batch_solve(b, ctypes.byref(opts) if opts is not None else None,
                               ctypes.addressof(st), ms.ctypes.data)
    _check(rc, allow)
    return rc, [st[i].as_dict() for i in range(count)], float(ms[0])


def hq_batch_set_variant(b: int, precision: int, variant: int) -> None:
    _check(load().hq_batch_set_variant(b, precision, variant))


def hq_batch_info(b: int) -> np.ndarray:
    out = np.zeros(8, dtype=np.int64)
    _check(load().hq_batch_info(b, out.ctypes.data))
    return out


def hq_batch_destroy(b: int) -> None:
    if b:
        load().hq_batch_destroy(b)


def hq_mlp_create(hidden: int = 256, seed: int = 1, stream=None) -> int:
    m = _vp()
    s = stream if isinstance(stream, int) or stream is None else stream.cuda_stream
    _check(load().hq_mlp_create(hidden, seed, s, ctypes.byref(m)))
    return m.value


def hq_mlp_num_params(m: int) -> int:
    return int(load().hq_mlp_num_params(m))


def hq_mlp_set_weights(m: int, w) -> None:
    p, mem = _ptr(w, np.float32, hq_mlp_num_params(m), "w")
    _check(load().hq_mlp_set_weights(m, p, hq_mlp_num_params(m), mem))


def hq_mlp_get_weights(m: int, out=None):
    if out is None:
        out = np.empty(hq_mlp_num_params(m), dtype=np.float32)
    p, mem = _ptr(out, np.float32, hq_mlp_num_params(m), "w")
    _check(load().hq_mlp_get_weights(m, p, hq_mlp_num_params(m), mem))
    return out


def _device_rows(X, target, name: str) -> tuple[int, int, int]:
    """(B, X address, target address) of B rows of 9 network inputs and B targets, both
    float32 CUDA tensors on the current device."""
    B = int(X.shape[0])
    px, mx = _ptr(X, np.float32, 9 * B, "X")
    pt, mt = _ptr(target, np.float32, B, name)
    if mx != HQ_DEVICE or mt != HQ_DEVICE:
        raise ValueError(f"X and {name} must be CUDA tensors")
    return B, px, pt


def hq_mlp_forward(m: int, X, y) -> None:
    """X: (B, 9) float32 CUDA tensor; y: (B,) float32 CUDA tensor."""
    B, px, py = _device_rows(X, y, "y")
    _check(load().hq_mlp_forward(m, px, B, py))


def hq_mlp_gradients(m: int, X, target, grad=None) -> float:
    loss = ctypes.c_float(0.0)
    B, px, pt = _device_rows(X, target, "target")
    pg, mg = _ptr(grad, np.float32, hq_mlp_num_params(m), "grad")
    if grad is not None and mg != HQ_DEVICE:
        raise ValueError("grad must be a CUDA tensor")
    _check(load().hq_mlp_gradients(m, px, pt, B, pg, ctypes.addressof(loss)))
    return float(loss.value)


def hq_mlp_train_step(m: int, X, target, lr: float, want_loss: bool = True):
    loss = ctypes.c_float(0.0)
    B, px, pt = _device_rows(X, target, "target")
    _check(load().hq_mlp_train_step(m, px, pt, B, lr, ctypes.addressof(loss) if want_loss else None))
    return float(loss.value) if want_loss else None


def hq_mlp_features(h: int, out=None, N: int | None = None):
    """Network inputs, one row per (layer n = 1..N-1, unit i): (N (N-1), 9) float32."""
    n = _sizes(h)[0]
    if N is not None and N != n:
        raise ValueError(f"hq_mlp_features: the solver has N = {n}, not {N}")
    if out is None:
        out = np.empty((n * (n - 1), 9), dtype=np.float32)
    p, mem = _ptr(out, np.float32, 9 * n * (n - 1), "X")
    _check(load().hq_mlp_features(h, p, mem))
    return out


def hq_mlp_predict(h: int, m: int, N: int) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """(q (N+1, N), layer law P(n), rho) of the model for the loaded instance."""
    if N != _sizes(h)[0]:
        raise ValueError(f"hq_mlp_predict: the solver has N = {_sizes(h)[0]}, not {N}")
    q = np.empty((N + 1, N))
    pn = np.empty(N + 1)
    rho = np.empty(N)
    _check(load().hq_mlp_predict(h, m, q.ctypes.data, pn.ctypes.data, rho.ctypes.data, HQ_HOST))
    return q, pn, rho


def hq_attach_mlp(h: int, m: int | None) -> None:
    _check(load().hq_attach_mlp(h, m))


def hq_mlp_destroy(m: int) -> None:
    if m:
        load().hq_mlp_destroy(m)


WARMSTART_WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data",
                                 "warmstart_mlp_h256.f32")


def load_warmstart_model(path: str = WARMSTART_WEIGHTS, hidden: int = 256) -> int:
    """A model handle with the weights trained by train_warmstart.py (raw float32 file)."""
    w = np.fromfile(path, dtype="<f4")
    m = hq_mlp_create(hidden, 1)
    if w.size != hq_mlp_num_params(m):
        hq_mlp_destroy(m)
        raise ValueError(f"{path}: {w.size} parameters, the network has {hq_mlp_num_params(m)}")
    hq_mlp_set_weights(m, np.ascontiguousarray(w))
    return m


def hq_launch_count(reset: bool = False) -> int:
    return int(load().hq_launch_count(1 if reset else 0))


# ---- convenience wrapper ---------------------------------------------------------------

class Solver:
    """Owns one hq_solver handle: create -> load -> solve -> results (host numpy)."""

    def __init__(self, N: int, J: int, mode: int = HQ_LOSS, C: int = 0, stream=None):
        self.N, self.J, self.mode, self.C = N, J, mode, C
        self.h = hq_create(N, J, mode, C, stream)

    @classmethod
    def for_instance(cls, inst, stream=None) -> "Solver":
        s = cls(inst.N, inst.J, inst.mode, inst.C, stream)
        s.load(inst.lam_j, inst.nu, inst.pref)
        return s

    def load(self, lam_j, nu, pref):
        if isinstance(lam_j, np.ndarray) or not hasattr(lam_j, "is_cuda"):
            lam_j = np.ascontiguousarray(lam_j, dtype=np.float64)
            nu = np.ascontiguousarray(nu, dtype=np.float64)
            pref = np.ascontiguousarray(pref, dtype=np.int32)
        hq_load(self.h, lam_j, nu, pref)

    def solve(self, tol=1e-10, tol_kind=HQ_TOL_RESIDUAL, precision="fp32+df64", max_sweeps=100000,
              check_every=8, warm_p=None, fp32_stall=0.0, warm_mlp=False, warm_product=False,
              omega=1.0, order="ascending", debug_barrier=0) -> tuple[int, dict]:
        o = hq_default_opts()
        o.sweep_order = ORDER[order] if isinstance(order, str) else int(order)
        o.debug_barrier = debug_barrier
        o.tol = tol
        o.tol_kind = tol_kind
        o.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
        o.max_sweeps = max_sweeps
        o.check_every = check_every
        o.fp32_stall = fp32_stall
        o.omega = omega
        keep = None
        if warm_p is not None:
            # keep the buffer handed to C (a converted copy, for a numpy input) alive
            keep = np.ascontiguousarray(warm_p, dtype=np.float64) if isinstance(warm_p, np.ndarray) else warm_p
            p, m = _ptr(keep, np.float64, 1 << self.N, "warm_p")
            o.warm_start = HQ_WARM_GIVEN
            o.warm_p = p
            o.warm_mem = m
        elif warm_mlp:
            o.warm_start = HQ_WARM_MLP
        elif warm_product:
            o.warm_start = HQ_WARM_PRODUCT
        rc, st = hq_solve(self.h, o)
        del keep
        return rc, st.as_dict()

    def stationary(self) -> np.ndarray:
        return hq_get_stationary(self.h, np.empty(1 << self.N))

    def conditional(self) -> np.ndarray:
        return hq_get_conditional(self.h, np.empty(1 << self.N))

    def layer_marginals(self) -> tuple[np.ndarray, float]:
        top = self.N + (self.C if self.mode == HQ_FINITE else 0)
        pn = np.empty(top + 1)
        tail = np.zeros(1)
        hq_get_layer_marginals(self.h, pn, tail)
        return pn, float(tail[0])

    def utilisation(self) -> np.ndarray:
        return hq_get_utilisation(self.h, np.empty(self.N))

    def response_pattern(self) -> np.ndarray:
        return hq_get_response_pattern(self.h, np.empty((self.J, self.N)))

    def workload(self) -> np.ndarray:
        return hq_get_workload(self.h, np.empty((self.N, self.J)))

    def summary(self) -> dict:
        s = hq_get_summary(self.h)
        return {"throughput": s[0], "p_block": s[1], "p_wait": s[2], "residual": s[3],
                "mean_busy": s[4]}

    def table(self) -> tuple[np.ndarray, np.ndarray]:
        info = hq_get_info(self.h)
        T = np.empty(int(info[5]))
        masks = np.empty(1 << self.N, dtype=np.uint32)
        hq_get_table(self.h, T, masks)
        return T, masks

    def close(self):
        if self.h:
            hq_destroy(self.h)
            self.h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# ---- discrete-event simulation of the loss system -------------------------------------

DES_KINDS = {"exponential": 0, "lognormal": 1, "gamma5": 2, "gamma05": 3, "uniform": 4}


def hq_des_simulate(N: int, J: int, lam_j, nu, pref, travel, kind, reps: int, arrivals: int,
                    warmup: int, seed: int, stream=None) -> dict:
    """Run hq_des_simulate on host arrays (numpy) or device tensors (torch, all on the
    same device); returns the per-replication outputs as arrays of the same kind."""
    k = DES_KINDS[kind] if isinstance(kind, str) else int(kind)
    if isinstance(lam_j, np.ndarray) or not hasattr(lam_j, "is_cuda"):
        lam_j = np.ascontiguousarray(lam_j, dtype=np.float64)
        nu = np.ascontiguousarray(nu, dtype=np.float64)
        pref = np.ascontiguousarray(pref, dtype=np.int32)
        travel = np.ascontiguousarray(travel, dtype=np.float64)
        for a, n in ((lam_j, J), (nu, N), (pref, J * N), (travel, J * N)):
            if a.size != n:
                raise ValueError("hq_des_simulate: input of the wrong size")
        out = dict(busy=np.empty((reps, N)), served=np.empty((reps, N), dtype=np.int64),
                   lost=np.empty(reps, dtype=np.int64), window=np.empty(reps), resp=np.empty(reps))
        mem = HQ_HOST
    else:
        import torch

        dev = lam_j.device
        out = dict(busy=torch.empty((reps, N), dtype=torch.float64, device=dev),
                   served=torch.empty((reps, N), dtype=torch.int64, device=dev),
                   lost=torch.empty(reps, dtype=torch.int64, device=dev),
                   window=torch.empty(reps, dtype=torch.float64, device=dev),
                   resp=torch.empty(reps, dtype=torch.float64, device=dev))
        mem = HQ_DEVICE
    pa = []
    for x, dt, n, name in ((lam_j, np.float64, J, "lambda_j"), (nu, np.float64, N, "nu"),
                           (pref, np.int32, J * N, "pref"), (travel, np.float64, J * N, "travel")):
        p, m = _ptr(x, dt, n, name)
        if m != mem:
            raise ValueError("hq_des_simulate: all inputs in host memory, or all CUDA tensors")
        pa.append(p)
    po = [_ptr(out[k2], dt, n, k2)[0]
          for k2, dt, n in (("busy", np.float64, reps * N), ("served", np.int64, reps * N),
                            ("lost", np.int64, reps), ("window", np.float64, reps), ("resp", np.float64, reps))]
    sp = stream.cuda_stream if stream is not None and hasattr(stream, "cuda_stream") else stream
    _check(load().hq_des_simulate(N, J, *pa, k, reps, arrivals, warmup, ctypes.c_uint64(seed), *po, mem, sp))
    return out
