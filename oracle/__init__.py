"""CPU oracle for the spatial hypercube queue solver (arXiv 2603.03019).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg of the
benchmark use this package; the GPU library never imports or calls it.

Two independent routes:
  * ``solve`` -- Algorithm 1 (Conditional Probability Update) in plain C, FP64,
    literal inner loop (``hq_oracle.c``), plus Eq. (10)/Proposition 2/Remark and
    the performance measures;
  * ``oracle.dense.dense_solve`` -- a dense direct solve of the global balance
    equations (1)-(2) built straight from Eq. (3) in numpy (N <= 12).

Also ``des_loss``: the discrete-event simulation of the loss system with general service
times (Section 5.5) in plain C (``des.c``).  Its sample path is defined with FP32
variates from series functions and an FP64 clock (the paper gives its simulation no
precision), the one place the oracle computes in FP32; it is pinned to Erlang-B, the
exact solution and the samplers' moments.

Arguments are plain arrays: N, J, lam_j (J,), nu (N,), pref (J, N) int32 with
pref[j, h] = zeta_j(h+1) (0-based unit ids), mode 0 loss / 1 finite / 2 infinite,
C the buffer size (finite mode).  Any object with those attributes can be passed
as ``inst``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

LOSS, FINITE, INFINITE = 0, 1, 2

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hq_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "des.c")]
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_LIB_OMP_PATH = os.path.join(_BUILD, "liboracle_omp.so")
_lock = threading.Lock()
_libs: dict = {}

_d = ctypes.c_double
_i = ctypes.c_int
_i64 = ctypes.c_int64
_pd = ctypes.POINTER(ctypes.c_double)
_pi32 = ctypes.POINTER(ctypes.c_int32)
_pu32 = ctypes.POINTER(ctypes.c_uint32)
_pu64 = ctypes.POINTER(ctypes.c_uint64)
_vp = ctypes.c_void_p


def _compile(path: str, omp: bool, force: bool) -> str:
    os.makedirs(_BUILD, exist_ok=True)
    stale = not os.path.exists(path) or any(os.path.getmtime(path) < os.path.getmtime(s) for s in _SRCS)
    if force or stale:
        tmp = path + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
               "-ffp-contract=off", *(["-fopenmp"] if omp else []), *_SRCS, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, path)
    return path


def build(force: bool = False) -> str:
    """Compile hq_oracle.c (gcc, -O2, no fast-math) twice: plainly into
    oracle/_build/liboracle.so (single-threaded) and with -fopenmp into
    liboracle_omp.so (the loops over the states of a layer on all host threads).  A
    toolchain without OpenMP support leaves only the plain library."""
    _compile(_LIB_PATH, False, force)
    try:
        _compile(_LIB_OMP_PATH, True, force)
    except (subprocess.CalledProcessError, OSError):
        pass
    return _LIB_PATH


def max_threads() -> int:
    """Host threads the OpenMP build would use (1 without it)."""
    return int(_load(0).or_threads(0))


def _load(threads: int = 1):
    """The plain library (threads == 1) or the OpenMP one (threads 0 = all host
    threads, or a count), falling back to the plain one if OpenMP is unavailable."""
    omp = threads != 1
    with _lock:
        build()
        path = _LIB_OMP_PATH if omp and os.path.exists(_LIB_OMP_PATH) else _LIB_PATH
        lib = _libs.get(path)
        if lib is not None:
            if path == _LIB_OMP_PATH:
                lib.or_threads(threads if threads > 1 else os.cpu_count() or 1)
            return lib
        lib = ctypes.CDLL(path)
        sig = {
            "or_create": (_vp, [_i, _i, _pd, _pd, _pi32, _i, _i]),
            "or_destroy": (None, [_vp]),
            "or_layer_size": (_i64, [_vp, _i]),
            "or_layer_states": (None, [_vp, _i, _pu32]),
            "or_build_up": (_i, [_vp, _i, _i]),
            "or_get_up_rows": (None, [_vp, _i, _pd]),
            "or_init": (None, [_vp, _pd]),
            "or_set_p": (None, [_vp, _pd]),
            "or_get_p": (None, [_vp, _pd]),
            "or_get_layer_scalars": (None, [_vp, _pd, _pd]),
            "or_layer_rates": (None, [_vp, _pd, _pd]),
            "or_inner_total": (ctypes.c_long, [_vp]),
            "or_update_layer": (_i, [_vp, _i, _d, _i, _pd, _pd]),
            "or_sweep": (_d, [_vp, _d, _i, _pd]),
            "or_solve": (_i, [_vp, _d, _d, _i, _i, _pd, _pd, ctypes.POINTER(_i)]),
            "or_birth_death": (None, [_i, _i, _i, _d, _d, _pd, _pd, _pd, _pd]),
            "or_stationary": (None, [_vp, _pd, _pd]),
            "or_outputs": (_d, [_vp, _pd, _d, _d, _pd, _pd, _pd]),
            "or_residual": (_d, [_vp, _pd, _d]),
            "or_first_idle": (_i, [_i, _pi32, ctypes.c_uint64]),
            "or_dispatch_rate": (_d, [_i, _i, _pd, _pi32, ctypes.c_uint64, _i]),
            "or_dispatch_rates_batch": (None, [_i, _i, _pd, _pi32, _i64, _pu64, _pi32, _pd]),
            "or_sampled_balance": (None, [_i, _i, _pd, _pd, _pi32, _i, _i64, _pu64, _pd, _pd, _d,
                                          _pd, _pd]),
            "or_threads": (_i, [_i]),
            "or_des_loss": (_i, [_i, _i, _pd, _pd, _pi32, _pd, _i, _i64, _i64, _i64, ctypes.c_uint64,
                                 _pd, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                 _pd, _pd]),
            "or_des_service": (ctypes.c_float, [_i, ctypes.c_float, ctypes.c_uint64, ctypes.c_uint64]),
            "or_des_uniform": (ctypes.c_float, [ctypes.c_uint64, _i64, ctypes.c_uint64]),
            "or_des_ln": (ctypes.c_float, [ctypes.c_float]),
            "or_des_exp": (ctypes.c_float, [ctypes.c_float]),
            "or_des_cos2pi": (ctypes.c_float, [ctypes.c_float]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _libs[path] = lib
        if path == _LIB_OMP_PATH:
            lib.or_threads(threads if threads > 1 else os.cpu_count() or 1)
        return lib


def _p(a, ptr):
    return a.ctypes.data_as(ptr)


def _args(inst=None, **kw):
    if inst is not None:
        for k in ("N", "J", "lam_j", "nu", "pref", "mode", "C"):
            kw.setdefault(k, getattr(inst, k))
    N, J = int(kw["N"]), int(kw["J"])
    lam_j = np.ascontiguousarray(kw["lam_j"], dtype=np.float64)
    nu = np.ascontiguousarray(kw["nu"], dtype=np.float64)
    pref = np.ascontiguousarray(kw["pref"], dtype=np.int32)
    mode = int(kw.get("mode", LOSS))
    C = int(kw.get("C", 0))
    return N, J, lam_j, nu, pref, mode, C


class Oracle:
    """Handle on the C oracle's state for one instance (keeps the rate table).
    threads: 1 = the plain single-threaded build; 0 = the OpenMP build on all host
    threads; k > 1 = the OpenMP build on k threads."""

    def __init__(self, inst=None, threads: int = 1, **kw):
        self.lib = _load(threads)
        (self.N, self.J, self.lam_j, self.nu, self.pref, self.mode, self.C) = _args(inst, **kw)
        self.ctx = self.lib.or_create(self.N, self.J, _p(self.lam_j, _pd), _p(self.nu, _pd),
                                      _p(self.pref, _pi32), self.mode, self.C)
        if not self.ctx:
            raise ValueError("oracle rejected the instance")
        self.S = 1 << self.N
        self.lam = float(self.lam_j.sum())
        self.nu_sum = float(self.nu.sum())
        self._table_built = False

    def close(self):
        if self.ctx:
            self.lib.or_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- rates ----------------------------------------------------------------------
    def build_table(self, n_lo: int = 0, n_hi: int | None = None):
        n_hi = self.N - 1 if n_hi is None else n_hi
        if self.lib.or_build_up(self.ctx, n_lo, n_hi) != 0:
            raise MemoryError("oracle rate table")
        self._table_built = True

    def layer_states(self, n: int) -> np.ndarray:
        L = self.lib.or_layer_size(self.ctx, n)
        out = np.empty(L, dtype=np.uint32)
        self.lib.or_layer_states(self.ctx, n, _p(out, _pu32))
        return out

    def up_rows(self, n: int) -> np.ndarray:
        """rows of source layer n: [k, u] = rate of the upward move state_k -> state_k + u."""
        L = self.lib.or_layer_size(self.ctx, n)
        out = np.empty((L, self.N), dtype=np.float64)
        self.lib.or_get_up_rows(self.ctx, n, _p(out, _pd))
        return out

    # -- Algorithm 1 ----------------------------------------------------------------
    def init(self, p0: np.ndarray | None = None):
        if p0 is None:
            self.lib.or_init(self.ctx, None)
        else:
            p0 = np.ascontiguousarray(p0, dtype=np.float64)
            self.lib.or_init(self.ctx, _p(p0, _pd))

    def sweep(self, delta: float = 1e-20, max_inner: int = 100000) -> tuple[float, float]:
        l1 = ctypes.c_double()
        step = self.lib.or_sweep(self.ctx, delta, max_inner, ctypes.byref(l1))
        return step, l1.value

    def update_layer(self, n: int, delta: float = 1e-20, max_inner: int = 100000):
        md, l1 = ctypes.c_double(), ctypes.c_double()
        r = self.lib.or_update_layer(self.ctx, n, delta, max_inner, ctypes.byref(md),
                                     ctypes.byref(l1))
        return r, md.value, l1.value

    def run(self, eps: float, delta: float = 1e-20, max_sweeps: int = 100000,
            max_inner: int = 100000):
        tl = np.zeros(max_sweeps)
        t1 = np.zeros(max_sweeps)
        conv = ctypes.c_int()
        k = self.lib.or_solve(self.ctx, eps, delta, max_sweeps, max_inner, _p(tl, _pd),
                              _p(t1, _pd), ctypes.byref(conv))
        return k, bool(conv.value), tl[:k], t1[:k]

    def conditional(self) -> np.ndarray:
        out = np.empty(self.S)
        self.lib.or_get_p(self.ctx, _p(out, _pd))
        return out

    def layer_scalars(self):
        ln = np.empty(self.N + 1)
        mn = np.empty(self.N + 1)
        self.lib.or_get_layer_scalars(self.ctx, _p(ln, _pd), _p(mn, _pd))
        return ln, mn

    def layer_rates(self):
        """lambda(n), mu(n) recomputed from the current p (Eq. 6-7)."""
        ln = np.empty(self.N + 1)
        mn = np.empty(self.N + 1)
        self.lib.or_layer_rates(self.ctx, _p(ln, _pd), _p(mn, _pd))
        return ln, mn

    def residual(self, P: np.ndarray, pq1: float = 0.0) -> float:
        """max_m |out_m - in_m| / max_m out_m of Eq. (1) for a given y-order P."""
        P = np.ascontiguousarray(P, dtype=np.float64)
        return float(self.lib.or_residual(self.ctx, _p(P, _pd), float(pq1)))

    # -- results --------------------------------------------------------------------
    def results(self, with_R: bool = True, with_residual: bool = True) -> dict:
        ln, mn = self.layer_rates()
        top = self.N + self.C if self.mode == FINITE else self.N
        pn = np.empty(top + 1)
        tail = ctypes.c_double(0.0)
        self.lib.or_birth_death(self.N, self.mode, self.C, self.lam, self.nu_sum, _p(ln, _pd),
                                _p(mn, _pd), _p(pn, _pd), ctypes.byref(tail))
        P = np.empty(self.S)
        self.lib.or_stationary(self.ctx, _p(pn, _pd), _p(P, _pd))
        rho_q = self.lam / self.nu_sum
        if self.mode == LOSS:
            q_busy, q_wait, pq1, p_block = 0.0, 0.0, 0.0, float(pn[self.N])
        elif self.mode == FINITE:
            q_busy = float(pn[self.N + 1:].sum())
            q_wait = float(pn[self.N:self.N + self.C].sum())
            pq1 = float(pn[self.N + 1])
            p_block = float(pn[self.N + self.C])
        else:
            q_busy = tail.value
            q_wait = float(pn[self.N]) + tail.value
            pq1 = float(pn[self.N]) * rho_q
            p_block = 0.0
        rho = np.empty(self.N)
        R = np.empty((self.J, self.N)) if with_R else None
        W = np.empty((self.N, self.J)) if with_R else None
        thr = self.lib.or_outputs(self.ctx, _p(P, _pd), q_busy, q_wait, _p(rho, _pd),
                                  _p(R, _pd) if with_R else None, _p(W, _pd) if with_R else None)
        out = dict(P=P, pn=pn, cond=self.conditional(), lam_n=ln, mu_n=mn, rho=rho, R=R, W=W,
                   throughput=thr, q_busy=q_busy, q_wait=q_wait, pq1=pq1, p_block=p_block,
                   queue_tail=tail.value)
        if with_residual:
            out["residual"] = self.lib.or_residual(self.ctx, _p(P, _pd), pq1)
        return out


def solve(inst=None, eps: float = 1e-12, delta: float = 1e-20, max_sweeps: int = 100000,
          max_inner: int = 100000, p0=None, sweeps: int | None = None, with_R: bool = True,
          threads: int = 1, **kw) -> dict:
    """Algorithm 1 to max|p^k - p^{k-1}| <= eps (or exactly ``sweeps`` sweeps), then the
    birth-death step and the performance measures.  threads as for ``Oracle``."""
    o = Oracle(inst, threads=threads, **kw)
    try:
        o.build_table()
        o.init(p0)
        if sweeps is not None:
            k, conv, tl, t1 = o.run(-1.0, delta, sweeps, max_inner)
        else:
            k, conv, tl, t1 = o.run(eps, delta, max_sweeps, max_inner)
        res = o.results(with_R=with_R)
        res.update(sweeps=k, converged=conv, trace_linf=tl, trace_l1=t1,
                   inner_total=int(o.lib.or_inner_total(o.ctx)))
        return res
    finally:
        o.close()


def solve_to_residual(inst=None, tol: float = 1e-10, check_every: int = 8,
                      max_sweeps: int = 100000, threads: int = 1, **kw) -> dict:
    """Algorithm 1 from the uniform start until the relative balance residual of Eq. (1)
    (evaluated on P after the birth-death step of Eq. (10), every ``check_every``
    sweeps) is at most ``tol``: the stopping rule the GPU solver applies, here for
    timing the oracle end to end.  The dispatch-rate table is built and timed apart
    (the paper times coefficient generation separately).  threads as for ``Oracle``."""
    import time

    o = Oracle(inst, threads=threads, **kw)
    try:
        t0 = time.perf_counter()
        o.build_table()
        t_table = time.perf_counter() - t0
        t0 = time.perf_counter()
        o.init(None)
        sweeps, res = 0, float("inf")
        while sweeps < max_sweeps:
            k, _, _, _ = o.run(-1.0, 1e-20, min(check_every, max_sweeps - sweeps), 100000)
            sweeps += k
            res = float(o.results(with_R=False)["residual"])
            if res <= tol:
                break
        t_iter = time.perf_counter() - t0
        return {"sweeps": sweeps, "residual": res, "converged": res <= tol,
                "seconds_table": t_table, "seconds_iterate": t_iter}
    finally:
        o.close()


def birth_death(N, mode, C, lam, nu_sum, lam_n, mu_n):
    lib = _load(1)
    lam_n = np.ascontiguousarray(lam_n, dtype=np.float64)
    mu_n = np.ascontiguousarray(mu_n, dtype=np.float64)
    top = N + C if mode == FINITE else N
    pn = np.empty(top + 1)
    tail = ctypes.c_double(0.0)
    lib.or_birth_death(N, mode, C, lam, nu_sum, _p(lam_n, _pd), _p(mu_n, _pd), _p(pn, _pd),
                       ctypes.byref(tail))
    return pn, tail.value


def first_idle(pref_row, B: int) -> int:
    lib = _load(1)
    row = np.ascontiguousarray(pref_row, dtype=np.int32)
    return lib.or_first_idle(len(row), _p(row, _pi32), B)


def dispatch_rates(inst=None, src=None, u=None, **kw) -> np.ndarray:
    """lambda_{lm} of Eq. (3) for sampled (source state, unit) pairs."""
    lib = _load(1)
    N, J, lam_j, nu, pref, mode, C = _args(inst, **kw)
    src = np.ascontiguousarray(src, dtype=np.uint64)
    u = np.ascontiguousarray(u, dtype=np.int32)
    out = np.empty(len(src))
    lib.or_dispatch_rates_batch(N, J, _p(lam_j, _pd), _p(pref, _pi32), len(src), _p(src, _pu64),
                                _p(u, _pi32), _p(out, _pd))
    return out


def sampled_balance(inst, B, Pself, Pnb, pq1=0.0):
    """outflow and inflow of Eq. (1) at sampled states, neighbour P given by the caller."""
    lib = _load(1)
    N, J, lam_j, nu, pref, mode, C = _args(inst)
    B = np.ascontiguousarray(B, dtype=np.uint64)
    Pself = np.ascontiguousarray(Pself, dtype=np.float64)
    Pnb = np.ascontiguousarray(Pnb, dtype=np.float64)
    out = np.empty(len(B))
    inn = np.empty(len(B))
    lib.or_sampled_balance(N, J, _p(lam_j, _pd), _p(nu, _pd), _p(pref, _pi32), mode, len(B),
                           _p(B, _pu64), _p(Pself, _pd), _p(Pnb, _pd), float(pq1), _p(out, _pd),
                           _p(inn, _pd))
    return out, inn


# ---- discrete-event simulation of the loss system (des.c) -----------------------------

DES_KINDS = {"exponential": 0, "lognormal": 1, "gamma5": 2, "gamma05": 3, "uniform": 4}


def des_loss(inst=None, travel=None, kind: str | int = "exponential", reps: int = 20,
             arrivals: int = 100_000, warmup: int = 1000, seed: int = 1, **kw) -> dict:
    """Simulate the loss system (Section 5.5): per replication and unit the busy time in
    the window and the calls served, per replication the calls lost, the window length
    and the summed travel time of served calls; plus the estimates built from them
    (utilisation, loss probability, mean response time), averaged over replications."""
    lib = _load(1)
    N, J, lam_j, nu, pref, mode, C = _args(inst, **kw)
    travel = np.ascontiguousarray(travel if travel is not None else np.zeros((J, N)), dtype=np.float64)
    k = DES_KINDS[kind] if isinstance(kind, str) else int(kind)
    busy = np.empty((reps, N))
    served = np.empty((reps, N), dtype=np.int64)
    lost = np.empty(reps, dtype=np.int64)
    window = np.empty(reps)
    resp = np.empty(reps)
    _pi64 = ctypes.POINTER(ctypes.c_int64)
    rc = lib.or_des_loss(N, J, _p(lam_j, _pd), _p(nu, _pd), _p(pref, _pi32), _p(travel, _pd), k, reps,
                         arrivals, warmup, ctypes.c_uint64(seed), _p(busy, _pd), _p(served, _pi64),
                         _p(lost, _pi64), _p(window, _pd), _p(resp, _pd))
    if rc != 0:
        raise ValueError("oracle DES rejected its arguments")
    return des_summary(busy, served, lost, window, resp, arrivals - warmup)


def des_summary(busy, served, lost, window, resp, counted) -> dict:
    """Estimates from the per-replication totals, pooled over replications (ratios of
    sums, which carry no 1/window bias): utilisation = total busy time / total window,
    loss probability, mean response time = total travel time / calls served; standard
    errors from the spread of the per-replication ratios."""
    busy, window, resp = np.asarray(busy), np.asarray(window), np.asarray(resp)
    served, lost = np.asarray(served), np.asarray(lost)
    reps = busy.shape[0]
    nserved = served.sum(axis=1)
    util = busy.sum(axis=0) / window.sum()
    mrt = float(resp.sum() / max(int(nserved.sum()), 1))
    if reps > 1:
        se = (busy / window[:, None]).std(axis=0, ddof=1) / np.sqrt(reps)
        mrt_se = float((resp / np.maximum(nserved, 1)).std(ddof=1) / np.sqrt(reps))
    else:
        se, mrt_se = np.full(busy.shape[1], np.nan), float("nan")
    return dict(busy=busy, served=served, lost=lost, window=window, resp=resp, util=util, util_se=se,
                p_lost=float(lost.sum() / (reps * counted)), mrt=mrt, mrt_se=mrt_se)
