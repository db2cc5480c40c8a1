"""Failure paths, made to fire without faulting, trapping or hanging the GPU.

* A grid barrier that never completes: hq_opts.debug_barrier makes one CTA skip its
  first barrier arrival and shortens every bounded wait to 2^20 polls, so the waits give
  up, set the error word and the kernel runs to its end; the solve must return
  HQ_ETIMEOUT within seconds, and the next normal solve on the same handle must be right.
* A non-finite iterate: a given start vector holding a NaN must end in HQ_EDIVERGED.
"""
import time

import numpy as np
import pytest

import oracle
from paper_2603_03019_gb300 import hq
from paper_2603_03019_gb300 import instances as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("order", ["ascending", "redblack"])
@pytest.mark.parametrize("prec", ["fp64", "fp32+ir"])
def test_solve_barrier_timeout_then_recovers(gpu_lib, prec, order):
    inst = I.geometric_instance(14, 80, 91, 0.7, nu_lo=0.5, nu_hi=1.5)
    s = hq.Solver.for_instance(inst)
    t0 = time.time()
    with pytest.raises(hq.HQError) as e:
        s.solve(tol=1e-12, precision=prec, order=order, debug_barrier=3)
    assert e.value.code == hq.HQ_ETIMEOUT
    assert time.time() - t0 < 30.0
    rc, st = s.solve(tol=1e-12, precision=prec, order=order)
    assert rc == hq.HQ_OK, st
    r = oracle.solve(inst, eps=1e-15)
    assert np.max(np.abs(s.stationary() - r["P"])) < 1e-10
    s.close()


def test_batch_barrier_timeout_then_recovers(gpu_lib):
    insts = [I.geometric_instance(n, 20, 60 + n, 0.6, nu_lo=0.5, nu_hi=1.5) for n in (7, 9, 11)]
    ss = [hq.Solver.for_instance(i) for i in insts]
    b = hq.hq_batch_create([x.h for x in ss])
    o = hq.hq_default_opts()
    o.tol, o.tol_kind, o.precision = 1e-13, hq.HQ_TOL_STEP, hq.HQ_PREC_FP64
    o.debug_barrier = 2
    t0 = time.time()
    with pytest.raises(hq.HQError) as e:
        hq.hq_batch_solve(b, len(insts), o)
    assert e.value.code == hq.HQ_ETIMEOUT
    assert time.time() - t0 < 30.0
    o.debug_barrier = 0
    rc, st, _ = hq.hq_batch_solve(b, len(insts), o)
    assert rc == hq.HQ_OK
    for x, i in zip(ss, insts):
        assert np.max(np.abs(x.stationary() - oracle.solve(i, eps=1e-15)["P"])) < 1e-10
    hq.hq_batch_destroy(b)
    for x in ss:
        x.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32+ir"])
def test_nan_start_diverges(gpu_lib, prec):
    inst = I.geometric_instance(10, 30, 93, 0.7, nu_lo=0.5, nu_hi=1.5)
    s = hq.Solver.for_instance(inst)
    warm = np.full(1 << inst.N, 0.01)
    warm[0b0000011110] = np.nan
    with pytest.raises(hq.HQError) as e:
        s.solve(tol=1e-12, precision=prec, warm_p=warm)
    assert e.value.code == hq.HQ_EDIVERGED
    rc, st = s.solve(tol=1e-12, precision=prec)
    assert rc == hq.HQ_OK
    s.close()
