"""Batched solves (hq_batch_*) against the CPU oracle and the one-instance solver.

A batch runs Algorithm 1 on instances of uneven N in one persistent launch per check;
each instance must come out as if it had been solved alone: against the oracle to
1e-10 max-abs on P, rho, R, W (converged FP64 / DF64 / FP32+DF64 forms, stopped on the
step), bitwise equal to the same instance batched with other company (FP64: the fold
of an instance's partials does not depend on what else is in the batch), and within
1e-13 of the one-instance kernel after the same number of sweeps (the two kernels fold
their partial sums in different orders).
"""
import numpy as np
import pytest

import oracle
from paper_2603_03019_gb300 import hq
from paper_2603_03019_gb300 import instances as I

pytestmark = pytest.mark.gpu

MIXED = [(5, 9, 0, 0, 21), (7, 20, 1, 3, 22), (9, 33, 2, 0, 23), (11, 40, 0, 0, 24),
         (12, 60, 0, 0, 25), (13, 64, 2, 0, 26)]


def _instances(cases=MIXED, load=0.7):
    return [I.geometric_instance(N, J, seed, load, nu_lo=0.5, nu_hi=1.5, mode=mode, C=C)
            for N, J, mode, C, seed in cases]


def _opts(prec, tol, max_sweeps=100000, check_every=8, omega=1.0):
    o = hq.hq_default_opts()
    o.omega = omega
    o.tol = tol
    o.tol_kind = hq.HQ_TOL_STEP
    o.precision = hq.PRECISION[prec]
    o.max_sweeps = max_sweeps
    o.check_every = check_every
    return o


def _batch_solve(insts, prec, tol, **kw):
    solvers = [hq.Solver.for_instance(i) for i in insts]
    b = hq.hq_batch_create([s.h for s in solvers])
    rc, stats, ms = hq.hq_batch_solve(b, len(insts), _opts(prec, tol, **kw))
    info = hq.hq_batch_info(b)
    out = []
    for s in solvers:
        out.append(dict(P=s.stationary(), cond=s.conditional(), rho=s.utilisation(),
                        R=s.response_pattern(), W=s.workload(), summary=s.summary()))
    hq.hq_batch_destroy(b)
    for s in solvers:
        s.close()
    return rc, stats, out, info


@pytest.mark.parametrize("prec,tol,omega", [("fp64", 1e-14, 1.0), ("df64", 1e-13, 1.0),
                                            ("fp32+df64", 1e-13, 1.0), ("fp64", 1e-14, -1.0),
                                            ("fp32+df64", 1e-13, -1.0)])
def test_batch_matches_oracle(gpu_lib, prec, tol, omega):
    insts = _instances()
    rc, stats, out, info = _batch_solve(insts, prec, tol, omega=omega)
    assert rc == hq.HQ_OK, stats
    assert info[0] == len(insts) and info[1] == 13
    assert info[4] in (1, -1)  # checks replayed a captured graph, or launched directly
    for inst, g, st in zip(insts, out, stats):
        assert st["converged"] == 1
        r = oracle.solve(inst, eps=1e-15)
        assert np.max(np.abs(g["P"] - r["P"])) < 1e-10, inst.name
        assert np.max(np.abs(g["rho"] - r["rho"])) < 1e-10
        assert np.max(np.abs(g["R"] - r["R"])) < 1e-10
        assert np.max(np.abs(g["W"] - r["W"])) < 1e-10
        assert abs(g["summary"]["throughput"] - r["throughput"]) < 1e-10
        assert st["final_residual"] < 1e-10


def test_batch_after_reloading_its_solvers(gpu_lib):
    """The solvers of a batch are loaded with other instances of the same sizes after the
    batch was made (the double-float tables are made on first use after every load): a
    double-float batched solve then matches the oracle on the new instances."""
    first = _instances()
    second = _instances(load=0.5)
    solvers = [hq.Solver.for_instance(i) for i in first]
    b = hq.hq_batch_create([s.h for s in solvers])
    rc, stats, _ = hq.hq_batch_solve(b, len(first), _opts("fp32+df64", 1e-13))
    assert rc == hq.HQ_OK
    for s, inst in zip(solvers, second):
        s.load(inst.lam_j, inst.nu, inst.pref)
    rc, stats, _ = hq.hq_batch_solve(b, len(second), _opts("df64", 1e-13))
    assert rc == hq.HQ_OK, stats
    for s, inst in zip(solvers, second):
        r = oracle.solve(inst, eps=1e-15)
        assert np.max(np.abs(s.stationary() - r["P"])) < 1e-10, inst.name
    hq.hq_batch_destroy(b)
    for s in solvers:
        s.close()


def test_batch_independent_of_company(gpu_lib):
    """FP64: an instance's result does not depend on the other instances of its batch."""
    insts = _instances()
    rc_all, st_all, out_all, _ = _batch_solve(insts, "fp64", 1e-13)
    for k in (0, 4):
        rc_one, st_one, out_one, _ = _batch_solve([insts[k]], "fp64", 1e-13)
        assert st_one[0]["sweeps_hi"] == st_all[k]["sweeps_hi"]
        assert np.array_equal(out_one[0]["P"], out_all[k]["P"])


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("df64", 1e-12)])
def test_batch_fixed_sweeps_match_single_kernel(gpu_lib, prec, tol):
    insts = _instances()
    rc, stats, out, _ = _batch_solve(insts, prec, 0.0, max_sweeps=3, check_every=3)
    assert rc == hq.HQ_ENOTCONVERGED
    for inst, g, st in zip(insts, out, stats):
        assert st["sweeps_hi"] == 3
        s = hq.Solver.for_instance(inst)
        s.solve(tol=0.0, tol_kind=hq.HQ_TOL_STEP, precision=prec, max_sweeps=3, check_every=3)
        ref = s.conditional()
        s.close()
        assert np.max(np.abs(g["cond"] - ref)) < tol, inst.name


def test_batch_tune_and_uneven_n12_18(gpu_lib):
    """32 deployments with N drawn from 12..18 (the batched workload's generator)."""
    insts = I.batch_n12_18(count=32)
    solvers = [hq.Solver.for_instance(i) for i in insts]
    b = hq.hq_batch_create([s.h for s in solvers])
    for prec in (hq.HQ_PREC_FP32, hq.HQ_PREC_DF64):
        v, ms = hq.hq_batch_tune(b, prec, 2)
        assert 0 <= v < 4 and np.all(ms > 0)
    info = hq.hq_batch_info(b)
    assert info[0] == 32 and 12 <= info[1] <= 18
    assert info[2] == sum((1 << i.N) - 2 for i in insts)
    rc, stats, ms = hq.hq_batch_solve(b, 32, _opts("fp32+df64", 1e-11))
    assert rc == hq.HQ_OK
    assert all(st["converged"] == 1 and st["sweeps_hi"] > 0 for st in stats)
    # the smallest instances against the oracle
    small = sorted(range(32), key=lambda c: insts[c].N)[:2]
    for c in small:
        r = oracle.solve(insts[c], eps=1e-14)
        assert np.max(np.abs(solvers[c].stationary() - r["P"])) < 1e-9, insts[c].name
        assert np.max(np.abs(solvers[c].utilisation() - r["rho"])) < 1e-9
    hq.hq_batch_destroy(b)
    for s in solvers:
        s.close()


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_batch_every_cta_shape_matches_oracle(gpu_lib, variant):
    """Each kernel variant the autotuner may pick (threads per CTA x CTAs per SM) solves
    the mixed batch to the oracle's answer."""
    insts = _instances()
    solvers = [hq.Solver.for_instance(i) for i in insts]
    b = hq.hq_batch_create([s.h for s in solvers])
    for prec in (hq.HQ_PREC_FP32, hq.HQ_PREC_DF64, hq.HQ_PREC_FP64):
        hq.hq_batch_set_variant(b, prec, variant)
    info = hq.hq_batch_info(b)
    assert list(info[5:8]) == [variant] * 3
    rc, stats, _ = hq.hq_batch_solve(b, len(insts), _opts("fp32+df64", 1e-13))
    assert rc == hq.HQ_OK
    for inst, s, st in zip(insts, solvers, stats):
        assert st["converged"] == 1
        r = oracle.solve(inst, eps=1e-15)
        assert np.max(np.abs(s.stationary() - r["P"])) < 1e-10, inst.name
    with pytest.raises(hq.HQError):
        hq.hq_batch_set_variant(b, hq.HQ_PREC_FP32, 4)
    hq.hq_batch_destroy(b)
    for s in solvers:
        s.close()


def test_batch_errors(gpu_lib):
    inst = _instances()[0]
    unloaded = hq.Solver(inst.N, inst.J, inst.mode, inst.C)
    with pytest.raises(hq.HQError) as e:
        hq.hq_batch_create([unloaded.h])
    assert e.value.code == hq.HQ_ESTATE
    unloaded.close()
    s = hq.Solver.for_instance(inst)
    b = hq.hq_batch_create([s.h])
    o = _opts("fp64", 1e-10)
    o.tol_kind = hq.HQ_TOL_RESIDUAL
    with pytest.raises(hq.HQError) as e:
        hq.hq_batch_solve(b, 1, o)
    assert e.value.code == hq.HQ_EINVAL
    with pytest.raises(hq.HQError):
        hq.hq_batch_create([])
    hq.hq_batch_destroy(b)
    s.close()
