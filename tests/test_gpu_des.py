"""The GPU discrete-event simulation (hq_des_simulate) against the CPU oracle's
simulation of the same replications, and against the exact stationary solution
(Section 5.5: the loss system's insensitivity to the service distribution)."""
import math

import numpy as np
import pytest

import oracle
from paper_2603_03019_gb300 import hq
from paper_2603_03019_gb300 import instances as I

pytestmark = pytest.mark.gpu

KINDS = ["exponential", "lognormal", "gamma5", "gamma05", "uniform"]


@pytest.mark.parametrize("kind", KINDS)
def test_replications_match_the_oracle(gpu_lib, kind):
    """Same seed, same counter-based streams, the same IEEE steps for every variate (the
    FP32 series functions are written out on both sides): every replication's integer
    counts are equal and its times agree to rounding."""
    inst = I.des_instance(4242, N=10, load=0.7)
    tt = I.travel_times(inst)
    reps, arr, warm, seed = 40, 20_000, 500, 99
    g = hq.hq_des_simulate(inst.N, inst.J, inst.lam_j, inst.nu, inst.pref, tt, kind, reps, arr, warm, seed)
    r = oracle.des_loss(inst, travel=tt, kind=kind, reps=reps, arrivals=arr, warmup=warm, seed=seed)
    assert np.array_equal(g["served"], r["served"])
    assert np.array_equal(g["lost"], r["lost"])
    for k in ("busy", "window", "resp"):
        assert np.allclose(g[k], r[k], rtol=1e-11, atol=0), (k, np.max(np.abs(g[k] - r[k])))


def test_device_inputs_and_ragged_sizes(gpu_lib):
    """Device tensors in and out; a replication count that is not a multiple of the
    block; N = 1 and J = 1; the smallest window (warmup = arrivals - 2)."""
    import torch

    dev = torch.device("cuda", 0)
    inst = I.des_instance(77, N=8, load=0.4, J=13)
    tt = I.travel_times(inst)
    args = [torch.tensor(inst.lam_j, device=dev), torch.tensor(inst.nu, device=dev),
            torch.tensor(inst.pref, device=dev), torch.tensor(tt, device=dev)]
    g = hq.hq_des_simulate(inst.N, inst.J, *args, "gamma5", 67, 3000, 2998, 5)
    r = oracle.des_loss(inst, travel=tt, kind="gamma5", reps=67, arrivals=3000, warmup=2998, seed=5)
    assert np.array_equal(g["served"].cpu().numpy(), r["served"])
    assert np.allclose(g["busy"].cpu().numpy(), r["busy"], rtol=1e-11, atol=1e-13)
    one = dict(lam_j=np.array([0.5]), nu=np.array([2.0]), pref=np.zeros((1, 1), np.int32))
    g1 = hq.hq_des_simulate(1, 1, one["lam_j"], one["nu"], one["pref"], np.ones((1, 1)), 0, 5, 1000, 10, 3)
    r1 = oracle.des_loss(N=1, J=1, mode=oracle.LOSS, C=0, travel=np.ones((1, 1)), kind=0, reps=5,
                         arrivals=1000, warmup=10, seed=3, **one)
    assert np.array_equal(g1["lost"], r1["lost"])
    assert np.allclose(g1["busy"], r1["busy"], rtol=1e-11)


def test_largest_n_and_more_nodes_than_guide_ranges(gpu_lib):
    """N = 32 (the largest the simulation takes) and J = 3,000 nodes, more than the
    1,024 ranges of the node search's guide table, so several nodes share a range and
    the search walks past its first candidate; some nodes have zero demand.  Counts
    equal to the oracle's, times to rounding."""
    inst = I.des_instance(3232, N=32, load=0.8, J=3000)
    lam = inst.lam_j.copy()
    lam[::7] = 0.0
    lam *= inst.lam_j.sum() / lam.sum()
    tt = I.travel_times(inst)
    for kind in ("lognormal", "gamma5"):
        g = hq.hq_des_simulate(inst.N, inst.J, lam, inst.nu, inst.pref, tt, kind, 33, 4000, 300, 8)
        r = oracle.des_loss(N=inst.N, J=inst.J, mode=oracle.LOSS, C=0, lam_j=lam, nu=inst.nu, pref=inst.pref,
                            travel=tt, kind=kind, reps=33, arrivals=4000, warmup=300, seed=8)
        assert np.array_equal(g["served"], r["served"])
        assert np.array_equal(g["lost"], r["lost"])
        for k in ("busy", "window", "resp"):
            assert np.allclose(g[k], r[k], rtol=1e-11, atol=0), (kind, k)


@pytest.mark.parametrize("kind", KINDS)
def test_against_the_gpu_solution(gpu_lib, kind):
    """N = 12, load 0.7: 2,048 replications of 20,000 calls against the hypercube
    solution solved on the GPU (FP64, 1e-12 residual).  Exponential service: the solution
    is exact, so utilisations, loss probability and mean response time agree within 5
    standard errors (plus 1e-3 for the start-up bias).  Other shapes: with unit-dependent
    dispatch the loss system is insensitive only approximately; Section 5.5 reports
    errors below 1.4 % for utilisation and 0.08 % (mean) for MRT, which is the bound held
    here (1.4 % per unit, 0.2 % for MRT)."""
    inst = I.des_instance(1212, N=12, load=0.7)
    tt = I.travel_times(inst)
    s = hq.Solver.for_instance(inst)
    rc, st = s.solve(tol=1e-12, precision="fp64")
    assert rc == hq.HQ_OK
    rho, R, summ = s.utilisation(), s.response_pattern(), s.summary()
    s.close()
    reps, arr, warm = 2048, 20_000, 1000
    g = hq.hq_des_simulate(inst.N, inst.J, inst.lam_j, inst.nu, inst.pref, tt, kind, reps, arr, warm, 31)
    e = oracle.des_summary(g["busy"], g["served"], g["lost"], g["window"], g["resp"], arr - warm)
    served = R.reshape(inst.J, inst.N) * inst.lam_j[:, None]
    mrt = float((served * tt).sum() / served.sum())
    lost = g["lost"] / (arr - warm)
    if kind == "exponential":
        assert np.all(np.abs(e["util"] - rho) < 5 * e["util_se"] + 1e-3), (e["util"] - rho, e["util_se"])
        assert abs(e["mrt"] - mrt) < 5 * e["mrt_se"] + 1e-3
        assert abs(lost.mean() - summ["p_block"]) < 5 * lost.std(ddof=1) / math.sqrt(reps) + 1e-3
    else:
        assert np.all(np.abs(e["util"] - rho) / e["util"] < 0.014), (kind, (e["util"] - rho) / e["util"])
        assert abs(e["mrt"] - mrt) / e["mrt"] < 0.002, (kind, e["mrt"], mrt)


def test_errors(gpu_lib):
    inst = I.des_instance(5, N=4, load=0.5, J=6)
    tt = I.travel_times(inst)
    bad = inst.pref.copy()
    bad[2, 1] = bad[2, 0]
    for args in ((bad, 0, 10, 1000, 10), (inst.pref, 5, 10, 1000, 10), (inst.pref, 0, 10, 1000, 999),
                 (inst.pref, 0, 0, 1000, 10)):
        with pytest.raises(hq.HQError) as ex:
            hq.hq_des_simulate(inst.N, inst.J, inst.lam_j, inst.nu, args[0], tt, args[1], args[2], args[3],
                               args[4], 1)
        assert ex.value.code == hq.HQ_EINVAL
    # rates outside [2^-60, 2^60]: a unit's and the total
    tiny_nu = inst.nu.copy()
    tiny_nu[1] = 2.0 ** -61
    for lam, nu in ((inst.lam_j, tiny_nu), (inst.lam_j * 2.0 ** -70, inst.nu)):
        with pytest.raises(hq.HQError) as ex:
            hq.hq_des_simulate(inst.N, inst.J, lam, nu, inst.pref, tt, 1, 10, 1000, 10, 1)
        assert ex.value.code == hq.HQ_EINVAL
