"""Pins of the discrete-event simulation oracle (oracle/des.c), no GPU.

The simulation is pinned to what the mathematics fixes, not to itself: the M/M/1/1 loss
probability, the Erlang-B loss probability of N identical units under every service
distribution (insensitivity of the M/G/N/N loss system), the exact stationary solution
of the hypercube model (solved by the oracle's Algorithm 1, a different code path) for
the utilisations and the mean response time (exact for exponential service, approximate
for the other shapes as Section 5.5 reports), and the first two moments of each service
sampler against its distribution's closed form.  Statistical checks use the standard
error across replications with a margin of 5 (the sizes keep each test to seconds).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2603_03019_gb300 import instances as I

KINDS = ["exponential", "lognormal", "gamma5", "gamma05", "uniform"]


def _erlang_b(n: int, a: float) -> float:
    b = 1.0
    for k in range(1, n + 1):
        b = a * b / (k + a * b)
    return b


def _hom_instance(N, J, load, seed=3):
    """N identical units (nu = 1); any preference lists."""
    r = np.random.default_rng(seed)
    lam_j = r.dirichlet(np.ones(J)) * load * N
    pref = np.array([r.permutation(N) for _ in range(J)], dtype=np.int32)
    return dict(N=N, J=J, lam_j=lam_j, nu=np.ones(N), pref=pref, mode=oracle.LOSS, C=0)


def test_mm11_loss_probability():
    """One unit, one node: P(lost) = rho / (1 + rho), utilisation the same (M/M/1/1)."""
    inst = dict(N=1, J=1, lam_j=np.array([0.7]), nu=np.array([1.3]), pref=np.zeros((1, 1), np.int32),
                mode=oracle.LOSS, C=0)
    r = oracle.des_loss(travel=np.ones((1, 1)), kind="exponential", reps=16, arrivals=50_000, warmup=100,
                        seed=11, **inst)
    rho = 0.7 / 1.3
    want = rho / (1 + rho)
    lost = r["lost"] / (50_000 - 100)
    se = lost.std(ddof=1) / math.sqrt(16)
    assert abs(lost.mean() - want) < 5 * se + 1e-3, (lost.mean(), want, se)
    assert abs(r["util"][0] - want) < 5 * r["util_se"][0] + 1e-3
    assert r["mrt"] == pytest.approx(1.0)


@pytest.mark.parametrize("kind", KINDS)
def test_erlang_b_under_every_service_distribution(kind):
    """N = 4 identical units: the number busy is Erlang-B whatever the service shape, so
    the loss probability is B(4, a) with a = lambda / nu."""
    inst = _hom_instance(4, 6, 0.6)
    a = float(inst["lam_j"].sum())
    r = oracle.des_loss(travel=np.zeros((6, 4)), kind=kind, reps=16, arrivals=40_000, warmup=500, seed=7,
                        **inst)
    lost = r["lost"] / (40_000 - 500)
    se = lost.std(ddof=1) / math.sqrt(16)
    want = _erlang_b(4, a)
    assert abs(lost.mean() - want) < 5 * se + 2e-3, (kind, lost.mean(), want, se)
    # with identical units the mean number busy is a (1 - B)
    assert abs(r["util"].sum() - a * (1 - want)) < 5 * math.sqrt((r["util_se"] ** 2).sum()) + 5e-3


@pytest.mark.parametrize("kind", KINDS)
def test_against_the_exact_solution(kind):
    """Heterogeneous units (N = 6, nu ~ U[0.8, 1.2]) with distance-ordered preference
    lists: utilisations and the mean response time of the simulation against the exact
    stationary solution of the exponential model (the oracle's Algorithm 1 to 1e-13).
    Exact for exponential service; for the other shapes the agreement is the approximate
    insensitivity Section 5.5 reports, well inside these 5-standard-error-plus-2e-3
    margins at this size."""
    inst = I.des_instance(515, N=6, load=0.5, J=20)
    tt = I.travel_times(inst)
    ex = oracle.solve(inst, eps=1e-13)
    r = oracle.des_loss(inst, travel=tt, kind=kind, reps=16, arrivals=60_000, warmup=500, seed=23)
    assert np.all(np.abs(r["util"] - ex["rho"]) < 5 * r["util_se"] + 2e-3), (kind, r["util"], ex["rho"])
    served = ex["R"] * inst.lam_j[:, None]
    mrt = float((served * tt).sum() / served.sum())
    assert abs(r["mrt"] - mrt) < 5 * r["mrt_se"] + 2e-3, (kind, r["mrt"], mrt)
    assert abs(r["p_lost"] - ex["p_block"]) < 5e-3


@pytest.mark.parametrize("kind,var_over_m2", [("exponential", 1.0), ("lognormal", 1.0), ("gamma5", 0.2),
                                              ("gamma05", 2.0), ("uniform", 1.0 / 3.0)])
def test_service_sampler_moments(kind, var_over_m2):
    """Mean m and variance of each service distribution (Section 5.5 sets every mean to
    1/nu_i): exponential m^2, log-normal with the exponential's variance m^2, gamma of
    shape 5 m^2/5, gamma of shape 1/2 2 m^2, uniform on [0, 2m] m^2/3."""
    lib = oracle._load(1)
    m = 0.8
    k = oracle.DES_KINDS[kind]
    n = 200_000
    x = np.array([lib.or_des_service(k, m, 0x1234 + 77 * i, 8 * i + 2) for i in range(n)])
    assert np.all(x >= 0)
    assert abs(x.mean() - m) < 5 * x.std() / math.sqrt(n), (kind, x.mean())
    # the sample variance's standard error needs the fourth moment: use the sample's own
    v = x.var()
    se_v = math.sqrt(max(((x - x.mean()) ** 4).mean() - v * v, 0.0) / n)
    assert abs(v - var_over_m2 * m * m) < 5 * se_v, (kind, v, var_over_m2 * m * m)


def test_uniforms_are_in_the_open_unit_interval_and_independent_of_schedule():
    """The counter-based stream: every draw in (0, 1], the same value whatever else was
    drawn before (a function of seed, replication and counter only), and distinct
    replications give distinct streams."""
    lib = oracle._load(1)
    a = [lib.or_des_uniform(9, 3, c) for c in range(1000)]
    b = [lib.or_des_uniform(9, 3, c) for c in reversed(range(1000))][::-1]
    assert a == b
    assert all(0.0 < u <= 1.0 for u in a)
    c = [lib.or_des_uniform(9, 4, c) for c in range(1000)]
    assert a != c
    assert abs(np.mean(a) - 0.5) < 5 * math.sqrt(1 / 12 / 1000)


def test_series_functions_are_accurate():
    """The FP32 logarithm, exponential and cosine the simulation forms its variates with,
    against numpy's FP64 functions over their whole input ranges: ln over the uniforms'
    range (2^-120, 1] and the means, e^y for |y| <= 20, cos(2 pi u) on [0, 1].  A dropped
    series term or a wrong constant costs orders of magnitude more than these bounds."""
    lib = oracle._load(1)
    r = np.random.default_rng(5)
    xs = np.concatenate([np.exp2(-r.uniform(0, 120, 4000)), r.uniform(0, 1, 4000), r.uniform(0.05, 20, 500),
                         [2.0 ** -24, 0.5, 1.0, np.sqrt(0.5), np.sqrt(2.0)]]).astype(np.float32)
    ln = np.array([lib.or_des_ln(float(x)) for x in xs])
    want = np.log(xs.astype(np.float64))
    err = np.abs(ln - want) / np.maximum(np.abs(want), 1e-30)
    assert np.max(err[np.abs(want) > 1e-3]) < 5e-7
    assert np.max(np.abs(ln - want)) < 1e-7 * 84
    assert lib.or_des_ln(1.0) == 0.0
    ys = np.concatenate([r.uniform(-20, 20, 4000), [0.0, -0.3466, 0.3466]]).astype(np.float32)
    ex = np.array([lib.or_des_exp(float(y)) for y in ys])
    assert np.max(np.abs(ex / np.exp(ys.astype(np.float64)) - 1.0)) < 5e-7
    assert lib.or_des_exp(0.0) == 1.0
    us = np.concatenate([r.uniform(0, 1, 4000), np.arange(9) / 8.0]).astype(np.float32)
    co = np.array([lib.or_des_cos2pi(float(u)) for u in us])
    assert np.max(np.abs(co - np.cos(2 * np.pi * us.astype(np.float64)))) < 2e-7
    assert lib.or_des_cos2pi(0.0) == 1.0 and lib.or_des_cos2pi(0.5) == -1.0


def test_summary_pools_ratios_of_sums_by_hand():
    """Two replications worked by hand: utilisation is total busy / total window (not
    the mean of the per-replication ratios), the mean response time total travel /
    total served, the loss probability total lost / total counted; the standard errors
    come from the per-replication ratios (two values a, b: |a - b| / 2)."""
    e = oracle.des_summary(busy=[[1.0, 2.0], [3.0, 4.0]], served=[[1, 1], [2, 0]], lost=[1, 3],
                           window=[10.0, 30.0], resp=[5.0, 9.0], counted=10)
    assert e["util"] == pytest.approx([0.1, 0.15], abs=1e-15)
    assert e["mrt"] == pytest.approx(3.5, abs=1e-15)
    assert e["p_lost"] == pytest.approx(0.2, abs=1e-15)
    assert e["util_se"] == pytest.approx([0.0, (0.2 - 4.0 / 30.0) / 2], abs=1e-15)
    assert e["mrt_se"] == pytest.approx(1.0, abs=1e-15)
