"""Pins of the CPU oracle against facts the paper and the mathematics fix.

Nothing here retypes the oracle's formulas: each expected value comes from a hand
derivation (tests/golden), a textbook closed form (Erlang), an exact special case
of the model, an invariant the paper proves, or the independent dense solve of
Eq. (1)-(2) -- which is itself pinned by the same closed forms below.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle.dense import dense_solve
from paper_2603_03019_gb300 import instances as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _inst(N, J, lam_j, nu, pref, mode=0, C=0):
    return I.Instance(N=N, J=J, lam_j=np.asarray(lam_j, float), nu=np.asarray(nu, float),
                      pref=np.asarray(pref, np.int32), mode=mode, C=C)


def _load_golden_n2():
    rows, nu, lam, pref = [], None, None, []
    with open(os.path.join(GOLDEN, "n2_two_nodes.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            t = line.split()
            if t[0] == "nu":
                nu = [float(x) for x in t[1:]]
            elif t[0] == "lam_j":
                lam = [float(x) for x in t[1:]]
            elif t[0] == "pref":
                pref.append([int(x) for x in t[1:]])
            else:
                rows.append((int(t[0]), Fraction(int(t[1]), int(t[2]))))
    return nu, lam, pref, rows


# ---- exact small cases ------------------------------------------------------------------

def test_golden_n2_hand_derived_oracle_and_dense():
    """Hand-derived 2-unit, 2-node solution (Eq. 1-3) -- pins the first-idle rule and
    the iteration: a swapped preference or transposed rate changes these fractions."""
    nu, lam, pref, rows = _load_golden_n2()
    inst = _inst(2, 2, lam, nu, pref)
    expect = np.zeros(4)
    for y, fr in rows:
        expect[y] = float(fr)
    r = oracle.solve(inst, eps=1e-15)
    d = dense_solve(inst)
    assert np.max(np.abs(r["P"] - expect)) < 1e-14
    assert np.max(np.abs(d["P"] - expect)) < 1e-15


def test_single_unit_is_mm1():
    """N=1: M/M/1/1 (loss), M/M/1/1+C (finite), M/M/1 (infinite)."""
    lam, nu = 0.7, 1.3
    r = lam / nu
    loss = oracle.solve(_inst(1, 1, [lam], [nu], [[0]]), eps=1e-15)
    assert abs(loss["P"][1] - lam / (lam + nu)) < 1e-15
    C = 4
    fin = oracle.solve(_inst(1, 1, [lam], [nu], [[0]], mode=1, C=C), eps=1e-15)
    z = sum(r ** k for k in range(C + 2))
    assert np.allclose(fin["pn"], [r ** k / z for k in range(C + 2)], rtol=1e-14, atol=0)
    inf = oracle.solve(_inst(1, 1, [lam], [nu], [[0]], mode=2), eps=1e-15)
    assert abs(inf["P"][0] - (1 - r)) < 1e-15
    assert abs(inf["P"][1] - (1 - r) * r) < 1e-15
    assert abs(inf["queue_tail"] - r * r) < 1e-15


@pytest.mark.parametrize("seed", [11, 12])
def test_common_first_choice_unit_is_mm11(seed):
    """If every node ranks the same unit first, that unit alternates idle (rate lambda)
    and busy (rate nu_u) whatever the others do: rho_u = lambda/(lambda+nu_u), any nu."""
    inst = I.geometric_instance(7, 15, seed, 0.6, nu_lo=0.4, nu_hi=2.0)
    u0 = int(inst.pref[0, 0])
    pref = inst.pref.copy()
    for j in range(inst.J):
        row = [u0] + [int(x) for x in pref[j] if x != u0]
        pref[j] = row
    inst.pref = pref
    r = oracle.solve(inst, eps=1e-14)
    assert abs(r["rho"][u0] - inst.lam / (inst.lam + inst.nu[u0])) < 1e-12


def test_ordered_hunting_prefix_matches_n2():
    """One node, ordered hunting 0,1,2,...: units 0 and 1 alone form the 2-unit system
    of the golden derivation with lam_b = 0 (later units never affect them)."""
    nu = [1.0, 2.0, 0.7, 1.4, 0.9]
    lam = 2.5
    inst = _inst(5, 1, [lam], nu, [[0, 1, 2, 3, 4]])
    r = oracle.solve(inst, eps=1e-15)
    P = r["P"]
    y = np.arange(32)
    both = P[(y & 3) == 3].sum()
    nu1, nu2, S = 1.0, 2.0, 3.0
    w = nu1 * nu2 * (2 * lam + S)
    x = nu2 * (lam ** 2 + S * lam)
    yv = nu1 * (lam ** 2)
    z = lam * (lam ** 2 + nu2 * lam)
    assert abs(both - z / (w + x + yv + z)) < 1e-13


# ---- homogeneous closed forms (Corollary; Erlang) -------------------------------------

def _erlang_b_dist(N, a):
    t = [Fraction(a) ** k / math.factorial(k) for k in range(N + 1)]
    z = sum(t)
    return [float(x / z) for x in t]


@pytest.mark.parametrize("N,load", [(4, 0.3), (7, 0.8), (9, 1.4)])
def test_homogeneous_loss_layers_are_erlang_b(N, load):
    inst = I.homogeneous_instance(N, 12, 5, load, nu=1.0)
    a = Fraction(inst.lam).limit_denominator(10 ** 12)
    r = oracle.solve(inst, eps=1e-14)
    expect = _erlang_b_dist(N, inst.lam)
    assert np.max(np.abs(r["pn"] - expect)) < 1e-13
    d = dense_solve(inst)
    layer = np.array([bin(v).count("1") for v in range(1 << N)])
    dl = np.array([d["P"][layer == n].sum() for n in range(N + 1)])
    assert np.max(np.abs(dl - expect)) < 1e-13
    del a


def test_homogeneous_finite_buffer_is_mmn_nc():
    N, C, nu = 5, 3, 1.0
    inst = I.homogeneous_instance(N, 9, 8, 0.9, nu=nu, mode=1, C=C)
    a = inst.lam / nu
    t = [a ** k / math.factorial(k) for k in range(N + 1)]
    t += [t[N] * (a / N) ** c for c in range(1, C + 1)]
    z = sum(t)
    expect = np.array(t) / z
    r = oracle.solve(inst, eps=1e-14)
    assert np.max(np.abs(r["pn"] - expect)) < 1e-13
    d = dense_solve(inst)
    assert np.max(np.abs(d["Pq"] - expect[N + 1:])) < 1e-13


def test_homogeneous_infinite_is_erlang_c():
    N, nu = 6, 1.0
    inst = I.homogeneous_instance(N, 10, 9, 0.85, nu=nu, mode=2)
    a = inst.lam / nu
    rho = a / N
    t = [a ** k / math.factorial(k) for k in range(N)]
    tN = a ** N / math.factorial(N)
    p0 = 1.0 / (sum(t) + tN / (1 - rho))
    r = oracle.solve(inst, eps=1e-14)
    assert abs(r["pn"][0] - p0) < 1e-13
    # Erlang-C waiting probability = P(all busy) / (1 - rho)
    assert abs(r["q_wait"] - p0 * tN / (1 - rho)) < 1e-13
    d = dense_solve(inst)
    assert abs(d["queue_tail"] - r["queue_tail"]) < 1e-13


def test_homogeneous_contraction_bound():
    """Corollary: with equal rates the layer-sup L1 step M_k contracts at least by
    Phi_N = 1 - prod(j nu) / prod(lambda + j nu)."""
    N, nu = 4, 1.0
    inst = I.homogeneous_instance(N, 6, 21, 0.1, nu=nu)
    lam = inst.lam
    phi = 1.0 - np.prod([j * nu for j in range(1, N + 1)]) / np.prod(
        [lam + j * nu for j in range(1, N + 1)])
    r = oracle.solve(inst, eps=1e-15, max_sweeps=200)
    M = r["trace_l1"]
    checked = 0
    for k in range(1, len(M)):
        if M[k - 1] > 1e-12:
            assert M[k] <= phi * M[k - 1] * (1 + 1e-9) + 1e-15
            checked += 1
    assert checked >= 3


# ---- heterogeneous: dense solve of Eq. (1)-(2) ----------------------------------------

@pytest.mark.parametrize("N,J,mode,C,seed", [
    (3, 4, 0, 0, 1), (5, 9, 0, 0, 2), (6, 20, 1, 2, 3), (7, 30, 2, 0, 4), (9, 40, 0, 0, 5),
    (8, 25, 1, 5, 6), (9, 12, 2, 0, 7)])
def test_oracle_matches_dense_solve(N, J, mode, C, seed):
    inst = I.geometric_instance(N, J, seed, 0.7, nu_lo=0.5, nu_hi=1.5, mode=mode, C=C)
    r = oracle.solve(inst, eps=1e-14)
    d = dense_solve(inst)
    assert r["converged"]
    assert np.max(np.abs(r["P"] - d["P"])) < 1e-12
    if mode == 1:
        assert np.max(np.abs(r["pn"][N + 1:] - d["Pq"])) < 1e-12
    if mode == 2:
        assert abs(r["queue_tail"] - d["queue_tail"]) < 1e-12


def test_small_loss_n10_within_1e10_of_dense():
    inst = I.small_loss_n10(1001)
    r = oracle.solve(inst, eps=1e-12)
    d = dense_solve(inst)
    assert np.max(np.abs(r["P"] - d["P"])) < 1e-10
    assert r["residual"] < 1e-10


def test_mutated_preferences_are_detected():
    """A transposed operand (nodes' lists reversed) must break agreement with the
    dense solve: the comparison above is sensitive to the dispatch rule."""
    inst = I.geometric_instance(6, 10, 3, 0.7, nu_lo=0.5, nu_hi=1.5)
    d = dense_solve(inst)
    bad = I.Instance(N=inst.N, J=inst.J, lam_j=inst.lam_j, nu=inst.nu,
                     pref=inst.pref[:, ::-1].copy())
    r = oracle.solve(bad, eps=1e-14)
    assert np.max(np.abs(r["P"] - d["P"])) > 1e-4


# ---- invariants the paper proves ------------------------------------------------------

def test_dispatch_rates_sum_to_lambda():
    """sum_u lambda_u(B) = lambda for every non-full state (each call goes somewhere)."""
    inst = I.geometric_instance(8, 33, 9, 0.5, nu_lo=0.5, nu_hi=1.5)
    o = oracle.Oracle(inst)
    o.build_table()
    for n in range(inst.N):
        rows = o.up_rows(n)
        states = o.layer_states(n)
        assert np.allclose(rows.sum(axis=1), inst.lam, rtol=1e-14, atol=0)
        busy = ((states[:, None] >> np.arange(inst.N)[None, :]) & 1).astype(bool)
        assert np.all(rows[busy] == 0.0)
    o.close()


def test_first_idle_examples():
    assert oracle.first_idle([2, 0, 1], 0b101) == 1
    assert oracle.first_idle([2, 0, 1], 0b000) == 2
    assert oracle.first_idle([2, 0, 1], 0b111) == -1
    assert oracle.first_idle([0, 1, 2], 0b011) == 2


def test_layer_normalisation_every_sweep():
    """Lemma 1 (normalisation): sum_m p_n^k(B_m) = 1 after every outer iteration."""
    inst = I.geometric_instance(9, 20, 13, 0.8, nu_lo=0.5, nu_hi=1.5)
    o = oracle.Oracle(inst)
    o.build_table()
    o.init()
    layer = np.array([bin(v).count("1") for v in range(1 << inst.N)])
    for _ in range(12):
        o.sweep()
        p = o.conditional()
        sums = np.array([p[layer == n].sum() for n in range(inst.N + 1)])
        assert np.max(np.abs(sums - 1.0)) < 1e-13
    o.close()


@pytest.mark.parametrize("mode,C", [(0, 0), (1, 3), (2, 0)])
def test_flow_balance_of_outputs(mode, C):
    """Dispatches to unit i equal its completions; each call is served or blocked."""
    inst = I.geometric_instance(8, 25, 17, 0.75, nu_lo=0.5, nu_hi=1.5, mode=mode, C=C)
    r = oracle.solve(inst, eps=1e-14)
    R, W, rho = r["R"], r["W"], r["rho"]
    assert np.allclose(inst.lam_j @ R, inst.nu * rho, rtol=1e-12, atol=1e-15)
    assert np.allclose(R.sum(axis=1), 1.0 - r["p_block"], rtol=1e-12, atol=1e-15)
    assert np.allclose(W.sum(axis=1), rho, rtol=1e-12, atol=1e-15)
    assert abs(r["throughput"] - inst.lam * (1.0 - r["p_block"])) < 1e-12
    total = r["P"].sum() + r["q_busy"]
    assert abs(total - 1.0) < 1e-13
    assert np.all(r["P"] > 0)
    layer = np.array([bin(v).count("1") for v in range(1 << inst.N)])
    busy_mean = (r["P"] * layer).sum() + inst.N * r["q_busy"]
    assert abs(rho.sum() - busy_mean) < 1e-12


def test_modes_share_conditionals():
    """The conditional p_n(B_m) do not depend on the buffer (only p(n) does)."""
    base = I.geometric_instance(7, 14, 23, 0.7, nu_lo=0.5, nu_hi=1.5)
    outs = []
    for mode, C in [(0, 0), (1, 4), (2, 0)]:
        inst = I.Instance(N=base.N, J=base.J, lam_j=base.lam_j, nu=base.nu, pref=base.pref,
                          mode=mode, C=C)
        outs.append(oracle.solve(inst, eps=1e-14)["cond"])
    assert np.max(np.abs(outs[0] - outs[1])) < 1e-15
    assert np.max(np.abs(outs[0] - outs[2])) < 1e-15


def test_residual_of_dense_solution_is_zero():
    inst = I.geometric_instance(7, 19, 29, 0.7, nu_lo=0.5, nu_hi=1.5, mode=2)
    d = dense_solve(inst)
    o = oracle.Oracle(inst)
    o.build_table()
    r = inst.lam / inst.nu.sum()
    assert o.residual(d["P"], d["P"][-1] * r) < 1e-13
    P = d["P"].copy()
    P[5] *= 1.001
    assert o.residual(P, d["P"][-1] * r) > 1e-5
    o.close()


def test_sampled_balance_matches_table_route():
    inst = I.geometric_instance(8, 21, 31, 0.7, nu_lo=0.5, nu_hi=1.5, mode=2)
    d = dense_solve(inst)
    P = d["P"]
    rng = np.random.default_rng(0)
    B = rng.integers(0, 1 << inst.N, 50).astype(np.uint64)
    nb = np.array([[P[int(b) ^ (1 << u)] for u in range(inst.N)] for b in B])
    pq1 = P[-1] * inst.lam / inst.nu.sum()
    out, inn = oracle.sampled_balance(inst, B, P[B.astype(np.int64)], nb, pq1)
    assert np.max(np.abs(out - inn)) / np.max(out) < 1e-13


def test_openmp_build_matches_the_plain_one():
    """The OpenMP build of the oracle (the loops over a layer's states on all host
    threads; only the order of the layer sums changes) gives the plain build's solution
    to rounding, and the residual-stopped solve used for timing reaches its tolerance."""
    import oracle as O

    inst = I.geometric_instance(12, 40, 31, 0.6, nu_lo=0.5, nu_hi=1.5, mode=2)
    a = O.solve(inst, eps=1e-14, threads=1)
    b = O.solve(inst, eps=1e-14, threads=0)
    assert a["sweeps"] == b["sweeps"]
    for k in ("P", "rho", "R", "W", "pn"):
        assert np.max(np.abs(a[k] - b[k])) < 1e-13, k
    r = O.solve_to_residual(inst, 1e-10, threads=0)
    assert r["converged"] and r["residual"] <= 1e-10 and r["sweeps"] % 8 == 0
