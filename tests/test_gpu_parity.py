"""GPU library (through its C ABI) against the CPU oracle.

Tolerances: 1e-10 max-abs on P, p(n), rho, R, W for the converged FP64 and DF64
(double-float, 48-bit) paths, as the solver's stated accuracy target; tighter
where the arithmetic allows (table 1e-13 relative: FP64 sums in another order;
a fixed number of sweeps 1e-12: same iteration, closed-form versus literal inner
loop).  FP32-only solves are held to 1e-5 (FP32 rounding, ~1e-7, amplified by the
iteration's conditioning).
"""
import math

import numpy as np
import pytest

import oracle
from oracle.dense import dense_solve
from paper_2603_03019_gb300 import hq
from paper_2603_03019_gb300 import instances as I

pytestmark = pytest.mark.gpu


def _layer_offsets(N):
    sizes = [math.comb(N, n) for n in range(N + 1)]
    off = np.concatenate([[0], np.cumsum(sizes)])
    toff = np.concatenate([[0], np.cumsum([n * sizes[n] for n in range(N + 1)])])
    return sizes, off, toff


def _solve_gpu(inst, **kw):
    s = hq.Solver.for_instance(inst)
    rc, st = s.solve(**kw)
    out = dict(rc=rc, stats=st, P=s.stationary(), cond=s.conditional(), rho=s.utilisation(),
               R=s.response_pattern(), W=s.workload(), summary=s.summary())
    out["pn"], out["tail"] = s.layer_marginals()
    s.close()
    return out


# ---- layout and dispatch table ---------------------------------------------------------

@pytest.mark.parametrize("N,J,seed", [(3, 2, 1), (8, 30, 2), (13, 40, 3), (14, 120, 4)])
def test_table_and_masks_match_oracle(gpu_lib, N, J, seed):
    inst = I.geometric_instance(N, J, seed, 0.6, nu_lo=0.5, nu_hi=1.5)
    s = hq.Solver.for_instance(inst)
    T, masks = s.table()
    s.close()
    o = oracle.Oracle(inst)
    o.build_table()
    sizes, off, toff = _layer_offsets(N)
    for n in range(N + 1):
        st = o.layer_states(n)
        assert np.array_equal(masks[off[n]:off[n + 1]], st), f"layer {n} order"
    pos = np.zeros(1 << N, dtype=np.int64)
    for n in range(N + 1):
        pos[o.layer_states(n)] = np.arange(sizes[n])
    for n in range(1, N + 1):
        rows = o.up_rows(n - 1)
        st = masks[off[n]:off[n + 1]].astype(np.int64)
        bits = ((st[:, None] >> np.arange(N)[None, :]) & 1).astype(bool)
        for k in range(sizes[n]):
            units = np.nonzero(bits[k])[0]
            for slot, u in enumerate(units):
                src = st[k] & ~(1 << u)
                want = rows[pos[src], u]
                got = T[toff[n] + slot * sizes[n] + k]
                assert abs(got - want) <= 1e-13 * max(1.0, abs(want)), (n, k, slot)
    o.close()


# ---- the iteration, sweep by sweep -----------------------------------------------------

@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("df64", 1e-12)])
@pytest.mark.parametrize("sweeps", [1, 3, 10])
@pytest.mark.parametrize("N,J", [(11, 37), (2, 3), (3, 5), (4, 7)])
def test_fixed_sweeps_match_algorithm1(gpu_lib, prec, tol, sweeps, N, J):
    """Sweep by sweep against the oracle's Algorithm 1, including the smallest N, where the
    layer finalised lazily at the start of a sweep (N-1) is the one that layer 1 reads
    (N=3) or the only one (N=2)."""
    inst = I.geometric_instance(N, J, 5, 0.8, nu_lo=0.5, nu_hi=1.5)
    g = _solve_gpu(inst, tol=0.0, tol_kind=hq.HQ_TOL_STEP, precision=prec, max_sweeps=sweeps,
                   check_every=sweeps)
    # N=2: layer 1 depends only on the empty and the full state, so the first sweep is
    # exact and every later step is 0, which meets the zero tolerance
    assert g["rc"] in ((hq.HQ_OK, hq.HQ_ENOTCONVERGED) if N == 2 else (hq.HQ_ENOTCONVERGED,))
    assert g["stats"]["sweeps_hi"] == sweeps
    r = oracle.solve(inst, sweeps=sweeps, with_R=False)
    assert np.max(np.abs(g["cond"] - r["cond"])) < tol


# ---- converged solutions, all queue modes ----------------------------------------------

CASES = [(6, 9, 0, 0, 11), (10, 50, 0, 0, 12), (9, 33, 1, 4, 13), (10, 41, 2, 0, 14),
         (13, 80, 0, 0, 15), (13, 64, 2, 0, 16)]


@pytest.mark.parametrize("prec", ["fp64", "df64", "fp32+df64", "fp32+fp64", "fp32+ir"])
@pytest.mark.parametrize("N,J,mode,C,seed", CASES)
def test_solve_matches_oracle(gpu_lib, N, J, mode, C, seed, prec):
    inst = I.geometric_instance(N, J, seed, 0.7, nu_lo=0.5, nu_hi=1.5, mode=mode, C=C)
    g = _solve_gpu(inst, tol=1e-13, tol_kind=hq.HQ_TOL_RESIDUAL, precision=prec)
    assert g["rc"] == hq.HQ_OK, g["stats"]
    r = oracle.solve(inst, eps=1e-15)
    assert np.max(np.abs(g["P"] - r["P"])) < 1e-10
    assert np.max(np.abs(g["pn"] - r["pn"])) < 1e-10
    assert np.max(np.abs(g["rho"] - r["rho"])) < 1e-10
    assert np.max(np.abs(g["R"] - r["R"])) < 1e-10
    assert np.max(np.abs(g["W"] - r["W"])) < 1e-10
    assert abs(g["summary"]["throughput"] - r["throughput"]) < 1e-10
    assert g["summary"]["residual"] < 1e-12
    if mode == 2:
        assert abs(g["tail"] - r["queue_tail"]) < 1e-10
    if N <= 10:
        d = dense_solve(inst)
        assert np.max(np.abs(g["P"] - d["P"])) < 1e-10


def test_small_loss_n10_matches_dense(gpu_lib):
    """N=10, J=50 loss system, tolerance 1e-12, against the dense direct solve."""
    inst = I.small_loss_n10(1001)
    g = _solve_gpu(inst, tol=1e-12, tol_kind=hq.HQ_TOL_STEP, precision="fp64")
    d = dense_solve(inst)
    assert g["rc"] == hq.HQ_OK
    assert np.max(np.abs(g["P"] - d["P"])) < 1e-10


def test_fp32_only_bound(gpu_lib):
    inst = I.geometric_instance(10, 40, 21, 0.7, nu_lo=0.5, nu_hi=1.5)
    g = _solve_gpu(inst, tol=1e-9, tol_kind=hq.HQ_TOL_STEP, precision="fp32", max_sweeps=2000)
    r = oracle.solve(inst, eps=1e-15)
    err = np.max(np.abs(g["P"] - r["P"]))
    assert err < 1e-5
    assert np.max(np.abs(g["rho"] - r["rho"])) < 1e-5


# ---- degenerate cases --------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["fp64", "fp32+ir"])
@pytest.mark.parametrize("mode,C", [(0, 0), (1, 3), (2, 0)])
def test_single_unit(gpu_lib, mode, C, prec):
    inst = I.Instance(N=1, J=1, lam_j=np.array([0.7]), nu=np.array([1.3]),
                      pref=np.array([[0]], np.int32), mode=mode, C=C)
    g = _solve_gpu(inst, precision=prec)
    r = oracle.solve(inst, eps=1e-15)
    assert np.max(np.abs(g["P"] - r["P"])) < 1e-14
    assert np.max(np.abs(g["pn"] - r["pn"])) < 1e-14
    assert np.max(np.abs(g["R"] - r["R"])) < 1e-14


@pytest.mark.parametrize("prec", ["fp64", "fp32+ir", "fp32+df64"])
def test_two_units_golden(gpu_lib, prec):
    inst = I.Instance(N=2, J=2, lam_j=np.array([1.0, 2.0]), nu=np.array([1.0, 2.0]),
                      pref=np.array([[0, 1], [1, 0]], np.int32))
    g = _solve_gpu(inst, tol=1e-15, tol_kind=hq.HQ_TOL_STEP, precision=prec)
    assert np.max(np.abs(g["P"] - np.array([18, 24, 15, 39]) / 96.0)) < 1e-14


def test_zero_rate_nodes_and_single_node(gpu_lib):
    inst = I.geometric_instance(9, 20, 31, 0.6, nu_lo=0.5, nu_hi=1.5)
    inst.lam_j[::3] = 0.0
    for prec in ("df64", "fp32+ir"):
        g = _solve_gpu(inst, tol=1e-13, precision=prec)
        r = oracle.solve(inst, eps=1e-15)
        assert np.max(np.abs(g["P"] - r["P"])) < 1e-10, prec
    one = I.Instance(N=7, J=1, lam_j=np.array([3.0]), nu=np.linspace(0.5, 1.5, 7),
                     pref=np.array([[3, 1, 4, 0, 5, 2, 6]], np.int32))
    g1 = _solve_gpu(one, tol=1e-13, precision="df64")
    r1 = oracle.solve(one, eps=1e-15)
    assert np.max(np.abs(g1["P"] - r1["P"])) < 1e-10
    assert abs(g1["rho"][3] - 3.0 / (3.0 + one.nu[3])) < 1e-10


def test_warm_start_from_solution(gpu_lib):
    inst = I.geometric_instance(12, 60, 41, 0.8, nu_lo=0.5, nu_hi=1.5)
    r = oracle.solve(inst, eps=1e-15)
    s = hq.Solver.for_instance(inst)
    rc, st = s.solve(tol=1e-11, precision="df64", warm_p=r["cond"], check_every=2)
    assert rc == hq.HQ_OK and st["sweeps_hi"] <= 4
    rc2, st2 = s.solve(tol=1e-11, precision="df64", check_every=2)
    assert st2["sweeps_hi"] > 3 * st["sweeps_hi"]
    s.close()


def test_errors_are_reported(gpu_lib):
    inst = I.geometric_instance(6, 8, 51, 0.6, nu_lo=0.5, nu_hi=1.5)
    s = hq.Solver(inst.N, inst.J)
    with pytest.raises(hq.HQError) as e:
        hq.hq_solve(s.h, None)
    assert e.value.code == hq.HQ_ESTATE
    bad = inst.pref.copy()
    bad[2, 1] = bad[2, 0]
    with pytest.raises(hq.HQError) as e:
        s.load(inst.lam_j, inst.nu, bad)
    assert e.value.code == hq.HQ_EINVAL
    with pytest.raises(hq.HQError) as e:
        s.load(inst.lam_j, -inst.nu, inst.pref)
    assert e.value.code == hq.HQ_EINVAL
    s.load(inst.lam_j, inst.nu, inst.pref)
    with pytest.raises(hq.HQError) as e:
        s.stationary()
    assert e.value.code == hq.HQ_ESTATE
    s.close()
    q = hq.Solver(inst.N, inst.J, hq.HQ_INFINITE)
    with pytest.raises(hq.HQError) as e:
        q.load(inst.lam_j * 10.0, inst.nu, inst.pref)
    assert e.value.code == hq.HQ_EUNSTABLE
    q.close()


def test_device_resident_inputs_and_outputs(gpu_lib):
    torch = pytest.importorskip("torch")
    inst = I.geometric_instance(12, 70, 61, 0.7, nu_lo=0.5, nu_hi=1.5)
    dev = torch.device("cuda:0")
    lam = torch.tensor(inst.lam_j, device=dev)
    nu = torch.tensor(inst.nu, device=dev)
    pref = torch.tensor(inst.pref, device=dev)
    s = hq.Solver(inst.N, inst.J, stream=torch.cuda.current_stream())
    s.load(lam, nu, pref)
    rc, st = s.solve(tol=1e-12)
    P = torch.empty(1 << inst.N, dtype=torch.float64, device=dev)
    hq.hq_get_stationary(s.h, P)
    torch.cuda.synchronize()
    r = oracle.solve(inst, eps=1e-15, with_R=False)
    assert np.max(np.abs(P.cpu().numpy() - r["P"])) < 1e-10
    s.close()


# ---- mid size: N=20 against the full oracle ------------------------------------------------

def test_mixed_n20_against_oracle(gpu_lib):
    # outputs that sum many states (rho, R) carry the residual times the chain's
    # relaxation factor (~1e2 here), so both sides stop well below 1e-10
    inst = I.mixed_n20(2001, 0.6)
    g = _solve_gpu(inst, tol=1e-13, precision="fp32+df64")
    assert g["rc"] == hq.HQ_OK
    r = oracle.solve(inst, eps=1e-15, threads=0)
    assert np.max(np.abs(g["P"] - r["P"])) < 1e-10
    assert np.max(np.abs(g["pn"] - r["pn"])) < 1e-10
    assert np.max(np.abs(g["rho"] - r["rho"])) < 1e-10
    assert np.max(np.abs(g["R"] - r["R"])) < 1e-10


# ---- full size: N=24, J=1000 infinite queue, the benchmark's launch configuration --------

@pytest.mark.parametrize("prec", ["fp32+df64", "fp32+ir"])
def test_large_n24_sampled(gpu_lib, prec):
    inst = I.large_infinite_n24()
    s = hq.Solver.for_instance(inst)
    rc, st = s.solve(tol=1e-10, precision=prec, omega=-1.0)
    assert rc == hq.HQ_OK, st
    P = s.stationary()
    T, masks = s.table()
    rho, R = s.utilisation(), s.response_pattern()
    pn, tail = s.layer_marginals()
    summ = s.summary()
    s.close()
    N = inst.N
    rng = np.random.default_rng(7)
    # sampled table entries against Eq. (3) evaluated by the oracle
    sizes, off, toff = _layer_offsets(N)
    for _ in range(300):
        n = int(rng.integers(1, N + 1))
        k = int(rng.integers(0, sizes[n]))
        m = int(masks[off[n] + k])
        units = [u for u in range(N) if (m >> u) & 1]
        slot = int(rng.integers(0, len(units)))
        u = units[slot]
        want = oracle.dispatch_rates(inst, src=[m & ~(1 << u)], u=[u])[0]
        got = T[toff[n] + slot * sizes[n] + k]
        assert abs(got - want) <= 1e-13 * max(1.0, want)
    # sampled global balance of Eq. (1) with the oracle's dispatch rule
    B = rng.integers(0, 1 << N, 1500).astype(np.uint64)
    B[:3] = [0, (1 << N) - 1, (1 << N) - 2]
    nb = np.stack([P[(B.astype(np.int64) ^ (1 << u))] for u in range(N)], axis=1)
    lam = inst.lam
    r_q = lam / inst.nu.sum()
    pq1 = P[-1] * r_q
    out, inn = oracle.sampled_balance(inst, B, P[B.astype(np.int64)], nb, pq1)
    y = np.arange(1 << N, dtype=np.int64)
    busy = np.zeros(1 << N)
    for u in range(N):
        busy += ((y >> u) & 1) * inst.nu[u]
    den = np.max(P * (lam + busy))
    assert np.max(np.abs(out - inn)) / den < 1e-10
    # invariants: normalisation and flow balance
    assert abs(P.sum() + tail - 1.0) < 1e-12
    # dispatches to unit i minus its completions is a sum of balance residuals over
    # the 2^(N-1) states where i is busy: bounded by 2^(N-1) * residual * max outflow
    bound = (1 << (N - 1)) * summ["residual"] * den
    assert np.max(np.abs(inst.lam_j @ R - inst.nu * rho)) <= bound
    assert np.allclose(R.sum(axis=1), 1.0, rtol=0, atol=1e-10)
    assert summ["residual"] < 1e-10


# ---- over-relaxation (not in the paper): same fixed point, fewer sweeps ------------------

@pytest.mark.parametrize("prec,omega", [("fp64", -1.0), ("fp32+df64", -1.0), ("df64", 1.3),
                                        ("fp32+ir", -1.0)])
@pytest.mark.parametrize("N,J,mode,C,seed", CASES)
def test_relaxed_solve_matches_oracle(gpu_lib, N, J, mode, C, seed, prec, omega):
    inst = I.geometric_instance(N, J, seed, 0.7, nu_lo=0.5, nu_hi=1.5, mode=mode, C=C)
    g = _solve_gpu(inst, tol=1e-13, tol_kind=hq.HQ_TOL_RESIDUAL, precision=prec, omega=omega)
    assert g["rc"] == hq.HQ_OK, g["stats"]
    assert g["stats"]["omega"] >= 1.0
    r = oracle.solve(inst, eps=1e-15)
    assert np.max(np.abs(g["P"] - r["P"])) < 1e-10
    assert np.max(np.abs(g["rho"] - r["rho"])) < 1e-10
    assert np.max(np.abs(g["R"] - r["R"])) < 1e-10


def test_relaxation_saves_sweeps_and_rejects_bad_omega(gpu_lib):
    inst = I.mixed_n20(2001, 0.6)
    s = hq.Solver.for_instance(inst)
    rc1, plain = s.solve(tol=1e-10, precision="fp64")
    P1 = s.stationary()
    rc2, relaxed = s.solve(tol=1e-10, precision="fp64", omega=-1.0)
    assert rc1 == rc2 == hq.HQ_OK
    assert relaxed["sweeps_hi"] < plain["sweeps_hi"] and relaxed["omega"] > 1.0
    assert np.max(np.abs(s.stationary() - P1)) < 1e-9
    for bad in (0.5, 2.0, 3.0):
        with pytest.raises(hq.HQError) as e:
            s.solve(tol=1e-10, precision="fp64", omega=bad)
        assert e.value.code == hq.HQ_EINVAL
    s.close()


# ---- iterative refinement (not in the paper): FP32 corrections against an FP64 base --------

def test_refinement_matches_fp64_and_rebases(gpu_lib):
    """FP32 correction sweeps reach the FP64 fixed point: the refined N=20 solution agrees
    with plain FP64 sweeps and the oracle; a stall threshold that declares every check
    stalled switches to refinement after 24 FP32 sweeps (the first check has no decay to
    judge, the next two stall in a row), far from the solution, so the first correction
    meets its FP32 floor early and the base must absorb it again."""
    inst = I.mixed_n20(2001, 0.6)
    s = hq.Solver.for_instance(inst)
    rc, ref = s.solve(tol=1e-13, precision="fp64", omega=-1.0)
    assert rc == hq.HQ_OK
    P64, rho64 = s.stationary(), s.utilisation()
    rc, st = s.solve(tol=1e-13, precision="fp32+ir", omega=-1.0)
    assert rc == hq.HQ_OK, st
    assert st["ir_bases"] >= 1 and st["sweeps_hi"] > 0 and st["sweeps_fp32"] > 0
    assert st["final_residual"] < 1e-13
    # rho sums 2^19 states: both solves' residuals (1e-13) times the chain's
    # relaxation factor (~1e2) each
    assert np.max(np.abs(s.stationary() - P64)) < 1e-11
    assert np.max(np.abs(s.utilisation() - rho64)) < 1e-10
    rc, st2 = s.solve(tol=1e-13, precision="fp32+ir", fp32_stall=1e-3, max_sweeps=800)
    assert rc == hq.HQ_OK, st2
    assert st2["sweeps_fp32"] == 24 and 2 <= st2["ir_bases"] <= 4
    assert np.max(np.abs(s.stationary() - P64)) < 1e-11
    r = oracle.solve(inst, eps=1e-15, threads=0)
    assert np.max(np.abs(P64 - r["P"])) < 1e-10
    ms = hq.hq_profile_sweep(s.h, hq.HQ_PREC_FP32_IR, 2)
    assert ms > 0
    s.close()

