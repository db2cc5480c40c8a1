"""The warm-start network's GPU kernels against its CPU reference, and the warm start.

Forward and gradient of the network (BF16 activations, BF16 tensor-core product, FP32
accumulation) against oracle/mlp.py evaluated with the same rounding points: the two
differ by FP32 accumulation order, and through it by rare flips of a BF16 rounding, so
the tolerance is 2 % of each parameter block's gradient norm (a transposed operand, a
dropped term or a wrong mask moves a block by far more).  Features and the product-form
start against their definitions.  A solve from the learned start reaches the same
stationary distribution as a cold solve; with the trained weights (if present) it needs
fewer sweeps on held-out instances.
"""
import math
import os

import numpy as np
import pytest

from oracle import mlp as ref
from paper_2603_03019_gb300 import hq
from paper_2603_03019_gb300 import instances as I

pytestmark = pytest.mark.gpu

H = 256


def _torch():
    import torch
    return torch, torch.device("cuda", 0)


def _blocks(H):
    sizes = [ref.F * H, H, H * H, H, H, 1]
    return np.cumsum([0] + sizes)


def test_forward_and_gradient_match_reference(gpu_lib):
    torch, dev = _torch()
    m = hq.hq_mlp_create(H, 11)
    w = hq.hq_mlp_get_weights(m)
    B = 300  # not a multiple of the 64-row tile
    r = np.random.default_rng(5)
    X = r.normal(0, 1, (B, ref.F)).astype(np.float32)
    t = r.normal(0, 1, B).astype(np.float32)
    Xd, td = torch.tensor(X, device=dev), torch.tensor(t, device=dev)
    y = torch.empty(B, device=dev)
    hq.hq_mlp_forward(m, Xd, y)
    y_ref = ref.forward(w, X, H, True)[0]
    assert np.max(np.abs(y.cpu().numpy() - y_ref)) < 2e-2 * max(1.0, np.max(np.abs(y_ref)))
    g = torch.empty(hq.hq_mlp_num_params(m), device=dev)
    loss = hq.hq_mlp_gradients(m, Xd, td, g)
    loss_ref, g_ref = ref.loss_and_grad(w, X, t, H, True)
    assert abs(loss - loss_ref) < 2e-2 * loss_ref
    gg = g.cpu().numpy().astype(np.float64)
    b = _blocks(H)
    for k in range(6):
        a, z = gg[b[k]:b[k + 1]], g_ref[b[k]:b[k + 1]]
        assert np.linalg.norm(a - z) <= 2e-2 * np.linalg.norm(z) + 1e-7, f"block {k}"
    assert gg @ g_ref / (np.linalg.norm(gg) * np.linalg.norm(g_ref)) > 0.999
    hq.hq_mlp_destroy(m)


def test_train_step_fits_a_teacher(gpu_lib):
    torch, dev = _torch()
    teacher = hq.hq_mlp_create(64, 3)
    student = hq.hq_mlp_create(64, 4)
    r = np.random.default_rng(6)
    X = torch.tensor(r.normal(0, 1, (4096, ref.F)).astype(np.float32), device=dev)
    t = torch.empty(4096, device=dev)
    hq.hq_mlp_forward(teacher, X, t)
    first = hq.hq_mlp_train_step(student, X, t, 3e-3)
    for _ in range(300):
        last = hq.hq_mlp_train_step(student, X, t, 3e-3)
    assert last < 0.1 * first, (first, last)
    hq.hq_mlp_destroy(teacher)
    hq.hq_mlp_destroy(student)


def test_features_and_layer_law(gpu_lib):
    inst = I.warmstart_instance(123, N=10, J=80)
    s = hq.Solver.for_instance(inst)
    X = hq.hq_mlp_features(s.h, N=inst.N)
    assert np.allclose(X, ref.features(inst), rtol=1e-6, atol=1e-6)
    m = hq.hq_mlp_create(H, 12)
    q, pn, rho = hq.hq_mlp_predict(s.h, m, inst.N)
    assert np.all(q[0] == 0) and np.all(q[-1] == 1) and np.all((q[1:-1] > 0) & (q[1:-1] < 1))
    P_ref, rho_ref = ref.layer_law(q, float(inst.lam_j.sum()), inst.nu)
    assert np.max(np.abs(pn - P_ref)) < 1e-12 and np.max(np.abs(rho - rho_ref)) < 1e-12
    hq.hq_mlp_destroy(m)
    s.close()


@pytest.mark.parametrize("seed", [14, 15, 16])
def test_learned_start_is_the_layer_product_form(gpu_lib, seed):
    """A learned-start solve stopped after two sweeps: two FP64 sweeps of Algorithm 1
    (oracle) from the oracle's layer-wise product form of the same predicted q if the
    residual test kept the learned start, else from the uniform start."""
    import oracle
    inst = I.warmstart_instance(200 + seed, N=9, J=60)
    m = hq.hq_mlp_create(H, seed)
    s = hq.Solver.for_instance(inst)
    q, _, _ = hq.hq_mlp_predict(s.h, m, inst.N)
    hq.hq_attach_mlp(s.h, m)
    rc, st = s.solve(tol=0.0, tol_kind=hq.HQ_TOL_STEP, precision="fp64", max_sweeps=2, check_every=1,
                     warm_mlp=True)
    g = s.conditional()
    s.close()
    hq.hq_mlp_destroy(m)
    assert st["sweeps_hi"] == 2
    # two sweeps of Algorithm 1 (oracle) from the start the solver kept
    o = oracle.Oracle(inst)
    o.build_table()
    o.init(ref.product_form_layers(q) if st["warm_used"] else None)
    o.sweep(1e-20)
    o.sweep(1e-20)
    want = o.conditional()
    o.close()
    assert np.max(np.abs(g - want)) < 1e-12


@pytest.mark.parametrize("seed", [14, 15, 16])
def test_analytic_start_is_the_layer_product_form(gpu_lib, seed):
    """The analytic control (first-choice utilisations, no network): two FP64 sweeps of
    Algorithm 1 (oracle) from the oracle's product form of the same q if the residual test
    kept it, else from the uniform start; and it solves to the same answer."""
    import oracle
    inst = I.warmstart_instance(200 + seed, N=9, J=60)
    s = hq.Solver.for_instance(inst)
    rc, st = s.solve(tol=0.0, tol_kind=hq.HQ_TOL_STEP, precision="fp64", max_sweeps=2, check_every=1,
                     warm_product=True)
    g = s.conditional()
    assert st["sweeps_hi"] == 2
    _, q = ref.first_choice_start(inst)
    # two sweeps of Algorithm 1 (oracle) from the start the solver kept
    o = oracle.Oracle(inst)
    o.build_table()
    o.init(ref.product_form_layers(q) if st["warm_used"] else None)
    o.sweep(1e-20)
    o.sweep(1e-20)
    want = o.conditional()
    o.close()
    assert np.max(np.abs(g - want)) < 1e-12
    rc, st = s.solve(tol=1e-13, precision="fp32+ir", omega=-1.0, warm_product=True)
    assert rc == hq.HQ_OK
    r = oracle.solve(inst, eps=1e-15)
    assert np.max(np.abs(s.stationary() - r["P"])) < 1e-10
    s.close()


def test_learned_start_reaches_the_same_solution(gpu_lib):
    inst = I.warmstart_instance(321, N=12, J=100)
    m = hq.hq_mlp_create(H, 13)  # untrained: the solve must still be exact
    s = hq.Solver.for_instance(inst)
    rc, cold = s.solve(tol=1e-12, precision="fp64")
    P_cold = s.stationary()
    hq.hq_attach_mlp(s.h, m)
    rc2, warm = s.solve(tol=1e-12, precision="fp64", warm_mlp=True)
    assert rc == rc2 == hq.HQ_OK
    assert np.max(np.abs(s.stationary() - P_cold)) < 1e-10
    assert warm["sweeps_hi"] >= 1
    s.close()
    hq.hq_mlp_destroy(m)


@pytest.mark.skipif(not os.path.exists(hq.WARMSTART_WEIGHTS), reason="trained weights not present")
def test_trained_network_gains(gpu_lib):
    """Held-out instances N=16..20.  What the trained network gains over the method
    without it: an estimate of every unit's utilisation in one forward pass that is on
    average less than half as far from the solved one as what the paper's uniform start
    implies (q_i(n) = n/N), and a solve from the learned start that reaches the same
    solution at about the cost of a cold one.  It does not shorten the solve: the
    iteration's rate, not its start, sets the sweep count, and the residual test (two
    FP64 residual evaluations) keeps the learned start only where it is closer than the
    uniform one."""
    m = hq.load_warmstart_model()
    cold_total, warm_total, err_net, err_uniform = 0, 0, [], []
    for N, seed in ((16, 777001), (18, 777002), (20, 777003)):
        inst = I.warmstart_instance(seed, N=N, J=300)
        s = hq.Solver.for_instance(inst)
        rc, c = s.solve(tol=1e-10, precision="fp32+df64")
        P, rho = s.stationary(), s.utilisation()
        q, pn, rho_net = hq.hq_mlp_predict(s.h, m, N)
        q_uni = np.outer(np.arange(N + 1) / N, np.ones(N))
        _, rho_uni = ref.layer_law(q_uni, float(inst.lam_j.sum()), inst.nu)
        err_net.append(np.max(np.abs(rho_net - rho)))
        err_uniform.append(np.max(np.abs(rho_uni - rho)))
        hq.hq_attach_mlp(s.h, m)
        rc2, w = s.solve(tol=1e-10, precision="fp32+df64", warm_mlp=True)
        assert rc == rc2 == hq.HQ_OK
        assert np.max(np.abs(s.stationary() - P)) < 1e-9
        cold_total += c["sweeps_fp32"] + c["sweeps_hi"]
        warm_total += w["sweeps_fp32"] + w["sweeps_hi"]
        s.close()
    hq.hq_mlp_destroy(m)
    assert np.mean(err_net) < 0.5 * np.mean(err_uniform), (err_net, err_uniform)
    # the start is not what limits the sweep count (the iteration's rate is): the learned
    # start costs at most its probes and a shifted check schedule
    assert warm_total <= 1.1 * cold_total + 6, (warm_total, cold_total)
