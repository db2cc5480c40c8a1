"""Pins of the warm-start network's CPU reference (oracle/mlp.py), no GPU.

The reference's gradient is pinned by central finite differences of its own exact
(FP64, no rounding) loss; the BF16 rounding by values whose rounding is known (ties to
even); the features by a hand-computed instance; the product form by special cases
(equal rates give the binomial layer law and uniform conditionals) and by its defining
ratio property.
"""
import math

import numpy as np

from oracle import mlp
from paper_2603_03019_gb300 import instances as I


def _params(H, seed):
    r = np.random.default_rng(seed)
    n = mlp.F * H + H + H * H + H + H + 1
    return r.normal(0, 0.5, n)


def test_gradient_matches_finite_differences():
    H, B = 16, 6
    w = _params(H, 1)
    r = np.random.default_rng(2)
    X = r.normal(0, 1, (B, mlp.F))
    t = r.normal(0, 1, B)
    loss, g = mlp.loss_and_grad(w, X, t, H, bf16_points=False)
    eps = 1e-6
    num = np.zeros_like(w)
    for i in range(w.size):
        wp, wm = w.copy(), w.copy()
        wp[i] += eps
        wm[i] -= eps
        num[i] = (mlp.loss_and_grad(wp, X, t, H, False)[0] - mlp.loss_and_grad(wm, X, t, H, False)[0]) / (2 * eps)
    assert np.max(np.abs(num - g)) <= 1e-6 * max(1.0, np.max(np.abs(g)))
    # a transposed or dropped term would not pass: the bias gradient alone is not enough
    assert np.linalg.norm(g) > 0 and abs(loss - np.mean((mlp.forward(w, X, H, False)[0] - t) ** 2)) < 1e-15


def test_bf16_rounding_ties_to_even():
    v = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -9, -2.5, 0.0], dtype=np.float32)
    want = np.array([1.0, 1.0, 1.0 + 2 ** -6, 1.0, -2.5, 0.0])
    assert np.array_equal(mlp.bf16(v), want)


def test_bf16_forward_close_to_exact():
    H, B = 64, 20
    w = _params(H, 3) * 0.3
    X = np.random.default_rng(4).normal(0, 1, (B, mlp.F)).astype(np.float32)
    y_exact = mlp.forward(w.astype(np.float32), X, H, False)[0]
    y_bf = mlp.forward(w.astype(np.float32), X, H, True)[0]
    assert np.max(np.abs(y_exact - y_bf)) < 0.05 * max(1.0, np.max(np.abs(y_exact)))


def test_features_by_hand():
    inst = I.geometric_instance(3, 2, 7, 0.5, nu_lo=0.5, nu_hi=1.5)
    inst.lam_j = np.array([0.3, 0.9])
    inst.nu = np.array([1.0, 2.0, 3.0])
    inst.pref = np.array([[2, 0, 1], [0, 1, 2]], dtype=np.int32)
    X = mlp.features(inst).astype(np.float64)
    lam, mean_nu = 1.2, 2.0
    s1 = np.array([0.9, 0.0, 0.3]) / lam
    s2 = np.array([0.3, 0.9, 0.0]) / lam
    s3 = np.array([0.0, 0.3, 0.9]) / lam
    u = np.stack([inst.nu / mean_nu, s1, s2, s3, np.array([0.9, 0.0, 0.3]) / inst.nu,
                  np.full(3, lam / 6.0), np.log(inst.nu / mean_nu), np.full(3, 3 / 16)], axis=1)
    assert X.shape == (6, 9)
    for n in (1, 2):
        for i in range(3):
            assert np.allclose(X[(n - 1) * 3 + i], np.concatenate([u[i], [n / 3]]), rtol=1e-6, atol=1e-7)


def test_first_choice_start_by_hand():
    inst = I.geometric_instance(3, 3, 7, 0.5, nu_lo=0.5, nu_hi=1.5)
    inst.lam_j = np.array([0.3, 0.9, 2.0])
    inst.nu = np.array([1.0, 2.0, 3.0])
    inst.pref = np.array([[2, 0, 1], [2, 1, 0], [0, 1, 2]], dtype=np.int32)
    rho0, q = mlp.first_choice_start(inst)
    # unit 0: node 2 (2.0 / 1.0, clipped to 0.98); unit 1: nobody (0, clipped to 0.02);
    # unit 2: nodes 0 and 1 ((0.3 + 0.9) / 3)
    assert np.allclose(rho0, [0.98, 0.02, 0.4], rtol=0, atol=1e-15)
    assert np.all(q[0] == 0) and np.all(q[3] == 1)
    assert np.allclose(q[1], rho0, rtol=1e-7) and np.array_equal(q[1], q[2])


def test_product_form_special_cases():
    N = 6
    q = np.full((N + 1, N), 0.5)
    p = mlp.product_form_layers(q)  # x_i(n) = 1: uniform conditionals
    for b in range(1 << N):
        assert abs(p[b] - 1.0 / math.comb(N, bin(b).count("1"))) < 1e-15
    # each layer's conditionals sum to one; within a layer, the ratio of two states is
    # the ratio of the swapped units' x(n); layers use their own x(n)
    N = 4
    q = np.array([[0, 0, 0, 0], [0.1, 0.2, 0.3, 0.4], [0.6, 0.5, 0.4, 0.5],
                  [0.9, 0.7, 0.8, 0.6], [1, 1, 1, 1]], dtype=float)
    p = mlp.product_form_layers(q)
    for n in range(N + 1):
        assert abs(sum(p[b] for b in range(16) if bin(b).count("1") == n) - 1.0) < 1e-14
    x2 = q[2] / (1 - q[2])
    assert abs(p[0b0011] / p[0b0101] - x2[1] / x2[2]) < 1e-12
    x1 = q[1] / (1 - q[1])
    assert abs(p[0b0001] / p[0b0010] - x1[0] / x1[1]) < 1e-12
    # the occupancy of a product form with equal x is n / N; the layer law of equal
    # rates is the Erlang-B (truncated Poisson) law
    qq = mlp.conditional_occupancy(mlp.product_form_layers(np.full((N + 1, N), 0.5)), N)
    assert np.allclose(qq, np.outer(np.arange(N + 1) / N, np.ones(N)), atol=1e-15)
    P, rho = mlp.layer_law(qq, 2.0, np.ones(N))
    erl = np.array([2.0 ** n / math.factorial(n) for n in range(N + 1)])
    assert np.allclose(P, erl / erl.sum(), atol=1e-15)
    assert np.allclose(rho, np.full(N, (P * np.arange(N + 1)).sum() / N), atol=1e-15)
