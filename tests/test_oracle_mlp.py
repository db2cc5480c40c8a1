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


# ---- pins of the BF16 rounding points, independent of the oracle's own arithmetic ------

def _flat(W1, b1, W2, b2, W3, b3):
    return np.concatenate([np.ravel(W1), b1, np.ravel(W2), b2, W3, [b3]]).astype(np.float64)


def test_bf16_points_are_no_ops_on_dyadic_values():
    """Small integers and halves everywhere: every input, weight, activation and error
    signal is exact in BF16 (8 significant bits) and FP32, so rounding at the BF16
    points must change nothing: forward, loss and gradient agree with the exact FP64
    network to 1e-12 (in fact exactly)."""
    r = np.random.default_rng(17)
    H, B = 16, 4
    W1 = r.integers(-1, 2, (mlp.F, H)).astype(np.float64)       # z1 integers in [-18, 19]
    b1 = r.integers(0, 2, H).astype(np.float64)
    W2 = np.zeros((H, H))
    for c in range(H):                                          # two entries per column
        rows = r.choice(H, 2, replace=False)
        W2[rows, c] = r.choice([-1.0, -0.5, 0.5, 1.0], 2)       # |z2| <= 38, step 1/2
    b2 = r.integers(0, 2, H).astype(np.float64)
    W3 = r.choice([-1.0, -0.5, 0.0, 0.5, 1.0], H)
    b3 = 0.25
    X = r.integers(0, 3, (B, mlp.F)).astype(np.float64)
    w = _flat(W1, b1, W2, b2, W3, b3)
    y_ex, c_ex = mlp.forward(w, X, H, False)
    # targets one small integer away from the output: e, dy = 2 e / B = e / 2 and
    # dz2 = dy W3 are dyadic with a few bits
    t = y_ex - r.integers(-2, 3, B)
    y_bf, c_bf = mlp.forward(w, X, H, True)
    for k in ("a1", "a2", "W2"):
        assert np.array_equal(mlp.bf16(c_ex[k]), c_ex[k]), k    # the values are BF16-exact
    assert np.max(np.abs(y_bf - y_ex)) <= 1e-12
    l_ex, g_ex = mlp.loss_and_grad(w, X, t, H, False)
    l_bf, g_bf = mlp.loss_and_grad(w, X, t, H, True)
    assert abs(l_bf - l_ex) <= 1e-12
    assert np.max(np.abs(g_bf - g_ex)) <= 1e-12
    assert np.count_nonzero(g_ex) > H                           # a non-trivial gradient


def test_bf16_points_two_hidden_units_by_hand():
    """Two hidden units, one input row, every BF16 rounding point deciding something.
    Worked by hand (BF16 keeps 8 significant bits: spacing 2^-7 on [1, 2), 2^-6 on
    [2, 4); ties go to the even significand):
      z1 = x W1 + b1 = [1 + 2^-8, 1]            (FP32, exact)
      a1 = bf16(relu z1) = [1, 1]               (1 + 2^-8 is a tie: down to even 1)
      bf16(W2) = [[1 + 2^-7, 0], [0, 3]]        (1 + 3 2^-9 is 3/4 of a step: up)
      z2 + b2 = [1 + 2^-7 + 2^-9, 3.5]
      a2 = [1 + 2^-7, 3.5]                      (a quarter step: down)
      y = a2 . W3 + b3 = (1 + 2^-7)(1 + 2^-8 + 2^-10) - 3.5 + 0.25
        = -2.25 + 2^-7 + 2^-8 + 2^-10 + 2^-15 + 2^-17
    The target is y - 2^-4, so e = 2^-4, loss = 2^-8, dy = 2 e = 2^-3 (B = 1):
      dz2 = bf16(dy W3) = bf16([2^-3 (1 + 2^-8 + 2^-10), -2^-3])
          = [2^-3 (1 + 2^-7), -2^-3]           (0.625 of a step: up)
      dW3 = dy a2 = [2^-3 (1 + 2^-7), 3.5 2^-3], db3 = 2^-3
      dW2 = a1^T dz2 (both rows [2^-3 (1 + 2^-7), -2^-3]), db2 = dz2
      da1 = dz2 bf16(W2)^T = [2^-3 (1 + 2^-7)^2, -3 2^-3] = dz1 (a1 > 0)
      dW1 = x^T dz1 (row 0 only), db1 = dz1."""
    H = 2
    W1 = np.zeros((mlp.F, H))
    W1[0] = [1 + 2.0 ** -8, 1.0]
    b1 = np.zeros(H)
    W2 = np.array([[1 + 3 * 2.0 ** -9, 0.0], [0.0, 3.0]])
    b2 = np.array([2.0 ** -9, 0.5])
    W3 = np.array([1 + 2.0 ** -8 + 2.0 ** -10, -1.0])
    b3 = 0.25
    X = np.zeros((1, mlp.F))
    X[0, 0] = 1.0
    w = _flat(W1, b1, W2, b2, W3, b3)
    y_hand = -2.25 + 2.0 ** -7 + 2.0 ** -8 + 2.0 ** -10 + 2.0 ** -15 + 2.0 ** -17
    y, c = mlp.forward(w, X, H, True)
    assert y[0] == y_hand
    assert np.array_equal(c["a1"], [[1.0, 1.0]])
    assert np.array_equal(c["W2"], [[1 + 2.0 ** -7, 0.0], [0.0, 3.0]])
    assert np.array_equal(c["a2"], [[1 + 2.0 ** -7, 3.5]])
    t = np.array([y_hand - 2.0 ** -4])
    loss, g = mlp.loss_and_grad(w, X, t, H, True)
    assert loss == 2.0 ** -8
    s = 2.0 ** -3
    u = 1 + 2.0 ** -7
    dz1 = [s * u * u, -3 * s]
    dW1 = np.zeros((mlp.F, H))
    dW1[0] = dz1
    want = _flat(dW1, dz1, [[s * u, -s], [s * u, -s]], [s * u, -s], [s * u, 3.5 * s], s)
    assert np.array_equal(g, want), np.nonzero(g != want)
    # the exact network differs at every step (the rounding points are not no-ops here)
    y_ex = mlp.forward(w, X, H, False)[0]
    assert abs(y_ex[0] - y_hand) > 2.0 ** -10
