"""CPU reference of the warm-start network (test infrastructure only).

Plain numpy, FP64 arithmetic, written from the network's definition: an MLP
x (9 inputs) -> relu(x W1 + b1) -> relu(a1 W2 + b2) -> a2 W3 + b3, trained on the mean
squared error of its output against logit(q_i(n)), q_i(n) = P(unit i busy | n busy),
one row per (layer, unit).  With ``bf16=True`` it rounds at the
points where the GPU kernels store BF16 (the hidden activations a1 and a2, the copy of
W2 used by the tensor-core product, and the layer-2 error signal dz2), and evaluates the
first layer in FP32 with one rounding per multiply-add, so that both sides take the
same quantisation decisions; with ``bf16=False`` it is the exact FP64 network, whose
gradient the finite-difference pin checks.

Parameter vector (flat): W1 [9 x H] row-major, b1 [H], W2 [H x H] row-major (input
index first), b2 [H], W3 [H], b3 [1].

Also: the network inputs of an instance (one row per layer n = 1..N-1 and unit i), the
layer-wise product-form start p_n(B) = prod_{i in B} x_i(n) / e_n(x(n)),
x_i(n) = q_i(n) / (1 - q_i(n)), and the layer law implied by q (Eq. 10 with
lambda(n) = lambda, mu(n) = sum_i nu_i q_i(n)), written from their definitions.  This
module shares no code with the CUDA library.
"""
from __future__ import annotations

import numpy as np

F = 9


def split(w: np.ndarray, H: int) -> dict:
    o = 0
    out = {}
    for name, shape in (("W1", (F, H)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H,)),
                        ("b3", (1,))):
        n = int(np.prod(shape))
        out[name] = np.asarray(w[o:o + n], dtype=np.float64).reshape(shape)
        o += n
    assert o == w.size
    return out


def bf16(x) -> np.ndarray:
    """Round float32 values to bfloat16 (nearest, ties to even), returned as float64."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _layer1_fp32(X, W1, b1):
    # z = b1; z = fma(x_f, W1[f], z) in FP32, f = 0..F-1 (each step rounded once to FP32)
    X32 = np.asarray(X, dtype=np.float32).astype(np.float64)
    z = np.broadcast_to(np.asarray(b1, dtype=np.float32).astype(np.float64), (X32.shape[0], W1.shape[1])).copy()
    W = np.asarray(W1, dtype=np.float32).astype(np.float64)
    for f in range(F):
        z = (X32[:, f:f + 1] * W[f][None, :] + z).astype(np.float32).astype(np.float64)
    return z


def forward(w, X, H: int, bf16_points: bool = True):
    p = split(np.asarray(w), H)
    X = np.asarray(X, dtype=np.float64)
    if bf16_points:
        z1 = _layer1_fp32(X, p["W1"], p["b1"])
        a1 = bf16(np.maximum(z1, 0.0))
        W2 = bf16(p["W2"])
        z2 = a1 @ W2
        a2 = bf16(np.maximum(z2 + p["b2"], 0.0))
    else:
        z1 = X @ p["W1"] + p["b1"]
        a1 = np.maximum(z1, 0.0)
        W2 = p["W2"]
        z2 = a1 @ W2
        a2 = np.maximum(z2 + p["b2"], 0.0)
    y = a2 @ p["W3"] + p["b3"][0]
    return y, dict(a1=a1, a2=a2, W2=W2, p=p)


def loss_and_grad(w, X, t, H: int, bf16_points: bool = True):
    """Mean squared error and its gradient with respect to the flat parameters."""
    X = np.asarray(X, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    B = X.shape[0]
    y, c = forward(w, X, H, bf16_points)
    e = y - t
    loss = float(np.mean(e * e))
    dy = 2.0 * e / B
    a1, a2, p = c["a1"], c["a2"], c["p"]
    dW3 = a2.T @ dy
    db3 = np.array([dy.sum()])
    dz2 = np.outer(dy, p["W3"]) * (a2 > 0)
    if bf16_points:
        dz2 = bf16(dz2)
    dW2 = a1.T @ dz2
    db2 = dz2.sum(axis=0)
    da1 = dz2 @ c["W2"].T
    dz1 = da1 * (a1 > 0)
    dW1 = X.T @ dz1
    db1 = dz1.sum(axis=0)
    g = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dW3, db3])
    return loss, g


def unit_features(inst) -> np.ndarray:
    """The 8 per-unit features of an instance (N x 8), from their definitions."""
    N = inst.N
    lam = float(np.sum(inst.lam_j))
    nu = np.asarray(inst.nu, dtype=np.float64)
    s = np.zeros((3, N))
    for j in range(inst.J):
        for h in range(min(3, N)):
            s[h, int(inst.pref[j, h])] += inst.lam_j[j]
    mean_nu = nu.sum() / N
    return np.stack([nu / mean_nu, s[0] / lam, s[1] / lam, s[2] / lam, s[0] / nu,
                     np.full(N, lam / nu.sum()), np.log(nu / mean_nu), np.full(N, N / 16.0)], axis=1)


def features(inst) -> np.ndarray:
    """Network inputs: row (n-1) N + i = unit i's features and n / N, n = 1..N-1."""
    N = inst.N
    u = unit_features(inst)
    rows = [np.concatenate([u[i], [n / N]]) for n in range(1, N) for i in range(N)]
    return np.asarray(rows).astype(np.float32)


def product_form_layers(q: np.ndarray) -> np.ndarray:
    """p_n(B) in y-order for q ((N+1) x N, row n = q_(.)(n)): brute force over the states;
    the empty and the full state get 1."""
    q = np.asarray(q, dtype=np.float64)
    N = q.shape[1]
    S = 1 << N
    w = np.ones(S)
    n_of = np.array([bin(b).count("1") for b in range(S)])
    for b in range(S):
        n = n_of[b]
        if 0 < n < N:
            qq = np.clip(q[n], 1e-4, 1 - 1e-4)
            x = qq / (1 - qq)
            for i in range(N):
                if (b >> i) & 1:
                    w[b] *= x[i]
    e = np.zeros(N + 1)
    np.add.at(e, n_of, w)
    return w / e[n_of]


def layer_law(q: np.ndarray, lam: float, nu: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """(P(n), rho) of the loss system with lambda(n) = lambda, mu(n) = sum_i nu_i q_i(n)."""
    q = np.asarray(q, dtype=np.float64)
    N = q.shape[1]
    mu = q @ np.asarray(nu, dtype=np.float64)
    w = np.ones(N + 1)
    for n in range(1, N + 1):
        w[n] = w[n - 1] * lam / mu[n]
    P = w / w.sum()
    return P, P @ q


def first_choice_start(inst) -> tuple[np.ndarray, np.ndarray]:
    """The analytic start (no network): rho0_i = lambda1_i / nu_i clipped to
    [0.02, 0.98], lambda1_i = sum of lambda_j over the nodes j whose first choice is
    unit i; q_i(n) = rho0_i for every layer 1..N-1 (0 in layer 0, 1 in layer N), with q
    passed through the same float32 logit as the GPU's logit buffer.  Returns (rho0, q)."""
    N = inst.N
    l1 = np.zeros(N)
    for j in range(inst.J):
        l1[int(inst.pref[j, 0])] += inst.lam_j[j]
    rho0 = np.clip(l1 / np.asarray(inst.nu, dtype=np.float64), 0.02, 0.98)
    y = np.log(rho0 / (1.0 - rho0)).astype(np.float32).astype(np.float64)
    q = np.zeros((N + 1, N))
    q[N] = 1.0
    q[1:N] = 1.0 / (1.0 + np.exp(-y))
    return rho0, q


def conditional_occupancy(cond: np.ndarray, N: int) -> np.ndarray:
    """q_i(n) = sum of p_n(B) over the states B of layer n with unit i busy."""
    S = 1 << N
    q = np.zeros((N + 1, N))
    for b in range(S):
        n = bin(b).count("1")
        for i in range(N):
            if (b >> i) & 1:
                q[n, i] += cond[b]
    return q
