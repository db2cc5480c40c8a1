"""Dense direct solve of the hypercube balance equations, Eq. (1)-(2) (arXiv 2603.03019).

TEST INFRASTRUCTURE ONLY (part of the CPU oracle).

The generator matrix is built straight from Eq. (3), in the "target" form the
paper's Algorithm 3 uses: for a state m and node j, walk zeta_j over the units
busy in m until the first idle one; every busy unit l met on the way is the unit
that a call from j would have been sent to in state m - l, so the transition
(m - l) -> m gains lambda f_j.  Downward moves m -> m - u have rate nu_u.  This is
a different route to the same rates than the C oracle's (which walks from the
source state), so agreement checks both.

Queues:
  * finite buffer C -- the C queued states of Section 2.2 are appended as extra
    states (Eq. 11 and the all-busy balance equation above it);
  * infinite buffer -- the queued states form the geometric chain
    P~{c} = P{all busy} (lambda / sum nu)^c; substituting it, the all-busy balance
    becomes P{all busy} sum nu = inflow from layer N-1 and the normalisation weighs
    P{all busy} by 1 / (1 - lambda / sum nu).  That exact reduction is what is solved.

The linear system replaces one balance equation by the normalisation (Section 2.1).
Solved with LAPACK through numpy (FP64).  Practical for N <= 12.
"""
from __future__ import annotations

import numpy as np

LOSS, FINITE, INFINITE = 0, 1, 2


def generator(N, J, lam_j, nu, pref, mode=LOSS, C=0):
    """Q[src, dst] = transition rate; diagonal = -(total outflow).  Returns (Q, weights)."""
    S = 1 << N
    full = S - 1
    extra = C if mode == FINITE else 0
    Q = np.zeros((S + extra, S + extra))
    m = np.arange(S, dtype=np.int64)
    pref = np.asarray(pref)
    for j in range(J):
        searching = np.ones(S, dtype=bool)
        for h in range(N):
            u = int(pref[j, h])
            busy = ((m >> u) & 1).astype(bool)
            hit = searching & busy
            tgt = m[hit]
            np.add.at(Q, (tgt ^ (1 << u), tgt), lam_j[j])
            searching &= busy
    for u in range(N):
        busy = ((m >> u) & 1).astype(bool)
        src = m[busy]
        Q[src, src ^ (1 << u)] += nu[u]
    lam = float(np.sum(lam_j))
    nus = float(np.sum(nu))
    w = np.ones(S + extra)
    if mode == FINITE:
        chain = [full] + [S + c for c in range(C)]
        for a, b in zip(chain[:-1], chain[1:]):
            Q[a, b] += lam
            Q[b, a] += nus
    elif mode == INFINITE:
        w[full] = 1.0 / (1.0 - lam / nus)
    Q[np.diag_indices_from(Q)] = 0.0
    Q[np.diag_indices_from(Q)] = -Q.sum(axis=1)
    return Q, w


def dense_solve(inst=None, **kw):
    """Stationary distribution by Gaussian elimination.  Returns dict with
    P (2^N, y-order), Pq (queued states P~{1..C} for finite mode), and the full vector."""
    if inst is not None:
        for k in ("N", "J", "lam_j", "nu", "pref", "mode", "C"):
            kw.setdefault(k, getattr(inst, k))
    N, J = int(kw["N"]), int(kw["J"])
    mode, C = int(kw.get("mode", LOSS)), int(kw.get("C", 0))
    Q, w = generator(N, J, np.asarray(kw["lam_j"], float), np.asarray(kw["nu"], float),
                     kw["pref"], mode, C)
    A = Q.T.copy()
    b = np.zeros(A.shape[0])
    A[-1, :] = w
    b[-1] = 1.0
    x = np.linalg.solve(A, b)
    S = 1 << N
    out = {"P": x[:S], "full": x}
    if mode == FINITE:
        out["Pq"] = x[S:]
    elif mode == INFINITE:
        lam = float(np.sum(kw["lam_j"]))
        r = lam / float(np.sum(kw["nu"]))
        out["queue_tail"] = x[S - 1] * r / (1.0 - r)
    return out
