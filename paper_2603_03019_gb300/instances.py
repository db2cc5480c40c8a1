"""Seeded synthetic EMS-shaped instances of the spatial hypercube queue.

This module only *produces inputs*: unit and demand-node positions, per-node
arrival rates lambda_j = lambda * f_j, service rates nu_i and the preference lists
zeta_j (units sorted by distance from node j, Section 2.1 of the paper).  It holds
none of the solution method's arithmetic, and both the GPU library and the CPU
oracle consume its arrays.

Random numbers come from a counter-based splitmix64 stream written out here, so
an instance is bit-identical on every machine and numpy version: value k of
stream (seed, tag) is splitmix64(mix(seed, tag) + (k + 1) * 0x9E3779B97F4A7C15).

The paper's datasets (St. Paul, MN: 71 nodes; Greenville County, SC: 99 nodes)
are not available; these instances stand in for them with the same kind of
structure (planar geometry, distance-ordered preference lists, skewed demand).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

LOSS, FINITE, INFINITE = 0, 1, 2
MODE_NAMES = {LOSS: "loss", FINITE: "finite", INFINITE: "infinite"}

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


class Stream:
    """Counter-based splitmix64 stream: draws never depend on call order across streams."""

    def __init__(self, seed: int, tag: int):
        with np.errstate(over="ignore"):
            base = np.array([(seed * 0x100000001B3 + tag * 0xC2B2AE3D27D4EB4F) & 0xFFFFFFFFFFFFFFFF],
                            dtype=np.uint64)
            self._key = int(_mix64(base)[0])
        self._ctr = 0

    def bits(self, n: int) -> np.ndarray:
        with np.errstate(over="ignore"):
            k = np.arange(self._ctr + 1, self._ctr + 1 + n, dtype=np.uint64)
            z = np.uint64(self._key) + k * _GOLDEN
            out = _mix64(z)
        self._ctr += n
        return out

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        u = (self.bits(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u

    def normal(self, n: int) -> np.ndarray:
        m = (n + 1) // 2
        u1 = 1.0 - self.uniform(m)  # (0, 1]
        u2 = self.uniform(m)
        r = np.sqrt(-2.0 * np.log(u1))
        z = np.concatenate([r * np.cos(2 * math.pi * u2), r * np.sin(2 * math.pi * u2)])
        return z[:n]

    def exponential(self, n: int) -> np.ndarray:
        return -np.log1p(-self.uniform(n))

    def integers(self, n: int, lo: int, hi_inclusive: int) -> np.ndarray:
        span = hi_inclusive - lo + 1
        return lo + np.minimum((self.uniform(n) * span).astype(np.int64), span - 1)


@dataclasses.dataclass
class Instance:
    """One hypercube-queue instance (paper notation in brackets).

    N units, J demand nodes; lam_j[j] = lambda f_j [per-node Poisson rate];
    nu[i] = nu_i [service rate]; pref[j, h] = zeta_j(h+1), 0-based unit ids, each
    row a permutation; mode LOSS (C=0), FINITE (buffer C) or INFINITE.
    """

    N: int
    J: int
    lam_j: np.ndarray
    nu: np.ndarray
    pref: np.ndarray
    mode: int = LOSS
    C: int = 0
    name: str = ""
    units_xy: np.ndarray | None = None
    nodes_xy: np.ndarray | None = None

    @property
    def lam(self) -> float:
        return float(np.sum(self.lam_j))

    @property
    def load(self) -> float:
        return self.lam / float(np.sum(self.nu))

    def describe(self) -> dict:
        return {"N": self.N, "J": self.J, "mode": MODE_NAMES[self.mode], "C": self.C,
                "load": round(self.load, 6), "name": self.name}


def distance_preferences(units_xy: np.ndarray, nodes_xy: np.ndarray) -> np.ndarray:
    """zeta_j: units sorted by Euclidean distance from node j (stable: ties go to the lower id)."""
    d = np.sqrt(((nodes_xy[:, None, :] - units_xy[None, :, :]) ** 2).sum(-1))
    return np.argsort(d, axis=1, kind="stable").astype(np.int32)


def geometric_instance(N: int, J: int, seed: int, load: float, *, nu_lo: float, nu_hi: float,
                       nu_dist: str = "uniform", nodes: str = "uniform", clusters: int = 4,
                       sigma: float = 0.1, mode: int = LOSS, C: int = 0, name: str = "") -> Instance:
    """Units and demand nodes in the unit square; lambda_j = Lambda * Dirichlet(1) weights
    with Lambda = load * sum(nu); nu_i uniform on [nu_lo, nu_hi] or log-uniform."""
    s_units = Stream(seed, 1)
    s_nodes = Stream(seed, 2)
    s_dem = Stream(seed, 3)
    s_nu = Stream(seed, 4)
    units_xy = s_units.uniform(2 * N).reshape(N, 2)
    if nodes == "uniform":
        nodes_xy = s_nodes.uniform(2 * J).reshape(J, 2)
    elif nodes == "clusters":
        centres = s_nodes.uniform(2 * clusters, 0.2, 0.8).reshape(clusters, 2)
        which = s_nodes.integers(J, 0, clusters - 1)
        nodes_xy = np.clip(centres[which] + sigma * s_nodes.normal(2 * J).reshape(J, 2), 0.0, 1.0)
    else:
        raise ValueError(nodes)
    if nu_dist == "uniform":
        nu = s_nu.uniform(N, nu_lo, nu_hi)
    elif nu_dist == "loguniform":
        nu = np.exp(s_nu.uniform(N, math.log(nu_lo), math.log(nu_hi)))
    else:
        raise ValueError(nu_dist)
    w = s_dem.exponential(J)
    w = w / w.sum()
    lam_total = load * float(nu.sum())
    lam_j = lam_total * w
    pref = distance_preferences(units_xy, nodes_xy)
    return Instance(N=N, J=J, lam_j=lam_j.astype(np.float64), nu=nu.astype(np.float64),
                    pref=pref, mode=mode, C=C, name=name, units_xy=units_xy, nodes_xy=nodes_xy)


# ---- the workloads the solver is measured and checked on --------------------------------

def small_loss_n10(seed: int = 1001) -> Instance:
    """N=10 units, J=50 nodes, loss system, nu ~ U[0.8,1.2], load 0.5 (dense-solve size)."""
    return geometric_instance(10, 50, seed, 0.5, nu_lo=0.8, nu_hi=1.2, name=f"loss_n10_j50_s{seed}")


def mixed_n20(seed: int = 2001, load: float = 0.6) -> Instance:
    """N=20 units, J=500 nodes, loss system, nu ~ U[0.5,1.5], load 0.3/0.6/0.9."""
    return geometric_instance(20, 500, seed, load, nu_lo=0.5, nu_hi=1.5,
                              name=f"loss_n20_j500_l{load}_s{seed}")


def large_infinite_n24(seed: int = 3001, N: int = 24, J: int = 1000) -> Instance:
    """N=24 units, J=1000 clustered nodes (4 Gaussian clusters, sigma 0.1), infinite queue,
    nu log-uniform on [1,3], load 0.8.  N and J may be shrunk for tests of the same shape."""
    return geometric_instance(N, J, seed, 0.8, nu_lo=1.0, nu_hi=3.0, nu_dist="loguniform",
                              nodes="clusters", mode=INFINITE, name=f"inf_n{N}_j{J}_s{seed}")


def batch_n12_18(count: int = 256, base_seed: int = 4000, J: int = 200) -> list[Instance]:
    """count deployments, N ~ U{12..18}, J=200, nu ~ U[0.7,1.3], load ~ U[0.4,0.9], loss."""
    out = []
    for c in range(count):
        s = Stream(base_seed + c, 9)
        N = int(s.integers(1, 12, 18)[0])
        load = float(s.uniform(1, 0.4, 0.9)[0])
        out.append(geometric_instance(N, J, base_seed + c, load, nu_lo=0.7, nu_hi=1.3,
                                      name=f"batch_n{N}_s{base_seed + c}"))
    return out


def warmstart_instance(seed: int, N: int = 16, J: int = 300) -> Instance:
    """Training/evaluation instances for the learned warm start: nu ~ U[0.5,1.5],
    load ~ U[0.3,0.9], loss system."""
    load = float(Stream(seed, 10).uniform(1, 0.3, 0.9)[0])
    return geometric_instance(N, J, seed, load, nu_lo=0.5, nu_hi=1.5, name=f"ws_n{N}_s{seed}")


def homogeneous_instance(N: int, J: int, seed: int, load: float, nu: float = 1.0,
                         mode: int = LOSS, C: int = 0) -> Instance:
    """Equal service rates (the Corollary's homogeneous setting)."""
    inst = geometric_instance(N, J, seed, load, nu_lo=nu, nu_hi=nu, mode=mode, C=C,
                              name=f"homog_n{N}_s{seed}")
    inst.nu = np.full(N, float(nu))
    inst.lam_j = inst.lam_j / inst.lam_j.sum() * load * N * nu
    return inst


# ---- inputs of the discrete-event simulation (Section 5.5) ------------------------------

def travel_times(inst: Instance) -> np.ndarray:
    """J x N response times: the Euclidean distance from unit i's station to node j in the
    unit square (a synthetic stand-in for the paper's road travel times)."""
    d = inst.nodes_xy[:, None, :] - inst.units_xy[None, :, :]
    return np.sqrt((d * d).sum(axis=2))


def des_instance(seed: int, N: int = 10, load: float = 0.5, J: int = 71) -> Instance:
    """Loss-system instances of the service-distribution check: N = 8..12 units, J = 71
    demand nodes uniform in the unit square (the St. Paul case has 71 census tracts),
    nu_i = 1 +- U[-0.2, 0.2] (the paper's heterogeneity adjustment), a given load."""
    return geometric_instance(N, J, seed, load, nu_lo=0.8, nu_hi=1.2,
                              name=f"des_n{N}_j{J}_l{load}_s{seed}")
