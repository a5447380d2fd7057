"""Seeded synthetic inputs for the commute-time anomaly-detection path.

This module is shared by the tests, the benchmark and the oracle checks. It
only draws node time series; it contains none of the method's arithmetic
(no distances, kernels, Laplacians, projections or scores).

Every series value is rounded to a multiple of 2**-16 with magnitude below
2**7. Such values are exactly representable in float32 and as int32 fixed
point, and the difference of two of them squared is exact in float64, so a
squared distance over T <= 2**12 samples is an exact float64 number whatever
order its terms are added in.

Workloads (all stand-ins for the paper's gridded precipitation graphs and its
synthetic graphs; none of the paper's datasets is used):

* ``iid_pair``: n nodes, T-sample N(0,1) series; graph 2 resamples the
  series of ``n_changed`` randomly chosen nodes from the same stream.
* ``field_sequence``: nodes on an R x C lat-lon grid; each time sample is an
  independent unit-variance Gaussian field with separable exponential
  covariance exp(-|dr|/l - |dc|/l), generated exactly as an AR(1) filter with
  rho = exp(-1/l) along rows and then along columns. Successive graphs add an
  AR(1) drift; an optional patch of nodes is shifted by ``patch_shift``
  (in field standard deviations) in one transition.
* ``ragged_pairs``: G independent pairs with n log-uniform in [n_lo, n_hi],
  N(0,1) series, 1-5 perturbed nodes per pair.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

GRID = 2.0 ** -16
LIMIT = 2.0 ** 7 - GRID


def to_grid(x: np.ndarray) -> np.ndarray:
    """Round to the nearest multiple of 2**-16, clipped to |x| < 2**7 (float64 out)."""
    y = np.rint(np.asarray(x, dtype=np.float64) / GRID) * GRID
    return np.clip(y, -LIMIT, LIMIT)


@dataclass
class GraphPairs:
    """A sequence of node-series matrices (each n x T, float64, C-contiguous).

    Consecutive entries of ``X`` form the graph pairs. ``planted`` lists, per
    transition, the node indices whose series were perturbed (ground truth
    for the semantic check; not used by any computation)."""
    X: List[np.ndarray]
    planted: List[np.ndarray] = field(default_factory=list)
    meta: dict = field(default_factory=dict)


def iid_pair(n: int = 1024, T: int = 64, n_changed: int = 10, seed: int = 0) -> GraphPairs:
    rng = np.random.default_rng(seed)
    X1 = to_grid(rng.standard_normal((n, T)))
    idx = np.sort(rng.choice(n, size=n_changed, replace=False))
    X2 = X1.copy()
    X2[idx] = to_grid(rng.standard_normal((n_changed, T)))
    return GraphPairs([np.ascontiguousarray(X1), np.ascontiguousarray(X2)], [idx],
                      dict(kind="iid_pair", n=n, T=T, n_changed=n_changed, seed=seed))


def _exp_field(rng: np.random.Generator, R: int, C: int, T: int, ell: float) -> np.ndarray:
    """Unit-variance field, separable exponential covariance, shape (R, C, T)."""
    rho = math.exp(-1.0 / ell)
    s = math.sqrt(1.0 - rho * rho)
    g = rng.standard_normal((R, C, T))
    for r in range(1, R):
        g[r] = rho * g[r - 1] + s * g[r]
    for c in range(1, C):
        g[:, c] = rho * g[:, c - 1] + s * g[:, c]
    return g


def field_sequence(R: int, C: int, T: int, n_graphs: int, ell: float = 5.0,
                   patch: int = 8, patch_transition: Optional[int] = 1,
                   patch_shift: float = 1.0, seasonal: float = 0.0,
                   seed: int = 1) -> GraphPairs:
    """Graph g's series: X_0 = field; X_{g+1} = X_g + delta_g with
    delta_g = 0.9 delta_{g-1} + 0.1 sqrt(1 - 0.81) field_g (delta_{-1} = 0).
    In transition ``patch_transition`` (graph index t -> t+1) a patch x patch
    block of grid cells centred in the grid gets +patch_shift on every sample.
    ``seasonal`` adds seasonal * sin(2 pi t / 365 + phase_row) to all nodes."""
    rng = np.random.default_rng(seed)
    n = R * C
    base = _exp_field(rng, R, C, T, ell).reshape(n, T)
    if seasonal:
        phase = np.repeat(np.linspace(0.0, math.pi, R), C)[:, None]
        base = base + seasonal * np.sin(2.0 * math.pi * np.arange(T)[None, :] / 365.0 + phase)
    xs = [base]
    delta = np.zeros_like(base)
    planted = []
    r0, c0 = (R - patch) // 2, (C - patch) // 2
    patch_nodes = np.array([(r0 + a) * C + (c0 + b) for a in range(patch) for b in range(patch)],
                           dtype=np.int64)
    for g in range(n_graphs - 1):
        delta = 0.9 * delta + 0.1 * math.sqrt(1.0 - 0.81) * _exp_field(rng, R, C, T, ell).reshape(n, T)
        nxt = xs[-1] + delta
        if patch_transition is not None and g == patch_transition:
            nxt = nxt.copy()
            nxt[patch_nodes] += patch_shift
            planted.append(patch_nodes)
        else:
            planted.append(np.zeros(0, dtype=np.int64))
        xs.append(nxt)
    X = [np.ascontiguousarray(to_grid(x)) for x in xs]
    return GraphPairs(X, planted, dict(kind="field_sequence", R=R, C=C, T=T, n=n, ell=ell,
                                       patch=patch, patch_transition=patch_transition,
                                       patch_shift=patch_shift, seasonal=seasonal, seed=seed))


def ragged_pairs(G: int = 64, n_lo: int = 256, n_hi: int = 4096, T: int = 64,
                 seed: int = 7) -> List[GraphPairs]:
    rng = np.random.default_rng(seed)
    ns = np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=G)).astype(np.int64)
    out = []
    for g in range(G):
        n = int(ns[g])
        X1 = to_grid(rng.standard_normal((n, T)))
        cnt = int(rng.integers(1, 6))
        idx = np.sort(rng.choice(n, size=cnt, replace=False))
        X2 = X1.copy()
        X2[idx] = to_grid(rng.standard_normal((cnt, T)))
        out.append(GraphPairs([np.ascontiguousarray(X1), np.ascontiguousarray(X2)], [idx],
                              dict(kind="ragged_pair", n=n, T=T, seed=seed, index=g)))
    return out


# Named workloads with the method parameters they are run with.
CONFIGS = {
    "iid_n1024": dict(make=lambda: iid_pair(1024, 64, 10, 0), k=32, d=8, topk=10),
    "field_n8192_seq4": dict(make=lambda: field_sequence(64, 128, 128, 4, patch=8,
                                                         patch_transition=1, seed=1),
                             k=64, d=12, topk=10),
    "field_n32768_pair": dict(make=lambda: field_sequence(128, 256, 256, 2, patch=8,
                                                          patch_transition=0, seed=2),
                              k=128, d=14, topk=10),
}
