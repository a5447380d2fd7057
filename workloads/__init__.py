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
* ``gmm_pair``: the paper's synthetic data (Sec. 4.2.1, "Synthetic Data"):
  n points of a 2-D mixture of 4 Gaussians, the same points with small
  Gaussian noise, and a sparse random matrix R whose symmetrised half
  (R + R^T) / 2 is added to the second graph; ground truth marks the added
  edges that join different clusters. The kernel matrices themselves are the
  method's graph build and are not formed here.
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


@dataclass
class GMMPair:
    """Points of the synthetic mixture pair (Sec. 4.2.1, "Synthetic Data").

    ``X``: the two n x 2 point sets (float64 on the 2**-16 grid); graph t is
    the kernel graph of X[t] and graph 2 additionally gets the edge weights
    ``w`` on the node pairs ``ij``. ``ij``: (m, 2) int64, i < j, ascending
    in (i, j); ``w``: (m,) float64, w = (R_ij + R_ji) / 2 > 0 with R_ij and
    R_ji independent draws of the paper's R (zero with probability 1 - p,
    else uniform on (0, 1], here on the 2**-16 grid, so w is exact).
    ``labels``: mixture component of each point. ``truth``: (m,) bool, the
    added edges that join different components (the anomalous edges); the
    anomalous nodes are their endpoints."""
    X: List[np.ndarray]
    labels: np.ndarray
    ij: np.ndarray
    w: np.ndarray
    truth: np.ndarray
    meta: dict = field(default_factory=dict)

    def anomalous_nodes(self) -> np.ndarray:
        t = self.ij[self.truth]
        return np.unique(t.reshape(-1))


def _upper_pair(flat: np.ndarray, n: int):
    """Row-major position in the strict upper triangle -> (i, j)."""
    i_all = np.arange(n - 1, dtype=np.int64)
    start = i_all * (2 * n - i_all - 1) // 2          # first position of row i
    i = np.searchsorted(start, flat, side="right") - 1
    j = flat - start[i] + i + 1
    return i, j


def _bernoulli_positions(rng: np.random.Generator, M: int, p: float) -> np.ndarray:
    """Sorted positions in [0, M) of independent Bernoulli(p) successes
    (geometric gaps between successes)."""
    out = []
    pos = -1
    while True:
        cnt = int(max(1024, 1.05 * p * max(M - pos, 0) + 64))
        gaps = rng.geometric(p, size=cnt)
        cs = pos + np.cumsum(gaps)
        keep = cs[cs < M]
        out.append(keep)
        if keep.size < cs.size:
            break
        pos = int(cs[-1])
    return np.concatenate(out).astype(np.int64)


def gmm_pair(n: int = 2000, p: float = 0.05, noise: float = 0.05, sep: float = 3.0,
             seed: int = 11) -> GMMPair:
    """Mixture of 4 unit-covariance Gaussians in the plane with means
    (+-sep, +-sep), equal weights; graph 2's points are graph 1's plus
    N(0, noise^2) per coordinate; R_ij ~ p-Bernoulli times U(0, 1] for every
    ordered pair i != j (the diagonal is left out: the graphs have no self
    edges)."""
    rng = np.random.default_rng(seed)
    labels = rng.integers(0, 4, size=n).astype(np.int64)
    means = np.array([[-sep, -sep], [-sep, sep], [sep, -sep], [sep, sep]])
    X1 = to_grid(means[labels] + rng.standard_normal((n, 2)))
    X2 = to_grid(X1 + noise * rng.standard_normal((n, 2)))
    M = n * (n - 1) // 2
    pos, val = [], []
    for _ in range(2):                                  # R_ij (i < j), then R_ji
        q = _bernoulli_positions(rng, M, p)
        u = rng.integers(1, (1 << 16) + 1, size=q.size).astype(np.float64) * GRID
        pos.append(q)
        val.append(u)
    (q1, q2), (u1, u2) = pos, val
    # union of the two sorted position lists, values added where both drew
    at = np.searchsorted(q1, q2)
    both = at < q1.size
    both[both] = q1[at[both]] == q2[both]
    u1 = u1.copy()
    u1[at[both]] += u2[both]
    allpos = np.concatenate([q1, q2[~both]])
    order = np.argsort(allpos, kind="stable")           # merge of two sorted runs
    uniq = allpos[order]
    w = np.concatenate([u1, u2[~both]])[order] * 0.5
    i, j = _upper_pair(uniq, n)
    ij = np.ascontiguousarray(np.stack([i, j], axis=1).astype(np.int64))
    truth = labels[i] != labels[j]
    return GMMPair([np.ascontiguousarray(X1), np.ascontiguousarray(X2)], labels, ij, w, truth,
                   dict(kind="gmm_pair", n=n, p=p, noise=noise, sep=sep, seed=seed))


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
