"""The seeded input generators follow the recipes they state (the field's
separable exponential covariance, the AR(1) drift, the planted patch shift,
the resampled nodes of the i.i.d. and ragged pairs, the 2^-16 grid). CPU."""
import math

import numpy as np

from workloads import GRID, LIMIT, field_sequence, iid_pair, ragged_pairs


def _corr(a, b):
    a = a - a.mean(axis=-1, keepdims=True)
    b = b - b.mean(axis=-1, keepdims=True)
    return float(np.mean((a * b).mean(-1) / np.sqrt((a * a).mean(-1) * (b * b).mean(-1))))


def _on_grid(x):
    return np.all(np.rint(x / GRID) * GRID == x) and np.all(np.abs(x) <= LIMIT)


def test_field_has_separable_exponential_covariance():
    R, C, T, ell = 24, 40, 3000, 5.0
    wl = field_sequence(R, C, T, 1, ell=ell, seed=3)
    F = wl.X[0].reshape(R, C, T)
    assert _on_grid(wl.X[0])
    assert abs(float(F.var(axis=-1).mean()) - 1.0) < 0.03
    rho = math.exp(-1.0 / ell)
    for dr, dc in [(0, 1), (1, 0), (1, 1), (0, 3), (2, 1)]:
        c = _corr(F[: R - dr, : C - dc], F[dr:, dc:])
        assert abs(c - rho ** (dr + dc)) < 0.015, (dr, dc, c)


def test_field_drift_and_planted_patch():
    R, C, T = 16, 24, 2000
    wl = field_sequence(R, C, T, 3, patch=4, patch_transition=1, patch_shift=1.0, seed=4)
    d0 = wl.X[1] - wl.X[0]                        # delta_0 = 0.1 sqrt(0.19) field
    assert abs(float(d0.std()) - 0.1 * math.sqrt(0.19)) < 0.003
    assert len(wl.planted[0]) == 0 and len(wl.planted[1]) == 16
    patch = wl.planted[1]
    r0, c0 = (R - 4) // 2, (C - 4) // 2
    assert sorted(patch.tolist()) == sorted((r0 + a) * C + c0 + b for a in range(4) for b in range(4))
    d1 = wl.X[2] - wl.X[1]                        # delta_1 (+1 on the patch)
    others = np.setdiff1d(np.arange(R * C), patch)
    assert abs(float(d1[patch].mean()) - 1.0) < 0.02
    assert abs(float(d1[others].mean())) < 0.02
    # delta_1 = 0.9 delta_0 + 0.1 sqrt(0.19) field_1 off the patch
    resid = d1[others] - 0.9 * d0[others]
    assert abs(float(resid.std()) - 0.1 * math.sqrt(0.19)) < 0.003


def test_iid_pair_resamples_only_the_planted_nodes():
    wl = iid_pair(500, 32, 7, seed=9)
    X1, X2 = wl.X
    assert _on_grid(X1) and _on_grid(X2)
    changed = np.nonzero(np.any(X1 != X2, axis=1))[0]
    assert changed.tolist() == wl.planted[0].tolist() and len(changed) == 7
    assert abs(float(X1.mean())) < 0.02 and abs(float(X1.std()) - 1.0) < 0.02


def test_ragged_pairs_sizes_and_perturbations():
    pairs = ragged_pairs(64, 256, 4096, 64, seed=7)
    ns = np.array([p.X[0].shape[0] for p in pairs])
    assert len(pairs) == 64 and ns.min() >= 256 and ns.max() <= 4096
    # log-uniform: the logs' mean near the midpoint, spread near (ln 16)^2 / 12
    lg = np.log(ns)
    assert abs(float(lg.mean()) - math.log(1024)) < 0.25
    assert abs(float(lg.var()) - math.log(16) ** 2 / 12) < 0.2
    for p in pairs:
        changed = np.nonzero(np.any(p.X[0] != p.X[1], axis=1))[0]
        assert 1 <= len(changed) <= 5 and changed.tolist() == p.planted[0].tolist()
