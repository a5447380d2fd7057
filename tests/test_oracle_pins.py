"""Pins of the float64 oracle against facts fixed by the paper and by the
mathematics (closed forms, invariants, brute force, hand-derived fixtures).
CPU only."""
import itertools
import math
import os
import statistics
from fractions import Fraction

import numpy as np
import pytest
import scipy.spatial.distance

from oracle import caddelag as O
from oracle import philox as P
from workloads import iid_pair, to_grid, field_sequence

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([int(v) for v in line.split()])
    return rows


def _random_graph(n, seed, lo=0.05):
    rng = np.random.default_rng(seed)
    W = rng.uniform(lo, 1.0, (n, n))
    A = np.triu(W, 1)
    return A + A.T


# ---------------------------------------------------------------- Philox

def test_philox_weyl_constants_closed_form():
    # golden ratio and sqrt(3) fractional parts, 32-bit (Philox key schedule)
    golden = (math.sqrt(5.0) - 1.0) / 2.0
    assert P.WEYL0 == int(golden * 2 ** 32)
    assert P.WEYL1 == int((math.sqrt(3.0) - 1.0) * 2 ** 32)


def test_philox_is_injective_and_balanced():
    n = 1 << 16
    c = np.arange(n, dtype=np.uint64)
    w = P.philox4x32(c, 7, 0, 0, 123, 456)
    # 128-bit outputs of distinct counters must be distinct (bijection)
    packed = set(zip(*(x.tolist() for x in w)))
    assert len(packed) == n
    bits = np.unpackbits(np.stack(w).view(np.uint8))
    m = bits.size
    # bit frequency within 6 sigma of 1/2
    assert abs(bits.mean() - 0.5) < 6 * 0.5 / math.sqrt(m)
    # each of the 128 output bit positions is balanced
    words = np.stack(w, axis=1)  # (n, 4)
    for wi in range(4):
        for b in range(32):
            f = ((words[:, wi] >> np.uint32(b)) & 1).mean()
            assert abs(f - 0.5) < 6 * 0.5 / math.sqrt(n)


def test_philox_key_and_counter_sensitivity():
    base = P.philox4x32(1, 2, 3, 4, 5, 6)
    for args in [(0, 2, 3, 4, 5, 6), (1, 2, 3, 5, 5, 6), (1, 2, 3, 4, 5, 7), (1, 2, 3, 4, 4, 6)]:
        other = P.philox4x32(*args)
        diff = sum(bin(int(a) ^ int(b)).count("1") for a, b in zip(base, other))
        assert 30 < diff < 98   # avalanche: about half of 128 bits flip


def test_philox_rounds_zero_is_identity_like():
    # with zero rounds the counter passes through unchanged (structure check)
    out = P.philox4x32(11, 22, 33, 44, 5, 6, rounds=0)
    assert [int(x) for x in out] == [11, 22, 33, 44]


def test_philox_single_round_by_hand():
    # one round written out with Python integers: products of words 0 and 2
    c0, c1, c2, c3, k0, k1 = 0x01234567, 0x89ABCDEF, 0xDEADBEEF, 0x0BADF00D, 0x13579BDF, 0x2468ACE0
    p0 = P.MUL0 * c0
    p1 = P.MUL1 * c2
    expect = [(p1 >> 32) ^ c1 ^ k0, p1 & 0xFFFFFFFF, (p0 >> 32) ^ c3 ^ k1, p0 & 0xFFFFFFFF]
    got = [int(x) for x in P.philox4x32(c0, c1, c2, c3, k0, k1, rounds=1)]
    assert got == expect


def test_edge_signs_are_iid_pm1():
    n = 300
    iu, ju = np.triu_indices(n, 1)
    bits = P.edge_sign_bits(99, iu, ju, 200)   # spans two 128-sign blocks
    s = np.where(bits, 1.0, -1.0)
    m = s.shape[0]
    # E[s_r s_t] = delta_rt: empirical Gram of the sign columns
    G = s.T @ s / m
    off = G - np.diag(np.diag(G))
    assert np.allclose(np.diag(G), 1.0)
    assert np.abs(off).max() < 6 / math.sqrt(m)
    assert abs(s.mean()) < 6 / math.sqrt(s.size)


# ---------------------------------------------------------------- graph

def test_squared_distances_match_scipy():
    rng = np.random.default_rng(1)
    X = rng.standard_normal((37, 11))
    d2 = O.squared_distances(X)
    ref = scipy.spatial.distance.cdist(X, X, "sqeuclidean")
    assert np.allclose(d2, ref, rtol=1e-13, atol=1e-13)
    assert np.array_equal(d2, d2.T)
    assert np.all(np.diag(d2) == 0.0)


def test_squared_distances_brute_force_scalar():
    X = to_grid(np.random.default_rng(2).standard_normal((5, 3)))
    d2 = O.squared_distances(X)
    for i, j in itertools.product(range(5), range(5)):
        acc = 0.0
        for t in range(3):
            diff = X[i, t] - X[j, t]
            acc = acc + diff * diff
        assert d2[i, j] == acc


def test_exact_grid_distances_bit_equal():
    X = iid_pair(300, 64, 5, 3).X[0]
    assert np.array_equal(O.squared_distances(X), O.squared_distances_exact_grid(X))
    Xf = field_sequence(8, 16, 40, 2, seed=4).X[1]
    assert np.array_equal(O.squared_distances(Xf), O.squared_distances_exact_grid(Xf))
    with pytest.raises(ValueError):
        O.squared_distances_exact_grid(X + 1e-9)


def test_median_sigma_brute_force():
    rng = np.random.default_rng(3)
    for n in (2, 3, 4, 9, 16):
        X = rng.standard_normal((n, 4))
        d = [math.dist(X[i], X[j]) for i in range(n) for j in range(i + 1, n)]
        s = O.median_sigma(O.squared_distances(X))
        assert math.isclose(s, statistics.median_low(d), rel_tol=1e-14)


def test_gaussian_graph_invariants_and_entries():
    X = iid_pair(64, 16, 3, 5).X[0]
    A, D, vol, sigma = O.gaussian_graph(X)
    assert np.array_equal(A, A.T)
    assert np.all(np.diag(A) == 0.0)
    off = A[~np.eye(64, dtype=bool)]
    assert np.all(off > 0.0) and np.all(off <= 1.0)
    assert np.allclose(D, A.sum(1), rtol=1e-15) and math.isclose(vol, D.sum(), rel_tol=1e-15)
    i, j = 3, 41
    d2 = sum((X[i, t] - X[j, t]) ** 2 for t in range(16))
    assert math.isclose(A[i, j], math.exp(-d2 / (2 * sigma * sigma)), rel_tol=1e-14)
    # half of the off-diagonal kernel values are >= exp(-1/2) (median rule)
    frac = np.mean(A[np.triu_indices(64, 1)] >= math.exp(-0.5) * (1 - 1e-15))
    assert 0.5 <= frac <= 0.5 + 2.0 / (64 * 63 / 2)


def test_graph_rows_match_full():
    X = iid_pair(50, 8, 2, 6).X[0]
    A, D, vol, sigma = O.gaussian_graph(X)
    rows = [0, 7, 49]
    assert np.array_equal(O.graph_rows(X, sigma, rows), A[rows])


def test_incidence_gives_laplacian():
    A = _random_graph(9, 4)
    B, w, _ = O.incidence(A)
    assert np.allclose(B.T @ (w[:, None] * B), O.laplacian(A), atol=1e-14)
    # every edge row has one head (+1) at the lower index and one tail (-1)
    assert np.all(B.sum(1) == 0) and np.all((B == 1).sum(1) == 1)
    assert np.all(np.argmax(B == 1, axis=1) < np.argmax(B == -1, axis=1))


# ---------------------------------------------------------------- commute times

def test_golden_triangle_commute_times():
    A = np.zeros((3, 3))
    rows = _read_golden("triangle_commute.txt")
    for i, j, a, num, den in rows:
        A[i, j] = A[j, i] = a
    C = O.commute_times_pinv(A)
    for i, j, a, num, den in rows:
        assert math.isclose(C[i, j], num / den, rel_tol=1e-13)
    # Foster: sum_{i<j} A_ij c_ij / vol = n - 1
    vol = A.sum()
    assert math.isclose(sum(A[i, j] * C[i, j] for i, j, *_ in rows) / vol, 2.0, rel_tol=1e-13)


def test_golden_path_commute_times():
    A = np.zeros((4, 4))
    for i, j, a in [(0, 1, 2), (1, 2, 1), (2, 3, 4)]:
        A[i, j] = A[j, i] = a
    C = O.commute_times_pinv(A)
    for i, j, num, den in _read_golden("path_commute.txt"):
        assert math.isclose(C[i, j], num / den, rel_tol=1e-13)


def test_complete_graph_commute_time_closed_form():
    for n in (3, 8, 33):
        A = np.ones((n, n)) - np.eye(n)
        C = O.commute_times_pinv(A)
        off = C[~np.eye(n, dtype=bool)]
        assert np.allclose(off, 2 * (n - 1), rtol=1e-12)
        # and through the embedding of the full projection Q = I_m
        B, w, _ = O.incidence(A)
        Y = B.T * np.sqrt(w)[None, :]
        Z = O.exact_embedding(A, Y)
        Ce = O.commute_times(Z, A.sum())
        assert np.allclose(Ce[~np.eye(n, dtype=bool)], 2 * (n - 1), rtol=1e-11)


def test_full_projection_embedding_reproduces_eq1():
    # with Q = I_m the embedding gives Z Z^T = L^+ B^T W B L^+ = L^+, i.e. Eq. 1
    A = _random_graph(12, 8)
    B, w, _ = O.incidence(A)
    Y = B.T * np.sqrt(w)[None, :]
    Z = O.exact_embedding(A, Y)
    assert np.allclose(O.commute_times(Z, A.sum()), O.commute_times_pinv(A), rtol=1e-10, atol=1e-10)


def test_foster_theorem_random_graph():
    A = _random_graph(30, 9)
    C = O.commute_times_pinv(A)
    vol = A.sum()
    iu = np.triu_indices(30, 1)
    assert math.isclose((A[iu] * C[iu]).sum() / vol, 29.0, rel_tol=1e-11)


def test_commute_times_are_squared_metric():
    A = _random_graph(15, 10)
    C = O.commute_times_pinv(A)
    R = np.sqrt(np.maximum(C, 0))
    assert np.allclose(C, C.T, atol=1e-12) and np.allclose(np.diag(C), 0, atol=1e-10)
    assert np.all(C[~np.eye(15, dtype=bool)] > 0)
    for i, j, l in itertools.permutations(range(15), 3):
        assert R[i, j] <= R[i, l] + R[l, j] + 1e-10


# ---------------------------------------------------------------- projection

def test_project_matches_incidence_form():
    X = iid_pair(40, 8, 2, 11).X[0]
    A, *_ = O.gaussian_graph(X)
    for k in (5, 130):
        Q = O.projection_matrix(40, 2024, k)
        assert np.allclose(O.project(A, 2024, k), O.project_explicit(A, Q), rtol=1e-13, atol=1e-14)


def test_c_projection_matches_numpy_and_incidence_form():
    X = iid_pair(150, 8, 2, 12).X[0]
    A, *_ = O.gaussian_graph(X)
    for k, seed in ((7, 3), (128, 2 ** 33 + 5), (200, 11)):
        Yc = O.project_rows_c(A, range(150), seed, k)
        assert np.allclose(Yc, O.project(A, seed, k), rtol=1e-13, atol=1e-13)
        assert np.allclose(Yc, O.project_explicit(A, O.projection_matrix(150, seed, k)), rtol=1e-12, atol=1e-13)
    assert np.allclose(O.project_rows_c(A[[5, 90]], [5, 90], 4, 16), O.project(A, 4, 16)[[5, 90]], rtol=1e-13)


def test_project_columns_sum_to_zero_and_rows():
    A = _random_graph(50, 12)
    Y = O.project(A, 5, 16)
    assert np.abs(Y.sum(0)).max() < 1e-12 * np.abs(Y).max() * 50
    assert np.array_equal(O.project_rows(A[[3, 17]], [3, 17], 5, 16), Y[[3, 17]])


def test_complete_graph_embedding_is_y_over_n():
    n = 17
    A = np.ones((n, n)) - np.eye(n)
    Y = O.project(A, 77, 8)
    Z = O.exact_embedding(A, Y)
    assert np.allclose(Z, Y / n, atol=1e-14)


def test_projection_is_unbiased_for_commute_times():
    # E[c_ij] over random sign matrices equals the exact commute time (JL mean)
    A = _random_graph(10, 13)
    exact = O.commute_times_pinv(A)
    acc = np.zeros_like(exact)
    reps = 60
    for s in range(reps):
        Z = O.exact_embedding(A, O.project(A, 1000 + s, 64))
        acc += O.commute_times(Z, A.sum())
    mean = acc / reps
    rel = np.abs(mean - exact)[~np.eye(10, dtype=bool)] / exact[~np.eye(10, dtype=bool)]
    # std of one estimate is about sqrt(2/k) = 0.18; of the mean 0.18/sqrt(60) = 0.023
    assert rel.max() < 0.12


# ---------------------------------------------------------------- solver (Alg. 2)

def test_exact_embedding_is_pseudoinverse_solution():
    A = _random_graph(40, 14)
    Y = O.project(A, 3, 6)
    Z = O.exact_embedding(A, Y)
    Lp = np.linalg.pinv(O.laplacian(A))
    D = A.sum(1)
    ref = O.dweighted_center(Lp @ Y, D)
    assert np.allclose(Z, ref, rtol=1e-10, atol=1e-12)
    assert O.residual_norm(A, Y, Z) < 1e-13
    assert np.abs(D @ Z).max() < 1e-12 * np.abs(Z).max() * D.sum()


def test_chain_closed_form_complete_graph():
    # K_n: S = (J - I)/(n-1), eigenvalue s = -1/(n-1) on the complement of 1,
    # P1 b = (1 - s^(2^d))/n b; after j updates y = (1 - s^(2^d j))/n b
    n, d, q = 7, 3, 4
    A = np.ones((n, n)) - np.eye(n)
    L = O.laplacian(A)
    P1, P2 = O.chain_product(L, d)
    s = -1.0 / (n - 1)
    b = np.random.default_rng(0).standard_normal(n)
    b -= b.mean()
    assert np.allclose(P1 @ b, (1 - s ** (2 ** d)) / n * b, atol=1e-14)
    y = O.estimate_solution(P1, P2, b, q)
    assert np.allclose(y, (1 - s ** (2 ** d * (q - 1))) / n * b, atol=1e-14)


def test_chain_error_operator_spectral_form():
    # I - P1 L = D^{-1/2} S^{2^d} D^{1/2} (telescoping product), via eigh of S
    A = _random_graph(25, 15)
    D = A.sum(1)
    d = 4
    P1, P2 = O.chain_product(O.laplacian(A), d)
    r = 1 / np.sqrt(D)
    lam, V = np.linalg.eigh(r[:, None] * A * r[None, :])
    S2d = (V * lam ** (2 ** d)) @ V.T
    E = (r[:, None] * S2d) * np.sqrt(D)[None, :]
    assert np.allclose(np.eye(25) - P2, E, atol=1e-12)
    # and P1 itself: D^{-1/2} V diag(prod (1 + lam^(2^i))) V^T D^{-1/2}
    f = np.prod([1 + lam ** (2 ** i) for i in range(d)], axis=0)
    assert np.allclose(P1, r[:, None] * ((V * f) @ V.T) * r[None, :], atol=1e-12)


def test_chain_levels_are_powers():
    A = _random_graph(12, 16)
    lv = O.chain_levels(A, 4)
    S = lv[0]
    assert np.allclose(lv[3], np.linalg.matrix_power(S, 8), atol=1e-14)


def test_chain_level0_is_the_normalised_adjacency():
    """Level 0 of Alg. 2's ChainProduct is S = D^{-1/2} A D^{-1/2}: symmetric,
    eigenvalue 1 with eigenvector D^{1/2} 1, the same spectrum as the random-
    walk matrix D^{-1} A (similar to S), all eigenvalues in [-1, 1]; on the
    unit-weight complete graph K_n it is (J - I) / (n - 1) exactly. A wrong
    normalisation (D^{-1} A, A D^{-1}, D^{-1/2} A, a missing square root)
    fails at least one of these; level i is S^{2^i} through S's own
    eigenbasis (not by repeated products)."""
    A = _random_graph(40, 21)
    D = A.sum(1)
    lv = O.chain_levels(A, 4)
    S = lv[0]
    assert np.allclose(S, S.T, rtol=4e-16, atol=0)        # (r_i A_ij) r_j vs (r_j A_ji) r_i
    v = np.sqrt(D)
    assert np.allclose(S @ v, v, rtol=0, atol=1e-14 * np.abs(v).max())
    lam = np.linalg.eigvalsh(S)
    rw = np.sort(np.linalg.eigvals(A / D[:, None]).real)
    assert np.allclose(lam, rw, atol=1e-12)
    assert abs(lam[-1] - 1.0) <= 1e-13 and lam[0] >= -1.0 - 1e-13
    lam_all, V = np.linalg.eigh(S)
    for i in (1, 2, 3):
        assert np.allclose(lv[i], (V * lam_all ** (2 ** i)) @ V.T, atol=1e-13)
    for n in (2, 5, 9):
        Kn = np.ones((n, n)) - np.eye(n)
        S0 = O.chain_levels(Kn, 1)[0]
        assert np.allclose(S0, Kn / (n - 1), rtol=0, atol=1e-15)


def test_literal_solver_converges_to_exact():
    A = _random_graph(60, 17, lo=0.3)
    Y = O.project(A, 8, 10)
    Zl = O.literal_embedding(A, Y, d=8, q=6)
    Ze = O.exact_embedding(A, Y)
    assert np.allclose(Zl, Ze, rtol=1e-10, atol=1e-13)


def test_literal_solver_keeps_dweighted_mean():
    A = _random_graph(30, 18)
    Y = O.project(A, 9, 4)
    P1, P2 = O.chain_product(O.laplacian(A), 5)
    y = O.estimate_solution(P1, P2, Y, 4)
    D = A.sum(1)
    assert np.abs(D @ y).max() < 1e-10 * np.abs(y).max() * D.sum()


def test_richardson_and_dimension_helpers():
    assert O.richardson_count(1e-4) == 10      # ceil(ln 1e4) = ceil(9.21)
    assert O.projection_dim(2000, 1e-2) == 13  # ceil(ln 2e5) = ceil(12.2)


# ---------------------------------------------------------------- scores (Alg. 4)

def test_scores_brute_force_and_invariants():
    n = 12
    A1 = _random_graph(n, 20)
    A2 = A1.copy()
    A2[2, 5] = A2[5, 2] = A1[2, 5] * 3
    A2[7, 9] = A2[9, 7] = A1[7, 9] * 0.2
    Y1 = O.project(A1, 4, 50)
    Y2 = O.project(A2, 4, 50)
    Z1, Z2 = O.exact_embedding(A1, Y1), O.exact_embedding(A2, Y2)
    v1, v2 = A1.sum(), A2.sum()
    F = O.node_scores(A1, A2, Z1, Z2, v1, v2)
    C1, C2 = O.commute_times(Z1, v1), O.commute_times(Z2, v2)
    for i in range(n):
        ref = 0.0
        for j in range(n):
            ref += abs(A1[i, j] - A2[i, j]) * abs(C2[i, j] - C1[i, j])
        assert math.isclose(F[i], ref, rel_tol=1e-12)
    assert np.all(F >= 0)
    dE = O.edge_scores(A1, A2, C1, C2)
    iu = np.triu_indices(n, 1)
    assert math.isclose(F.sum(), 2 * dE[iu].sum(), rel_tol=1e-12)
    # only nodes incident to changed edges score (edge scores vanish elsewhere)
    assert set(np.nonzero(F)[0]) == {2, 5, 7, 9}
    # same graph twice: all scores are zero
    assert np.all(O.node_scores(A1, A1, Z1, Z1, v1, v1) == 0.0)
    # centring shift leaves scores unchanged
    F2 = O.node_scores(A1, A2, Z1 + 3.0, Z2 - 1.0, v1, v2)
    assert np.allclose(F, F2, rtol=1e-9)


def test_c_node_scores_match_brute_force_and_numpy():
    """The oracle's C node scores (oracle/cscore.c) against scalar loops over
    the definition (Alg. 4: F_i = sum_j |A1 - A2|_ij |c2 - c1|_ij with
    c = vol ||z_i - z_j||^2) on a tiny pair, and against ``node_scores`` on a
    larger one, on a subset of rows and on all of them."""
    n, k = 9, 3
    A1 = _random_graph(n, 24)
    A2 = A1.copy()
    A2[1, 6] = A2[6, 1] = A1[1, 6] * 2.5
    A2[0, 3] = A2[3, 0] = 0.0
    rng = np.random.default_rng(25)
    Z1, Z2 = rng.standard_normal((n, k)), rng.standard_normal((n, k))
    v1, v2 = 3.5, 0.75
    Fc = O.node_scores_c(A1, A2, range(n), Z1, Z2, v1, v2)
    for i in range(n):
        ref = 0.0
        for j in range(n):
            if j == i:
                continue
            c1 = v1 * sum((Z1[i, r] - Z1[j, r]) ** 2 for r in range(k))
            c2 = v2 * sum((Z2[i, r] - Z2[j, r]) ** 2 for r in range(k))
            ref += abs(A1[i, j] - A2[i, j]) * abs(c2 - c1)
        assert math.isclose(Fc[i], ref, rel_tol=1e-14, abs_tol=0.0)
    assert set(np.nonzero(Fc)[0]) == {0, 1, 3, 6}
    n, k = 300, 37
    A1 = _random_graph(n, 26)
    A2 = _random_graph(n, 27)
    Z1, Z2 = rng.standard_normal((n, k)), rng.standard_normal((n, k))
    F = O.node_scores(A1, A2, Z1, Z2, 2.0, 5.0)
    assert np.allclose(O.node_scores_c(A1, A2, range(n), Z1, Z2, 2.0, 5.0), F, rtol=1e-13, atol=0)
    rows = [299, 0, 17, 17, 150]
    assert np.allclose(O.node_scores_c(A1[rows], A2[rows], rows, Z1, Z2, 2.0, 5.0), F[rows], rtol=1e-13, atol=0)


def test_grid_distance_counts_locate_the_lower_median():
    """The streamed counts against sorted brute-force distances: the lower
    median's integer key k (||x_i - x_j||^2 2^32) has count_below <= rank <
    count_at_most, a key between two distance values has count_below ==
    count_at_most, and the counts at the smallest and beyond the largest key
    are 0 and m. Row blocks smaller than n exercise the block seams."""
    wl = iid_pair(157, 9, 1, seed=41)
    X = wl.X[0]
    n = X.shape[0]
    d2 = O.squared_distances(X)
    iu = np.triu_indices(n, 1)
    keys = np.sort(np.rint(d2[iu] * 2.0 ** 32).astype(np.int64))
    m = keys.size
    rank = (m - 1) // 2
    med = int(keys[rank])
    lt, le = O.grid_distance_counts(X, med, row_block=40, threads=3)
    assert lt == int(np.count_nonzero(keys < med)) and le == int(np.count_nonzero(keys <= med))
    assert lt <= rank < le
    assert math.sqrt(med * 2.0 ** -32) == O.median_sigma(d2)
    gap = next(int(a) + 1 for a, v in zip(keys[rank:], keys[rank + 1:]) if v > a + 1)   # a < gap < v
    lt2, le2 = O.grid_distance_counts(X, gap, row_block=64)
    assert lt2 == le2 == int(np.count_nonzero(keys < gap))
    assert O.grid_distance_counts(X, int(keys[0]) - 1) == (0, 0)
    assert O.grid_distance_counts(X, int(keys[-1]) + 1) == (m, m)
    # values near 2^7 over 300 samples: (max |a|)^2 T >= 2^53, the 12-bit pieces
    rng = np.random.default_rng(44)
    W = np.rint(rng.uniform(-127.0, 127.0, (90, 300)) * 65536.0) / 65536.0
    assert (np.abs(W).max() * 65536.0) ** 2 * 300 >= 2.0 ** 53
    kw = np.sort(np.rint(O.squared_distances_exact_grid(W)[np.triu_indices(90, 1)] * 2.0 ** 32).astype(np.int64))
    medw = int(kw[(kw.size - 1) // 2])
    assert O.grid_distance_counts(W, medw, row_block=17) == (int(np.count_nonzero(kw < medw)),
                                                             int(np.count_nonzero(kw <= medw)))


def test_streamed_degrees_equal_the_dense_graph():
    """Degrees streamed over row blocks (each upper-triangle value added to
    both rows) against D = A 1 of the dense Gaussian graph (Sec. 3.2)."""
    wl = field_sequence(9, 21, 30, 1, seed=43)
    X = wl.X[0]
    A, D, vol, sig = O.gaussian_graph(X)
    Ds = O.gaussian_degrees_streamed(X, sig, row_block=50, threads=2)
    np.testing.assert_allclose(Ds, D, rtol=1e-13, atol=0)
    # the same pass with the median counts of grid_distance_counts
    key = int(round(sig * sig * 2.0 ** 32))
    D2, lt, le = O.gaussian_degrees_streamed(X, sig, row_block=37, key=key)
    assert np.array_equal(D2, Ds) or np.allclose(D2, Ds, rtol=1e-15, atol=0)
    assert (lt, le) == O.grid_distance_counts(X, key, row_block=64)
    m = X.shape[0] * (X.shape[0] - 1) // 2
    assert lt <= (m - 1) // 2 < le


def test_top_anomalies_ties_and_order():
    F = np.array([1.0, 3.0, 3.0, 2.0, 3.0, 0.5])
    assert list(O.top_anomalies(F, 4)) == [1, 2, 4, 3]
    ref = sorted(range(6), key=lambda i: (-F[i], i))[:4]
    assert list(O.top_anomalies(F, 4)) == ref
    assert O.min_relative_gap(F, 4) == 0.0


def test_pipeline_finds_planted_nodes():
    wl = iid_pair(200, 32, 4, 21)
    out = O.caddelag_pair(wl.X[0], wl.X[1], k=32, seed=5, topk=4)
    assert set(out["top"].tolist()) == set(wl.planted[0].tolist())


# ------------------------------------------------------------------ anomalous edge set (Sec. 3.3)

def _brute_min_set(v, delta):
    """Smallest number of edges whose removal leaves the rest below delta, by
    enumeration of all subsets."""
    import itertools
    m = v.size
    for size in range(m + 1):
        for sub in itertools.combinations(range(m), size):
            if v.sum() - v[list(sub)].sum() < delta:
                return size
    return None


def test_anomalous_edges_minimal_by_brute_force():
    rng = np.random.default_rng(3)
    for trial in range(30):
        n = 5
        E = np.triu(rng.exponential(size=(n, n)), 1)
        total = E.sum()
        delta = rng.uniform(0.05, 0.95) * total
        out = O.anomalous_edges(E, delta)
        iu, ju = np.triu_indices(n, 1)
        assert len(out["edges"]) == _brute_min_set(E[iu, ju], delta)
        assert out["remaining"] < delta
        # removing the smallest chosen edge from the set breaks the bound
        if len(out["edges"]):
            keep = out["values"].sum() - out["values"].min()
            assert total - keep >= delta


def test_anomalous_edges_limits_and_ties():
    E = np.triu(np.ones((4, 4)), 1)          # six equal edges
    out = O.anomalous_edges(E, 10.0)          # total 6 < 10: nothing to take
    assert len(out["edges"]) == 0 and out["remaining"] == 6.0
    out = O.anomalous_edges(E, 3.5)           # take 3, ties to the lower (i, j)
    assert [tuple(e) for e in out["edges"]] == [(0, 1), (0, 2), (0, 3)]
    assert out["remaining"] == 3.0
    out = O.anomalous_edges(E, 1e-9)          # every edge
    assert len(out["edges"]) == 6 and out["remaining"] == 0.0


def test_edge_scores_sum_to_node_scores():
    wl = iid_pair(60, 8, 3, seed=2)
    g = [O.embed(X, 8, 1) for X in wl.X]
    E = O.upper_edge_scores(g[0]["A"], g[1]["A"], g[0]["Z"], g[1]["Z"], g[0]["vol"], g[1]["vol"])
    F = O.node_scores(g[0]["A"], g[1]["A"], g[0]["Z"], g[1]["Z"], g[0]["vol"], g[1]["vol"])
    np.testing.assert_allclose((E + E.T).sum(axis=1), F, rtol=1e-12)
    part, vals = O.node_top_edges(E, [0, 5], 3)
    Ef = E + E.T
    for t, i in enumerate([0, 5]):
        row = [(Ef[i, j], -j) for j in range(60) if j != i]
        best = sorted(row, reverse=True)[:3]
        assert list(part[t]) == [-b[1] for b in best]


# ------------------------------------------------------------------ synthetic mixture data (Sec. 4.2.1)

def test_exp_graph_closed_form_triangle():
    """A 3-4-5 right triangle: the synthetic-data kernel exp(-d) by hand."""
    X = np.array([[0.0, 0.0], [3.0, 0.0], [0.0, 4.0]])
    A, D, vol, s = O.exp_graph(X, 1.0)
    e3, e4, e5 = math.exp(-3.0), math.exp(-4.0), math.exp(-5.0)
    np.testing.assert_allclose(A, [[0, e3, e4], [e3, 0, e5], [e4, e5, 0]], rtol=1e-15, atol=0)
    np.testing.assert_allclose(D, [e3 + e4, e3 + e5, e4 + e5], rtol=1e-15)
    assert math.isclose(vol, 2 * (e3 + e4 + e5), rel_tol=1e-15)
    assert s == 1.0
    # the median rule picks the lower median of {3, 4, 5}
    assert O.exp_graph(X, 0.0)[3] == 4.0
    # width 2 on X is width 1 on X / 2 (halving is exact)
    assert np.array_equal(O.exp_graph(X, 2.0)[0], O.exp_graph(X / 2, 1.0)[0])


def test_degrees_and_edge_weights_brute_force():
    A = _random_graph(7, 2)
    np.fill_diagonal(A, 0.0)
    ij = np.array([[0, 3], [2, 6], [1, 5], [4, 5]], dtype=np.int64)
    w = np.array([0.5, 0.25, 0.125, 0.75])
    B = O.add_edge_weights(A, ij, w)
    for a in range(7):
        for b in range(7):
            add = sum(w[e] for e in range(4) if {a, b} == {int(ij[e, 0]), int(ij[e, 1])})
            assert B[a, b] == A[a, b] + add
    D, vol = O.degrees(B)
    for a in range(7):
        assert math.isclose(D[a], math.fsum(B[a]), rel_tol=1e-15)
    assert math.isclose(vol, math.fsum(B.reshape(-1)), rel_tol=1e-14)


def test_gmm_workload_matches_its_model():
    from workloads import gmm_pair
    n, p = 300, 0.05
    g = gmm_pair(n, p=p, seed=4)
    m = n * (n - 1) // 2
    # an unordered pair carries weight unless both of its two draws were zero
    q = 1 - (1 - p) ** 2
    assert abs(len(g.w) - q * m) < 5 * math.sqrt(m * q * (1 - q))
    assert np.all(g.ij[:, 0] < g.ij[:, 1])
    flat = g.ij[:, 0] * n + g.ij[:, 1]
    assert np.all(np.diff(flat) > 0)
    assert np.all(g.w > 0) and np.all(g.w <= 1.0)
    assert np.array_equal(g.w * 2 ** 17, np.rint(g.w * 2 ** 17))
    assert np.array_equal(g.truth, g.labels[g.ij[:, 0]] != g.labels[g.ij[:, 1]])
    # mixture components sit at (+-3, +-3); the noise is small
    for c, mu in enumerate([(-3, -3), (-3, 3), (3, -3), (3, 3)]):
        pts = g.X[0][g.labels == c]
        assert np.all(np.abs(pts.mean(0) - mu) < 0.5)
    assert np.abs(g.X[1] - g.X[0]).max() < 0.05 * 6


def _auc(score, pos):
    """Probability that a random positive outranks a random negative (ties 1/2)."""
    s_pos, s_neg = score[pos], score[~pos]
    order = np.sort(s_neg)
    below = np.searchsorted(order, s_pos, side="left")
    equal = np.searchsorted(order, s_pos, side="right") - below
    return float((below + 0.5 * equal).sum() / (s_pos.size * s_neg.size))


def test_gmm_detector_separates_cross_cluster_edges():
    """Sec. 4.2.1's synthetic design: added edges that join two clusters change
    the commute times, added edges inside a cluster barely do. Among the added
    edges, Delta E ranks the cross-cluster ones first, while |Delta A| alone
    (the added weight, independent of the clusters) does not. This holds with
    the exact commute times of Eq. 1 (pseudoinverse, independent of the
    oracle's solver) and with the oracle's own k = 128 embedding."""
    from workloads import gmm_pair
    n, k = 300, 128
    g = gmm_pair(n, seed=9)
    A1, _, vol1, _ = O.exp_graph(g.X[0], 1.0)
    Q, _, _, _ = O.exp_graph(g.X[1], 1.0)
    A2 = O.add_edge_weights(Q, g.ij, g.w)
    _, vol2 = O.degrees(A2)
    i, j = g.ij[:, 0], g.ij[:, 1]
    dA = np.abs(A1 - A2)[i, j]
    C1x, C2x = O.commute_times_pinv(A1), O.commute_times_pinv(A2)
    e_exact = dA * np.abs(C2x - C1x)[i, j]
    Z1 = O.exact_embedding(A1, O.project(A1, 3, k))
    Z2 = O.exact_embedding(A2, O.project(A2, 3, k))
    E = O.upper_edge_scores(A1, A2, Z1, Z2, vol1, vol2)
    e_orc = E[i, j]
    auc_dA, auc_x, auc_o = _auc(dA, g.truth), _auc(e_exact, g.truth), _auc(e_orc, g.truth)
    assert abs(auc_dA - 0.5) < 0.06
    assert auc_x > auc_dA + 0.15
    assert auc_o > auc_dA + 0.08


def test_gmm_commute_time_error_matches_jl_spread():
    """Alg. 3's projected commute times against Eq. 1's exact ones on a mixture
    graph: c_est / c = ||Q v||^2 / ||v||^2 for the edge-space vector v of the
    pair, which for +-1/sqrt(k) signs and v spread over many edges is close to
    normal with mean 1 and standard deviation sqrt(2 / k), so the median
    absolute relative error is about 0.674 sqrt(2 / k)."""
    from workloads import gmm_pair
    n, k = 240, 64
    g = gmm_pair(n, seed=2)
    A, _, vol, _ = O.exp_graph(g.X[0], 1.0)
    C = O.commute_times_pinv(A)
    Z = O.exact_embedding(A, O.project(A, 8, k))
    Ce = O.commute_times(Z, vol)
    iu, ju = np.triu_indices(n, 1)
    rel = Ce[iu, ju] / C[iu, ju] - 1.0
    assert abs(np.mean(rel)) < 0.05
    med = np.median(np.abs(rel))
    expect = 0.6745 * math.sqrt(2.0 / k)
    assert 0.75 * expect < med < 1.25 * expect


def test_richardson_error_matches_the_spectral_form():
    """Alg. 2's EstimateSolution: with chi = P1 b = P1 L z*, the error after j
    updates is (I - P1 L)^j z*, and I - P1 L = D^{-1/2} S^{2^d} D^{1/2}. So, with
    w = D^{1/2} z* written in the eigenvectors of S = D^{-1/2} A D^{-1/2}, the
    D-norm error after q - 1 updates is |Lambda^{2^d (q-1)} c| / |c|, bounded by
    the second largest |eigenvalue| to the power 2^d (q-1): the depth d and the
    update count q trade off exactly as the telescoping product says."""
    n = 30
    A = _random_graph(n, 21, lo=0.2)
    D = A.sum(1)
    r = 1.0 / np.sqrt(D)
    lam, V = np.linalg.eigh(r[:, None] * A * r[None, :])
    lam2 = np.sort(np.abs(lam))[-2]                      # the largest is 1
    b = O.project(A, 5, 3)
    zs = O.exact_embedding(A, b)
    c = V.T @ (np.sqrt(D)[:, None] * zs)
    L = O.laplacian(A)

    def dnorm(x):
        return float(np.sqrt(np.einsum("ij,i,ij->", x, D, x)))

    for d in (1, 2, 3):
        P1, P2 = O.chain_product(L, d)
        for q in (2, 3, 4):
            y = O.estimate_solution(P1, P2, b, q)
            err = dnorm(zs - y) / dnorm(zs)
            p = 2 ** d * (q - 1)
            pred = float(np.linalg.norm((lam[:, None] ** p) * c) / np.linalg.norm(c))
            assert abs(err - pred) <= 1e-8 * pred + 1e-13, (d, q, err, pred)
            assert err <= lam2 ** p * (1 + 1e-9) + 1e-13


def test_projected_commute_times_error_scales_with_k():
    """The JL estimate's relative error shrinks as sqrt(2/k) (Sec. 4.2.2: the
    embedding dimension dominates the accuracy): the median relative error of
    the projected commute times is near 0.674 sqrt(2/k) for k = 16, 64, 256."""
    n = 60
    A = _random_graph(n, 22)
    exact = O.commute_times_pinv(A)
    off = ~np.eye(n, dtype=bool)
    meds = []
    for k in (16, 64, 256):
        Z = O.exact_embedding(A, O.project(A, 77, k))
        rel = np.abs(O.commute_times(Z, A.sum()) - exact)[off] / exact[off]
        med = float(np.median(rel))
        meds.append(med)
        assert 0.6 * 0.674 * math.sqrt(2 / k) < med < 1.5 * 0.674 * math.sqrt(2 / k), (k, med)
    assert meds[0] > meds[1] > meds[2]
