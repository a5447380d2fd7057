"""CADDeLaG hot path in plain float64 (TEST INFRASTRUCTURE; see package header).

Notation follows the paper: n nodes, A the symmetric adjacency matrix with
zero diagonal, D = A 1 the degrees, vol = sum_i D_i the graph volume,
L = D - A the Laplacian, B the signed edge-vertex incidence matrix and W the
diagonal matrix of edge weights (Sec. 2), k the projection dimension, d the
chain length and q the Richardson count (Alg. 2, Alg. 3).

Readings of passages the paper leaves open (each is also listed in the
design notes of the repository):

* Edges are the unordered pairs i < j (m = n(n-1)/2); the head of edge (i, j)
  is i, its tail j, so that B^T W B = L exactly (Sec. 2).
* ``y = W^{1/2} B q`` (Alg. 1, Alg. 3) is read as y = B^T W^{1/2} q with
  q in {+-1/sqrt(k)}^m, i.e. Y = (Q W^{1/2} B)^T for k stacked rows of Q.
* The matrix C in ChainProduct (Alg. 2) is read as D^{-1/2}, so that
  P1 = D^{-1/2} prod_{i<d} (I + S^{2^i}) D^{-1/2} approximates L^+ and
  P2 = P1 L approximates the identity on the complement of the all-ones
  vector; the chain has d factors and d - 1 squarings (Alg. 2, not Eq. 3).
* L is singular; the solution Z is normalised to D-weighted zero column
  means, the fixed point the Richardson iteration of Alg. 2 keeps.
* Commute times carry each graph's own volume: c_ij = vol ||z_i - z_j||^2
  (Eq. 1 and Alg. 1).
* Top anomalies are ordered by node score descending, ties by lower index.
"""
from __future__ import annotations

import math
import os
from typing import Optional, Sequence

import numpy as np
import scipy.linalg

from .philox import edge_sign_bits


# --------------------------------------------------------------------------
# Graph (Sec. 4.2.1, climate graph kernel; Sec. 2 zero diagonal, D = A 1)
# --------------------------------------------------------------------------

def squared_distances(X: np.ndarray, rows: Optional[Sequence[int]] = None) -> np.ndarray:
    """||x_i - x_j||^2 for the rows ``rows`` (default all) against all nodes.

    Plain definition: differences, squares and sums in float64, sample index
    ascending, each operation rounded on its own (no fused multiply-add).
    Pinned by brute force against scipy's pdist and by exactness on
    grid-rounded inputs."""
    X = np.asarray(X, dtype=np.float64)
    R = X if rows is None else X[np.asarray(rows)]
    d2 = np.zeros((R.shape[0], X.shape[0]))
    for t in range(X.shape[1]):
        diff = R[:, t][:, None] - X[:, t][None, :]
        d2 += diff * diff
    return d2


def squared_distances_exact_grid(X: np.ndarray, row_block: int = 4096) -> np.ndarray:
    """Same values as ``squared_distances`` for inputs on the 2**-16 grid.

    For such inputs x = a 2**-16 with integer a, so ||x_i - x_j||^2 =
    (|a_i|^2 + |a_j|^2 - 2 a_i.a_j) 2**-32 is an integer multiple of 2**-32.
    The integer Gram matrix is formed exactly from float64 matrix products of
    12-bit pieces of a (every product and partial sum below 2**53) and
    combined in int64. Whenever every partial sum of the plain definition is
    itself exact (squared distances below 2**21), both results are the same
    float64 number; the tests assert bit equality on such inputs.
    Raises ValueError for inputs off the grid."""
    X = np.asarray(X, dtype=np.float64)
    a = X * 65536.0
    if not np.array_equal(a, np.rint(a)) or np.abs(a).max() >= 2.0 ** 23:
        raise ValueError("input is not on the 2**-16 grid")
    ai = a.astype(np.int64)
    hi = (ai >> 12).astype(np.float64)       # floor division: a = hi*4096 + lo
    lo = (ai & 4095).astype(np.float64)
    norms = (ai * ai).sum(axis=1)            # int64, exact
    n = X.shape[0]
    out = np.empty((n, n))
    for r0 in range(0, n, row_block):
        r1 = min(n, r0 + row_block)
        g_hh = (hi[r0:r1] @ hi.T).astype(np.int64)
        g_hl = (hi[r0:r1] @ lo.T).astype(np.int64)
        g_lh = (lo[r0:r1] @ hi.T).astype(np.int64)
        g_ll = (lo[r0:r1] @ lo.T).astype(np.int64)
        gram = (g_hh << 24) + ((g_hl + g_lh) << 12) + g_ll
        d2i = norms[r0:r1, None] + norms[None, :] - 2 * gram
        out[r0:r1] = d2i.astype(np.float64) * 2.0 ** -32
    return out


def _grid_upper_blocks(X: np.ndarray, row_block: int, threads: int, fn):
    """Stream the exact squared distances of node series on the 2**-16 grid
    (x = a 2**-16, integer a) over row blocks of the upper triangle: for rows
    r0 .. r1 - 1 and columns j > r0, the integers D_ij = |a_i - a_j|^2 (the
    integer Gram from float64 products of 12-bit pieces, exact, as in
    ``squared_distances_exact_grid``) and the mask j > i go to
    fn(r0, r1, D, upper); the results come back in block order. A single
    float64 product a_i . a_j replaces the pieces when (max |a|)^2 T < 2^53
    (every partial sum exact). Blocks run on threads (NumPy and BLAS release
    the GIL)."""
    import concurrent.futures as cf
    X = np.asarray(X, dtype=np.float64)
    a = X * 65536.0
    if not np.array_equal(a, np.rint(a)) or np.abs(a).max() >= 2.0 ** 23:
        raise ValueError("input is not on the 2**-16 grid")
    ai = a.astype(np.int64)
    hi = (ai >> 12).astype(np.float64)
    lo = (ai & 4095).astype(np.float64)
    norms = (ai * ai).sum(axis=1)
    n = X.shape[0]
    # one float64 product is exact when every partial sum of a_i . a_j stays
    # below 2^53: (max |a|)^2 T < 2^53; else the 12-bit pieces
    amax = int(np.abs(ai).max()) if ai.size else 0
    direct = amax * amax * X.shape[1] < 2 ** 53

    def block(r0):
        r1 = min(n, r0 + row_block)
        c0 = r0 + 1                                   # columns j > i start after the block's first row
        if direct:
            g = (a[r0:r1] @ a[c0:].T).astype(np.int64)
        else:
            g = ((hi[r0:r1] @ hi[c0:].T).astype(np.int64) << 24) + \
                (((hi[r0:r1] @ lo[c0:].T) + (lo[r0:r1] @ hi[c0:].T)).astype(np.int64) << 12) + \
                (lo[r0:r1] @ lo[c0:].T).astype(np.int64)
        D = norms[r0:r1, None] + norms[None, c0:] - 2 * g
        upper = np.arange(c0, n)[None, :] > np.arange(r0, r1)[:, None]
        return fn(r0, r1, D, upper)

    starts = list(range(0, n - 1, row_block))
    workers = threads or min(4, os.cpu_count() or 1)
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        return list(ex.map(block, starts))


def grid_distance_counts(X: np.ndarray, key: int, row_block: int = 512, threads: int = 0):
    """For node series on the 2**-16 grid: the numbers of pairs i < j whose
    exact squared distance, as the integer D_ij = ||x_i - x_j||^2 2**32, is
    below ``key`` and at most ``key``. The lower median of the distances
    (Sec. 4.2.1 kernel width: rank (m - 1) // 2 of the m = n (n - 1) / 2
    sorted distances) is the key with count_below <= rank < count_at_most.
    Streamed (no n x n matrix is held)."""
    parts = _grid_upper_blocks(X, row_block, threads, lambda r0, r1, D, up: (
        int(np.count_nonzero((D < key) & up)), int(np.count_nonzero((D <= key) & up))))
    return sum(p[0] for p in parts), sum(p[1] for p in parts)


def gaussian_degrees_streamed(X: np.ndarray, sigma: float, row_block: int = 512, threads: int = 0,
                              key: Optional[int] = None):
    """D_i = sum_{j != i} exp(-||x_i - x_j||^2 / (2 sigma^2)) (Sec. 3.2: D = A 1)
    for node series on the 2**-16 grid, streamed over the upper triangle
    (each pair's value added to both of its rows; no n x n matrix is held).
    With ``key``, also the two counts of ``grid_distance_counts`` from the
    same pass: returns (D, count_below, count_at_most)."""
    n = X.shape[0]
    two_s2 = 2.0 * (sigma * sigma)

    def fn(r0, r1, Dk, up):
        A = np.exp(-((Dk.astype(np.float64) * 2.0 ** -32) / two_s2))
        A[~up] = 0.0
        cnt = (int(np.count_nonzero((Dk < key) & up)), int(np.count_nonzero((Dk <= key) & up))) if key is not None \
            else (0, 0)
        return r0, r1, A.sum(axis=1), A.sum(axis=0), cnt

    D = np.zeros(n)
    lt = le = 0
    for r0, r1, rs, cs, cnt in _grid_upper_blocks(X, row_block, threads, fn):
        D[r0:r1] += rs
        D[r0 + 1:] += cs
        lt += cnt[0]
        le += cnt[1]
    return (D, lt, le) if key is not None else D


def median_sigma(d2: np.ndarray) -> float:
    """Lower median of the distances ||x_i - x_j|| over i < j.

    sigma = sorted(d)[floor((m - 1) / 2)], m = n(n - 1)/2 (the kernel width
    rule of the workloads; the paper fixes sigma by hand for its climate
    graph). Pinned by brute force on small inputs."""
    n = d2.shape[0]
    m = n * (n - 1) // 2
    d = np.empty(m)
    o = 0
    for i in range(n - 1):                   # upper triangle, row by row
        d[o:o + n - 1 - i] = d2[i, i + 1:]
        o += n - 1 - i
    np.sqrt(d, out=d)
    h = (m - 1) // 2
    return float(np.partition(d, h)[h])


def gaussian_graph(X: np.ndarray, sigma: Optional[float] = None, d2: Optional[np.ndarray] = None):
    """Dense Gaussian-kernel graph A_ij = exp(-||x_i - x_j||^2 / (2 sigma^2)),
    A_ii = 0, D = A 1, vol = sum D (Sec. 4.2.1 kernel; Sec. 2 zero diagonal;
    Sec. 3.2 D = A 1). sigma <= 0 or None selects the median rule.
    Returns (A, D, vol, sigma)."""
    if d2 is None:
        d2 = squared_distances(X)
    if sigma is None or sigma <= 0:
        sigma = median_sigma(d2)
    two_s2 = 2.0 * (sigma * sigma)
    A = np.exp(-(d2 / two_s2))
    np.fill_diagonal(A, 0.0)
    D = A.sum(axis=1)
    vol = float(D.sum())
    return A, D, vol, float(sigma)


def graph_rows(X: np.ndarray, sigma: float, rows: Sequence[int]) -> np.ndarray:
    """Rows ``rows`` of the Gaussian-kernel graph for a given sigma."""
    rows = np.asarray(rows)
    d2 = squared_distances(X, rows)
    A = np.exp(-(d2 / (2.0 * (sigma * sigma))))
    A[np.arange(rows.size), rows] = 0.0
    return A


def exp_graph(X: np.ndarray, sigma: Optional[float] = 1.0, d2: Optional[np.ndarray] = None):
    """Graph of the synthetic experiments (Sec. 4.2.1, "Synthetic Data"):
    A_ij = exp(-d(i, j) / sigma) with d the Euclidean distance; the paper
    writes exp(-d(i, j)), i.e. sigma = 1. A_ii = 0, D = A 1, vol = sum D.
    sigma <= 0 or None selects the median rule. Returns (A, D, vol, sigma)."""
    if d2 is None:
        d2 = squared_distances(X)
    if sigma is None or sigma <= 0:
        sigma = median_sigma(d2)
    A = np.exp(-(np.sqrt(d2) / sigma))
    np.fill_diagonal(A, 0.0)
    D, vol = degrees(A)
    return A, D, vol, float(sigma)


def degrees(A: np.ndarray):
    """D = A 1 and vol = sum_i D_i (Sec. 3.2; Eq. 1) of a given adjacency
    matrix. Returns (D, vol)."""
    D = A.sum(axis=1)
    return D, float(D.sum())


def add_edge_weights(A: np.ndarray, ij: np.ndarray, w: np.ndarray) -> np.ndarray:
    """A + W with W_ij = W_ji = w_e for each listed pair e = (i, j), i != j
    (distinct unordered pairs): the perturbation A_2 = Q + (R + R^T) / 2 of
    the synthetic experiments (Sec. 4.2.1), w holding (R_ij + R_ji) / 2."""
    n = A.shape[0]
    W = np.zeros((n, n))
    W[ij[:, 0], ij[:, 1]] = w
    W[ij[:, 1], ij[:, 0]] = w
    return A + W


# --------------------------------------------------------------------------
# Laplacian and incidence matrix (Sec. 2, Eq. 1-2)
# --------------------------------------------------------------------------

def laplacian(A: np.ndarray) -> np.ndarray:
    """L = D - A."""
    return np.diag(A.sum(axis=1)) - A


def incidence(A: np.ndarray):
    """Signed edge-vertex incidence matrix B (m x n) over the unordered pairs
    i < j with head i (+1) and tail j (-1), and the edge weights w (W = diag w).
    Sec. 2; B^T diag(w) B = L is checked in the tests."""
    n = A.shape[0]
    iu, ju = np.triu_indices(n, 1)
    m = iu.size
    B = np.zeros((m, n))
    B[np.arange(m), iu] = 1.0
    B[np.arange(m), ju] = -1.0
    return B, A[iu, ju].copy(), (iu, ju)


def commute_times_pinv(A: np.ndarray) -> np.ndarray:
    """Eq. 1: c(i, j) = V_G (l+_ii + l+_jj - 2 l+_ij) with L^+ the
    Moore-Penrose pseudoinverse (via a symmetric eigendecomposition)."""
    L = laplacian(A)
    w, V = np.linalg.eigh(L)
    tol = w.max() * L.shape[0] * np.finfo(float).eps
    inv = np.where(w > tol, 1.0 / np.where(w > tol, w, 1.0), 0.0)
    Lp = (V * inv) @ V.T
    dg = np.diag(Lp)
    vol = A.sum()
    return vol * (dg[:, None] + dg[None, :] - 2.0 * Lp)


# --------------------------------------------------------------------------
# Random projection (Alg. 1 and Alg. 3; Sec. 4.1 complexity: Map + ReduceByKey)
# --------------------------------------------------------------------------

def projection_matrix(n: int, seed: int, k: int) -> np.ndarray:
    """Q (k x m): Q[r, e] = +-1/sqrt(k) for edge e = (i, j), i < j, in
    triu order, signs from ``edge_sign_bits``."""
    iu, ju = np.triu_indices(n, 1)
    bits = edge_sign_bits(seed, iu, ju, k)
    return np.where(bits, 1.0, -1.0).T / math.sqrt(k)


def project_explicit(A: np.ndarray, Q: np.ndarray) -> np.ndarray:
    """Y = (Q W^{1/2} B)^T built from explicit B, W and Q (small n only)."""
    B, w, _ = incidence(A)
    return B.T @ (np.sqrt(w)[:, None] * Q.T)


def project_rows(A_rows: np.ndarray, rows: Sequence[int], seed: int, k: int) -> np.ndarray:
    """Rows ``rows`` of Y = (Q W^{1/2} B)^T, edge by edge, without forming B
    or Q; ``A_rows[t]`` is row ``rows[t]`` of the adjacency matrix:
    Y[i, r] = (1/sqrt(k)) sum_{j != i} o_ij s_r(min(i,j), max(i,j)) sqrt(A_ij)
    with orientation o_ij = +1 if i < j (i is the head) and -1 otherwise, and
    s_r(.,.) = +-1 the sign of ``edge_sign_bits``. Pinned against
    ``project_explicit`` (the incidence-matrix form) in the tests."""
    A_rows = np.atleast_2d(A_rows)
    n = A_rows.shape[1]
    rows = list(rows)
    Y = np.zeros((len(rows), k))
    for t, i in enumerate(rows):
        j = np.arange(n)
        j = j[j != i]
        lo = np.minimum(i, j)
        hi = np.maximum(i, j)
        sgn = np.where(edge_sign_bits(seed, lo, hi, k), 1.0, -1.0)
        orient = np.where(j > i, 1.0, -1.0)
        Y[t] = (orient * np.sqrt(A_rows[t, j])) @ sgn
    return Y / math.sqrt(k)


def project(A: np.ndarray, seed: int, k: int) -> np.ndarray:
    """All rows of Y (see ``project_rows``)."""
    n = A.shape[0]
    return project_rows(A, range(n), seed, k)


def project_rows_c(A_rows: np.ndarray, rows: Sequence[int], seed: int, k: int) -> np.ndarray:
    """``project_rows`` computed by the oracle's plain C version (oracle/cproj.c,
    same definition, OpenMP over rows) for large graphs. Pinned against
    ``project_rows`` and ``project_explicit`` in the tests."""
    import ctypes
    from . import cbuild
    lib = ctypes.CDLL(cbuild.build())
    A_rows = np.ascontiguousarray(np.atleast_2d(A_rows), dtype=np.float64)
    rows = np.ascontiguousarray(np.asarray(list(rows), dtype=np.int64))
    n = A_rows.shape[1]
    if k > 1024:
        raise ValueError("k <= 1024")
    Y = np.empty((rows.size, k))
    P = ctypes.c_void_p
    lib.cdl_oracle_project_rows.argtypes = [P, P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                                            ctypes.c_uint64, P]
    lib.cdl_oracle_project_rows(A_rows.ctypes.data, rows.ctypes.data, rows.size, n, k, seed, Y.ctypes.data)
    return Y


# --------------------------------------------------------------------------
# SDD solver (Alg. 2) and embedding (Alg. 3)
# --------------------------------------------------------------------------

def split_sdd(M: np.ndarray):
    """Sec. 3.1: M = D - A with D = diag(M) and A the negated off-diagonal."""
    Dv = np.diag(M).copy()
    A = -(M - np.diag(Dv))
    return Dv, A


def chain_product(M: np.ndarray, d: int):
    """Alg. 2, ChainProduct(M, d): S = D^{-1/2} A D^{-1/2};
    P = (I + S)(I + S^2) ... (I + S^{2^{d-1}}) C with C = D^{-1/2};
    returns (P1, P2) = (D^{-1/2} P, D^{-1/2} P L), L = D - A."""
    Dv, A = split_sdd(M)
    n = M.shape[0]
    r = 1.0 / np.sqrt(Dv)
    S = r[:, None] * A * r[None, :]
    I = np.eye(n)
    P = I.copy()
    level = S.copy()
    for i in range(d):
        P = P @ (I + level)
        if i + 1 < d:
            level = level @ level
    P = P * r[None, :]          # right factor C = D^{-1/2}
    P1 = r[:, None] * P
    L = np.diag(Dv) - A
    P2 = P1 @ L
    return P1, P2


def chain_levels(A: np.ndarray, d: int):
    """The d chain levels S^{2^i}, i = 0 .. d-1, of Alg. 2 (S = D^{-1/2} A D^{-1/2})."""
    D = A.sum(axis=1)
    r = 1.0 / np.sqrt(D)
    S = r[:, None] * A * r[None, :]
    out = [S]
    for _ in range(d - 1):
        out.append(out[-1] @ out[-1])
    return out


def estimate_solution(P1: np.ndarray, P2: np.ndarray, b: np.ndarray, q: int) -> np.ndarray:
    """Alg. 2, EstimateSolution: chi = P1 b; y_1 = 0;
    y_{j+1} = y_j - P2 y_j + chi for j = 1 .. q-1; returns y_q. b may hold
    several right-hand sides as columns (Sec. 4.1, multi-RHS loop)."""
    chi = P1 @ b
    y = np.zeros_like(chi)
    for _ in range(q - 1):
        y = y - P2 @ y + chi
    return y


def richardson_count(delta: float) -> int:
    """q = ceil(log(1/delta)) of Alg. 2 (natural logarithm; the paper does not
    name the base)."""
    return int(math.ceil(math.log(1.0 / delta)))


def projection_dim(n: int, eps: float) -> int:
    """k_RP = ceil(log(n/eps)) of Alg. 1 and Alg. 3 (natural logarithm)."""
    return int(math.ceil(math.log(n / eps)))


def dweighted_center(Z: np.ndarray, D: np.ndarray) -> np.ndarray:
    """Shift each column to D-weighted zero mean: Z - 1 (D^T Z) / vol."""
    return Z - (D @ Z)[None, :] / D.sum()


def exact_embedding(A: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """Z = L^+ Y, D-weighted zero column means (the fixed point of Alg. 2's
    Richardson iteration). Y must be orthogonal to the ones vector; then
    (L + c 1 1^T) Z = Y with c = vol / n^2 > 0 has the unique solution L^+ Y
    (dense Cholesky)."""
    n = A.shape[0]
    D = A.sum(axis=1)
    vol = D.sum()
    M = np.diag(D) - A + vol / (n * n)
    Z = scipy.linalg.cho_solve(scipy.linalg.cho_factor(M, lower=False), Y)
    return dweighted_center(Z, D)


def literal_embedding(A: np.ndarray, Y: np.ndarray, d: int, q: int) -> np.ndarray:
    """Alg. 3 with Alg. 2 taken literally: ChainProduct(L, d) and q-step
    EstimateSolution on all k right-hand sides at once, then the D-weighted
    centring (which the exact iteration preserves)."""
    L = laplacian(A)
    P1, P2 = chain_product(L, d)
    Z = estimate_solution(P1, P2, Y, q)
    return dweighted_center(Z, A.sum(axis=1))


def residual_norm(A: np.ndarray, Y: np.ndarray, Z: np.ndarray) -> float:
    """||Y - L Z||_F / ||Y||_F in float64."""
    D = A.sum(axis=1)
    R = Y - (D[:, None] * Z - A @ Z)
    return float(np.linalg.norm(R) / np.linalg.norm(Y))


# --------------------------------------------------------------------------
# Commute times and CAD scores (Eq. 1, Alg. 1, Alg. 4, Sec. 2 CAD score)
# --------------------------------------------------------------------------

def commute_times(Z: np.ndarray, vol: float, rows: Optional[Sequence[int]] = None) -> np.ndarray:
    """c_ij = vol ||z_i - z_j||^2 (Alg. 1 accumulation, scaled by the volume
    of Eq. 1), direct differences, for rows ``rows`` against all nodes."""
    R = Z if rows is None else Z[np.asarray(rows)]
    c = np.zeros((R.shape[0], Z.shape[0]))
    for r in range(Z.shape[1]):
        diff = R[:, r][:, None] - Z[:, r][None, :]
        c += diff * diff
    return vol * c


def edge_scores(A1, A2, C1, C2) -> np.ndarray:
    """Delta E = |A1 - A2| (Hadamard) |C2 - C1| (Sec. 2; Alg. 4)."""
    return np.abs(A1 - A2) * np.abs(C2 - C1)


def node_scores(A1, A2, Z1, Z2, vol1, vol2, rows: Optional[Sequence[int]] = None,
                block: int = 512) -> np.ndarray:
    """F_i = sum_j Delta E_ij (Alg. 4) for rows ``rows`` (default all).
    A1 and A2 are full n x n matrices, or hold exactly the requested rows."""
    n = Z1.shape[0]
    rows = np.arange(n) if rows is None else np.asarray(rows)
    full = A1.shape[0] == n and rows.size == n
    F = np.empty(rows.size)
    for b0 in range(0, rows.size, block):
        rr = rows[b0:b0 + block]
        a1 = A1[rr] if full else A1[b0:b0 + block]
        a2 = A2[rr] if full else A2[b0:b0 + block]
        c1 = commute_times(Z1, vol1, rr)
        c2 = commute_times(Z2, vol2, rr)
        F[b0:b0 + rr.size] = edge_scores(a1, a2, c1, c2).sum(axis=1)
    return F


def node_scores_c(A1_rows, A2_rows, rows: Sequence[int], Z1, Z2, vol1: float, vol2: float) -> np.ndarray:
    """``node_scores`` for rows ``rows`` computed by the oracle's plain C
    version (oracle/cscore.c: the same definition, direct differences, OpenMP
    over rows) for large graphs. A1_rows and A2_rows hold exactly the
    requested rows. Pinned against ``node_scores`` in the tests."""
    import ctypes
    from . import cbuild
    lib = ctypes.CDLL(cbuild.build())
    A1_rows = np.ascontiguousarray(np.atleast_2d(A1_rows), dtype=np.float64)
    A2_rows = np.ascontiguousarray(np.atleast_2d(A2_rows), dtype=np.float64)
    rows = np.ascontiguousarray(np.asarray(list(rows), dtype=np.int64))
    Z1 = np.ascontiguousarray(Z1, dtype=np.float64)
    Z2 = np.ascontiguousarray(Z2, dtype=np.float64)
    n, k = Z1.shape
    if A1_rows.shape != (rows.size, n) or A2_rows.shape != (rows.size, n) or Z2.shape != (n, k):
        raise ValueError("shape mismatch")
    F = np.empty(rows.size)
    P = ctypes.c_void_p
    lib.cdl_oracle_node_scores.argtypes = [P, P, P, ctypes.c_int64, ctypes.c_int64, P, P, ctypes.c_int32,
                                           ctypes.c_double, ctypes.c_double, P]
    lib.cdl_oracle_node_scores(A1_rows.ctypes.data, A2_rows.ctypes.data, rows.ctypes.data, rows.size, n,
                               Z1.ctypes.data, Z2.ctypes.data, k, float(vol1), float(vol2), F.ctypes.data)
    return F


def upper_edge_scores(A1, A2, Z1, Z2, vol1, vol2) -> np.ndarray:
    """Delta E_ij for every edge i < j (Sec. 2; Alg. 4), as an n x n array
    holding the upper triangle (zero on and below the diagonal)."""
    C1 = commute_times(Z1, vol1)
    C2 = commute_times(Z2, vol2)
    return np.triu(edge_scores(A1, A2, C1, C2), 1)


def anomalous_edges(E_upper: np.ndarray, delta: float):
    """CAD's anomalous edge set (Sec. 3.3): the smallest set of edges whose
    removal leaves the total change of the remaining edges below delta.
    Edges are taken one at a time in descending Delta E (ties: lower (i, j)
    first), subtracting each from the total, until the remainder is below
    delta. Returns dict(edges: (s, 2) int64 (i, j) pairs in (i, j) order,
    values, total, remaining)."""
    n = E_upper.shape[0]
    iu, ju = np.triu_indices(n, 1)
    v = E_upper[iu, ju]
    total = float(np.sum(v))
    order = np.lexsort((ju, iu, -v))
    rem = total
    s = 0
    while not (rem < delta) and s < v.size:
        rem -= v[order[s]]
        s += 1
    chosen = order[:s]
    pairs = np.stack([iu[chosen], ju[chosen]], axis=1).astype(np.int64)
    vals = v[chosen]
    srt = np.lexsort((pairs[:, 1], pairs[:, 0]))
    return dict(edges=pairs[srt], values=vals[srt], total=total, remaining=rem)


def node_top_edges(E_upper: np.ndarray, nodes: Sequence[int], m: int):
    """For each node, its m largest Delta E partners (ties: lower partner
    first); -1 past the end."""
    Ef = E_upper + E_upper.T
    n = Ef.shape[0]
    out = np.full((len(nodes), m), -1, dtype=np.int64)
    vals = np.zeros((len(nodes), m))
    for t, i in enumerate(nodes):
        j = np.array([x for x in range(n) if x != i])
        o = np.lexsort((j, -Ef[i, j]))[:m]
        out[t, :o.size] = j[o]
        vals[t, :o.size] = Ef[i, j[o]]
    return out, vals


def top_anomalies(F: np.ndarray, k: int) -> np.ndarray:
    """Indices of the k highest node scores, ties broken by lower index."""
    F = np.asarray(F)
    return np.lexsort((np.arange(F.size), -F))[:k].astype(np.int64)


def min_relative_gap(F: np.ndarray, k: int) -> float:
    """Smallest relative gap between consecutive scores among the k+1 highest:
    the top-k set is decided only where this exceeds the score tolerance."""
    s = np.sort(np.asarray(F))[::-1][:k + 1]
    gaps = (s[:-1] - s[1:]) / np.maximum(np.abs(s[:-1]), 1e-300)
    return float(gaps.min()) if gaps.size else float("inf")


# --------------------------------------------------------------------------
# Whole pair (Alg. 4)
# --------------------------------------------------------------------------

def embed(X: np.ndarray, k: int, seed: int, d: int = 0, q: int = 0, mode: str = "exact",
          d2: Optional[np.ndarray] = None, sigma: Optional[float] = None):
    """CommuteTimeEmbedding (Alg. 3) of the Gaussian-kernel graph of X.
    mode "exact" returns L^+ Y; mode "literal" runs Alg. 2 with (d, q).
    Returns dict(A, D, vol, sigma, Y, Z)."""
    A, D, vol, sigma = gaussian_graph(X, sigma, d2)
    Y = project(A, seed, k)
    if mode == "exact":
        Z = exact_embedding(A, Y)
    elif mode == "literal":
        Z = literal_embedding(A, Y, d, q)
    else:
        raise ValueError(mode)
    return dict(A=A, D=D, vol=vol, sigma=sigma, Y=Y, Z=Z)


def caddelag_pair(X1, X2, k: int, seed: int, topk: int, d: int = 0, q: int = 0,
                  mode: str = "exact"):
    """Alg. 4 on one graph pair with a shared projection seed: embeddings of
    both graphs, node scores F and the top anomalies."""
    g1 = embed(X1, k, seed, d, q, mode)
    g2 = embed(X2, k, seed, d, q, mode)
    F = node_scores(g1["A"], g2["A"], g1["Z"], g2["Z"], g1["vol"], g2["vol"])
    return dict(g1=g1, g2=g2, F=F, top=top_anomalies(F, topk))
