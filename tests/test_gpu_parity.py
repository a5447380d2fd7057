"""Parity of the CUDA path (called through the C ABI) with the float64 oracle
on seeded inputs: graph build, projection, chain levels (including the
tcgen05 GEMM against an exact product of its own inputs), solve, scores, the
whole pair, and argument validation. Sizes span several tiles and ragged
tails; the oracle finishes each case in seconds."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import caddelag as O          # noqa: E402
from workloads import iid_pair, field_sequence, to_grid   # noqa: E402

pytestmark = pytest.mark.gpu

# The kernel values come from a float-float exponential (float64 argument
# reduction, degree-12 series in float-float): relative error below 1e-14
# for the arguments d^2 / (2 sigma^2) < 60 that occur here; numpy's exp is
# within one float64 ulp.
A_RTOL = 2e-14


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from gpu_util import Ctx, lib
    c = Ctx(lib())
    yield c
    c.close()


def _h(t):
    from gpu_util import host
    return host(t)


# ------------------------------------------------------------------ graph

@pytest.mark.parametrize("n,T", [(2, 3), (3, 1), (65, 7), (300, 64), (1000, 40)])
def test_graph_matches_oracle(G, n, T):
    X = iid_pair(n, T, 1, seed=n).X[0]
    A, D, vol, sig = G.graph(X)
    Ao, Do, volo, sigo = O.gaussian_graph(X)
    assert _h(sig)[0] == sigo                       # exact selection on exact distances
    np.testing.assert_allclose(_h(A), Ao, rtol=A_RTOL, atol=0)
    np.testing.assert_allclose(_h(D), Do, rtol=1e-13)
    assert math.isclose(_h(vol)[0], volo, rel_tol=1e-13)


@pytest.mark.parametrize("kind", ["three_points", "lattice"])
def test_graph_select_with_tied_distances(G, kind):
    """The median select when many distances are equal. Three distinct points
    repeated: the keys matching the median's first two digits are far more
    than the m / 64 the select copies for its last passes, so those passes
    read the whole triangle again. Points on an integer lattice: hundreds of
    keys tie at the median, fewer than the copy holds."""
    rng = np.random.default_rng(7)
    n, T = 700, 5
    if kind == "three_points":
        P = np.array([[0.0] * T, [1.0] * T, [0.5, -2.0, 3.0, 0.25, 1.5]])
        X = P[rng.integers(0, 3, n)]
    else:
        X = rng.integers(-10, 11, (n, T)).astype(np.float64)   # 717 keys tie at the median
    A, D, vol, sig = G.graph(X)
    Ao, Do, volo, sigo = O.gaussian_graph(X)
    assert _h(sig)[0] == sigo
    np.testing.assert_allclose(_h(A), Ao, rtol=A_RTOL, atol=0)


def test_graph_off_grid_uses_float64_path(G):
    rng = np.random.default_rng(5)
    X = rng.standard_normal((130, 7)) * 3.0 + 1e-9   # off the 2^-16 grid
    A, D, vol, sig = G.graph(X)
    Ao, Do, volo, sigo = O.gaussian_graph(X)
    assert _h(sig)[0] == sigo
    np.testing.assert_allclose(_h(A), Ao, rtol=A_RTOL, atol=0)


def test_graph_given_sigma(G):
    X = iid_pair(100, 9, 1, seed=2).X[0]
    A, D, vol, sig = G.graph(X, sigma=1.75)
    Ao, Do, volo, _ = O.gaussian_graph(X, sigma=1.75)
    assert _h(sig)[0] == 1.75
    np.testing.assert_allclose(_h(A), Ao, rtol=A_RTOL, atol=0)


def test_graph_with_tiny_kernel_values(G):
    """A sigma small enough that a fifth of the kernel values lie in [2^-100,
    2^-74], where splitting a float64 into two floats needs a subnormal low
    part: values, degrees (the smallest about 6e-17) and the projection (square
    roots of A) still match the oracle."""
    X = iid_pair(300, 8, 1, seed=4).X[0]
    sigma = 0.375
    A, D, vol, sig = G.graph(X, sigma=sigma)
    Ao, Do, volo, _ = O.gaussian_graph(X, sigma=sigma)
    a = Ao[np.triu_indices(300, 1)]
    assert np.mean((a > 2.0 ** -100) & (a < 2.0 ** -74)) > 0.2
    # the arguments t = d2 / (2 sigma^2) reach about 150 here: the two sides round t
    # differently (d2 times the rounded 1 / (2 sigma^2), against the rounded
    # quotient), each within 2^-53 relative, which moves exp(-t) by up to t 2^-52
    Ah = _h(A)
    off = ~np.eye(300, dtype=bool)
    t = -np.log(Ao[off])
    assert np.all(np.abs(Ah[off] - Ao[off]) <= (A_RTOL + t * 2.0 ** -52) * Ao[off])
    assert np.all(np.diag(Ah) == 0.0)
    np.testing.assert_allclose(_h(D), Do, rtol=1e-13)
    Y = _h(G.project(torch.from_numpy(Ao).cuda(), 32, 9))
    Yo = O.project(Ao, 9, 32)
    assert np.abs(Y - Yo).max() <= 1e-12 * np.abs(Yo).max()


def test_graph_field_workload(G):
    X = field_sequence(16, 32, 48, 2, patch=4, seed=3).X[1]
    A, D, vol, sig = G.graph(X)
    Ao, Do, volo, sigo = O.gaussian_graph(X)
    assert _h(sig)[0] == sigo
    np.testing.assert_allclose(_h(A), Ao, rtol=A_RTOL, atol=0)


# ------------------------------------------------------------------ projection

@pytest.mark.parametrize("n,k,seed", [(50, 1, 1), (97, 5, 2), (300, 32, 3), (200, 130, 2 ** 40 + 7),
                                      # k of the benchmarks and beyond: ragged row blocks and edge
                                      # tiles, two 128-row Philox blocks per edge
                                      (300, 128, 4), (211, 192, 5), (77, 256, 2 ** 33 + 1)])
def test_projection_matches_oracle(G, n, k, seed):
    X = iid_pair(n, 16, 1, seed=n + k).X[0]
    Ao, *_ = O.gaussian_graph(X)
    Y = _h(G.project(torch.from_numpy(Ao).cuda(), k, seed))
    Yo = O.project(Ao, seed, k)
    assert np.abs(Y - Yo).max() <= 1e-12 * np.abs(Yo).max()
    assert np.abs(Y.sum(0)).max() <= 1e-11 * np.abs(Yo).max()


def test_projection_scales_with_weights_k128(G):
    """The piece grids follow sqrt(max A): weights four times larger (max A
    above 1) give exactly twice the projection at the benchmark's k = 128."""
    X = iid_pair(260, 16, 1, seed=41).X[0]
    Ao, *_ = O.gaussian_graph(X)
    A = torch.from_numpy(Ao).cuda()
    Y = _h(G.project(A, 128, 9))
    Y4 = _h(G.project(4.0 * A, 128, 9))
    assert np.array_equal(Y4, 2.0 * Y)


# ------------------------------------------------------------------ chain

def _deflated_levels(Ao, d):
    D = Ao.sum(1)
    u = np.sqrt(D / D.sum())
    return [L - np.outer(u, u) for L in O.chain_levels(Ao, d)]


DT = {"f64": 0, "f32": 1, "bf16": 2, "fp8": 3, "fp8t": 4}


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-12), ("f32", 2e-5), ("bf16", 3e-2), ("fp8", 0.2),
                                       ("fp8t", 0.1)])
@pytest.mark.parametrize("n", [300, 1000])
def test_chain_levels_match_oracle(G, dtype, tol, n):
    cdl = G.cdl
    dt = DT[dtype]
    X = iid_pair(n, 32, 1, seed=7).X[0]
    A, D, vol, _ = G.graph(X)
    d = 4
    ch = G.chain(A, D, vol, d, dt)
    try:
        ref = _deflated_levels(_h(A), d)
        scale = np.linalg.norm(ref[0])
        for i in range(d):
            Lg = G.level_values(ch, i, {"f64": np.float64, "f32": np.float32, "bf16": "bf16", "fp8": "fp8",
                                        "fp8t": "fp8t"}[dtype])
            assert np.all(Lg[n:, :] == 0) and np.all(Lg[:, n:] == 0)   # zero padding
            assert np.array_equal(Lg, Lg.T)                             # exact symmetry
            err = np.linalg.norm(Lg[:n, :n] - ref[i]) / scale
            assert err <= tol, (i, err)
    finally:
        cdl.cdl_chain_free(ch)


@pytest.mark.parametrize("n", [300, 1000, 2100])
def test_tcgen05_square_is_exact_product_of_its_inputs(G, n):
    """One bf16 squaring against the float64 product of the same bf16 input:
    the only errors allowed are float32 accumulation and the final bf16
    rounding (n = 2100 pads to 2304: 9 x 9 blocks, crossing the 8 x 8
    super-block grouping, diagonal and off-diagonal blocks)."""
    cdl = G.cdl
    X = iid_pair(n, 24, 1, seed=11).X[0]
    A, D, vol, _ = G.graph(X)
    ch = G.chain(A, D, vol, 2, cdl.CDL_BF16)
    try:
        L0 = G.level(ch, 0, "bf16").double().cpu().numpy()
        L1 = G.level(ch, 1, "bf16").double().cpu().numpy()
    finally:
        cdl.cdl_chain_free(ch)
    R = L0 @ L0
    bound = 2.0 ** -8 * np.abs(R) + L0.shape[0] * 2.0 ** -23 * (np.abs(L0) @ np.abs(L0)) + 1e-30
    assert np.all(np.abs(L1 - R) <= bound)
    assert np.array_equal(L1, L1.T)


@pytest.mark.parametrize("n", [300, 1000, 2100])
def test_tcgen05_fp8_tile_square_is_exact_product_of_its_inputs(G, n):
    """One e4m3 squaring with 128 x 128 tile scales (tcgen05 kind::mxf8f6f4,
    the tensor core applying each operand tile's e8m0 scale) against the
    float64 product of the same dequantized input: the bf16 copy may differ
    by the float32 accumulation and bf16 rounding; each output tile's scale is
    the least power of two 2^e with tile maximum <= 448 * 2^e, and its e4m3
    values are the tile divided by the scale, rounded (2^-4 relative, or one
    subnormal step of the tile). A tile scale applied to the wrong 128
    columns of an operand would be off by powers of two and fail the bounds;
    n = 1000 and 2100 have several tiles per row with different scales."""
    cdl = G.cdl
    X = iid_pair(n, 24, 1, seed=17).X[0]
    A, D, vol, _ = G.graph(X)
    ch = G.chain(A, D, vol, 2, cdl.CDL_FP8E4M3_T128)
    try:
        V0 = G.level_values(ch, 0, "fp8t")
        V1 = G.level_values(ch, 1, "fp8t")
        S0 = G.tile_scales(ch, 0)
        S1 = G.tile_scales(ch, 1)
        L16 = G.level16(ch, 1)
    finally:
        cdl.cdl_chain_free(ch)
    R = V0 @ V0
    acc = V0.shape[0] * 2.0 ** -23 * (np.abs(V0) @ np.abs(V0))
    assert np.all(np.abs(L16 - R) <= 2.0 ** -8 * np.abs(R) + acc + 1e-30)
    s1 = np.kron(S1, np.ones((128, 128)))
    assert np.all(np.abs(V1 - R) <= 2.0 ** -4 * np.abs(R) + s1 * 2.0 ** -9 + acc + 1e-30)
    nt = S1.shape[0]
    for I in range(nt):
        for J in range(nt):
            blk = np.s_[I * 128:(I + 1) * 128, J * 128:(J + 1) * 128]
            m = np.abs(R[blk]).max()
            sc = S1[I, J]
            assert sc > 0 and math.frexp(sc)[0] == 0.5, (I, J, sc)          # a power of two
            if m > 0:
                slack = 2.0 ** -20 * m + acc[blk].max()
                assert m <= 448 * sc + slack and m > 224 * sc - slack, (I, J, m, sc)
            assert np.abs(V1[blk]).max() <= 448 * sc * (1 + 1e-6)
    # the level-0 scales are powers of two too
    assert all(math.frexp(v)[0] == 0.5 for v in np.unique(S0))
    assert np.array_equal(S1, S1.T)
    assert np.array_equal(V1, V1.T) and np.array_equal(L16, L16.T)


@pytest.mark.parametrize("n", [300, 1000, 2100])
def test_tcgen05_fp8_square_is_exact_product_of_its_inputs(G, n):
    """One e4m3 squaring (kind::f8f6f4) against the float64 product of the same
    dequantized e4m3 input: the bf16 copy of the output may differ only by
    float32 accumulation and bf16 rounding; the e4m3 output additionally by
    e4m3 rounding (2^-4 relative, or one subnormal step) and must respect the
    per-level bound (no overflow)."""
    cdl = G.cdl
    X = iid_pair(n, 24, 1, seed=13).X[0]
    A, D, vol, _ = G.graph(X)
    ch = G.chain(A, D, vol, 2, cdl.CDL_FP8E4M3)
    try:
        V0 = G.level_values(ch, 0, "fp8")
        V1 = G.level_values(ch, 1, "fp8")
        st, sc1 = cdl.cdl_chain_level_scale(ch, 1)
        st2, p16, npad = cdl.cdl_chain_level(ch, 1)
        L16 = G.level16(ch, 1)
    finally:
        cdl.cdl_chain_free(ch)
    R = V0 @ V0
    acc = V0.shape[0] * 2.0 ** -23 * (np.abs(V0) @ np.abs(V0))
    assert np.all(np.abs(L16 - R) <= 2.0 ** -8 * np.abs(R) + acc + 1e-30)
    assert np.all(np.abs(V1 - R) <= 2.0 ** -4 * np.abs(R) + sc1 * 2.0 ** -9 + acc + 1e-30)
    assert np.abs(V1).max() <= 448 * sc1 * (1 + 1e-6)
    assert np.array_equal(V1, V1.T) and np.array_equal(L16, L16.T)


def test_simt_f32_square_is_exact_product_of_its_inputs(G):
    cdl = G.cdl
    n = 700
    X = iid_pair(n, 24, 1, seed=12).X[0]
    A, D, vol, _ = G.graph(X)
    ch = G.chain(A, D, vol, 2, cdl.CDL_F32)
    try:
        L0 = G.level(ch, 0, np.float32).double().cpu().numpy()
        L1 = G.level(ch, 1, np.float32).double().cpu().numpy()
    finally:
        cdl.cdl_chain_free(ch)
    R = L0 @ L0
    bound = 2.0 ** -24 * np.abs(R) + L0.shape[0] * 2.0 ** -23 * (np.abs(L0) @ np.abs(L0)) + 1e-30
    assert np.all(np.abs(L1 - R) <= bound)


# ------------------------------------------------------------------ solve

@pytest.mark.parametrize("full", [False, True])
@pytest.mark.parametrize("dtype,tol", [("f64", 1e-11), ("f32", 1e-10), ("bf16", 1e-10), ("fp8", 1e-10)])
@pytest.mark.parametrize("n,k", [(300, 8), (1000, 32)])
def test_solve_matches_exact_embedding(G, dtype, tol, n, k, full):
    cdl = G.cdl
    dt = DT[dtype]
    X = iid_pair(n, 32, 1, seed=n + 1).X[0]
    Ao, Do, volo, _ = O.gaussian_graph(X)
    Yo = O.project(Ao, 9, k)
    Zo = O.exact_embedding(Ao, Yo)
    A = torch.from_numpy(Ao).cuda()
    D = torch.from_numpy(Do).cuda()
    vol = torch.tensor([volo], dtype=torch.float64, device="cuda")
    ch = G.chain(A, D, vol, 6, dt)
    try:
        Z, stats = G.solve(ch, A, torch.from_numpy(Yo).cuda(), max_iter=30, rel_tol=tol,
                           flags=cdl.CDL_SOLVE_FULL_RESIDUAL if full else 0)
    finally:
        cdl.cdl_chain_free(ch)
    Zg = _h(Z)
    assert stats.rel_res <= tol and stats.iters >= 1
    assert O.residual_norm(Ao, Yo, Zg) <= 3 * tol
    assert np.linalg.norm(Zg - Zo) <= 100 * tol * np.linalg.norm(Zo)
    assert np.abs(Do @ Zg).max() <= 1e-12 * np.abs(Zg).max() * Do.sum()


def test_solve_reports_not_converged(G):
    cdl = G.cdl
    X = iid_pair(300, 16, 1, seed=4).X[0]
    Ao, Do, volo, _ = O.gaussian_graph(X)
    A = torch.from_numpy(Ao).cuda()
    D = torch.from_numpy(Do).cuda()
    vol = torch.tensor([volo], dtype=torch.float64, device="cuda")
    ch = G.chain(A, D, vol, 1, cdl.CDL_BF16)
    try:
        Y = torch.from_numpy(O.project(Ao, 1, 4)).cuda()
        Z, stats = G.solve(ch, A, Y, max_iter=1, rel_tol=1e-14, expect=cdl.CDL_ERR_NOT_CONVERGED)
    finally:
        cdl.cdl_chain_free(ch)
    assert stats.iters == 1 and stats.rel_res > 1e-14


@pytest.mark.parametrize("dtype", ["bf16", "fp8t"])
@pytest.mark.parametrize("k", [136, 192, 300])
def test_solve_more_than_128_columns(G, dtype, k):
    """Tensor-core chains apply a level to at most 128 right-hand sides at a
    time; more columns are solved as independent column blocks (Alg. 2 acts on
    each column on its own). k = 136 and 300 leave ragged blocks, 192 is the
    projection dimension of the n = 131072 configuration. Checked against the
    exact embedding L^+ Y, column by column and as a whole."""
    cdl = G.cdl
    n, tol = 700, 1e-10
    X = iid_pair(n, 32, 1, seed=k).X[0]
    Ao, Do, volo, _ = O.gaussian_graph(X)
    Yo = O.project(Ao, 5, k)
    Zo = O.exact_embedding(Ao, Yo)
    A = torch.from_numpy(Ao).cuda()
    D = torch.from_numpy(Do).cuda()
    vol = torch.tensor([volo], dtype=torch.float64, device="cuda")
    ch = G.chain(A, D, vol, 7, DT[dtype])
    try:
        Z, stats = G.solve(ch, A, torch.from_numpy(Yo).cuda(), max_iter=30, rel_tol=tol)
    finally:
        cdl.cdl_chain_free(ch)
    Zg = _h(Z)
    assert stats.rel_res <= tol and stats.iters >= 1
    res = O.residual_norm(Ao, Yo, Zg)
    assert res <= 3 * tol and abs(res - stats.rel_res) <= 0.1 * tol + 0.5 * stats.rel_res
    for c in range(k):                     # every column block solved, none left at zero
        assert np.linalg.norm(Zg[:, c] - Zo[:, c]) <= 100 * tol * np.linalg.norm(Zo[:, c])
    assert np.abs(Do @ Zg).max() <= 1e-12 * np.abs(Zg).max() * Do.sum()
    assert 0 < stats.history[stats.iters - 1] <= tol


def test_pair_k192_bf16_matches_oracle(G):
    """The whole pair (Alg. 4) with k = 192 on a bf16 chain, against the
    oracle's exact embeddings."""
    cdl = G.cdl
    wl = iid_pair(600, 32, 4, seed=192)
    k, seed, topk = 192, 11, 10
    F, top, s1, s2 = G.pair(wl.X[0], wl.X[1], k, 8, cdl.CDL_BF16, cdl.CDL_F32, seed, topk, max_iter=40,
                            rel_tol=1e-12)
    ref = O.caddelag_pair(wl.X[0], wl.X[1], k, seed, topk)
    Fo, topo = ref["F"], ref["top"]
    assert s1.rel_res <= 1e-12 and s2.rel_res <= 1e-12
    assert np.max(np.abs(F - Fo) / Fo) <= 1e-6
    if O.min_relative_gap(Fo, topk) > 1e-5:
        assert list(top) == list(topo)


# ------------------------------------------------------------------ scores

SCORE_DT = {"f64": "CDL_F64", "f32": "CDL_F32", "bf16": "CDL_BF16"}


@pytest.mark.parametrize("score", ["f64", "f32", "bf16"])
def test_scores_match_oracle(G, score):
    cdl = G.cdl
    wl = iid_pair(333, 24, 6, seed=8)
    g = [O.embed(X, 16, 3) for X in wl.X]
    Fo = O.node_scores(g[0]["A"], g[1]["A"], g[0]["Z"], g[1]["Z"], g[0]["vol"], g[1]["vol"])
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    v1 = torch.tensor([g[0]["vol"]], dtype=torch.float64, device="cuda")
    v2 = torch.tensor([g[1]["vol"]], dtype=torch.float64, device="cuda")
    sd = getattr(cdl, SCORE_DT[score])
    F, top = G.score(t(g[0]["A"]), t(g[1]["A"]), t(g[0]["Z"]), t(g[1]["Z"]), v1, v2, 8, sd)
    rel = np.abs(_h(F) - Fo) / Fo
    # float32 pipes with grid-split differences and compensated sums, or exact
    # bf16 slices on the tensor cores: each commute-time difference to about
    # 2^-45 of its terms' scale
    assert rel.max() <= (1e-12 if score == "f64" else 1e-10), rel.max()
    if O.min_relative_gap(Fo, 8) > 1e-6:
        assert list(_h(top)) == list(O.top_anomalies(Fo, 8))


@pytest.mark.parametrize("score", ["f64", "f32", "bf16"])
def test_scores_with_cancelling_sums(G, score):
    """Ragged-pair statistics (n = 407, 2 perturbed nodes, k = 32): for many
    node pairs the k-term commute-time difference cancels by a factor of 10^3;
    a plain float32 sum misses such nodes' scores by 1e-5."""
    from workloads import ragged_pairs
    cdl = G.cdl
    wl = ragged_pairs(G=6, n_lo=256, n_hi=1200, T=64, seed=7)[4]
    g = [O.embed(X, 32, 7) for X in wl.X]
    Fo = O.node_scores(g[0]["A"], g[1]["A"], g[0]["Z"], g[1]["Z"], g[0]["vol"], g[1]["vol"])
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    v1 = torch.tensor([g[0]["vol"]], dtype=torch.float64, device="cuda")
    v2 = torch.tensor([g[1]["vol"]], dtype=torch.float64, device="cuda")
    sd = getattr(cdl, SCORE_DT[score])
    F, top = G.score(t(g[0]["A"]), t(g[1]["A"]), t(g[0]["Z"]), t(g[1]["Z"]), v1, v2, 5, sd)
    rel = np.abs(_h(F) - Fo) / Fo
    # float64 sums carry 2^-53 of the cancelling terms (up to 10^3 times the
    # difference): about 1e-11 on the worst node
    assert rel.max() <= 1e-10, rel.max()


@pytest.mark.parametrize("n,k", [(130, 8), (1000, 128), (777, 96), (2, 1)])
def test_scores_bf16_shapes(G, n, k):
    """Tensor-core scores over ragged shapes: n not a multiple of the 128 x 64
    tiles (partner blocks past n), k padded to the 64-wide K blocks, the
    smallest graph; embeddings of unequal scale in the two graphs."""
    cdl = G.cdl
    rng = np.random.default_rng(n + k)
    X1 = iid_pair(n, 12, 1, seed=n).X[0]
    X2 = X1.copy()
    X2[: max(1, n // 50)] += 0.25
    A1, _, vol1, _ = O.gaussian_graph(X1)
    A2, _, vol2, _ = O.gaussian_graph(X2)
    Z1 = rng.standard_normal((n, k)) * 1e-2
    Z2 = Z1 + rng.standard_normal((n, k)) * 1e-4
    Fo = O.node_scores(A1, A2, Z1, Z2, vol1, vol2)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    v1 = torch.tensor([vol1], dtype=torch.float64, device="cuda")
    v2 = torch.tensor([vol2], dtype=torch.float64, device="cuda")
    F, top = G.score(t(A1), t(A2), t(Z1), t(Z2), v1, v2, min(n, 4), cdl.CDL_BF16)
    F = _h(F)
    ok = Fo > 0
    assert np.all(F[~ok] == 0.0)
    assert np.max(np.abs(F[ok] - Fo[ok]) / Fo[ok]) <= 1e-10


# ------------------------------------------------------------------ whole pair (Alg. 4)

@pytest.fixture(scope="module")
def iid1024():
    wl = iid_pair(1024, 64, 10, 0)
    out = O.caddelag_pair(wl.X[0], wl.X[1], k=32, seed=0, topk=10)
    return wl, out


@pytest.mark.parametrize("chain,score,tol,host_io", [
    ("f64", "f64", 1e-9, False),
    ("f64", "f64", 1e-9, True),
    ("f32", "f64", 1e-9, False),
    ("bf16", "f32", 1e-6, False),
    ("bf16", "f32", 1e-6, True),
    ("bf16", "bf16", 1e-6, False),
    ("fp8", "f32", 1e-6, False),
    ("fp8t", "f32", 1e-6, False),
])
def test_pair_iid_n1024_matches_oracle(G, iid1024, chain, score, tol, host_io):
    cdl = G.cdl
    wl, out = iid1024
    dt = DT
    F, top, s1, s2 = G.pair(wl.X[0], wl.X[1], 32, 8, dt[chain], dt[score], 0, 10, host_io=host_io)
    Fo = out["F"]
    rel = np.abs(F - Fo) / Fo
    assert rel.max() <= tol, rel.max()
    assert s1.rel_res <= 1e-10 and s2.rel_res <= 1e-10
    gap = O.min_relative_gap(Fo, 10)
    assert gap > 10 * tol
    assert list(top) == list(out["top"])
    assert set(top.tolist()) == set(wl.planted[0].tolist())


def test_pair_field_bf16_finds_patch(G):
    cdl = G.cdl
    wl = field_sequence(32, 64, 64, 2, patch=4, patch_transition=0, seed=5)
    out = O.caddelag_pair(wl.X[0], wl.X[1], k=32, seed=1, topk=16)
    F, top, s1, s2 = G.pair(wl.X[0], wl.X[1], 32, 10, cdl.CDL_BF16, cdl.CDL_F32, 1, 16)
    rel = np.abs(F - out["F"]) / out["F"]
    assert rel.max() <= 1e-6, rel.max()
    if O.min_relative_gap(out["F"], 16) > 1e-5:
        assert list(top) == list(out["top"])
    assert len(set(top.tolist()) & set(wl.planted[0].tolist())) >= 12


def test_pair_field_fp8_tiles_finds_patch(G):
    """The field graph whose dynamic range defeats one scale per level: with
    one scale per 128 x 128 tile the e4m3 chain preconditions the refinement
    to the same tolerance and scores."""
    cdl = G.cdl
    wl = field_sequence(32, 64, 64, 2, patch=4, patch_transition=0, seed=5)
    out = O.caddelag_pair(wl.X[0], wl.X[1], k=32, seed=1, topk=16)
    F, top, s1, s2 = G.pair(wl.X[0], wl.X[1], 32, 10, cdl.CDL_FP8E4M3_T128, cdl.CDL_F32, 1, 16, max_iter=40)
    assert s1.rel_res <= 1e-10 and s2.rel_res <= 1e-10
    rel = np.abs(F - out["F"]) / out["F"]
    assert rel.max() <= 1e-6, rel.max()
    assert len(set(top.tolist()) & set(wl.planted[0].tolist())) >= 12


# ------------------------------------------------------------------ validation

def test_invalid_arguments(G):
    cdl = G.cdl
    n, T = 64, 8
    X = torch.zeros((n, T), dtype=torch.float64, device="cuda")
    A = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    D = torch.zeros(n, dtype=torch.float64, device="cuda")
    s = torch.zeros(2, dtype=torch.float64, device="cuda")
    Xh = np.zeros((n, T))
    args = (s[0:1].data_ptr(), s[1:2].data_ptr())
    assert cdl.cdl_build_graph(G.h, X, 1, T, 0.0, cdl.CDL_F64, A, D, *args) == cdl.CDL_ERR_INVALID_ARG
    assert cdl.cdl_build_graph(G.h, X, n, 0, 0.0, cdl.CDL_F64, A, D, *args) == cdl.CDL_ERR_INVALID_ARG
    assert cdl.cdl_build_graph(G.h, Xh, n, T, 0.0, cdl.CDL_F64, A, D, *args) == cdl.CDL_ERR_INVALID_ARG
    assert cdl.cdl_build_graph(G.h, X, n, T, 0.0, cdl.CDL_F32, A, D, *args) == cdl.CDL_ERR_UNSUPPORTED
    assert cdl.cdl_build_graph(G.h, X.data_ptr() + 4, n, T, 0.0, cdl.CDL_F64, A, D, *args) == \
        cdl.CDL_ERR_INVALID_ARG
    st, ch = cdl.cdl_chain_build(G.h, A, cdl.CDL_F64, D, s, n, 3, 7)     # no such dtype
    assert st == cdl.CDL_ERR_INVALID_ARG
    assert cdl.cdl_project(G.h, A, cdl.CDL_F64, n, 0, 1, A) == cdl.CDL_ERR_INVALID_ARG
    assert cdl.cdl_project(G.h, A, cdl.CDL_F64, n, 1025, 1, A) == cdl.CDL_ERR_INVALID_ARG
    F = torch.zeros(n, dtype=torch.float64, device="cuda")
    assert cdl.cdl_cad_score(G.h, A, A, cdl.CDL_F64, A, A, s, s, n, 4, cdl.CDL_FP8E4M3, 2, F, F) == \
        cdl.CDL_ERR_INVALID_ARG
    assert cdl.cdl_cad_score(G.h, A, A, cdl.CDL_F64, A, A, s, s, n, 4, cdl.CDL_F64, n + 1, F, F) == \
        cdl.CDL_ERR_INVALID_ARG
    assert cdl.cdl_sync(G.h) == cdl.CDL_OK


def test_chain_reuse_and_mismatch(G):
    cdl = G.cdl
    X = iid_pair(200, 8, 1, seed=1).X[0]
    A, D, vol, _ = G.graph(X)
    ch = G.chain(A, D, vol, 3, cdl.CDL_F32)
    try:
        ch2 = G.chain(A, D, vol, 3, cdl.CDL_F32, chain=ch)   # same shape: storage reused
        assert ch2.value == ch.value
        st, _ = cdl.cdl_chain_build(G.h, A, cdl.CDL_F64, D, vol.data_ptr(), 200, 4, cdl.CDL_F32, 0, ch)
        assert st == cdl.CDL_ERR_INVALID_ARG
    finally:
        cdl.cdl_chain_free(ch)


def test_workspace_cap_gives_oom():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from gpu_util import lib
    cdl = lib()
    st, h = cdl.cdl_ctx_create(0, torch.cuda.current_stream().cuda_stream, 1 << 20)
    assert st == 0
    try:
        n, T = 600, 8
        X = torch.from_numpy(iid_pair(n, T, 1, seed=1).X[0]).cuda()
        A = torch.zeros((n, n), dtype=torch.float64, device="cuda")
        D = torch.zeros(n, dtype=torch.float64, device="cuda")
        s = torch.zeros(2, dtype=torch.float64, device="cuda")
        assert cdl.cdl_build_graph(h, X, n, T, 0.0, cdl.CDL_F64, A, D, s[0:1].data_ptr(),
                                   s[1:2].data_ptr()) == cdl.CDL_OK
        st, ch = cdl.cdl_chain_build(h, A, cdl.CDL_F64, D, s[0:1].data_ptr(), n, 8, cdl.CDL_F64)
        assert st == cdl.CDL_ERR_OOM
    finally:
        cdl.cdl_ctx_destroy(h)


def test_launch_counter_and_timing(G):
    cdl = G.cdl
    cdl.cdl_ctx_reset_counters(G.h)
    cdl.cdl_ctx_set_timing(G.h, True)
    X = iid_pair(256, 8, 1, seed=1).X[0]
    G.graph(X)
    st, n = cdl.cdl_ctx_launch_count(G.h)
    assert st == 0 and n >= 10
    st, ms, launches, work = cdl.cdl_ctx_timing(G.h, cdl.CDL_KC_DISTANCE)
    # fixed-point check, digit planes, norms, tensor-core Gram, float64 fallback (returns at once)
    assert st == 0 and launches == 5 and ms > 0 and work == 0.5 * 256 * 255 * 8
    cdl.cdl_ctx_set_timing(G.h, False)


@pytest.mark.parametrize("n,k", [(1000, 32), (700, 96), (1300, 128)])
def test_exact_slice_residual(G, n, k):
    """The tensor chains' full residual (A Z from exact bf16 slices on the
    tensor cores): after each of a few refinement steps, the reported
    residual norm equals the float64 residual of the returned Z computed on
    the host in extended precision, to 1e-15 of ||Y||."""
    cdl = G.cdl
    X = iid_pair(n, 32, 1, seed=23).X[0]
    A, D, vol, _ = G.graph(X)
    ch = G.chain(A, D, vol, 6, cdl.CDL_BF16)
    try:
        Y = G.project(A, k, 9)
        An, Dn, Yn = _h(A).astype(np.longdouble), _h(D).astype(np.longdouble), _h(Y).astype(np.longdouble)
        ny = np.sqrt((Yn ** 2).sum())
        for it in (1, 2, 3):
            Z, st = G.solve(ch, A, Y, max_iter=it, rel_tol=0.0, flags=cdl.CDL_SOLVE_FULL_RESIDUAL)
            Zn = _h(Z).astype(np.longdouble)
            R = Yn - (Dn[:, None] * Zn - An @ Zn)
            rel = float(np.sqrt((R ** 2).sum()) / ny)
            assert abs(st.rel_res - rel) <= 1e-15, (it, st.rel_res, rel)
    finally:
        cdl.cdl_chain_free(ch)
