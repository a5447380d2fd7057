"""Scores over the changed edges only (Sec. 3.3: commute times are needed
only where Delta A != 0). With a sigma shared by both graphs, A1 and A2
differ only in the rows and columns of the nodes whose series changed; the
sparse pass must give the dense pass's scores (to summation order) and the
oracle's."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import caddelag as O           # noqa: E402
from workloads import iid_pair   # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from gpu_util import Ctx, lib
    c = Ctx(lib())
    yield c
    c.close()


def _changed(G, X1, X2):
    from gpu_util import dev
    n, T = X1.shape
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    st, m = G.cdl.cdl_changed_nodes(G.h, dev(X1), dev(X2), n, T, out)
    G.check(st)
    return out, m


@pytest.mark.parametrize("n,k_changed", [(1000, 7), (333, 1), (257, 0)])
def test_changed_nodes(G, n, k_changed):
    wl = iid_pair(n, 24, max(k_changed, 1), seed=31)
    X2 = wl.X[1] if k_changed else wl.X[0].copy()
    out, m = _changed(G, wl.X[0], X2)
    expect = np.nonzero(np.any(wl.X[0] != X2, axis=1))[0]
    assert m == len(expect) and list(out.cpu().numpy()[:m]) == list(expect)


def _shared_sigma_pair(G, X1, X2, k, d, seed, chain):
    """Both graphs with graph 1's median sigma; embeddings by the chain solve."""
    A1, D1, v1, s1 = G.graph(X1)
    sig = float(s1.item())
    A2, D2, v2, _ = G.graph(X2, sigma=sig)
    out = []
    for A, D, v in ((A1, D1, v1), (A2, D2, v2)):
        ch = G.chain(A, D, v, d, chain)
        try:
            Y = G.project(A, k, seed)
            Z, st = G.solve(ch, A, Y, max_iter=40, rel_tol=1e-12)
        finally:
            G.cdl.cdl_chain_free(ch)
        out.append((A, Z, v))
    return out, sig


@pytest.mark.parametrize("score", ["f32", "f64"])
def test_sparse_scores_equal_dense(G, score):
    cdl = G.cdl
    wl = iid_pair(1200, 32, 9, seed=41)
    (g1, g2), sig = _shared_sigma_pair(G, wl.X[0], wl.X[1], 32, 8, 3, cdl.CDL_BF16)
    sd = cdl.CDL_F32 if score == "f32" else cdl.CDL_F64
    Fd, td = G.score(g1[0], g2[0], g1[1], g2[1], g1[2], g2[2], 10, sd)
    lst, m = _changed(G, wl.X[0], wl.X[1])
    n, k = g1[1].shape
    Fs = torch.empty(n, dtype=torch.float64, device="cuda")
    ts = torch.empty(10, dtype=torch.int64, device="cuda")
    G.check(cdl.cdl_cad_score_changed(G.h, g1[0], g2[0], cdl.CDL_F64, g1[1], g2[1], g1[2].data_ptr(),
                                      g2[2].data_ptr(), n, k, sd, lst, m, 10, Fs, ts))
    G.check(cdl.cdl_sync(G.h))
    Fd, Fs = Fd.cpu().numpy(), Fs.cpu().numpy()
    np.testing.assert_allclose(Fs, Fd, rtol=1e-12, atol=0)
    assert list(ts.cpu().numpy()) == list(td.cpu().numpy())
    # and the oracle's dense definition with the same shared sigma
    A1o, _, vol1, _ = O.gaussian_graph(wl.X[0], sig)
    A2o, _, vol2, _ = O.gaussian_graph(wl.X[1], sig)
    Z1o = O.exact_embedding(A1o, O.project(A1o, 3, 32))
    Z2o = O.exact_embedding(A2o, O.project(A2o, 3, 32))
    Fo = O.node_scores(A1o, A2o, Z1o, Z2o, vol1, vol2)
    assert (np.abs(Fs - Fo) / Fo).max() <= 1e-6
    assert np.all(A1o[np.ix_(~np.isin(np.arange(n), wl.planted[0]), ~np.isin(np.arange(n), wl.planted[0]))]
                  == A2o[np.ix_(~np.isin(np.arange(n), wl.planted[0]), ~np.isin(np.arange(n), wl.planted[0]))])


def test_sparse_scores_no_change_and_all_changed(G):
    cdl = G.cdl
    wl = iid_pair(300, 16, 3, seed=5)
    A1, D1, v1, s1 = G.graph(wl.X[0])
    sig = float(s1.item())
    Z = torch.randn(300, 16, dtype=torch.float64, device="cuda") * 1e-3
    F = torch.empty(300, dtype=torch.float64, device="cuda")
    top = torch.empty(4, dtype=torch.int64, device="cuda")
    none = torch.empty(1, dtype=torch.int32, device="cuda")
    G.check(cdl.cdl_cad_score_changed(G.h, A1, A1, cdl.CDL_F64, Z, Z, v1.data_ptr(), v1.data_ptr(), 300, 16,
                                      cdl.CDL_F32, none, 0, 4, F, top))
    assert torch.count_nonzero(F).item() == 0
    A2, D2, v2, _ = G.graph(wl.X[1], sigma=sig)
    Z2 = Z * 1.3 + 1e-4
    allc = torch.arange(300, dtype=torch.int32, device="cuda")
    G.check(cdl.cdl_cad_score_changed(G.h, A1, A2, cdl.CDL_F64, Z, Z2, v1.data_ptr(), v2.data_ptr(), 300, 16,
                                      cdl.CDL_F32, allc, 300, 4, F, top))
    Fd, _ = G.score(A1, A2, Z, Z2, v1, v2, 4, cdl.CDL_F32)
    np.testing.assert_allclose(F.cpu().numpy(), Fd.cpu().numpy(), rtol=1e-12)


def test_pair_driver_changed_only(G):
    """cdl_caddelag_pair with a shared sigma scores only the changed edges
    when asked, with the same result as its dense scoring."""
    cdl = G.cdl
    wl = iid_pair(1500, 32, 12, seed=8)
    A, D, v, s = G.graph(wl.X[0])
    sig = float(s.item())
    n, T = wl.X[0].shape
    from gpu_util import dev, host
    res = []
    for flags in (0, cdl.CDL_SCORE_CHANGED_ONLY):
        o = cdl.cdl_pair_opts(32, 10, cdl.CDL_BF16, cdl.CDL_F32, 1, sig, cdl.cdl_solve_opts(40, 1e-12, 0), 10, 0, 0,
                              flags)
        F = torch.empty(n, dtype=torch.float64, device="cuda")
        top = torch.empty(10, dtype=torch.int64, device="cuda")
        G.check(cdl.cdl_caddelag_pair(G.h, dev(wl.X[0]), dev(wl.X[1]), n, T, o, F, top, None, None))
        res.append((host(F), host(top)))
    np.testing.assert_allclose(res[1][0], res[0][0], rtol=1e-12)
    assert list(res[1][1]) == list(res[0][1])
    o = cdl.cdl_pair_opts(32, 10, cdl.CDL_BF16, cdl.CDL_F32, 1, 0.0, cdl.cdl_solve_opts(40, 1e-12, 0), 10, 0, 0,
                          cdl.CDL_SCORE_CHANGED_ONLY)
    F = torch.empty(n, dtype=torch.float64, device="cuda")
    top = torch.empty(10, dtype=torch.int64, device="cuda")
    assert cdl.cdl_caddelag_pair(G.h, dev(wl.X[0]), dev(wl.X[1]), n, T, o, F, top, None, None) == \
        cdl.CDL_ERR_INVALID_ARG
