"""CAD's anomalous edge set (Sec. 3.3) and per-node top edges against the
float64 oracle: on identical embeddings the set and the partner lists must
match exactly; on the whole pair (GPU embeddings, 1e-9-level differences in
Delta E) they must match wherever the oracle's cut is decided."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import caddelag as O         # noqa: E402
from workloads import iid_pair           # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from gpu_util import Ctx, lib
    c = Ctx(lib())
    yield c
    c.close()


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _edges(G, A1, A2, Z1, Z2, vol1, vol2, delta, score, nodes, m, cap=1 << 16):
    cdl = G.cdl
    n, k = Z1.shape
    ij = torch.full((cap, 2), -7, dtype=torch.int64, device="cuda")
    val = torch.zeros(cap, dtype=torch.float64, device="cuda")
    nd = _t(np.asarray(nodes, dtype=np.int64)) if len(nodes) else torch.zeros(1, dtype=torch.int64, device="cuda")
    part = torch.zeros((max(len(nodes), 1), max(m, 1)), dtype=torch.int64, device="cuda")
    pv = torch.zeros((max(len(nodes), 1), max(m, 1)), dtype=torch.float64, device="cuda")
    F = torch.empty(n, dtype=torch.float64, device="cuda")
    v1 = torch.tensor([vol1], dtype=torch.float64, device="cuda")
    v2 = torch.tensor([vol2], dtype=torch.float64, device="cuda")
    st, res = cdl.cdl_cad_edges(G.h, A1, A2, cdl.CDL_F64, Z1, Z2, v1, v2, n, k, score, delta, cap, ij, val, nd,
                                len(nodes), m, part, pv, F)
    G.check(st)
    s = min(res.n_edges, cap)
    return res, ij[:s].cpu().numpy(), val[:s].cpu().numpy(), part.cpu().numpy(), pv.cpu().numpy(), F.cpu().numpy()


@pytest.mark.parametrize("score,tol", [("f64", 1e-12), ("f32", 1e-10)])
def test_edges_on_oracle_embeddings(G, score, tol):
    """Same A and Z on both sides: Delta E agrees to rounding, so the set is
    exact wherever the oracle's values at the cut are separated."""
    cdl = G.cdl
    wl = iid_pair(700, 32, 6, seed=12)
    g = [O.embed(X, 32, 2) for X in wl.X]
    E = O.upper_edge_scores(g[0]["A"], g[1]["A"], g[0]["Z"], g[1]["Z"], g[0]["vol"], g[1]["vol"])
    iu, ju = np.triu_indices(700, 1)
    v = np.sort(E[iu, ju])[::-1]
    total = v.sum()
    sd = cdl.CDL_F64 if score == "f64" else cdl.CDL_F32
    nodes = list(O.top_anomalies(E.sum(1) + E.sum(0), 5))
    for s_target in (1, 37, 500):
        # delta halfway between the remainders after s - 1 and s edges
        rem_prev, rem = total - v[:s_target - 1].sum(), total - v[:s_target].sum()
        delta = 0.5 * (rem_prev + rem)
        out = O.anomalous_edges(E, delta)
        assert len(out["edges"]) == s_target
        res, ij, val, part, pv, F = _edges(G, _t(g[0]["A"]), _t(g[1]["A"]), _t(g[0]["Z"]), _t(g[1]["Z"]),
                                           g[0]["vol"], g[1]["vol"], delta, sd, nodes, 8)
        assert res.n_edges == s_target and res.remaining < delta
        assert np.array_equal(ij, out["edges"])
        np.testing.assert_allclose(val, out["values"], rtol=tol)
        np.testing.assert_allclose(res.total, out["total"], rtol=1e-12)
    po, pvo = O.node_top_edges(E, nodes, 8)
    assert np.array_equal(part[:len(nodes)], po)
    np.testing.assert_allclose(pv[:len(nodes)], pvo, rtol=tol)
    np.testing.assert_allclose(F, E.sum(1) + E.sum(0), rtol=tol)


def test_edges_limits(G):
    cdl = G.cdl
    wl = iid_pair(300, 16, 2, seed=4)
    g = [O.embed(X, 16, 1) for X in wl.X]
    args = (_t(g[0]["A"]), _t(g[1]["A"]), _t(g[0]["Z"]), _t(g[1]["Z"]), g[0]["vol"], g[1]["vol"])
    E = O.upper_edge_scores(g[0]["A"], g[1]["A"], g[0]["Z"], g[1]["Z"], g[0]["vol"], g[1]["vol"])
    total = E.sum()
    res, ij, *_ = _edges(G, *args, 2 * total, cdl.CDL_F64, [], 0)            # nothing needed
    assert res.n_edges == 0 and len(ij) == 0 and np.isinf(res.threshold)
    res, ij, val, *_ = _edges(G, *args, 1e-300, cdl.CDL_F64, [], 0, cap=50)   # every positive edge; capacity 50
    assert res.n_edges == np.count_nonzero(E) and len(ij) == 50
    full = O.anomalous_edges(E, 1e-300)["edges"]
    assert np.array_equal(ij, full[:50])
    n, k = g[0]["Z"].shape
    v = torch.ones(1, dtype=torch.float64, device="cuda")
    st, _ = cdl.cdl_cad_edges(G.h, args[0], args[1], cdl.CDL_F64, args[2], args[3], v, v, n, k, cdl.CDL_F64, 0.0, 0,
                              None, None, None, 0, 0, None, None, None)
    assert st == cdl.CDL_ERR_INVALID_ARG


def test_edges_whole_pair(G):
    """GPU embeddings (bf16 chain, refined to 1e-12): the edge set matches the
    oracle's where its cut is decided; the planted nodes lead the lists."""
    cdl = G.cdl
    wl = iid_pair(1024, 64, 10, 0)
    out = O.caddelag_pair(wl.X[0], wl.X[1], k=32, seed=0, topk=10)
    g1, g2 = out["g1"], out["g2"]
    E = O.upper_edge_scores(g1["A"], g2["A"], g1["Z"], g2["Z"], g1["vol"], g2["vol"])
    gpu = []
    for X in wl.X:
        A, D, vol, _ = G.graph(X)
        ch = G.chain(A, D, vol, 8, cdl.CDL_BF16)
        try:
            Y = G.project(A, 32, 0)
            Z, _ = G.solve(ch, A, Y, max_iter=40, rel_tol=1e-12)
        finally:
            cdl.cdl_chain_free(ch)
        gpu.append((A, Z, float(vol.item())))
    iu, ju = np.triu_indices(1024, 1)
    v = np.sort(E[iu, ju])[::-1]
    total = v.sum()
    s_target = 200
    delta = 0.5 * ((total - v[:s_target - 1].sum()) + (total - v[:s_target].sum()))
    res, ij, val, part, pv, F = _edges(G, gpu[0][0], gpu[1][0], gpu[0][1], gpu[1][1], gpu[0][2], gpu[1][2], delta,
                                       cdl.CDL_F32, list(out["top"][:3]), 5)
    gap = (v[s_target - 1] - v[s_target]) / v[s_target - 1]
    assert gap > 1e-6     # the cut is decided at this tolerance
    assert res.n_edges == s_target
    assert np.array_equal(ij, O.anomalous_edges(E, delta)["edges"])
    planted = set(wl.planted[0].tolist())
    assert all(i in planted or j in planted for i, j in ij)
