"""The larger-than-memory form at its own size: one graph pair at n = 131072
(a 256 x 512 grid, T = 365 daily samples of the spatially correlated field
plus a seasonal sinusoid, a planted 16 x 16 patch), k = 192, d = 10, bf16
chain levels partly in pinned host memory, float64-class refinement to
1e-10, top-100 anomalies. Neither 137 GB float64 graph is stored: the pair
regenerates them in row panels (cdl_caddelag_pair with
CDL_PAIR_REGEN_GRAPHS).

No exact solve is possible at this size on the host (a dense Cholesky of a
137 GB matrix), so the oracle checks what it can compute from the node
series and the GPU's embeddings (Z parity itself is bounded only through
the residual):
  * sigma: the GPU's value is sqrt of an exact squared distance whose
    streamed counts place it at the lower median's rank;
  * degrees and vol streamed over the upper triangle;
  * sampled rows: the projection Y (plain C oracle), the float64 residual
    Y - D Z + A Z of the GPU's Z (relative to the same rows of Y), the node
    scores recomputed from the GPU's Z;
  * the top-100: every sampled node outside it scores below its last entry,
    the order holds wherever the oracle's scores decide it, and the planted
    patch fills it."""
import gc
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import caddelag as O            # noqa: E402
from workloads import field_sequence        # noqa: E402

pytestmark = [pytest.mark.gpu, pytest.mark.fullsize]

K, DCH, SEED, TOPK, TOL = 192, 10, 2024, 100, 1e-10


def field_pair_n131072():
    return field_sequence(256, 512, 365, 2, patch=16, patch_transition=0, seasonal=0.5, seed=5)


def test_field_pair_n131072_regenerated_graphs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from gpu_util import Ctx, lib, dev
    gc.collect()
    torch.cuda.empty_cache()
    G = Ctx(lib())
    cdl = G.cdl
    wl = field_pair_n131072()
    n, T = wl.X[0].shape
    flags = cdl.CDL_PAIR_REGEN_GRAPHS | cdl.CDL_CHAIN_HOST_LEVELS | cdl.CDL_CHAIN_RESIDENT(255)
    try:
        opts = cdl.cdl_pair_opts(K, DCH, cdl.CDL_BF16, cdl.CDL_BF16, SEED, 0.0, cdl.cdl_solve_opts(40, TOL, 0), TOPK,
                                 0, flags)
        F = torch.empty(n, dtype=torch.float64, device="cuda")
        top = torch.empty(TOPK, dtype=torch.int64, device="cuda")
        s1, s2 = cdl.cdl_solve_stats(), cdl.cdl_solve_stats()
        G.check(cdl.cdl_caddelag_pair(G.h, dev(wl.X[0]), dev(wl.X[1]), n, T, opts, F, top, s1, s2))
        G.check(cdl.cdl_sync(G.h))
        Z1 = np.empty((n, K))
        Z2 = np.empty((n, K))
        sc = np.empty(4)
        G.check(cdl.cdl_pair_embeddings(G.h, Z1, Z2, sc))
        F = F.cpu().numpy()
        top = [int(i) for i in top.cpu().numpy()]
    finally:
        G.close()
        torch.cuda.empty_cache()
    assert s1.rel_res <= TOL and s2.rel_res <= TOL
    vol = sc[:2]
    sig = sc[2:]
    m = n * (n - 1) // 2
    rank = (m - 1) // 2
    rng = np.random.default_rng(3)
    rows = np.unique(np.concatenate([rng.choice(n, 40, replace=False), wl.planted[0][:4]]))
    Arows = []
    for g, X in enumerate(wl.X):
        # sigma: the lower median of the n (n - 1) / 2 exact distances
        key = int(round(sig[g] * sig[g] * 2.0 ** 32))
        assert math.sqrt(key * 2.0 ** -32) == sig[g]
        # and the degrees and the volume, in the same streamed pass
        D, lt, le = O.gaussian_degrees_streamed(X, sig[g], key=key)
        assert lt <= rank < le, (g, lt, rank, le)
        assert math.isclose(vol[g], D.sum(), rel_tol=1e-12)
        # sampled rows of A, Y and the float64 residual of the GPU's Z
        Ar = O.graph_rows(X, sig[g], rows)
        np.testing.assert_allclose(Ar.sum(axis=1), D[rows], rtol=1e-13)
        Yr = O.project_rows_c(Ar, rows, SEED, K)
        Zg = Z1 if g == 0 else Z2
        R = Yr - (D[rows, None] * Zg[rows] - Ar @ Zg)
        assert np.linalg.norm(R) <= 20 * TOL * np.linalg.norm(Yr), np.linalg.norm(R) / np.linalg.norm(Yr)
        assert np.abs(D @ Zg).max() <= 1e-10 * np.abs(Zg).max() * D.sum()   # D-weighted zero column means
        Arows.append(Ar)
        del D
        gc.collect()
    # node scores from the GPU's embeddings: the sampled rows and the top-100
    chk = np.unique(np.concatenate([rows, top]))
    A1c = O.graph_rows(wl.X[0], sig[0], chk)
    A2c = O.graph_rows(wl.X[1], sig[1], chk)
    Fo = O.node_scores_c(A1c, A2c, chk, Z1, Z2, vol[0], vol[1])
    rel = np.abs(F[chk] - Fo) / Fo
    assert rel.max() <= 1e-9, rel.max()
    fo = dict(zip(chk.tolist(), Fo.tolist()))
    tv = [fo[i] for i in top]
    for t in range(TOPK - 1):
        if abs(tv[t] - tv[t + 1]) > 1e-8 * max(tv[t], tv[t + 1]):
            assert tv[t] > tv[t + 1]
    others = [fo[i] for i in rows.tolist() if i not in set(top)]
    assert max(others) < tv[-1]
    assert len(set(top) & set(wl.planted[0].tolist())) >= 90
