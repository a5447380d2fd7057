"""Graph sequence on the plain float32 GPU path (chain in float32 on CUDA
cores): 4 graphs of the 64 x 128 correlated field (n = 8192, T = 128), each
embedded once and reused by its two pairs (k = 64, d = 12); node scores of the
3 transitions against the float64 oracle; the planted patch of transition 2
ranks on top."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import caddelag as O             # noqa: E402
from workloads import field_sequence          # noqa: E402

pytestmark = pytest.mark.gpu


def test_field_sequence_n8192_f32_path():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from gpu_util import Ctx, lib
    G = Ctx(lib())
    cdl = G.cdl
    wl = field_sequence(64, 128, 128, 4, patch=8, patch_transition=1, seed=1)
    k, d, seed, topk = 64, 12, 5, 10
    emb = []
    try:
        for X in wl.X:
            A, D, vol, sig = G.graph(X)
            ch = G.chain(A, D, vol, d, cdl.CDL_F32)
            try:
                Y = G.project(A, k, seed)
                Z, st = G.solve(ch, A, Y, max_iter=20, rel_tol=1e-10)
                assert st.rel_res <= 1e-10
            finally:
                cdl.cdl_chain_free(ch)
            emb.append((A, vol, Z, float(sig.item())))
        for t in range(3):
            (A1, v1, Z1, s1), (A2, v2, Z2, s2) = emb[t], emb[t + 1]
            F, top = G.score(A1, A2, Z1, Z2, v1, v2, topk, cdl.CDL_F32)
            F = F.cpu().numpy()
            # oracle on the same inputs: exact graphs (sigma checked), exact embeddings
            Ao = []
            for X, s in ((wl.X[t], s1), (wl.X[t + 1], s2)):
                d2 = O.squared_distances_exact_grid(X)
                assert O.median_sigma(d2) == s
                Ao.append(O.gaussian_graph(X, d2=d2))
            Zo = [O.exact_embedding(a[0], O.project(a[0], seed, k)) for a in Ao]
            Fo = O.node_scores(Ao[0][0], Ao[1][0], Zo[0], Zo[1], Ao[0][2], Ao[1][2])
            rel = np.abs(F - Fo) / Fo
            assert rel.max() <= 1e-6, (t, rel.max())
            if O.min_relative_gap(Fo, topk) > 1e-5:
                assert list(top.cpu().numpy()) == list(O.top_anomalies(Fo, topk))
            if t == 1:
                assert set(top.cpu().numpy().tolist()) <= set(wl.planted[1].tolist())
    finally:
        G.close()
