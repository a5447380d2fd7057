"""Graphs too large to keep (the larger-than-memory form, Sec. 1 and Sec.
3.2): cdl_caddelag_pair with CDL_PAIR_REGEN_GRAPHS regenerates each graph
from its node series in row panels wherever it is needed. Checked against
the float64 oracle (node scores 1e-6, top anomalies where decided), against
the stored-graph pair (the same sigma, scores to summation order), with
several panels and a ragged last one, with k = 192 (two column blocks) and
with levels split between device and pinned host memory. Also: chain levels
kept partly on the device equal the device-resident ones bit for bit."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import caddelag as O           # noqa: E402
from workloads import iid_pair, field_sequence   # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from gpu_util import Ctx, lib
    c = Ctx(lib())
    yield c
    c.close()


def _regen_flags(cdl, panel_log2, resident=None):
    f = cdl.CDL_PAIR_REGEN_GRAPHS | cdl.CDL_PAIR_PANEL_LOG2(panel_log2)
    if resident is not None:
        f |= cdl.CDL_CHAIN_HOST_LEVELS | cdl.CDL_CHAIN_RESIDENT(resident)
    return f


@pytest.mark.parametrize("n,panel_log2,resident", [(1500, 8, None), (1500, 9, 3), (700, 8, 1)])
def test_regen_pair_matches_oracle_and_stored_pair(G, n, panel_log2, resident):
    cdl = G.cdl
    wl = iid_pair(n, 40, 6, seed=n + 3)
    k, d, seed, topk = 32, 8, 4, 10
    Fr, tr, r1, r2 = G.pair(wl.X[0], wl.X[1], k, d, cdl.CDL_BF16, cdl.CDL_BF16, seed, topk, max_iter=40,
                            rel_tol=1e-11, chain_flags=_regen_flags(cdl, panel_log2, resident))
    Fs, ts, s1, s2 = G.pair(wl.X[0], wl.X[1], k, d, cdl.CDL_BF16, cdl.CDL_BF16, seed, topk, max_iter=40,
                            rel_tol=1e-11)
    assert r1.rel_res <= 1e-11 and r2.rel_res <= 1e-11
    # the same graphs (exact distances and sigma, the same exponential): the
    # embeddings agree to the refinement tolerance, the scores far below 1e-6
    assert np.max(np.abs(Fr - Fs) / Fs) <= 1e-8
    out = O.caddelag_pair(wl.X[0], wl.X[1], k, seed, topk)
    rel = np.abs(Fr - out["F"]) / out["F"]
    assert rel.max() <= 1e-6, rel.max()
    if O.min_relative_gap(out["F"], topk) > 1e-5:
        assert list(tr) == list(out["top"])
    assert len(set(tr.tolist()) & set(wl.planted[0].tolist())) >= 5


def test_regen_pair_k192_field_graph(G):
    """k = 192 (two column blocks in the solve, K = 384 score Gram) on a small
    field pair with a planted patch; n = 1100 leaves a last panel narrower
    than the others (npad - r0 < P)."""
    cdl = G.cdl
    wl = field_sequence(20, 55, 48, 2, patch=4, patch_transition=0, seed=9)
    k, d, seed, topk = 192, 8, 6, 16
    Fr, tr, r1, r2 = G.pair(wl.X[0], wl.X[1], k, d, cdl.CDL_BF16, cdl.CDL_BF16, seed, topk, max_iter=40,
                            rel_tol=1e-11, chain_flags=_regen_flags(cdl, 9, 2))
    assert r1.rel_res <= 1e-11 and r2.rel_res <= 1e-11
    out = O.caddelag_pair(wl.X[0], wl.X[1], k, seed, topk)
    rel = np.abs(Fr - out["F"]) / out["F"]
    assert rel.max() <= 1e-6, rel.max()
    if O.min_relative_gap(out["F"], topk) > 1e-5:
        assert list(tr) == list(out["top"])
    assert len(set(tr.tolist()) & set(wl.planted[0].tolist())) >= 12


def test_regen_pair_host_io(G):
    cdl = G.cdl
    wl = iid_pair(600, 24, 3, seed=8)
    a = G.pair(wl.X[0], wl.X[1], 16, 6, cdl.CDL_BF16, cdl.CDL_BF16, 2, 5, chain_flags=_regen_flags(cdl, 8))
    b = G.pair(wl.X[0], wl.X[1], 16, 6, cdl.CDL_BF16, cdl.CDL_BF16, 2, 5, host_io=True,
               chain_flags=_regen_flags(cdl, 8))
    assert np.array_equal(a[0], b[0]) and list(a[1]) == list(b[1])


def test_regen_pair_refuses_what_it_cannot_do(G):
    cdl = G.cdl
    wl = iid_pair(300, 16, 2, seed=3)
    Xoff = wl.X[0] + 1e-9                                  # off the 2^-16 grid
    n, T = Xoff.shape
    from gpu_util import dev
    opts = cdl.cdl_pair_opts(8, 4, cdl.CDL_BF16, cdl.CDL_BF16, 1, 0.0, cdl.cdl_solve_opts(10, 1e-10, 0), 3, 0,
                             _regen_flags(cdl, 8))
    F = torch.empty(n, dtype=torch.float64, device="cuda")
    top = torch.empty(3, dtype=torch.int64, device="cuda")
    s1, s2 = cdl.cdl_solve_stats(), cdl.cdl_solve_stats()
    assert cdl.cdl_caddelag_pair(G.h, dev(Xoff), dev(wl.X[1]), n, T, opts, F, top, s1, s2) == \
        cdl.CDL_ERR_UNSUPPORTED
    bad = cdl.cdl_pair_opts(8, 4, cdl.CDL_F32, cdl.CDL_F32, 1, 0.0, cdl.cdl_solve_opts(10, 1e-10, 0), 3, 0,
                            _regen_flags(cdl, 8))
    assert cdl.cdl_caddelag_pair(G.h, dev(wl.X[0]), dev(wl.X[1]), n, T, bad, F, top, s1, s2) == \
        cdl.CDL_ERR_UNSUPPORTED
    assert cdl.cdl_sync(G.h) == 0


@pytest.mark.parametrize("resident", [1, 3, 8])
def test_partly_resident_levels_equal_device_levels(G, resident):
    cdl = G.cdl
    n, d = 1500, 8
    wl = iid_pair(n, 32, 4, seed=22)
    A, D, vol, _ = G.graph(wl.X[0])
    dev = G.chain(A, D, vol, d, cdl.CDL_BF16)
    mixed = G.chain(A, D, vol, d, cdl.CDL_BF16, flags=cdl.CDL_CHAIN_HOST_LEVELS | cdl.CDL_CHAIN_RESIDENT(resident))
    try:
        for i in range(d):
            ref = G.level(dev, i, "bf16").double().cpu().numpy()
            got = G.level(mixed, i, "bf16").double().cpu().numpy() if i < resident else G.host_level(mixed, i)
            np.testing.assert_array_equal(got, ref)
        Y = G.project(A, 32, 5)
        Zd, sd = G.solve(dev, A, Y, max_iter=20, rel_tol=1e-11)
        Zm, sm = G.solve(mixed, A, Y, max_iter=20, rel_tol=1e-11)
        assert torch.equal(Zd, Zm) and sd.iters == sm.iters
    finally:
        cdl.cdl_chain_free(dev)
        cdl.cdl_chain_free(mixed)
