"""Opt-in chain truncation: squaring stops once a level's max row sum is at
most 2^-24 (it and every later level cannot change a float32 x + S~ x). The
kept levels equal the full chain's, the refinement reaches the same
tolerance and the scores match the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import caddelag as O                 # noqa: E402
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


@pytest.mark.parametrize("dtype", ["bf16", "f32", "fp8t"])
def test_truncated_chain_keeps_levels_and_solves(G, dtype):
    cdl = G.cdl
    dt = {"bf16": cdl.CDL_BF16, "f32": cdl.CDL_F32, "fp8t": cdl.CDL_FP8E4M3_T128}[dtype]
    view = {"bf16": "bf16", "f32": np.float32, "fp8t": "fp8t"}[dtype]
    wl = iid_pair(1024, 64, 10, 0)
    A, D, vol, _ = G.graph(wl.X[0])
    full = G.chain(A, D, vol, 10, dt)
    trunc = G.chain(A, D, vol, 10, dt, flags=cdl.CDL_CHAIN_TRUNCATE)
    try:
        st, d_eff = cdl.cdl_chain_depth(trunc)
        assert st == 0 and 1 <= d_eff < 10
        st, d_full = cdl.cdl_chain_depth(full)
        assert d_full == 10
        for i in range(d_eff):
            assert np.array_equal(G.level_values(trunc, i, view), G.level_values(full, i, view))
        # the first level not kept is below the bound in the full chain
        Lnext = G.level_values(full, d_eff, view)
        assert np.abs(Lnext).sum(axis=1).max() <= 2.0 ** -24 * (1 + 1e-3)
        st, _, _ = cdl.cdl_chain_level(trunc, d_eff)
        assert st == cdl.CDL_ERR_INVALID_ARG
        Y = G.project(A, 32, 0)
        Zf, sf = G.solve(full, A, Y, max_iter=30, rel_tol=1e-11)
        Zt, stt = G.solve(trunc, A, Y, max_iter=30, rel_tol=1e-11)
        assert stt.rel_res <= 1e-11 and stt.iters <= sf.iters + 1
        assert torch.norm(Zt - Zf) <= 1e-9 * torch.norm(Zf)
    finally:
        cdl.cdl_chain_free(full)
        cdl.cdl_chain_free(trunc)


def test_truncated_pair_matches_oracle(G):
    cdl = G.cdl
    wl = field_sequence(32, 64, 64, 2, patch=4, patch_transition=0, seed=5)
    out = O.caddelag_pair(wl.X[0], wl.X[1], k=32, seed=1, topk=16)
    F, top, s1, s2 = G.pair(wl.X[0], wl.X[1], 32, 10, cdl.CDL_BF16, cdl.CDL_F32, 1, 16,
                            chain_flags=cdl.CDL_CHAIN_TRUNCATE)
    assert s1.rel_res <= 1e-10 and s2.rel_res <= 1e-10
    rel = np.abs(F - out["F"]) / out["F"]
    assert rel.max() <= 1e-6, rel.max()
    assert len(set(top.tolist()) & set(wl.planted[0].tolist())) >= 12


def test_truncate_with_host_levels_is_refused(G):
    cdl = G.cdl
    wl = iid_pair(300, 16, 2, seed=3)
    A, D, vol, _ = G.graph(wl.X[0])
    st, ch = cdl.cdl_chain_build(G.h, A, cdl.CDL_F64, D, vol.data_ptr(), 300, 4, cdl.CDL_BF16,
                                 cdl.CDL_CHAIN_TRUNCATE | cdl.CDL_CHAIN_HOST_LEVELS, None)
    assert st == cdl.CDL_ERR_UNSUPPORTED and not ch
