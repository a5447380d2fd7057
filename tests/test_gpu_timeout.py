"""Bounded device waits: a tensor-core squaring whose first tile load is
withheld (test hook) must give up after its wait limit, report
CDL_ERR_TIMEOUT through cdl_sync, and leave the context usable."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from workloads import iid_pair   # noqa: E402

pytestmark = pytest.mark.gpu


def test_withheld_tile_load_times_out_and_context_recovers():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from gpu_util import Ctx, lib
    G = Ctx(lib())
    cdl = G.cdl
    try:
        X = iid_pair(256, 16, 1, seed=3).X[0]
        A, D, vol, _ = G.graph(X)
        n = 256
        assert cdl.cdl_ctx_set_debug(G.h, cdl.CDL_DEBUG_WITHHOLD_TC_LOAD) == 0
        st, ch = cdl.cdl_chain_build(G.h, A, cdl.CDL_F64, D, vol.data_ptr(), n, 2, cdl.CDL_BF16)
        assert st == cdl.CDL_OK                         # the launch itself succeeds
        assert cdl.cdl_sync(G.h) == cdl.CDL_ERR_TIMEOUT  # the bounded wait expired
        assert cdl.cdl_sync(G.h) == cdl.CDL_OK           # the status word was cleared
        assert cdl.cdl_ctx_set_debug(G.h, 0) == 0
        ch = G.chain(A, D, vol, 2, cdl.CDL_BF16, chain=ch)
        try:
            L0 = G.level(ch, 0, "bf16").double().cpu().numpy()
            L1 = G.level(ch, 1, "bf16").double().cpu().numpy()
        finally:
            cdl.cdl_chain_free(ch)
        R = L0 @ L0
        bound = 2.0 ** -8 * np.abs(R) + L0.shape[0] * 2.0 ** -23 * (np.abs(L0) @ np.abs(L0)) + 1e-30
        assert np.all(np.abs(L1 - R) <= bound)
        assert cdl.cdl_ctx_set_debug(G.h, 99) == cdl.CDL_ERR_INVALID_ARG
    finally:
        G.close()
