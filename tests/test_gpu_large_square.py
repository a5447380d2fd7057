"""The bf16 chain squaring with K pacing (orders from 65536 on: every CTA's
producer waits until all CTAs have reached the k-block step two steps
behind its own, so CTAs sharing row panels read them from L2): one
squaring at n = 65536 against a float64 product of the same bf16 input on
sampled rows, with the error bound of the small-size exact-product test
(float32 accumulation, then one bf16 rounding), and the sampled rows equal
to the sampled columns (the symmetric output is written once per pair of
blocks and mirrored)."""
import gc

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from workloads import iid_pair     # noqa: E402

pytestmark = [pytest.mark.gpu, pytest.mark.fullsize]


def test_paced_square_n65536_matches_product_of_its_input():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from gpu_util import Ctx, lib
    gc.collect()
    torch.cuda.empty_cache()
    G = Ctx(lib())
    cdl = G.cdl
    n = 65536
    X = iid_pair(n, 16, 1, seed=13).X[0]
    ch = None
    try:
        A, D, vol, _ = G.graph(X)
        ch = G.chain(A, D, vol, 2, cdl.CDL_BF16)
        del A
        torch.cuda.empty_cache()
        L0 = G.level(ch, 0, "bf16")
        L1 = G.level(ch, 1, "bf16")
        npad = L0.shape[0]
        rng = np.random.default_rng(5)
        rows = np.unique(np.concatenate([rng.choice(n, 12, replace=False), [0, 127, 128, n - 1]]))
        ridx = torch.from_numpy(rows).cuda()
        Lr = L0[ridx].double()                        # sampled rows, exact bf16 values
        R = torch.empty((len(rows), npad), dtype=torch.float64, device="cuda")
        Ra = torch.empty_like(R)
        for c0 in range(0, npad, 8192):               # float64 products by column blocks
            Lc = L0[:, c0:c0 + 8192].double()
            R[:, c0:c0 + 8192] = Lr @ Lc
            Ra[:, c0:c0 + 8192] = Lr.abs() @ Lc.abs()
            del Lc
        got = L1[ridx].double()
        cols = L1[:, ridx].double().T
        # level 0 has negative entries (the deflated first eigenvector), so
        # the float32 accumulation bound uses |L0| |L0|
        bound = 2.0 ** -8 * R.abs() + npad * 2.0 ** -23 * Ra + 1e-30
        bad = int(((got - R).abs() > bound).sum().item())
        mirrored = bool(torch.equal(got, cols))
        nz = int((got != 0).sum().item())
    finally:
        if ch is not None:
            cdl.cdl_chain_free(ch)
        G.close()
        torch.cuda.empty_cache()
    assert bad == 0
    assert mirrored
    assert nz > 0
