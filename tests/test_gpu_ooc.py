"""Chain levels in pinned host memory (the larger-than-memory form): the
levels streamed through two device slots equal the device-resident ones bit
for bit, so do the solve and the whole pair, and the pair still matches the
float64 oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import caddelag as O           # noqa: E402
from workloads import iid_pair              # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from gpu_util import Ctx, lib
    c = Ctx(lib())
    yield c
    c.close()


@pytest.mark.parametrize("n,d", [(1500, 8), (700, 3), (300, 1)])
def test_host_levels_equal_device_levels(G, n, d):
    cdl = G.cdl
    wl = iid_pair(n, 32, 4, seed=21)
    A, D, vol, _ = G.graph(wl.X[0])
    dev = G.chain(A, D, vol, d, cdl.CDL_BF16)
    host = G.chain(A, D, vol, d, cdl.CDL_BF16, flags=cdl.CDL_CHAIN_HOST_LEVELS)
    try:
        for i in range(d):
            np.testing.assert_array_equal(G.host_level(host, i), G.level(dev, i, "bf16").double().cpu().numpy())
        Y = G.project(A, 32, 5)
        Zd, sd = G.solve(dev, A, Y, max_iter=20, rel_tol=1e-11)
        Zh, sh = G.solve(host, A, Y, max_iter=20, rel_tol=1e-11)
        assert torch.equal(Zd, Zh)
        assert sd.iters == sh.iters and sd.rel_res == sh.rel_res
        # rebuilding the host chain for another graph reuses its storage
        A2, D2, vol2, _ = G.graph(wl.X[1])
        host2 = G.chain(A2, D2, vol2, d, cdl.CDL_BF16, chain=host, flags=cdl.CDL_CHAIN_HOST_LEVELS)
        dev2 = G.chain(A2, D2, vol2, d, cdl.CDL_BF16, chain=dev)
        assert host2.value == host.value
        np.testing.assert_array_equal(G.host_level(host2, d - 1), G.level(dev2, d - 1, "bf16").double().cpu().numpy())
    finally:
        cdl.cdl_chain_free(dev)
        cdl.cdl_chain_free(host)


def test_host_levels_pair_matches_oracle(G):
    cdl = G.cdl
    wl = iid_pair(1024, 64, 10, 0)
    out = O.caddelag_pair(wl.X[0], wl.X[1], k=32, seed=0, topk=10)
    Fh, th, s1, s2 = G.pair(wl.X[0], wl.X[1], 32, 8, cdl.CDL_BF16, cdl.CDL_F32, 0, 10,
                            chain_flags=cdl.CDL_CHAIN_HOST_LEVELS)
    Fd, td, _, _ = G.pair(wl.X[0], wl.X[1], 32, 8, cdl.CDL_BF16, cdl.CDL_F32, 0, 10)
    assert np.array_equal(Fh, Fd) and list(th) == list(td)
    rel = np.abs(Fh - out["F"]) / out["F"]
    assert rel.max() <= 1e-6
    assert list(th) == list(out["top"])


def test_host_levels_need_bf16(G):
    cdl = G.cdl
    wl = iid_pair(300, 16, 2, seed=3)
    A, D, vol, _ = G.graph(wl.X[0])
    for dt in (cdl.CDL_F32, cdl.CDL_F64, cdl.CDL_FP8E4M3):
        st, ch = cdl.cdl_chain_build(G.h, A, cdl.CDL_F64, D, vol.data_ptr(), 300, 4, dt,
                                     cdl.CDL_CHAIN_HOST_LEVELS, None)
        assert st == cdl.CDL_ERR_UNSUPPORTED and not ch
    st, ch = cdl.cdl_chain_build(G.h, A, cdl.CDL_F64, D, vol.data_ptr(), 300, 4, cdl.CDL_BF16, 4, None)
    assert st == cdl.CDL_ERR_INVALID_ARG


def test_host_link_copy_timing(G):
    """Host-link copies are timed as their own class (CDL_KC_HOST_LINK): one
    copy out per level while the chain is built, loads while it is applied,
    every copy one level of bytes, and none of them counted as a kernel
    launch (the build issues the same kernels as with device levels)."""
    cdl = G.cdl
    n, d = 700, 3
    npad = (n + 255) // 256 * 256
    lb = npad * npad * 2
    wl = iid_pair(n, 32, 4, seed=22)
    A, D, vol, _ = G.graph(wl.X[0])
    cdl.cdl_ctx_set_timing(G.h, 1)
    try:
        cdl.cdl_ctx_reset_counters(G.h)
        dev = G.chain(A, D, vol, d, cdl.CDL_BF16)
        _, dev_launches = cdl.cdl_ctx_launch_count(G.h)
        _, _, dev_copies, _ = cdl.cdl_ctx_timing(G.h, cdl.CDL_KC_HOST_LINK)
        assert dev_copies == 0
        cdl.cdl_ctx_reset_counters(G.h)
        host = G.chain(A, D, vol, d, cdl.CDL_BF16, flags=cdl.CDL_CHAIN_HOST_LEVELS)
        _, host_launches = cdl.cdl_ctx_launch_count(G.h)
        st, ms, copies, work = cdl.cdl_ctx_timing(G.h, cdl.CDL_KC_HOST_LINK)
        assert st == 0 and host_launches == dev_launches
        assert copies == d and work == d * lb and ms > 0
        Y = G.project(A, 32, 5)
        cdl.cdl_ctx_reset_counters(G.h)
        _, s = G.solve(host, A, Y, max_iter=2, rel_tol=0.0)
        st, ms, copies, work = cdl.cdl_ctx_timing(G.h, cdl.CDL_KC_HOST_LINK)
        assert st == 0 and s.iters == 2
        # each application reads the d levels (two of them may still sit in the slots)
        assert 2 * d - 2 <= copies <= 2 * d + 1 and work == copies * lb and ms > 0
    finally:
        cdl.cdl_ctx_set_timing(G.h, 0)
        cdl.cdl_chain_free(dev)
        cdl.cdl_chain_free(host)
