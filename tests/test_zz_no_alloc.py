"""cdl_build_graph_static: the graph build for callers that cannot let a
library allocate device memory (for example when all device memory belongs
to the caller's own pool allocator). It must give the same results as
cdl_build_graph while using only the library's static scratch array, on
consecutive calls that reuse that array with different inputs."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from workloads import iid_pair, field_sequence   # noqa: E402

pytestmark = pytest.mark.gpu


def _outputs(n):
    A = torch.empty((n, n), dtype=torch.float64, device="cuda")
    D = torch.empty(n, dtype=torch.float64, device="cuda")
    s = torch.zeros(2, dtype=torch.float64, device="cuda")
    return A, D, s


def test_static_graph_build_matches_allocating_entry_point():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from gpu_util import lib
    cdl = lib()
    stream = torch.cuda.current_stream()
    st, ctx = cdl.cdl_ctx_create(0, stream.cuda_stream, 0)
    assert st == 0
    try:
        rng = np.random.default_rng(34)
        wide = np.rint(rng.uniform(-127.0, 127.0, (1500, 300)) * 65536.0) / 65536.0   # large grid values
        inputs = [iid_pair(1000, 64, 3, seed=31).X[1],             # exact integer distances
                  field_sequence(16, 48, 100, 2, seed=32).X[1],     # second call, other sizes
                  np.random.default_rng(33).standard_normal((700, 9)) + 1e-7,   # off-grid path
                  iid_pair(4000, 200, 3, seed=35).X[0],             # many tiles, ragged n and T
                  wide,                                             # all three digits in use
                  iid_pair(130, 1, 1, seed=36).X[0]]                # T = 1
        for X in inputs:
            n, T = X.shape
            Xd = torch.from_numpy(X).cuda()
            A0, D0, s0 = _outputs(n)
            assert cdl.cdl_build_graph(ctx, Xd, n, T, 0.0, cdl.CDL_F64, A0, D0, s0[0:1].data_ptr(),
                                       s0[1:2].data_ptr()) == 0
            A1, D1, s1 = _outputs(n)
            assert cdl.cdl_build_graph_static(Xd, n, T, 0.0, A1, D1, s1[0:1].data_ptr(), s1[1:2].data_ptr(),
                                              stream.cuda_stream) == 0
            torch.cuda.synchronize()
            # the allocating entry point forms distances on the tensor cores and the
            # kernel values tile by tile (half the exponentials, degrees from tile
            # sums), the static one distances in int64 and values row by row: the
            # distances and values are exact or the same arithmetic, the degree sums
            # differ in order only
            assert torch.equal(s0[1:2], s1[1:2])             # sigma
            assert torch.equal(A0, A1)
            assert torch.allclose(s0[0:1], s1[0:1], rtol=1e-13, atol=0)   # vol
            assert torch.allclose(D0, D1, rtol=1e-13, atol=0)
    finally:
        cdl.cdl_ctx_destroy(ctx)


def test_static_graph_build_rejects_oversized_input():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from gpu_util import lib
    cdl = lib()
    n, T = 8192, 256                      # n * T = 2^21 > 2^20
    X = torch.zeros((n, T), dtype=torch.float64, device="cuda")
    A = torch.empty((1, 1), dtype=torch.float64, device="cuda")
    s = torch.zeros(2, dtype=torch.float64, device="cuda")
    assert cdl.cdl_build_graph_static(X, n, T, 0.0, A, s, s[0:1].data_ptr(), s[1:2].data_ptr(), None) == \
        cdl.CDL_ERR_INVALID_ARG


def _cudart():
    import ctypes
    import glob
    import os
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    for cand in ["libcudart.so"] + sorted(glob.glob(os.path.join(home, "lib64", "libcudart.so*"))) + \
            sorted(glob.glob(os.path.join(home, "targets", "*", "lib", "libcudart.so*"))):
        try:
            return ctypes.CDLL(cand)
        except OSError:
            continue
    pytest.skip("libcudart not found")


def test_static_graph_build_accepts_managed_memory():
    """Inputs and outputs in managed memory (cudaMallocManaged, made by the
    caller) give the same results as device memory, as for the entry points
    that take a context."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import ctypes
    from gpu_util import lib
    cdl = lib()
    rt = _cudart()
    X = iid_pair(500, 24, 2, seed=37).X[0]
    n, T = X.shape
    stream = torch.cuda.current_stream()
    Xd = torch.from_numpy(X).cuda()
    A0, D0, s0 = _outputs(n)
    assert cdl.cdl_build_graph_static(Xd, n, T, 0.0, A0, D0, s0[0:1].data_ptr(), s0[1:2].data_ptr(),
                                      stream.cuda_stream) == 0
    torch.cuda.synchronize()
    sizes = {"X": n * T * 8, "A": n * n * 8, "D": n * 8, "s": 2 * 8}
    ptr = {}
    try:
        for k, b in sizes.items():
            p = ctypes.c_void_p()
            assert rt.cudaMallocManaged(ctypes.byref(p), ctypes.c_size_t(b), ctypes.c_uint(1)) == 0
            ptr[k] = p.value
        assert rt.cudaDeviceSynchronize() == 0
        ctypes.memmove(ptr["X"], X.ctypes.data, sizes["X"])
        assert cdl.cdl_build_graph_static(ptr["X"], n, T, 0.0, ptr["A"], ptr["D"], ptr["s"], ptr["s"] + 8,
                                          stream.cuda_stream) == 0
        torch.cuda.synchronize()
        assert rt.cudaDeviceSynchronize() == 0

        def view(k, count):
            return np.ctypeslib.as_array(ctypes.cast(ptr[k], ctypes.POINTER(ctypes.c_double)), (count,)).copy()
        assert np.array_equal(view("A", n * n).reshape(n, n), A0.cpu().numpy())
        assert np.array_equal(view("D", n), D0.cpu().numpy())
        assert np.array_equal(view("s", 2), s0.cpu().numpy())
    finally:
        for p in ptr.values():
            rt.cudaFree(ctypes.c_void_p(p))
