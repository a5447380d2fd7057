"""Helpers for the GPU tests: device buffers via torch, calls via the C ABI."""
import numpy as np

import torch


def lib():
    from paper_1802_05421_gb300 import build
    build.build()
    from paper_1802_05421_gb300 import cdl
    return cdl


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


class _CAI:
    """Zero-copy view of library-owned device memory (e.g. a chain level)."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = dict(shape=shape, typestr=typestr, data=(ptr, False),
                                             version=3, strides=None)


def view_device(ptr, shape, dtype):
    if dtype == "bf16":
        return torch.as_tensor(_CAI(ptr, shape, "<i2"), device="cuda").view(torch.bfloat16)
    if dtype == "fp8":
        return torch.as_tensor(_CAI(ptr, shape, "|u1"), device="cuda").view(torch.float8_e4m3fn)
    return torch.as_tensor(_CAI(ptr, shape, np.dtype(dtype).str), device="cuda")


class Ctx:
    def __init__(self, cdl):
        self.cdl = cdl
        st, self.h = cdl.cdl_ctx_create(0, torch.cuda.current_stream().cuda_stream, 0)
        assert st == 0, cdl.cdl_status_string(st)

    def close(self):
        self.cdl.cdl_ctx_destroy(self.h)

    def check(self, st):
        assert st == 0, (self.cdl.cdl_status_string(st), self.cdl.cdl_last_error_detail())

    def graph(self, X, sigma=0.0):
        cdl = self.cdl
        n, T = X.shape
        Xd = dev(X)
        A = torch.empty((n, n), dtype=torch.float64, device="cuda")
        D = torch.empty(n, dtype=torch.float64, device="cuda")
        sc = torch.zeros(2, dtype=torch.float64, device="cuda")
        self.check(cdl.cdl_build_graph(self.h, Xd, n, T, sigma, cdl.CDL_F64, A, D, sc[0:1].data_ptr(),
                                       sc[1:2].data_ptr()))
        self.check(cdl.cdl_sync(self.h))
        return A, D, sc[0:1], sc[1:2]

    def project(self, A, k, seed):
        n = A.shape[0]
        Y = torch.empty((n, k), dtype=torch.float64, device="cuda")
        self.check(self.cdl.cdl_project(self.h, A, self.cdl.CDL_F64, n, k, seed, Y))
        self.check(self.cdl.cdl_sync(self.h))
        return Y

    def chain(self, A, D, vol, d, dtype, chain=None, flags=0):
        n = A.shape[0]
        st, ch = self.cdl.cdl_chain_build(self.h, A, self.cdl.CDL_F64, D, vol.data_ptr(), n, d, dtype,
                                          flags, chain)
        self.check(st)
        self.check(self.cdl.cdl_sync(self.h))
        return ch

    def level(self, ch, i, dtype):
        st, ptr, npad = self.cdl.cdl_chain_level(ch, i)
        self.check(st)
        return view_device(ptr, (npad, npad), dtype)

    def host_level(self, ch, i):
        """Level i of a chain with host levels, as a bf16-valued float64 array."""
        import ctypes
        st, ptr, npad = self.cdl.cdl_chain_level(ch, i)
        self.check(st)
        raw = np.ctypeslib.as_array((ctypes.c_uint16 * (npad * npad)).from_address(ptr)).copy()
        return (raw.astype(np.uint32) << 16).view(np.float32).astype(np.float64).reshape(npad, npad)

    def level16(self, ch, i):
        """bf16 view of level i read by the apply, as float64 on the host."""
        st, ptr = self.cdl.cdl_chain_apply_level(ch, i)
        self.check(st)
        st, _, npad = self.cdl.cdl_chain_level(ch, i)
        return view_device(ptr, (npad, npad), "bf16").double().cpu().numpy()

    def level_values(self, ch, i, dtype):
        """Level i as float64 values on the host (fp8 levels times their
        scale; "fp8t" levels times their 128 x 128 tile scales)."""
        if dtype == "fp8t":
            v = self.level(ch, i, "fp8").double().cpu().numpy()
            st, ptr, nt = self.cdl.cdl_chain_tile_scales(ch, i)
            self.check(st)
            sc = view_device(ptr, (nt, nt), np.float32).double().cpu().numpy()
            return v * np.kron(sc, np.ones((128, 128)))
        v = self.level(ch, i, dtype).double().cpu().numpy()
        st, sc = self.cdl.cdl_chain_level_scale(ch, i)
        self.check(st)
        return v * sc

    def tile_scales(self, ch, i):
        st, ptr, nt = self.cdl.cdl_chain_tile_scales(ch, i)
        self.check(st)
        return view_device(ptr, (nt, nt), np.float32).double().cpu().numpy()

    def solve(self, ch, A, Y, max_iter=20, rel_tol=1e-10, expect=0, flags=0):
        cdl = self.cdl
        n, k = Y.shape
        Z = torch.empty((n, k), dtype=torch.float64, device="cuda")
        opts = cdl.cdl_solve_opts(max_iter, rel_tol, flags)
        stats = cdl.cdl_solve_stats()
        st = cdl.cdl_chain_solve(self.h, ch, A, cdl.CDL_F64, Y, k, opts, Z, stats)
        assert st == expect, cdl.cdl_status_string(st)
        self.check(cdl.cdl_sync(self.h))
        return Z, stats

    def score(self, A1, A2, Z1, Z2, vol1, vol2, topk, score_dtype):
        cdl = self.cdl
        n, k = Z1.shape
        F = torch.empty(n, dtype=torch.float64, device="cuda")
        top = torch.empty(max(topk, 1), dtype=torch.int64, device="cuda")
        self.check(cdl.cdl_cad_score(self.h, A1, A2, cdl.CDL_F64, Z1, Z2, vol1.data_ptr(), vol2.data_ptr(),
                                     n, k, score_dtype, topk, F, top))
        self.check(cdl.cdl_sync(self.h))
        return F, top[:topk]

    def pair(self, X1, X2, k, d, chain_dtype, score_dtype, seed, topk, max_iter=30, rel_tol=1e-10,
             host_io=False, sigma=0.0, chain_flags=0):
        cdl = self.cdl
        n, T = X1.shape
        opts = cdl.cdl_pair_opts(k, d, chain_dtype, score_dtype, seed, sigma,
                                 cdl.cdl_solve_opts(max_iter, rel_tol, 0), topk, int(host_io), chain_flags)
        s1, s2 = cdl.cdl_solve_stats(), cdl.cdl_solve_stats()
        if host_io:
            F = np.empty(n)
            top = np.empty(max(topk, 1), dtype=np.int64)
            self.check(cdl.cdl_caddelag_pair(self.h, np.ascontiguousarray(X1), np.ascontiguousarray(X2), n, T,
                                             opts, F, top, s1, s2))
            return F, top[:topk], s1, s2
        F = torch.empty(n, dtype=torch.float64, device="cuda")
        top = torch.empty(max(topk, 1), dtype=torch.int64, device="cuda")
        self.check(cdl.cdl_caddelag_pair(self.h, dev(X1), dev(X2), n, T, opts, F, top, s1, s2))
        self.check(cdl.cdl_sync(self.h))
        return host(F), host(top)[:topk], s1, s2
