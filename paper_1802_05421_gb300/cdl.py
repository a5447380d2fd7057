"""ctypes binding of libcdl (the C ABI declared in include/cdl.h).

Argument marshalling only: every function here forwards to the C entry point
of the same name and returns its integer status. Array arguments may be
given as integers (raw pointers), as objects with ``data_ptr()`` (torch
tensors) or ``ctypes.data`` (NumPy arrays), or as None (NULL). The library
must have been built (``python -m paper_1802_05421_gb300.build``); importing
this module without it raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcdl.so")

CDL_OK = 0
CDL_ERR_INVALID_ARG = -1
CDL_ERR_OOM = -2
CDL_ERR_CUDA = -3
CDL_ERR_NOT_CONVERGED = -4
CDL_ERR_TIMEOUT = -5
CDL_ERR_UNSUPPORTED = -6

CDL_F64, CDL_F32, CDL_BF16, CDL_FP8E4M3, CDL_FP8E4M3_T128 = 0, 1, 2, 3, 4
CDL_SOLVE_FULL_RESIDUAL = 1
CDL_CHAIN_DEFAULT = 0
CDL_CHAIN_HOST_LEVELS = 1
CDL_CHAIN_TRUNCATE = 2
CDL_CHAIN_RESIDENT_SHIFT, CDL_CHAIN_RESIDENT_MASK = 8, 0xFF00
CDL_PAIR_REGEN_GRAPHS = 4
CDL_PAIR_PANEL_SHIFT, CDL_PAIR_PANEL_MASK = 16, 0xFF0000


def CDL_CHAIN_RESIDENT(r):
    """Chain flag bits: keep levels 0 .. r - 1 in device memory (with CDL_CHAIN_HOST_LEVELS)."""
    return (int(r) << CDL_CHAIN_RESIDENT_SHIFT) & CDL_CHAIN_RESIDENT_MASK


def CDL_PAIR_PANEL_LOG2(p):
    """Pair flag bits: regenerated graphs in row panels of 2^p rows."""
    return (int(p) << CDL_PAIR_PANEL_SHIFT) & CDL_PAIR_PANEL_MASK
CDL_SCORE_CHANGED_ONLY = 1
CDL_KERNEL_GAUSSIAN, CDL_KERNEL_EXP = 0, 1
CDL_DEBUG_WITHHOLD_TC_LOAD = 1
CDL_DEBUG_BATCH_VARIANT = 2

(CDL_KC_DISTANCE, CDL_KC_SELECT, CDL_KC_KERNEL, CDL_KC_CHAIN_INIT, CDL_KC_SQUARE, CDL_KC_APPLY,
 CDL_KC_RESIDUAL, CDL_KC_PROJECT, CDL_KC_SCORE, CDL_KC_TOPK, CDL_KC_MISC, CDL_KC_HOST_LINK, CDL_KC_COUNT) = range(13)
KERNEL_CLASSES = ["distance", "select", "kernel", "chain_init", "square", "apply", "residual",
                  "project", "score", "topk", "misc"]


class cdl_solve_opts(ctypes.Structure):
    _fields_ = [("max_iter", ctypes.c_int32), ("rel_tol", ctypes.c_double), ("flags", ctypes.c_int32)]


class cdl_solve_stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("rel_res", ctypes.c_double),
                ("history", ctypes.c_double * 64)]


class cdl_pair_opts(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("d", ctypes.c_int32), ("chain_dtype", ctypes.c_int),
                ("score_dtype", ctypes.c_int), ("seed", ctypes.c_uint64), ("sigma", ctypes.c_double), ("solve", cdl_solve_opts),
                ("topk", ctypes.c_int32), ("host_io", ctypes.c_int32), ("chain_flags", ctypes.c_int32),
                ("score_flags", ctypes.c_int32)]


class cdl_batch_opts(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("d", ctypes.c_int32), ("chain_dtype", ctypes.c_int),
                ("score_dtype", ctypes.c_int), ("seed", ctypes.c_uint64), ("sigma", ctypes.c_double),
                ("solve", cdl_solve_opts), ("topk", ctypes.c_int32), ("host_io", ctypes.c_int32),
                ("use_graph", ctypes.c_int32)]


class cdl_batch_info(ctypes.Structure):
    _fields_ = [("ready", ctypes.c_int32), ("square_max_npad_128", ctypes.c_int32),
                ("project_rows_per_block", ctypes.c_int32), ("residual_tile_m", ctypes.c_int32),
                ("residual_tile_n", ctypes.c_int32), ("slots_captured", ctypes.c_int32),
                ("slots_seen", ctypes.c_int32), ("n_square_variants", ctypes.c_int32),
                ("n_project_variants", ctypes.c_int32), ("square_variant_max_npad_128", ctypes.c_int32 * 8),
                ("square_variant_ms", ctypes.c_double * 8), ("project_variant_rows", ctypes.c_int32 * 8),
                ("project_variant_ms", ctypes.c_double * 8), ("device_bytes", ctypes.c_uint64)]


class cdl_edge_result(ctypes.Structure):
    _fields_ = [("n_edges", ctypes.c_int64), ("n_ties_taken", ctypes.c_int64), ("threshold", ctypes.c_double),
                ("remaining", ctypes.c_double), ("total", ctypes.c_double)]


if not os.path.exists(LIB_PATH):
    raise ImportError(f"libcdl.so not built at {LIB_PATH}; run python -m paper_1802_05421_gb300.build")
_lib = ctypes.CDLL(LIB_PATH)

_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32
_D = ctypes.c_double
_SIGS = {
    "cdl_ctx_create": [ctypes.POINTER(_P), ctypes.c_int, _P, ctypes.c_size_t],
    "cdl_ctx_destroy": [_P],
    "cdl_sync": [_P],
    "cdl_ctx_set_timing": [_P, ctypes.c_int],
    "cdl_ctx_timing": [_P, ctypes.c_int, ctypes.POINTER(_D), ctypes.POINTER(_I64), ctypes.POINTER(_D)],
    "cdl_ctx_reset_counters": [_P],
    "cdl_ctx_launch_count": [_P, ctypes.POINTER(_I64)],
    "cdl_ctx_set_debug": [_P, ctypes.c_int],
    "cdl_build_graph": [_P, _P, _I64, _I32, _D, ctypes.c_int, _P, _P, _P, _P],
    "cdl_build_graph_static": [_P, _I64, _I32, _D, _P, _P, _P, _P, _P],
    "cdl_build_graph_kernel": [_P, _P, _I64, _I32, _I32, _D, ctypes.c_int, _P, _P, _P, _P],
    "cdl_graph_degrees": [_P, _P, ctypes.c_int, _I64, _P, _P],
    "cdl_graph_add_edges": [_P, _P, ctypes.c_int, _I64, _I64, _P, _P, ctypes.POINTER(_I64)],
    "cdl_chain_build": [_P, _P, ctypes.c_int, _P, _P, _I64, _I32, ctypes.c_int, _I32, ctypes.POINTER(_P)],
    "cdl_chain_free": [_P],
    "cdl_chain_depth": [_P, ctypes.POINTER(_I32)],
    "cdl_chain_level": [_P, _I32, ctypes.POINTER(_P), ctypes.POINTER(_I64)],
    "cdl_chain_level_scale": [_P, _I32, ctypes.POINTER(_D)],
    "cdl_chain_apply_level": [_P, _I32, ctypes.POINTER(_P)],
    "cdl_chain_tile_scales": [_P, _I32, ctypes.POINTER(_P), ctypes.POINTER(_I64)],
    "cdl_project": [_P, _P, ctypes.c_int, _I64, _I32, ctypes.c_uint64, _P],
    "cdl_chain_solve": [_P, _P, _P, ctypes.c_int, _P, _I32, ctypes.POINTER(cdl_solve_opts), _P,
                        ctypes.POINTER(cdl_solve_stats)],
    "cdl_cad_score": [_P, _P, _P, ctypes.c_int, _P, _P, _P, _P, _I64, _I32, ctypes.c_int, _I32, _P, _P],
    "cdl_cad_edges": [_P, _P, _P, ctypes.c_int, _P, _P, _P, _P, _I64, _I32, ctypes.c_int, _D, _I64, _P, _P, _P, _I32,
                      _I32, _P, _P, _P, ctypes.POINTER(cdl_edge_result)],
    "cdl_changed_nodes": [_P, _P, _P, _I64, _I32, _P, ctypes.POINTER(_I32)],
    "cdl_cad_score_changed": [_P, _P, _P, ctypes.c_int, _P, _P, _P, _P, _I64, _I32, ctypes.c_int, _P, _I32, _I32,
                              _P, _P],
    "cdl_pair_embeddings": [_P, _P, _P, _P],
    "cdl_caddelag_pair": [_P, _P, _P, _I64, _I32, ctypes.POINTER(cdl_pair_opts), _P, _P,
                          ctypes.POINTER(cdl_solve_stats), ctypes.POINTER(cdl_solve_stats)],
    "cdl_caddelag_batched": [_P, _I32, _P, _I32, _P, _P, ctypes.POINTER(cdl_batch_opts), _P, _P, _P],
    "cdl_batch_plan_info": [_P, ctypes.POINTER(cdl_batch_info)],
}
for _name, _args in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = ctypes.c_int
_lib.cdl_status_string.argtypes = [ctypes.c_int]
_lib.cdl_status_string.restype = ctypes.c_char_p
_lib.cdl_last_error_detail.argtypes = []
_lib.cdl_last_error_detail.restype = ctypes.c_char_p


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    if isinstance(x, ctypes.c_void_p):
        return x.value
    raise TypeError(f"cannot pass {type(x)} as a pointer")


def cdl_status_string(status: int) -> str:
    return _lib.cdl_status_string(status).decode()


def cdl_last_error_detail() -> str:
    return _lib.cdl_last_error_detail().decode()


def cdl_ctx_create(device: int = 0, stream=None, ws_cap_bytes: int = 0):
    """Returns (status, ctx handle)."""
    h = _P()
    st = _lib.cdl_ctx_create(ctypes.byref(h), device, _ptr(stream), ws_cap_bytes)
    return st, h


def cdl_ctx_destroy(ctx) -> int:
    return _lib.cdl_ctx_destroy(ctx)


def cdl_sync(ctx) -> int:
    return _lib.cdl_sync(ctx)


def cdl_ctx_set_timing(ctx, enable: bool) -> int:
    return _lib.cdl_ctx_set_timing(ctx, int(enable))


def cdl_ctx_timing(ctx, kernel_class: int):
    """Returns (status, total_ms, launches, work)."""
    ms, n, w = _D(), _I64(), _D()
    st = _lib.cdl_ctx_timing(ctx, kernel_class, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(w))
    return st, ms.value, n.value, w.value


def cdl_ctx_reset_counters(ctx) -> int:
    return _lib.cdl_ctx_reset_counters(ctx)


def cdl_ctx_set_debug(ctx, flags: int) -> int:
    return _lib.cdl_ctx_set_debug(ctx, flags)


def cdl_ctx_launch_count(ctx):
    n = _I64()
    st = _lib.cdl_ctx_launch_count(ctx, ctypes.byref(n))
    return st, n.value


def cdl_build_graph(ctx, X, n, T, sigma, a_dtype, A, D, vol, sigma_out) -> int:
    return _lib.cdl_build_graph(ctx, _ptr(X), n, T, sigma, a_dtype, _ptr(A), _ptr(D), _ptr(vol),
                                _ptr(sigma_out))


def cdl_build_graph_kernel(ctx, X, n, T, kernel, sigma, a_dtype, A, D, vol, sigma_out) -> int:
    return _lib.cdl_build_graph_kernel(ctx, _ptr(X), n, T, kernel, sigma, a_dtype, _ptr(A), _ptr(D),
                                       _ptr(vol), _ptr(sigma_out))


def cdl_graph_degrees(ctx, A, a_dtype, n, D, vol) -> int:
    return _lib.cdl_graph_degrees(ctx, _ptr(A), a_dtype, n, _ptr(D), _ptr(vol))


def cdl_graph_add_edges(ctx, A, a_dtype, n, m, ij, w):
    """Returns (status, number of skipped invalid entries)."""
    bad = _I64(0)
    st = _lib.cdl_graph_add_edges(ctx, _ptr(A), a_dtype, n, m, _ptr(ij), _ptr(w), ctypes.byref(bad))
    return st, bad.value


def cdl_build_graph_static(X, n, T, sigma, A, D, vol, sigma_out, stream=None) -> int:
    return _lib.cdl_build_graph_static(_ptr(X), n, T, sigma, _ptr(A), _ptr(D), _ptr(vol), _ptr(sigma_out),
                                       _ptr(stream))


def cdl_chain_build(ctx, A, a_dtype, D, vol, n, d, chain_dtype, flags=0, chain=None):
    """Returns (status, chain handle). Pass ``chain`` to rebuild into it."""
    h = chain if chain is not None else _P()
    st = _lib.cdl_chain_build(ctx, _ptr(A), a_dtype, _ptr(D), _ptr(vol), n, d, chain_dtype, flags,
                              ctypes.byref(h))
    return st, h


def cdl_chain_depth(chain):
    """Returns (status, d_eff)."""
    d = _I32()
    st = _lib.cdl_chain_depth(chain, ctypes.byref(d))
    return st, d.value


def cdl_chain_free(chain) -> int:
    return _lib.cdl_chain_free(chain)


def cdl_chain_level(chain, i):
    """Returns (status, device pointer, npad)."""
    p, npad = _P(), _I64()
    st = _lib.cdl_chain_level(chain, i, ctypes.byref(p), ctypes.byref(npad))
    return st, p.value, npad.value


def cdl_chain_apply_level(chain, i):
    """Returns (status, device pointer of the bf16 apply view of level i)."""
    p = _P()
    st = _lib.cdl_chain_apply_level(chain, i, ctypes.byref(p))
    return st, p.value


def cdl_chain_tile_scales(chain, i):
    """Returns (status, device pointer to the nt x nt float32 tile scales, nt)."""
    p = _P()
    nt = _I64()
    st = _lib.cdl_chain_tile_scales(chain, i, ctypes.byref(p), ctypes.byref(nt))
    return st, p.value, nt.value


def cdl_chain_level_scale(chain, i):
    """Returns (status, scale of level i)."""
    sc = _D()
    st = _lib.cdl_chain_level_scale(chain, i, ctypes.byref(sc))
    return st, sc.value


def cdl_project(ctx, A, a_dtype, n, k, seed, Y) -> int:
    return _lib.cdl_project(ctx, _ptr(A), a_dtype, n, k, seed, _ptr(Y))


def cdl_chain_solve(ctx, chain, A, a_dtype, Y, k, opts: cdl_solve_opts, Z, stats=None) -> int:
    return _lib.cdl_chain_solve(ctx, chain, _ptr(A), a_dtype, _ptr(Y), k, ctypes.byref(opts), _ptr(Z),
                                ctypes.byref(stats) if stats is not None else None)


def cdl_cad_score(ctx, A1, A2, a_dtype, Z1, Z2, vol1, vol2, n, k, score_dtype, topk, F,
                  top_idx) -> int:
    return _lib.cdl_cad_score(ctx, _ptr(A1), _ptr(A2), a_dtype, _ptr(Z1), _ptr(Z2), _ptr(vol1),
                              _ptr(vol2), n, k, score_dtype, topk, _ptr(F), _ptr(top_idx))


def cdl_cad_edges(ctx, A1, A2, a_dtype, Z1, Z2, vol1, vol2, n, k, score_dtype, delta, max_edges, edge_ij, edge_dE,
                  nodes, n_nodes, top_per_node, partner, partner_dE, F):
    """Returns (status, cdl_edge_result)."""
    res = cdl_edge_result()
    st = _lib.cdl_cad_edges(ctx, _ptr(A1), _ptr(A2), a_dtype, _ptr(Z1), _ptr(Z2), _ptr(vol1), _ptr(vol2), n, k,
                            score_dtype, delta, max_edges, _ptr(edge_ij), _ptr(edge_dE), _ptr(nodes), n_nodes,
                            top_per_node, _ptr(partner), _ptr(partner_dE), _ptr(F), ctypes.byref(res))
    return st, res


def cdl_changed_nodes(ctx, X1, X2, n, T, changed):
    """Returns (status, n_changed)."""
    m = _I32()
    st = _lib.cdl_changed_nodes(ctx, _ptr(X1), _ptr(X2), n, T, _ptr(changed), ctypes.byref(m))
    return st, m.value


def cdl_cad_score_changed(ctx, A1, A2, a_dtype, Z1, Z2, vol1, vol2, n, k, score_dtype, changed, n_changed, topk,
                          F, top_idx) -> int:
    return _lib.cdl_cad_score_changed(ctx, _ptr(A1), _ptr(A2), a_dtype, _ptr(Z1), _ptr(Z2), _ptr(vol1), _ptr(vol2),
                                      n, k, score_dtype, _ptr(changed), n_changed, topk, _ptr(F), _ptr(top_idx))


def cdl_caddelag_pair(ctx, X1, X2, n, T, opts: cdl_pair_opts, F, top_idx, stats1=None,
                      stats2=None) -> int:
    return _lib.cdl_caddelag_pair(ctx, _ptr(X1), _ptr(X2), n, T, ctypes.byref(opts), _ptr(F),
                                  _ptr(top_idx),
                                  ctypes.byref(stats1) if stats1 is not None else None,
                                  ctypes.byref(stats2) if stats2 is not None else None)


def cdl_pair_embeddings(ctx, Z1, Z2, scalars) -> int:
    return _lib.cdl_pair_embeddings(ctx, _ptr(Z1), _ptr(Z2), _ptr(scalars))


def cdl_caddelag_batched(ctx, G, n, T, X1, X2, opts: cdl_batch_opts, F, top_idx, stats=None) -> int:
    """n: int64 array of G orders (NumPy); stats: a ctypes array of 2G
    cdl_solve_stats or None."""
    return _lib.cdl_caddelag_batched(ctx, G, _ptr(n), T, _ptr(X1), _ptr(X2), ctypes.byref(opts), _ptr(F),
                                     _ptr(top_idx), ctypes.cast(stats, _P) if stats is not None else None)


def cdl_batch_plan_info(ctx):
    """Returns (status, cdl_batch_info)."""
    info = cdl_batch_info()
    st = _lib.cdl_batch_plan_info(ctx, ctypes.byref(info))
    return st, info


def exported_symbols():
    """Names of the C entry points bound here (for the export check)."""
    return sorted(list(_SIGS) + ["cdl_status_string", "cdl_last_error_detail"])
