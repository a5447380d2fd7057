"""The C ABI library builds, loads without a GPU and exports every entry
point include/cdl.h declares (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cdl.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cdl_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1802_05421_gb300 import build as B
    path = B.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["cdl_build_graph", "cdl_chain_build", "cdl_chain_solve", "cdl_project",
                     "cdl_cad_score", "cdl_caddelag_pair", "cdl_ctx_create", "cdl_sync"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header(lib):
    from paper_1802_05421_gb300 import cdl
    assert set(cdl.exported_symbols()) == set(declared_functions())


def test_status_strings(lib):
    from paper_1802_05421_gb300 import cdl
    assert cdl.cdl_status_string(0) == "CDL_OK"
    assert cdl.cdl_status_string(-4) == "CDL_ERR_NOT_CONVERGED"
    assert cdl.cdl_status_string(-99) == "CDL_ERR_UNKNOWN"


def test_null_arguments_are_rejected_without_a_gpu(lib):
    from paper_1802_05421_gb300 import cdl
    assert cdl._lib.cdl_ctx_create(None, 0, None, 0) == cdl.CDL_ERR_INVALID_ARG
    assert cdl.cdl_build_graph(None, None, 10, 4, 0.0, cdl.CDL_F64, None, None, None, None) == \
        cdl.CDL_ERR_INVALID_ARG
    assert cdl.cdl_sync(None) == cdl.CDL_ERR_INVALID_ARG
    assert cdl.cdl_ctx_destroy(None) == cdl.CDL_OK
    assert cdl.cdl_chain_free(None) == cdl.CDL_OK


def declared_constants():
    """Every enumerator of include/cdl.h with its value (explicit decimal or
    hexadecimal values only, which is how the header writes them)."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    out = {}
    for body in re.findall(r"enum\s*(?:\w+\s*)?\{(.*?)\}", text, flags=re.S):
        for name, value in re.findall(r"\b(CDL_[A-Z0-9_]+)\s*=\s*(-?(?:0x[0-9A-Fa-f]+|\d+))", body):
            out[name] = int(value, 0)
    return out


def test_binding_constants_match_the_header():
    from paper_1802_05421_gb300 import cdl
    consts = declared_constants()
    assert len(consts) >= 30 and consts["CDL_KC_HOST_LINK"] == 11
    wrong = {k: (v, getattr(cdl, k, None)) for k, v in consts.items() if getattr(cdl, k, None) != v}
    assert not wrong, wrong
    assert len(cdl.KERNEL_CLASSES) == consts["CDL_KC_HOST_LINK"]   # the kernel classes precede the copy class


def test_every_entry_point_rejects_null_arguments_without_a_gpu(lib):
    """Each entry point called with null pointers and zero sizes returns
    CDL_ERR_INVALID_ARG before touching CUDA; the two release calls accept
    null. Context creation on a machine without a usable device reports
    CDL_ERR_CUDA with the runtime's message and leaves the handle null."""
    from paper_1802_05421_gb300 import cdl
    release = {"cdl_ctx_destroy", "cdl_chain_free"}
    wrong = {}
    for name, args in cdl._SIGS.items():
        vals = []
        for a in args:
            if a is ctypes.c_double:
                vals.append(0.0)
            elif a in (ctypes.c_int, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t, ctypes.c_uint64):
                vals.append(0)
            else:
                vals.append(None)
        r = getattr(cdl._lib, name)(*vals)
        want = cdl.CDL_OK if name in release else cdl.CDL_ERR_INVALID_ARG
        if r != want:
            wrong[name] = r
    assert not wrong, wrong
    import torch
    if not torch.cuda.is_available():
        h = ctypes.c_void_p()
        assert cdl._lib.cdl_ctx_create(ctypes.byref(h), 0, None, 0) == cdl.CDL_ERR_CUDA
        assert h.value is None and cdl.cdl_last_error_detail()
