"""GB300 (sm_103a) implementation of the CADDeLaG hot path behind a C ABI.

The compute lives in ``libcdl.so`` (CUDA kernels under ``csrc/``, entry points
declared in ``include/cdl.h``); ``cdl`` is its ctypes binding. Build with
``python -m paper_1802_05421_gb300.build``.
"""
import os

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libcdl.so")


def load():
    """Import and return the ctypes binding (raises if the library is missing)."""
    from . import cdl
    return cdl
