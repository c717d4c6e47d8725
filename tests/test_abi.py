"""Host-side checks of the C ABI (no GPU): the library builds for sm_103a,
loads, and exports every symbol include/nne.h declares."""
import os
import re

import pytest

from paper_2501_13237_gb300 import build, nne

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return nne.load()


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "nne.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(nne_[a-z0-9_]+)\s*\(", txt)))


def test_header_declares_the_binding_symbols():
    assert declared_symbols() == sorted(nne.SYMBOLS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_no_gpu_call_fails_cleanly(lib):
    # Without a GPU, context creation must return an error status, not crash.
    import ctypes as C
    h = C.c_void_p()
    rc = lib.nne_ctx_create(0, None, 0, C.byref(h))
    import torch
    if not torch.cuda.is_available():
        assert rc != 0 and lib.nne_last_error()
