"""The C ABI library builds, loads and exports every entry point include/ckinv.h declares
(CPU only: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ckinv.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ckinv_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1312_1869_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_entry_points():
    names = declared_functions()
    for n in ["ckinv_sketch", "ckinv_tsqr", "ckinv_solve", "ckinv_nll_grad", "ckinv_create", "ckinv_destroy"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_1312_1869_gb300 import ckinv as ck
    assert set(declared_functions()) <= set(ck._SIGS)


def test_version_and_struct_layouts(lib):
    from paper_1312_1869_gb300 import ckinv as ck
    assert ck.version().startswith("ckinv")
    assert ctypes.sizeof(ck.PlanDesc) == 48
    assert ctypes.sizeof(ck.KernelDesc) == 32


def test_context_creation_without_a_gb300_fails_cleanly():
    import torch
    from paper_1312_1869_gb300 import ckinv as ck
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(ck.CKInvError) as e:
        ck.Context(0)
    assert e.value.status in (ck.EUNSUPPORTED, ck.ECUDA)
