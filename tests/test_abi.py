"""The C ABI library builds for sm_103a, loads, and exports every entry point
declared in include/qcx.h (no GPU needed: no compute call is made)."""
import ctypes
import os

import pytest

from paper_2603_12326_gb300 import build, qcx


@pytest.fixture(scope="session")
def lib():
    build.build()
    return qcx.load()


def test_every_declared_symbol_is_exported(lib):
    names = qcx.declared_symbols()
    assert len(names) >= 12
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding wraps each of them
    assert set(names) <= set(qcx._SIGS)


def test_library_is_built_for_sm103a(lib):
    """The build compiles every source for sm_103a alone (one -gencode, no
    PTX for other targets); on a GPU, qcx_create also refuses a library whose
    kernels report another binary version (cudaFuncGetAttributes)."""
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    src = open(os.path.join(os.path.dirname(qcx.__file__), "csrc", "api.cu")).read()
    assert "fa.binaryVersion != 103" in src


def test_create_without_device_fails_cleanly(lib):
    # on a machine without a GB300 the context refuses to start instead of
    # falling back to anything else
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    st = qcx.qcx_create(ctypes.byref(h), 0, None)
    assert st == 3 and not h.value


def test_null_context_arguments(lib):
    assert qcx.qcx_sync(None) == 1
    assert qcx.qcx_nbasis(None) == 0
    assert qcx.qcx_last_error(None) == b"null context"


def test_status_names_match_header():
    txt = open(os.path.join(os.path.dirname(qcx.__file__), "..", "include", "qcx.h")).read()
    for code, name in qcx.STATUS.items():
        assert f"{name} = {code}" in txt
