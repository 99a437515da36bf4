"""The C-ABI library builds, loads and exports every declared entry point (no GPU)."""
import os
import re

import pytest

import paper_2201_10956_gb300 as epi
from paper_2201_10956_gb300 import build as B

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                      "epi3.h")


def declared():
    with open(HEADER) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(epi3_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return epi.load()


def test_header_declares_binding_symbols():
    assert sorted(epi.SYMBOLS) == declared()


def test_library_exports_every_declared_symbol(lib):
    for name in declared():
        assert hasattr(lib, name), name


def test_build_targets_sm103a_only():
    # one -gencode, sm_103a: the build passes nothing else to nvcc
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert not any("gencode" in f or "arch" in f for f in B.FLAGS)


def test_argument_errors_without_gpu(lib):
    import ctypes
    import numpy as np
    h = ctypes.c_void_p()
    g = np.zeros((4, 8), dtype=np.uint8)
    p = np.zeros(8, dtype=np.uint8)
    P = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    assert lib.epi3_create(ctypes.byref(h), None, P(p), 4, 8, 0, None) == epi.ERR_ARG
    assert lib.epi3_create(ctypes.byref(h), P(g), P(p), 2, 8, 0, None) == epi.ERR_ARG
    assert "n_snps" in epi.last_error()
    assert lib.epi3_create(ctypes.byref(h), P(g), P(p), 4, 0, 0, None) == epi.ERR_ARG
    assert lib.epi3_create(ctypes.byref(h), P(g), P(p), 4, 8, 7, None) == epi.ERR_ARG
    assert lib.epi3_scan(None, 1, P(p), P(p)) == epi.ERR_ARG
    assert h.value is None


def test_no_cpu_fallback(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    import numpy as np
    with pytest.raises(epi.Epi3Error) as ei:
        epi.Handle(np.zeros((4, 8), np.uint8), np.zeros(8, np.uint8))
    assert ei.value.code == epi.ERR_UNSUPPORTED
