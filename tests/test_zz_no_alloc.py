"""epi3_scan_noalloc: the scan for callers that cannot allocate device memory.

Such callers (fixed-budget hosts, frameworks whose own allocator owns the GPU) get the
whole scan with its scratch in the library's static device array.  These tests call the
entry point through the C ABI and check that its answer equals the CPU oracle's and the
allocating path's (epi3_create + epi3_scan): identical triplets and bit-identical FP64
scores, on two calls in a row with different data sets, so the second call also shows
that stale contents of the shared array do not leak.  Bad genotype and phenotype values
must be refused.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import gen
import oracle
import oracle_pins as pins
from paper_2201_10956_gb300 import build as B
import paper_2201_10956_gb300 as epi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    return epi.load()


def noalloc_call(lib, g, ph, k):
    import torch
    gd = torch.from_numpy(np.ascontiguousarray(g)).cuda()
    pd = torch.from_numpy(np.ascontiguousarray(ph)).cuda()
    trip = torch.full((k, 3), -1, dtype=torch.int32, device="cuda")
    sc = torch.full((k,), -1.0, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    rc = lib.epi3_scan_noalloc(ctypes.c_void_p(gd.data_ptr()), ctypes.c_void_p(pd.data_ptr()),
                               g.shape[0], g.shape[1], k, ctypes.c_void_p(trip.data_ptr()),
                               ctypes.c_void_p(sc.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    return rc, trip.cpu().numpy(), sc.cpu().numpy()


def noalloc_scan(lib, g, ph, k):
    rc, trip, sc = noalloc_call(lib, g, ph, k)
    assert rc == epi.OK, epi.last_error()
    return trip, sc


def allocating_scan(g, ph, k):
    with epi.Handle(g, ph) as h:
        return h.scan(k)


def test_noalloc_matches_allocating_scan_twice(lib):
    d1 = gen.make_config("tiny", seed=3)
    g2, ph2 = pins.tiny_data(200, 1000, 421, seed=77)       # ragged class sizes
    for g, ph, k in ((d1.genotypes, d1.phenotype, 10), (g2, ph2, 25)):
        tr, sc = noalloc_scan(lib, g, ph, k)
        otr, osc, _ = oracle.scan_topk(g, ph, k)
        assert np.array_equal(tr, otr), (tr[:3], otr[:3])
        assert np.array_equal(sc, osc)
        rtr, rsc = allocating_scan(g, ph, k)
        assert np.array_equal(tr, rtr), (tr[:3], rtr[:3])
        assert np.array_equal(sc, rsc)


def test_noalloc_refuses_bad_values(lib):
    g, ph = pins.tiny_data(20, 300, 150, seed=5)
    bad = g.copy()
    bad[7, 123] = 3                                         # genotype outside 0..2
    rc, _, _ = noalloc_call(lib, bad, ph, 5)
    assert rc == epi.ERR_ARG and "genotype" in epi.last_error()
    badp = ph.copy()
    badp[17] = 2                                            # phenotype outside 0..1
    rc, _, _ = noalloc_call(lib, g, badp, 5)
    assert rc == epi.ERR_ARG and "phenotype" in epi.last_error()
    # the array is usable again right after a refused call
    tr, sc = noalloc_scan(lib, g, ph, 5)
    otr, osc, _ = oracle.scan_topk(g, ph, 5)
    assert np.array_equal(tr, otr) and np.array_equal(sc, osc)


def test_noalloc_rejects_sizes_beyond_the_static_array(lib):
    import torch
    m, n = 4096, 8192                                      # ~8.4 MB of planes alone
    gd = torch.zeros((m, n), dtype=torch.uint8, device="cuda")
    pd = torch.zeros((n,), dtype=torch.uint8, device="cuda")
    out_t = torch.empty((1, 3), dtype=torch.int32, device="cuda")
    out_s = torch.empty((1,), dtype=torch.float64, device="cuda")
    rc = lib.epi3_scan_noalloc(ctypes.c_void_p(gd.data_ptr()), ctypes.c_void_p(pd.data_ptr()),
                               m, n, 1, ctypes.c_void_p(out_t.data_ptr()),
                               ctypes.c_void_p(out_s.data_ptr()), None)
    assert rc == epi.ERR_ARG
    assert "scratch" in epi.last_error()
