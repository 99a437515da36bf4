"""Interaction orders beyond three (needs an sm_103 GPU): epi3_scan_order at orders 4, 5 and 6
(Eq. 1 for four, five and six SNPs: 81, 243 and 729 cells per class) against the CPU oracle's
generic-order scan -- identical SNP sets and bit-identical FP64 scores -- on tiny inputs with
ragged class sizes, one class only, exact ties from a duplicated SNP column, and the minimum
number of SNPs; orders 2 and 3 route to the pairwise and triplet scans, other orders are
refused."""
import numpy as np
import pytest

import oracle
import oracle_pins as pins
from paper_2201_10956_gb300 import build as B
import paper_2201_10956_gb300 as epi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    return epi.load()


@pytest.mark.parametrize("m,n,n1,k", [(4, 50, 20, 1), (12, 129, 64, 30), (20, 300, 133, 64),
                                      (30, 257, 0, 10), (24, 1000, 999, 100), (40, 700, 300, 512)])
def test_order4_matches_oracle(m, n, n1, k):
    g, ph = pins.tiny_data(m, n, n1, seed=700 + m)
    with epi.Handle(g, ph) as h:
        sets, sc = h.scan_order(4, k)
    osets, osc, _ = oracle.scan_order_topk(g, ph, 4, k)
    assert np.array_equal(sets, osets), (sets[:3], osets[:3])
    assert np.array_equal(sc, osc)


def test_order4_exact_ties_and_planted():
    g, ph = pins.tiny_data(26, 800, 380, seed=711)
    g[25] = g[24]                           # sets ending in 24 or 25 tie exactly
    with epi.Handle(g, ph) as h:
        sets, sc = h.scan_order(4, 200)
    osets, osc, _ = oracle.scan_order_topk(g, ph, 4, 200)
    assert np.array_equal(sets, osets) and np.array_equal(sc, osc)


def test_orders_2_and_3_route_to_the_pair_and_triplet_scans():
    g, ph = pins.tiny_data(30, 400, 190, seed=712)
    with epi.Handle(g, ph) as h:
        p2, s2 = h.scan_order(2, 20)
        p3, s3 = h.scan_order(3, 20)
        with pytest.raises(epi.Epi3Error) as ei:
            h.scan_order(7, 3)
        assert ei.value.code == epi.ERR_UNSUPPORTED
        with pytest.raises(epi.Epi3Error) as ei:
            h.scan_order(1, 3)
        assert ei.value.code == epi.ERR_UNSUPPORTED
    o2, os2, _ = oracle.scan_order_topk(g, ph, 2, 20)
    o3, os3, _ = oracle.scan_order_topk(g, ph, 3, 20)
    assert np.array_equal(p2, o2) and np.array_equal(s2, os2)
    assert np.array_equal(p3, o3) and np.array_equal(s3, os3)


@pytest.mark.parametrize("order,m,n,n1,k", [(5, 5, 40, 17, 1), (5, 16, 300, 133, 40),
                                            (5, 22, 257, 0, 25), (5, 20, 1000, 999, 100),
                                            (6, 6, 90, 44, 1), (6, 14, 129, 64, 64),
                                            (6, 17, 700, 300, 512)])
def test_orders_5_and_6_match_oracle(order, m, n, n1, k):
    g, ph = pins.tiny_data(m, n, n1, seed=730 + 10 * order + m)
    with epi.Handle(g, ph) as h:
        sets, sc = h.scan_order(order, k)
    osets, osc, _ = oracle.scan_order_topk(g, ph, order, k)
    assert np.array_equal(sets, osets), (sets[:3], osets[:3])
    assert np.array_equal(sc, osc)


@pytest.mark.parametrize("order", [5, 6])
def test_orders_5_and_6_exact_ties(order):
    g, ph = pins.tiny_data(15, 600, 280, seed=740 + order)
    g[14] = g[13]                           # sets ending in 13 or 14 tie exactly
    with epi.Handle(g, ph) as h:
        sets, sc = h.scan_order(order, 150)
        with pytest.raises(epi.Epi3Error) as ei:
            h.scan_order(order, 4000)       # above EPI3_MAX_TOPK
        assert ei.value.code == epi.ERR_ARG
    osets, osc, _ = oracle.scan_order_topk(g, ph, order, 150)
    assert np.array_equal(sets, osets) and np.array_equal(sc, osc)
