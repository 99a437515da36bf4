"""Pairwise (second-order) scan vs the oracle (needs an sm_103 GPU): the top-k pairs and
their FP64 K2 must equal the oracle's exhaustive pair scan bit for bit."""
import numpy as np
import pytest

import gen
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


@pytest.mark.parametrize("m,n,n1,k", [(3, 5, 2, 3), (7, 130, 64, 21), (40, 512, 256, 50),
                                      (97, 257, 0, 100), (65, 300, 300, 7), (130, 1000, 401, 512),
                                      (70, 33, 11, 2415)])
def test_pair_scan_matches_oracle(m, n, n1, k):
    g, ph = pins.tiny_data(m, n, n1, seed=2000 + m + n)
    k = min(k, m * (m - 1) // 2, epi.MAX_TOPK)
    with epi.Handle(g, ph) as h:
        pr, sc = h.scan_pairs(k)
    opr, osc, _ = oracle.scan_pairs_topk(g, ph, k)
    assert np.array_equal(pr, opr) and np.array_equal(sc, osc)


def test_pair_scan_ties_and_many_blocks():
    # 2100 SNPs: C(2100, 2) = 2.2 M pairs, several selection passes; copies of one SNP give
    # exactly equal scores that must come out in (i, j) order
    d = gen.make_dataset(2100, 600, 250, (0.05, 0.5), 1, seed=31)
    g = d.genotypes.copy()
    for c in range(1000, 1010):
        g[c] = g[5]
    with epi.Handle(g, d.phenotype) as h:
        pr, sc = h.scan_pairs(512)
    opr, osc, _ = oracle.scan_pairs_topk(g, d.phenotype, 512)
    assert np.array_equal(pr, opr) and np.array_equal(sc, osc)


def test_pair_scan_medium_config_and_device_outputs():
    import torch
    d = gen.make_config("medium")
    opr, osc, _ = oracle.scan_pairs_topk(d.genotypes, d.phenotype, 64)
    with epi.Handle(torch.from_numpy(d.genotypes).cuda(), torch.from_numpy(d.phenotype).cuda()) as h:
        pr, sc = h.scan_pairs(64)
        assert np.array_equal(pr.cpu().numpy(), opr) and np.array_equal(sc.cpu().numpy(), osc)


def test_pair_scan_bad_arguments():
    g, ph = pins.tiny_data(6, 40, 20, seed=3)
    with epi.Handle(g, ph) as h:
        for k in (0, 16, epi.MAX_TOPK + 1):
            with pytest.raises(epi.Epi3Error) as ei:
                h.scan_pairs(k)
            assert ei.value.code == epi.ERR_ARG
        pr, sc = h.scan_pairs(15)   # C(6, 2): every pair, still usable after the errors
    opr, osc, _ = oracle.scan_pairs_topk(g, ph, 15)
    assert np.array_equal(pr, opr) and np.array_equal(sc, osc)
