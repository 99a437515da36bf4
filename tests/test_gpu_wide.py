"""Scans wider than the one-hot tensor form's tile list (needs an sm_103 GPU).

The one-hot tensor form (paths mma, mma16, mma4) lists one tile per (i, j block, k block) and
refuses data sets whose list would pass 2^26 tiles (from 9378 SNPs on).  The sample-compacted
tensor form (mma4c) decodes its tiles from a per-first-SNP table and serves any SNP count, so a
12 000-SNP scan with path auto still runs on the tensor cores.  Here, at 12 000 SNPs:

* path auto picks the compacted tensor form, and the one-hot form says it does not serve the
  shape;
* the whole scan's top-10 is rescored by the oracle and beats every sampled triplet
  (Eq. 1, lowest K2 first, ties by index);
* two pair-range slices that reach the largest indices (pairs with j < 24, whose third SNPs run
  to 11 999, and pairs with j >= 11 990) equal the oracle's exhaustive ranking of the same
  triplets, element by element.
"""
import numpy as np
import pytest

import gen
import oracle
import paper_2201_10956_gb300 as epi

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

M, N, N1 = 12000, 4096, 2048


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_10956_gb300 import build as B
    B.build()
    epi.load()


@pytest.fixture(scope="module")
def data():
    return gen.make_dataset(M, N, N1, maf_range=(0.05, 0.5), n_planted=1, planted_maf=0.4,
                            odds_ratio=10.0, seed=12, name="wide")


def pairs_of(m):
    """Pairs i<j of m SNPs: pair (i, j) has index j (j - 1) / 2 + i, so the pairs with j < m
    are the indices below this."""
    return m * (m - 1) // 2


def triplets_of_pairs(m, j_lo, j_hi):
    """Every triplet i<j<k of m SNPs with j_lo <= j < j_hi, sorted by (i, j, k)."""
    out = []
    for j in range(j_lo, min(j_hi, m - 1)):
        i, k = np.meshgrid(np.arange(j, dtype=np.int32), np.arange(j + 1, m, dtype=np.int32),
                           indexing="ij")
        out.append(np.stack([i.ravel(), np.full(i.size, j, np.int32), k.ravel()], axis=1))
    t = np.concatenate(out).astype(np.int32)
    return t[np.lexsort((t[:, 2], t[:, 1], t[:, 0]))]


def oracle_topk(g, ph, trip, k):
    s = oracle.scores(g, ph, trip)
    order = np.lexsort((trip[:, 2], trip[:, 1], trip[:, 0], s))[:k]
    return trip[order], s[order]


def test_auto_scans_wide_data_on_the_tensor_cores(data):
    g, ph = data.genotypes, data.phenotype
    k = 10
    with epi.Handle(g, ph) as h:
        tr, sc = h.scan(k)
        st = h.stats()
        assert st["path"] == epi.PATH_MMA4C, st["path"]
        assert st["n_triplets"] == gen.n_triplets(M)
        h.set_option("path", "mma4")
        with pytest.raises(epi.Epi3Error) as ei:
            h.scan(k)
        assert ei.value.code == epi.ERR_UNSUPPORTED
    samp = gen.random_triplets(M, 200_000, seed=7)
    planted = np.array(data.planted, dtype=np.int32).reshape(-1, 3)
    ref = oracle.scores(g, ph, np.concatenate([tr, samp, planted]))
    assert np.array_equal(ref[:k], sc)
    assert np.all(np.diff(sc) >= 0)
    assert np.all(tr[:, 0] < tr[:, 1]) and np.all(tr[:, 1] < tr[:, 2])
    assert np.all(tr[:, 2] < M)
    got = {tuple(t) for t in tr}
    assert all(tuple(t) in got for t in samp[ref[k:k + len(samp)] < sc[-1]])
    assert tuple(planted[0]) in got


@pytest.mark.parametrize("j_lo,j_hi", [(0, 24), (11990, M)])
def test_wide_range_slices_equal_the_oracle(data, j_lo, j_hi):
    g, ph = data.genotypes, data.phenotype
    k = 16
    pb, pe = pairs_of(j_lo), pairs_of(min(j_hi, M - 1))
    with epi.Handle(g, ph) as h:
        h.set_option("path", "mma4c")
        tr, sc = h.scan_range(pb, pe, k)
        assert h.stats()["path"] == epi.PATH_MMA4C
    otr, osc = oracle_topk(g, ph, triplets_of_pairs(M, j_lo, j_hi), k)
    assert np.array_equal(tr, otr), (tr[:4], otr[:4])
    assert np.array_equal(sc, osc)
