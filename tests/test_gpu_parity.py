"""GPU path vs the CPU oracle, through the C ABI (needs an sm_103 GPU).

Bars: contingency tables bit-exact; FP32 K2 within 1e-5 relative of the oracle's
FP64 K2 (and within the library's proven bound); FP64-rescored top-k triplets and
scores identical to the oracle's (same Eq. 1 evaluation order, same log table).
"""
import itertools

import numpy as np
import pytest

import gen
import oracle
import oracle_pins as pins
from paper_2201_10956_gb300 import build as B
import paper_2201_10956_gb300 as epi

pytestmark = pytest.mark.gpu

REL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    return epi.load()


def all_trip(m):
    return np.array(list(itertools.combinations(range(m), 3)), dtype=np.int32).reshape(-1, 3)


def check_scores(h, g, ph, trip):
    s32, s64 = h.scores(trip)
    ref = oracle.scores(g, ph, trip)
    assert np.array_equal(s64, ref), np.max(np.abs(s64 - ref))
    rel = np.abs(s32.astype(np.float64) - ref) / ref
    assert rel.max() <= REL, rel.max()
    st = h.stats()
    bound = st["k2_rel_bound"] * ref + st["k2_abs_bound"]
    assert np.all(np.abs(s32 - ref) <= bound)


PATHS = ["popc", "popc8"]


def check_scan(h, g, ph, k, paths=PATHS):
    for path in paths:
        h.set_option("path", path)
        _check_scan(h, g, ph, k)


def _check_scan(h, g, ph, k):
    tr, sc = h.scan(k)
    otr, osc, _ = oracle.scan_topk(g, ph, k)
    assert np.array_equal(tr, otr), (tr[:5], otr[:5])
    assert np.array_equal(sc, osc)


def test_tiny_config_full_parity():
    d = gen.make_config("tiny")
    with epi.Handle(d.genotypes, d.phenotype) as h:
        assert h.shape() == (64, 512, 256, 256)
        trip = all_trip(64)
        ref = oracle.tables(d.genotypes, d.phenotype, trip)
        assert np.array_equal(h.tables(trip), ref)
        assert np.array_equal(h.tables(trip, epi.PATH_POPC8), ref)
        check_scores(h, d.genotypes, d.phenotype, trip)
        check_scan(h, d.genotypes, d.phenotype, 10)
        st = h.stats()
        assert st["n_triplets"] == 41664


@pytest.mark.parametrize("m,n,n1", [(3, 1, 0), (4, 1, 1), (5, 31, 7), (6, 32, 16), (7, 33, 0),
                                    (8, 127, 127), (9, 128, 64), (10, 129, 1), (13, 130, 65),
                                    (12, 257, 100), (11, 385, 300)])
def test_ragged_shapes(m, n, n1):
    g, ph = pins.tiny_data(m, n, n1, seed=100 + m + n)
    with epi.Handle(g, ph) as h:
        trip = all_trip(m)
        ref = pins.numpy_tables(g, ph, trip).astype(np.int32)
        assert np.array_equal(h.tables(trip), ref)
        assert np.array_equal(h.tables(trip, epi.PATH_POPC8), ref)
        check_scores(h, g, ph, trip)
        check_scan(h, g, ph, min(10, len(trip)))


def test_multi_tile_exhaustive():
    # several k-chunks per pair, both classes spanning several 128-sample groups
    g, ph = pins.tiny_data(300, 700, 333, seed=7)
    with epi.Handle(g, ph) as h:
        for k in (1, 17, 64):
            check_scan(h, g, ph, k)


def test_out_of_order_triplets_take_roles():
    g, ph = pins.tiny_data(9, 200, 90, seed=8)
    with epi.Handle(g, ph) as h:
        trip = all_trip(9)[:, [2, 0, 1]]
        ref = oracle.tables(g, ph, trip)
        assert np.array_equal(h.tables(trip), ref)
        assert np.array_equal(h.tables(trip, epi.PATH_POPC8), ref)


def test_exact_ties_break_by_index():
    d = gen.make_dataset(60, 600, 300, (0.3, 0.5), 1, seed=5, odds_ratio=10.0)
    g = d.genotypes.copy()
    i, j, k = d.planted[0]
    free = [c for c in range(60) if c not in (i, j, k)]
    g[free[-1]] = g[k]
    g[free[0]] = g[i]
    with epi.Handle(g, d.phenotype) as h:
        otr, osc, _ = oracle.scan_topk(g, d.phenotype, 8)
        for path in PATHS:
            h.set_option("path", path)
            tr, sc = h.scan(8)
            assert np.array_equal(tr, otr) and np.array_equal(sc, osc)
            assert sc[0] == sc[1]


@pytest.mark.parametrize("path", PATHS)
def test_scan_range_slices_merge_to_full_scan(path):
    g, ph = pins.tiny_data(80, 300, 150, seed=9)
    k = 12
    with epi.Handle(g, ph) as h:
        h.set_option("path", path)
        full_t, full_s = h.scan(k)
        npairs = 80 * 79 // 2
        cuts = [0, 5, 400, 1000, 2500, npairs]
        rows = []
        for a, b in zip(cuts[:-1], cuts[1:]):
            t, s = h.scan_range(a, b, k)
            rows += [(float(x), *map(int, y)) for x, y in zip(s, t)]
        rows.sort()
        assert [r[1:] for r in rows[:k]] == [tuple(map(int, t)) for t in full_t]
        assert np.array_equal(np.array([r[0] for r in rows[:k]]), full_s)


def test_device_pointer_mode_matches_host_mode():
    import torch
    d = gen.make_config("tiny", seed=2)
    with epi.Handle(d.genotypes, d.phenotype) as h:
        tr_h, sc_h = h.scan(10)
        tab_h = h.tables(all_trip(20))
    g = torch.from_numpy(d.genotypes).cuda()
    p = torch.from_numpy(d.phenotype).cuda()
    with epi.Handle(g, p) as h:
        tr_d, sc_d = h.scan(10)
        tab_d = h.tables(all_trip(20))
        torch.cuda.synchronize()
        assert np.array_equal(tr_d.cpu().numpy(), tr_h)
        assert np.array_equal(sc_d.cpu().numpy(), sc_h)
        assert np.array_equal(tab_d.cpu().numpy(), tab_h)


def test_bad_values_are_rejected():
    g, ph = pins.tiny_data(5, 40, 20, seed=1)
    g2 = g.copy()
    g2[3, 7] = 3
    with pytest.raises(epi.Epi3Error) as ei:
        epi.Handle(g2, ph)
    assert ei.value.code == epi.ERR_ARG and "genotype" in str(ei.value)
    ph2 = ph.copy()
    ph2[0] = 2
    with pytest.raises(epi.Epi3Error) as ei:
        epi.Handle(g, ph2)
    assert ei.value.code == epi.ERR_ARG and "phenotype" in str(ei.value)
    with epi.Handle(g, ph) as h:
        with pytest.raises(epi.Epi3Error) as ei:
            h.scan(11)  # C(5,3) = 10
        assert ei.value.code == epi.ERR_ARG
        with pytest.raises(epi.Epi3Error) as ei:
            h.tables([[0, 1, 5]])
        assert ei.value.code == epi.ERR_ARG


def test_injected_allocation_failure(monkeypatch):
    g, ph = pins.tiny_data(5, 40, 20, seed=1)
    monkeypatch.setenv("EPI3_FAULT", "alloc")
    with pytest.raises(epi.Epi3Error) as ei:
        epi.Handle(g, ph)
    assert ei.value.code == epi.ERR_OOM
    monkeypatch.delenv("EPI3_FAULT")
    with epi.Handle(g, ph) as h:
        monkeypatch.setenv("EPI3_FAULT", "launch")
        with pytest.raises(epi.Epi3Error) as ei:
            h.scan(3)
        assert ei.value.code == epi.ERR_CUDA
        monkeypatch.delenv("EPI3_FAULT")
        assert h.scan(3)[0].shape == (3, 3)


def sampled_parity(d, n_sample, k, seed=0, path="popc8"):
    """Full-size workload: exact tables and scores on a random sample, the GPU's
    top-k rescored by the oracle, and no sampled triplet beating the k-th."""
    g, ph = d.genotypes, d.phenotype
    with epi.Handle(g, ph) as h:
        h.set_option("path", path)
        tr, sc = h.scan(k)
        st = h.stats()
        samp = gen.random_triplets(d.n_snps, n_sample, seed=seed)
        planted = np.array(d.planted, dtype=np.int32).reshape(-1, 3)
        test_t = np.concatenate([samp, tr, planted])
        ref_tab = oracle.tables(g, ph, test_t[:20000])
        assert np.array_equal(h.tables(test_t[:20000]), ref_tab)
        assert np.array_equal(h.tables(test_t[:20000], epi.PATH_POPC8), ref_tab)
        s32, s64 = h.scores(test_t)
    ref = oracle.scores(g, ph, test_t)
    assert np.array_equal(s64, ref)
    assert (np.abs(s32 - ref) / ref).max() <= REL
    # the GPU answer is sorted, rescored exactly, and nothing sampled beats its k-th
    assert np.array_equal(ref[n_sample:n_sample + k], sc)
    assert np.all(np.diff(sc) >= 0)
    assert np.all(tr[:, 0] < tr[:, 1]) and np.all(tr[:, 1] < tr[:, 2])
    better = ref[:n_sample] < sc[-1]
    got = {tuple(t) for t in tr}
    assert all(tuple(t) in got for t in samp[better])
    return st


@pytest.mark.parametrize("path", PATHS)
def test_medium_config_sampled(path):
    d = gen.make_config("medium")
    st = sampled_parity(d, 200_000, 10, path=path)
    assert st["n_triplets"] == gen.n_triplets(1024)


@pytest.mark.slow
@pytest.mark.parametrize("path", ["popc8", "auto"])
def test_large_config_sampled(path):
    d = gen.make_config("large")
    sampled_parity(d, 100_000, 10, seed=1, path=path)


def triplets_with(m, p):
    """Every triplet i<j<k of m SNPs that contains SNP p."""
    rest = np.array([x for x in range(m) if x != p], dtype=np.int32)
    a, b = np.triu_indices(m - 1, 1)
    t = np.stack([rest[a], rest[b], np.full(a.size, p, dtype=np.int32)], axis=1)
    return np.sort(t, axis=1).astype(np.int32)


@pytest.mark.slow
@pytest.mark.parametrize("path", ["popc8", "auto"])
def test_stress_config_sampled(path):
    d = gen.make_config("stress")
    sampled_parity(d, 200_000, 64, seed=2, path=path)
    # every triplet containing one SNP of each planted triplet (4 x C(4095, 2) = 3.4e7), scored
    # by the oracle: none outside the answer scores below its 64th
    g, ph = d.genotypes, d.phenotype
    with epi.Handle(g, ph) as h:
        h.set_option("path", path)
        tr, sc = h.scan(64)
    got = {tuple(t) for t in tr}
    for p in sorted({t[0] for t in d.planted}):
        trip = triplets_with(d.n_snps, p)
        s64 = oracle.scores(g, ph, trip)
        for t in trip[s64 < sc[-1]]:
            assert tuple(t) in got
        assert not np.any(s64 < sc[0])


@pytest.mark.slow
def test_stress_config_has_near_ties():
    # the precision-stress workload is meant to put top candidates within 1e-4 relative of each
    # other: the oracle-rescored top-64 must hold many distinct scores closer than 1e-4
    # relative, which the FP32 band and the FP64 rescoring then have to order exactly (exact
    # ties are covered by test_exact_ties_break_by_index and the tensor-form tie tests)
    d = gen.make_config("stress")
    with epi.Handle(d.genotypes, d.phenotype) as h:
        tr, sc = h.scan(64)
    ref = oracle.scores(d.genotypes, d.phenotype, tr)
    assert np.array_equal(ref, sc)
    gap = np.diff(sc) / sc[1:]
    near = np.count_nonzero((gap >= 0) & (gap < 1e-4))
    assert near >= 8, (near, gap)
