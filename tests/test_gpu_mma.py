"""Tensor-core (tcgen05) scan and the 8-cell POPC scan vs the oracle (needs an sm_103 GPU).

The scan kernels' own FP32 scores for every triplet (epi3_scan_scores) must equal the FP32
score of the exact table (epi3_scores) bit for bit -- so every table the kernel counted is
exact -- and the FP64-rescored top-k must equal the oracle's.
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

KERNEL_PATHS = [("popc", epi.PATH_POPC), ("popc8", epi.PATH_POPC8), ("mma", epi.PATH_MMA),
                ("mma16", epi.PATH_MMA16), ("mma4", epi.PATH_MMA4), ("mma4c", epi.PATH_MMA4C)]
TENSOR = {"mma": epi.PATH_MMA, "mma16": epi.PATH_MMA16, "mma4": epi.PATH_MMA4,
          "mma4c": epi.PATH_MMA4C}


@pytest.fixture(scope="module", autouse=True)
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    return epi.load()


def all_trip(m):
    return np.array(list(itertools.combinations(range(m), 3)), dtype=np.int32).reshape(-1, 3)


def check_every_triplet(h, g, ph, path_id):
    m = g.shape[0]
    cube = h.scan_scores(path_id)
    trip = all_trip(m)
    got = cube[trip[:, 0], trip[:, 1], trip[:, 2]]
    s32, _ = h.scores(trip)
    bad = np.nonzero(~(got == s32))[0]
    assert bad.size == 0, (path_id, bad.size, trip[bad[:5]], got[bad[:5]], s32[bad[:5]])


@pytest.mark.parametrize("name,path_id", KERNEL_PATHS)
@pytest.mark.parametrize("m,n,n1", [(3, 5, 2), (7, 130, 64), (40, 512, 256), (70, 1000, 401),
                                    (97, 257, 0), (65, 300, 300), (130, 200, 77)])
def test_scan_kernel_tables_exact(name, path_id, m, n, n1):
    g, ph = pins.tiny_data(m, n, n1, seed=1000 + m + n)
    with epi.Handle(g, ph) as h:
        check_every_triplet(h, g, ph, path_id)
        h.set_option("path", name)
        k = min(10, m * (m - 1) * (m - 2) // 6)
        tr, sc = h.scan(k)
        otr, osc, _ = oracle.scan_topk(g, ph, k)
        assert np.array_equal(tr, otr) and np.array_equal(sc, osc)


@pytest.mark.parametrize("name,path_id", KERNEL_PATHS[2:])
def test_tensor_counts_exact_at_large_counts(name, path_id):
    # nearly monomorphic SNPs: one cell holds almost every sample of a class, so the
    # accumulators reach ~N_c (here 16000 and 24000)
    rng = np.random.default_rng(5)
    m, n, n1 = 12, 40000, 24000
    g = np.zeros((m, n), dtype=np.uint8)
    g[rng.random((m, n)) < 0.002] = 1
    ph = np.zeros(n, dtype=np.uint8)
    ph[rng.choice(n, n1, replace=False)] = 1
    with epi.Handle(g, ph) as h:
        check_every_triplet(h, g, ph, path_id)
        h.set_option("path", name)
        tr, sc = h.scan(5)
    otr, osc, _ = oracle.scan_topk(g, ph, 5)
    assert np.array_equal(tr, otr) and np.array_equal(sc, osc)


@pytest.mark.parametrize("name", sorted(TENSOR))
def test_tensor_scan_tiny_config(name):
    d = gen.make_config("tiny")
    with epi.Handle(d.genotypes, d.phenotype) as h:
        h.set_option("path", name)
        tr, sc = h.scan(10)
        assert h.stats()["path"] == TENSOR[name]
    otr, osc, _ = oracle.scan_topk(d.genotypes, d.phenotype, 10)
    assert np.array_equal(tr, otr) and np.array_equal(sc, osc)


@pytest.mark.parametrize("name", sorted(TENSOR))
def test_tensor_scan_range_slices(name):
    g, ph = pins.tiny_data(90, 400, 170, seed=19)
    k = 9
    with epi.Handle(g, ph) as h:
        h.set_option("path", name)
        full_t, full_s = h.scan(k)
        npairs = 90 * 89 // 2
        rows = []
        for a, b in zip([0, 7, 900, 2500], [7, 900, 2500, npairs]):
            t, s = h.scan_range(a, b, k)
            rows += [(float(x), *map(int, y)) for x, y in zip(s, t)]
        rows.sort()
        assert [r[1:] for r in rows[:k]] == [tuple(map(int, t)) for t in full_t]


@pytest.mark.parametrize("name", sorted(TENSOR))
def test_tensor_scan_medium_sampled(name):
    d = gen.make_config("medium")
    g, ph = d.genotypes, d.phenotype
    with epi.Handle(g, ph) as h:
        h.set_option("path", "popc8")
        ref_t, ref_s = h.scan(10)
        h.set_option("path", name)
        tr, sc = h.scan(10)
    assert np.array_equal(tr, ref_t) and np.array_equal(sc, ref_s)
    assert np.array_equal(oracle.scores(g, ph, tr), sc)


@pytest.mark.parametrize("name,form", [("mma", "plain"), ("mma", "split"), ("mma4", "plain"),
                                       ("mma4", "split"), ("mma4c", "auto")])
def test_bounded_wait_times_out_and_context_survives(monkeypatch, name, form):
    # a device wait that can only run out: the kernel must report EPI3_ERR_TIMEOUT after its
    # 1 s limit, release its resources, and leave the context usable (both kernel forms)
    g, ph = pins.tiny_data(40, 300, 120, seed=77)
    with epi.Handle(g, ph) as h:
        h.set_option("path", name)
        h.set_option("mma_form", form)
        monkeypatch.setenv("EPI3_FAULT", "timeout")
        with pytest.raises(epi.Epi3Error) as ei:
            h.scan(5)
        assert ei.value.code == epi.ERR_TIMEOUT
        monkeypatch.delenv("EPI3_FAULT")
        tr, sc = h.scan(5)
    otr, osc, _ = oracle.scan_topk(g, ph, 5)
    assert np.array_equal(tr, otr) and np.array_equal(sc, osc)


@pytest.mark.parametrize("name", sorted(TENSOR))
def test_tensor_exact_ties_and_copies(name):
    # eight copies of one SNP and two of another: many triplets with exactly equal K2 at and
    # around the k-th place, which the band, the pruning and the (K2, i, j, k) order must keep
    d = gen.make_dataset(70, 900, 400, (0.2, 0.5), 1, seed=21, odds_ratio=6.0)
    g = d.genotypes.copy()
    for c in range(40, 48):
        g[c] = g[3]
    g[60] = g[61]
    with epi.Handle(g, d.phenotype) as h:
        h.set_option("path", name)
        tr, sc = h.scan(64)
    otr, osc, _ = oracle.scan_topk(g, d.phenotype, 64)
    assert np.array_equal(tr, otr) and np.array_equal(sc, osc)


def test_pruned_scan_with_a_crowded_band():
    # no planted signal, narrow MAF range: the k-th best lies in the bulk of the K2
    # distribution, so many tables fall inside the pruning bound and need the exact score
    d = gen.make_dataset(90, 3000, 1500, (0.3, 0.35), 0, seed=23)
    with epi.Handle(d.genotypes, d.phenotype) as h:
        h.set_option("path", "mma4")
        tr, sc = h.scan(512)
        st = h.stats()
    assert 0.0 < st["k2_prune_bound"] < 64.0
    otr, osc, _ = oracle.scan_topk(d.genotypes, d.phenotype, 512)
    assert np.array_equal(tr, otr) and np.array_equal(sc, osc)


@pytest.mark.parametrize("name", sorted(TENSOR))
def test_tensor_scan_full_size_matches_popc8(name):
    # the 2048 x 16384 workload: every tensor kind's top-10 equals the 8-cell POPC scan's
    # (itself checked against the oracle) and the oracle's FP64 scores of those triplets
    d = gen.make_config("large")
    g, ph = d.genotypes, d.phenotype
    with epi.Handle(g, ph) as h:
        h.set_option("path", "popc8")
        ref_t, ref_s = h.scan(10)
        h.set_option("path", name)
        tr, sc = h.scan(10)
    assert np.array_equal(tr, ref_t) and np.array_equal(sc, ref_s)
    assert np.array_equal(oracle.scores(g, ph, tr), sc)
    assert tuple(tr[0]) in [tuple(p) for p in d.planted]


@pytest.mark.parametrize("name", ["mma4", "mma4c", "popc8"])
def test_largest_sample_count(name):
    # 131 072 samples, the most a handle takes: the widest log-factorial table, the loosest
    # pruning bound and 512 K-steps per class boundary; top-k still equals the oracle's
    g, ph = pins.tiny_data(9, 131072, 50000, seed=91)
    with epi.Handle(g, ph) as h:
        h.set_option("path", name)
        tr, sc = h.scan(20)
        if name.startswith("mma4"):
            assert 0.0 < h.stats()["k2_prune_bound"] < 256.0
    otr, osc, _ = oracle.scan_topk(g, ph, 20)
    assert np.array_equal(tr, otr) and np.array_equal(sc, osc)


@pytest.mark.parametrize("m,n,n1", [(40, 512, 256), (70, 3000, 1200), (33, 20000, 7000)])
def test_both_kernel_forms(m, n, n1):
    # the plain (14 warps) and register-split (16 warps) forms of the tensor scan: every
    # triplet's table exact in both, identical top-k, and the stats report the launched form
    g, ph = pins.tiny_data(m, n, n1, seed=400 + m)
    otr, osc, _ = oracle.scan_topk(g, ph, 12)
    with epi.Handle(g, ph) as h:
        h.set_option("path", "mma4")
        for form, threads in (("plain", 448), ("split", 512)):
            h.set_option("mma_form", form)
            check_every_triplet(h, g, ph, epi.PATH_MMA4)
            tr, sc = h.scan(12)
            assert h.stats()["block"] == threads
            assert np.array_equal(tr, otr) and np.array_equal(sc, osc)
        # the compacted form's two epilogues (one triplet per lane at a time, or a lane's two
        # triplets in f32x2 instructions)
        h.set_option("path", "mma4c")
        for form, want in (("plain", 1), ("split", 2)):
            h.set_option("mma_form", form)
            check_every_triplet(h, g, ph, epi.PATH_MMA4C)
            tr, sc = h.scan(12)
            assert h.stats()["form"] == want
            assert np.array_equal(tr, otr) and np.array_equal(sc, osc)
        with pytest.raises(epi.Epi3Error) as ei:
            h.set_option("mma_form", "wide")
        assert ei.value.code == epi.ERR_ARG


@pytest.mark.parametrize("form", ["plain", "split"])
def test_compacted_form_derives_each_first_snp_genotype(form):
    # the compacted form counts the two least frequent genotypes of each first SNP and derives
    # the third.  Here the most frequent genotype of several SNPs differs between the classes
    # (controls mostly 0, cases mostly 1) or is genotype 2, and those SNPs dominate the top of
    # the ranking: the pruned scan's top-k (every table cell of one class meeting the same
    # cell of the other in the bound) must still equal the oracle's
    rng = np.random.default_rng(77)
    m, n, n1 = 150, 6000, 2600
    g = rng.binomial(2, rng.uniform(0.05, 0.5, size=m)[:, None], size=(m, n)).astype(np.uint8)
    ph = np.zeros(n, np.uint8)
    ph[rng.choice(n, n1, replace=False)] = 1
    case = ph == 1
    for s in (3, 40, 41, 97):       # majority 0 in controls, 1 in cases
        g[s, ~case] = rng.choice(3, size=(~case).sum(), p=[0.6, 0.3, 0.1])
        g[s, case] = rng.choice(3, size=case.sum(), p=[0.25, 0.55, 0.2])
    for s in (10, 120):             # majority 2 in both classes
        g[s] = rng.choice(3, size=n, p=[0.15, 0.25, 0.6])
    otr, osc, _ = oracle.scan_topk(g, ph, 24)
    with epi.Handle(g, ph) as h:
        h.set_option("path", "mma4c")
        h.set_option("mma_form", form)
        tr, sc = h.scan(24)
        assert h.stats()["k2_prune_bound"] > 0
    assert np.array_equal(tr, otr), (tr[:6], otr[:6])
    assert np.array_equal(sc, osc)
