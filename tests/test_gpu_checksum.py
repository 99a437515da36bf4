"""Every table of a full scan, at any size (needs an sm_103 GPU): epi3_scan_checksum sums a hash
of each counted table, so two counting forms agree table by table iff their sums agree (up to
a 2^-64 collision).  On small inputs and over all 1.8e8 tables of the 1024 x 8192 workload the
sum is checked against the same hash of the oracle's tables; at the larger workloads the
tensor-core forms are also checked against the 8-cell POPC form over all C(M, 3) tables."""
import concurrent.futures as cf

import numpy as np
import pytest

import gen
import oracle
import oracle_pins as pins
from paper_2201_10956_gb300 import build as B
import paper_2201_10956_gb300 as epi

pytestmark = pytest.mark.gpu

PATHS = {"popc": epi.PATH_POPC, "popc8": epi.PATH_POPC8, "mma": epi.PATH_MMA,
         "mma16": epi.PATH_MMA16, "mma4": epi.PATH_MMA4, "mma4c": epi.PATH_MMA4C}
M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


@pytest.fixture(scope="module", autouse=True)
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    return epi.load()


def mix64(z):
    # splitmix64 finaliser, elementwise on uint64 (arithmetic mod 2^64)
    z = z + np.uint64(0x9E3779B97F4A7C15)
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def checksum_of(trip, tab):
    """The library's table hash (documented with epi3_scan_checksum) of [n, 3] triplets and
    their [n, 2, 27] tables, summed mod 2^64."""
    with np.errstate(over="ignore"):
        t = np.ascontiguousarray(np.asarray(tab).transpose(2, 1, 0)).astype(np.uint64)  # [27][2][n]
        f = np.zeros(len(trip), dtype=np.uint64)
        for q in range(27):
            f *= np.uint64(0x100000001B3)
            f += t[q, 0]
            f += t[q, 1] << np.uint64(32)
        tr = trip.astype(np.uint64)
        key = (tr[:, 0] << np.uint64(42)) | (tr[:, 1] << np.uint64(21)) | tr[:, 2]
        h = mix64(f ^ mix64(key))
        return int(h.sum(dtype=np.uint64)), len(trip)


@pytest.mark.parametrize("m,n,n1", [(12, 300, 140), (40, 700, 300), (33, 20000, 7000),
                                    (9, 257, 0)])
def test_checksum_equals_oracle_tables(m, n, n1):
    g, ph = pins.tiny_data(m, n, n1, seed=900 + m)
    trip = pins.all_triplets(m)
    want = checksum_of(trip, oracle.tables(g, ph, trip))
    with epi.Handle(g, ph) as h:
        for name, pid in PATHS.items():
            assert h.scan_checksum(pid) == want, name
        h.set_option("path", "mma4")
        for form in ("plain", "split"):
            h.set_option("mma_form", form)
            assert h.scan_checksum(epi.PATH_MMA4) == want, form
            assert h.scan_checksum(epi.PATH_MMA4C) == want, form
        # the handle still scans normally afterwards
        tr, sc = h.scan(5)
    otr, osc, _ = oracle.scan_topk(g, ph, 5)
    assert np.array_equal(tr, otr) and np.array_equal(sc, osc)


def test_checksum_sees_one_changed_genotype():
    g, ph = pins.tiny_data(20, 400, 200, seed=5)
    g2 = g.copy()
    g2[7, 123] = (g2[7, 123] + 1) % 3
    with epi.Handle(g, ph) as h1, epi.Handle(g2, ph) as h2:
        a, b = h1.scan_checksum(epi.PATH_MMA4), h2.scan_checksum(epi.PATH_MMA4)
    assert a[1] == b[1] == 20 * 19 * 18 // 6 and a[0] != b[0]


def triplets_of_first(m, i0, i1):
    """Every triplet (i, j, k), i0 <= i < i1, i < j < k < m, in (i, j, k) order."""
    out = []
    for i in range(i0, i1):
        a, b = np.triu_indices(m - i - 1, 1)
        out.append(np.stack([np.full(a.size, i), a + i + 1, b + i + 1], axis=1).astype(np.int32))
    return np.concatenate(out) if out else np.zeros((0, 3), np.int32)


def oracle_checksum_all(g, ph, chunk=1_500_000):
    """checksum_of over all C(M, 3) oracle tables, streamed in chunks of first SNPs (the oracle
    counts on every host core while earlier chunks are hashed on worker threads)."""
    m = g.shape[0]
    bounds, i, acc = [0], 0, 0
    while i < m - 2:
        acc += (m - i - 1) * (m - i - 2) // 2
        i += 1
        if acc >= chunk or i == m - 2:
            bounds.append(i)
            acc = 0
    total, count = 0, 0
    with cf.ThreadPoolExecutor(max_workers=4) as ex:
        futs = []
        for a, b in zip(bounds[:-1], bounds[1:]):
            trip = triplets_of_first(m, a, b)
            futs.append(ex.submit(checksum_of, trip, oracle.tables(g, ph, trip)))
            if len(futs) > 6:
                h, n = futs.pop(0).result()
                total, count = (total + h) % (1 << 64), count + n
        for fu in futs:
            h, n = fu.result()
            total, count = (total + h) % (1 << 64), count + n
    return total, count


@pytest.mark.slow
def test_medium_workload_all_tables_equal_oracle():
    # all 178,433,024 tables of the 1024 x 8192 workload, counted sample by sample by the oracle
    # (a few minutes on the host cores), against every counting form of the library
    d = gen.make_config("medium")
    want = oracle_checksum_all(d.genotypes, d.phenotype)
    assert want[1] == 1024 * 1023 * 1022 // 6
    with epi.Handle(d.genotypes, d.phenotype) as h:
        assert h.scan_checksum(epi.PATH_POPC8) == want
        for form in ("plain", "split"):
            h.set_option("mma_form", form)
            assert h.scan_checksum(epi.PATH_MMA4) == want, form
            assert h.scan_checksum(epi.PATH_MMA4C) == want, form


@pytest.mark.parametrize("config", ["medium", "large", "stress"])
def test_full_size_tables_agree(config):
    # all C(M, 3) tables of the workload: every tensor-core kind and both kernel forms against
    # the 8-cell POPC form
    d = gen.make_config(config)
    m = d.genotypes.shape[0]
    with epi.Handle(d.genotypes, d.phenotype) as h:
        ref = h.scan_checksum(epi.PATH_POPC8)
        assert ref[1] == m * (m - 1) * (m - 2) // 6
        for name in ("mma4", "mma", "mma4c"):
            assert h.scan_checksum(PATHS[name]) == ref, name
        h.set_option("mma_form", "split" if config == "large" else "plain")  # the other form
        assert h.scan_checksum(epi.PATH_MMA4) == ref
        h.set_option("mma_form", "split")
        assert h.scan_checksum(epi.PATH_MMA4C) == ref
        h.set_option("mma_form", "plain")
        assert h.scan_checksum(epi.PATH_MMA4C) == ref


@pytest.mark.parametrize("name", ["popc8", "mma4", "mma4c"])
def test_retried_scan_restarts_the_checksum(monkeypatch, name):
    # a 128-entry candidate list overflows, so the scan is retried with a larger one; the
    # retry counts every table again and the checksum must count it once
    g, ph = pins.tiny_data(90, 1500, 700, seed=17)
    trip = pins.all_triplets(90)
    want = checksum_of(trip, oracle.tables(g, ph, trip))
    monkeypatch.setenv("EPI3_FAULT", "cand")
    with epi.Handle(g, ph) as h:
        assert h.scan_checksum(PATHS[name]) == want
        h.set_option("path", name)
        tr, sc = h.scan(20)
    otr, osc, _ = oracle.scan_topk(g, ph, 20)
    assert np.array_equal(tr, otr) and np.array_equal(sc, osc)
