"""Batched scan of many uneven cohorts (needs an sm_103 GPU): every cohort's answer must be
the oracle's, whichever form the tuner (or EPI3_BATCH_PATH) gives each cohort."""
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


def small_cohorts(seed=3):
    rng = np.random.default_rng(seed)
    out = []
    for c in range(7):
        m = int(rng.integers(20, 140))
        n = int(rng.integers(60, 1500))
        n1 = int(rng.integers(0, n + 1)) if c != 3 else 0
        out.append(pins.tiny_data(m, n, n1, seed=seed * 100 + c))
    return out


@pytest.mark.parametrize("force", [None, "mma", "mma4c", "popc8"])
def test_batch_matches_oracle(monkeypatch, force):
    if force:
        monkeypatch.setenv("EPI3_BATCH_PATH", force)
    data = small_cohorts()
    k = 7
    with epi.Batch(data) as b:
        paths = b.paths()
        if force:
            want = {"mma": epi.PATH_MMA4, "mma4c": epi.PATH_MMA4C, "popc8": epi.PATH_POPC8}[force]
            assert np.all(paths == want)
        for rep in range(2):  # the second scan replays the captured graph
            tr, sc = b.scan(k)
            for c, (g, ph) in enumerate(data):
                otr, osc, _ = oracle.scan_topk(g, ph, k)
                assert np.array_equal(tr[c], otr), (force, c)
                assert np.array_equal(sc[c], osc), (force, c)
        st = b.stats()
        assert st["n_triplets"] == sum(g.shape[0] * (g.shape[0] - 1) * (g.shape[0] - 2) // 6
                                       for g, _ in data)


def test_batch_top_k_change_and_one_shot():
    data = small_cohorts(seed=4)
    with epi.Batch(data) as b:
        tr3, sc3 = b.scan(3)
        tr9, sc9 = b.scan(9)
    assert np.array_equal(tr9[:, :3], tr3) and np.array_equal(sc9[:, :3], sc3)
    tr, sc = epi.scan_batch(data, 9)
    assert np.array_equal(tr, tr9) and np.array_equal(sc, sc9)


def test_batch_device_inputs():
    import torch
    data = small_cohorts(seed=5)
    with epi.Batch(data) as b:
        tr_h, sc_h = b.scan(5)
    dev = [(torch.from_numpy(g).cuda(), torch.from_numpy(p).cuda()) for g, p in data]
    with epi.Batch(dev) as b:
        tr_d, sc_d = b.scan(5)
        torch.cuda.synchronize()
    assert np.array_equal(tr_d.cpu().numpy(), tr_h) and np.array_equal(sc_d.cpu().numpy(), sc_h)


@pytest.mark.slow
def test_batch_config_48_cohorts():
    # the 48-cohort workload: per cohort the oracle rescores the answer exactly, and no triplet
    # of an oracle-scored sample (1e5 random triplets plus every triplet containing the first
    # SNP of the planted triplet) outside the answer scores below its 5th
    cohorts = gen.make_batch(seed=1)
    data = [(d.genotypes, d.phenotype) for d in cohorts]
    with epi.Batch(data) as b:
        tr, sc = b.scan(5)
        paths = b.paths()
    assert set(paths.tolist()) <= {epi.PATH_MMA4, epi.PATH_MMA4C, epi.PATH_POPC8}
    for c, d in enumerate(cohorts):
        g, ph = d.genotypes, d.phenotype
        assert np.array_equal(oracle.scores(g, ph, tr[c]), sc[c])
        assert np.all(np.diff(sc[c]) >= 0)
        assert np.all(tr[c][:, 0] < tr[c][:, 1]) and np.all(tr[c][:, 1] < tr[c][:, 2])
        samp = np.concatenate([gen.random_triplets(d.n_snps, 100_000, seed=c),
                               triplets_with(d.n_snps, int(d.planted[0][0]))])
        ref = oracle.scores(g, ph, samp)
        got = {tuple(t) for t in tr[c]}
        for t in samp[ref < sc[c][-1]]:
            assert tuple(t) in got, (c, t)
        # ties with the 5th score are broken by (i, j, k): none of the sample may precede it
        last = tuple(tr[c][-1])
        for t in samp[ref == sc[c][-1]]:
            assert tuple(t) in got or tuple(t) > last, (c, t)
        with epi.Handle(g, ph) as h:
            htr, hsc = h.scan(5)
        assert np.array_equal(htr, tr[c]) and np.array_equal(hsc, sc[c])


def triplets_with(m, p):
    """Every triplet i<j<k of m SNPs that contains SNP p."""
    rest = np.array([x for x in range(m) if x != p], dtype=np.int32)
    a, b = np.triu_indices(m - 1, 1)
    t = np.stack([rest[a], rest[b], np.full(a.size, p, dtype=np.int32)], axis=1)
    return np.sort(t, axis=1).astype(np.int32)
