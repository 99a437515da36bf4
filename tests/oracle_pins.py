"""Checks that pin the CPU oracle to facts fixed by the paper and by mathematics.

Each check takes an ``oracle.Oracle`` instance so the same checks can run
against deliberately broken copies of the oracle (tests/test_oracle_mutants.py)
and prove that they catch plausible mistakes.  None of these checks reuses the
oracle's own code path as its expected value:

* counts: an independent numpy ``bincount`` of the cell index (Sec. III,
  Fig. 1), brute force over every triplet of tiny inputs;
* K2: exact big-integer factorials, exp(K2) = prod (r+1)! / (r0! r1!) (Eq. 1),
  and hand-worked tables (tests/golden/k2_hand.json);
* log-factorials: math.lgamma;
* ranking: numpy lexsort over every triplet, exact FP64 ties from duplicated
  SNP columns, and recovery of a strongly planted triplet (lowest K2 wins,
  Sec. III);
* pairs (Eq. 1 for two SNPs, 9 cells): numpy bincount, big-integer K2, and the
  triplet K2 of a monomorphic third SNP, which must equal the pair K2 exactly;
* any order (Eq. 1 for k SNPs, 3^k cells, k up to 6): numpy bincount of the base-3 cell,
  big-integer K2, summing out a SNP gives the lower-order table, orders 2 and 3
  equal the pair and triplet functions bit for bit, a monomorphic last SNP
  gives the lower-order K2 exactly (orders 4, 5, 6), and numpy lexsort over every
  4-, 5- and 6-SNP set of small cases.
"""
from __future__ import annotations

import itertools
import json
import math
import os

import numpy as np

import gen

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def tiny_data(m, n, n_cases, seed, maf=(0.05, 0.5)):
    rng = np.random.default_rng(seed)
    p = rng.uniform(maf[0], maf[1], size=m)
    g = rng.binomial(2, p[:, None], size=(m, n)).astype(np.uint8)
    ph = np.zeros(n, dtype=np.uint8)
    ph[rng.choice(n, size=n_cases, replace=False)] = 1
    return g, ph


def all_triplets(m):
    return np.array(list(itertools.combinations(range(m), 3)), dtype=np.int32).reshape(-1, 3)


def numpy_tables(g, ph, trip):
    """Independent counting: bincount of class*27 + 9 gX + 3 gY + gZ."""
    out = np.empty((len(trip), 2, 27), dtype=np.int64)
    for t, (x, y, z) in enumerate(trip):
        idx = ph.astype(np.int64) * 27 + 9 * g[x].astype(np.int64) + 3 * g[y] + g[z]
        out[t] = np.bincount(idx, minlength=54).reshape(2, 27)
    return out


def exact_k2(table):
    """log of prod_cells (r+1)! / (r0! r1!), an integer, with Python big ints."""
    num = 1
    for c in range(27):
        r0, r1 = int(table[0][c]), int(table[1][c])
        num *= math.factorial(r0 + r1 + 1) // (math.factorial(r0) * math.factorial(r1))
    return math.log(num)


def check_lf(o):
    lf = o.log_factorials(30000)
    assert lf[0] == 0.0 and lf[1] == 0.0
    n = np.array([2, 3, 10, 100, 1000, 5000, 16385, 20001, 30000])
    ref = np.array([math.lgamma(float(v) + 1.0) for v in n])
    assert np.allclose(lf[n], ref, rtol=1e-12, atol=0), (lf[n], ref)


def check_hand_values(o):
    with open(os.path.join(GOLDEN, "k2_hand.json")) as f:
        cases = json.load(f)["cases"]
    tabs = np.zeros((len(cases), 2, 27), dtype=np.int32)
    for t, c in enumerate(cases):
        for cell, (r0, r1) in c["cells"].items():
            tabs[t, 0, int(cell)] = r0
            tabs[t, 1, int(cell)] = r1
    got = o.k2(tabs)
    want = np.array([c["k2"] for c in cases])
    assert np.allclose(got, want, rtol=1e-14, atol=1e-15), (got, want)


def check_k2_bigint(o, seed=3):
    rng = np.random.default_rng(seed)
    tabs = []
    for scale in (1, 3, 30, 300, 3000):
        for _ in range(6):
            t = rng.integers(0, scale + 1, size=(2, 27))
            t[:, rng.random(27) < 0.3] = 0          # some empty cells
            tabs.append(t)
    tabs.append(np.zeros((2, 27), dtype=np.int64))
    one = np.zeros((2, 27), dtype=np.int64)
    one[1, 26] = 20000                                 # one pure cell, large N
    tabs.append(one)
    tabs = np.array(tabs, dtype=np.int32)
    got = o.k2(tabs)
    want = np.array([exact_k2(t) for t in tabs])
    assert np.allclose(got, want, rtol=1e-12, atol=1e-12), np.max(np.abs(got - want))


def check_tables_bruteforce(o):
    for (m, n, n1, seed) in [(5, 1, 0, 1), (6, 33, 10, 2), (9, 64, 40, 3), (12, 100, 37, 4),
                             (7, 65, 65, 5), (8, 97, 0, 6)]:
        g, ph = tiny_data(m, n, n1, seed)
        trip = all_triplets(m)
        got = o.tables(g, ph, trip)
        assert np.array_equal(got, numpy_tables(g, ph, trip)), (m, n)
        # SNPs given out of order: X, Y, Z take the listed roles
        perm = trip[:, [2, 0, 1]]
        assert np.array_equal(o.tables(g, ph, perm), numpy_tables(g, ph, perm))


def check_invariants(o, seed=11):
    g, ph = tiny_data(10, 90, 41, seed)
    trip = all_triplets(10)
    tab = o.tables(g, ph, trip).astype(np.int64)          # [t, 2, 27]
    n1 = int(ph.sum())
    assert np.all(tab[:, 0].sum(1) == 90 - n1) and np.all(tab[:, 1].sum(1) == n1)
    cube = tab.reshape(-1, 2, 3, 3, 3)                    # [t, c, gX, gY, gZ]

    def pair_table(a, b):
        idx = ph.astype(np.int64) * 9 + 3 * g[a].astype(np.int64) + g[b]
        return np.bincount(idx, minlength=18).reshape(2, 3, 3)

    for t, (x, y, z) in enumerate(trip):
        assert np.array_equal(cube[t].sum(3), pair_table(x, y))
        assert np.array_equal(cube[t].sum(2), pair_table(x, z))
        assert np.array_equal(cube[t].sum(1), pair_table(y, z))
        single = np.bincount(ph.astype(np.int64) * 3 + g[x], minlength=6).reshape(2, 3)
        assert np.array_equal(cube[t].sum((2, 3)), single)


def check_symmetries(o, seed=12):
    g, ph = tiny_data(9, 120, 50, seed)
    trip = all_triplets(9)
    base = o.scores(g, ph, trip)
    ref = np.array([exact_k2(t) for t in numpy_tables(g, ph, trip)])
    assert np.allclose(base, ref, rtol=1e-13)
    for perm in itertools.permutations(range(3)):
        assert np.allclose(o.scores(g, ph, trip[:, list(perm)]), base, rtol=1e-12)
    g2 = g.copy()
    g2[4] = 2 - g2[4]                                     # relabel 0 <-> 2 at one SNP
    assert np.allclose(o.scores(g2, ph, trip), base, rtol=1e-12)
    assert np.allclose(o.scores(g, 1 - ph, trip), base, rtol=1e-12)   # swap classes


def check_monomorphic(o, seed=13):
    g, ph = tiny_data(6, 77, 30, seed)
    g[5] = 0                                              # SNP 5 monomorphic
    trip = np.array([[0, 1, 5], [2, 3, 5], [1, 4, 5]], dtype=np.int32)
    got = o.scores(g, ph, trip)
    for t, (x, y, _) in enumerate(trip):
        idx = ph.astype(np.int64) * 9 + 3 * g[x].astype(np.int64) + g[y]
        pt = np.bincount(idx, minlength=18).reshape(2, 9)
        num = 1
        for c in range(9):
            r0, r1 = int(pt[0, c]), int(pt[1, c])
            num *= math.factorial(r0 + r1 + 1) // (math.factorial(r0) * math.factorial(r1))
        assert math.isclose(got[t], math.log(num), rel_tol=1e-13)


def check_degenerate(o):
    # a single class: every term is log(r + 1)
    for n1 in (0, 40):
        g, ph = tiny_data(5, 40, n1, 21)
        trip = all_triplets(5)
        tab = numpy_tables(g, ph, trip)
        want = np.array([sum(math.log(int(t[0, c] + t[1, c]) + 1) for c in range(27)) for t in tab])
        assert np.allclose(o.scores(g, ph, trip), want, rtol=1e-13)
    # M = 3: the scan returns the only triplet with its score
    g, ph = tiny_data(3, 50, 20, 22)
    tr, sc, _ = o.scan_topk(g, ph, 1)
    assert tr.tolist() == [[0, 1, 2]]
    assert math.isclose(sc[0], exact_k2(numpy_tables(g, ph, [[0, 1, 2]])[0]), rel_tol=1e-13)
    # one sample
    g, ph = tiny_data(4, 1, 1, 23)
    assert np.allclose(o.scores(g, ph, all_triplets(4)), math.log(2.0), rtol=1e-15)


def check_scan_bruteforce(o):
    for (m, n, n1, seed, k) in [(11, 70, 30, 31, 7), (14, 129, 64, 32, 20), (9, 31, 31, 33, 84)]:
        g, ph = tiny_data(m, n, n1, seed)
        trip = all_triplets(m)
        s = np.array([exact_k2(t) for t in numpy_tables(g, ph, trip)])
        s_oracle = o.scores(g, ph, trip)
        assert np.allclose(s_oracle, s, rtol=1e-13)
        order = np.lexsort((trip[:, 2], trip[:, 1], trip[:, 0], s_oracle))
        tr, sc, _ = o.scan_topk(g, ph, k)
        assert np.array_equal(tr, trip[order[:k]])
        assert np.array_equal(sc, s_oracle[order[:k]])
        assert np.all(np.diff(sc) >= 0)


def check_ties(o):
    # duplicated columns give bit-identical tables, hence exactly equal K2;
    # equal K2 is ordered by (i, j, k).
    d = gen.make_dataset(30, 600, 300, (0.3, 0.5), 1, seed=5, odds_ratio=10.0)
    g = d.genotypes.copy()
    i, j, k = d.planted[0]
    free = [c for c in range(30) if c not in (i, j, k)]
    dup = free[-1]
    g[dup] = g[k]
    tr, sc, _ = o.scan_topk(g, d.phenotype, 4)
    want = sorted([tuple(sorted((i, j, k))), tuple(sorted((i, j, dup)))])
    assert [tuple(t) for t in tr[:2]] == want
    assert sc[0] == sc[1]
    assert sc[2] > sc[1]


def check_planted_recovery(o):
    # A strongly planted interaction scores lowest (Sec. III: lowest K2 wins).
    for seed in range(1, 6):
        d = gen.make_dataset(40, 800, 400, (0.3, 0.5), 1, seed=seed, odds_ratio=10.0)
        tr, sc, _ = o.scan_topk(d.genotypes, d.phenotype, 3)
        assert tuple(tr[0]) == d.planted[0], (seed, tr[0], d.planted[0])


# ---------------------------------------------------------------- pairs (Eq. 1, two SNPs)
def all_pairs(m):
    return np.array(list(itertools.combinations(range(m), 2)), dtype=np.int32).reshape(-1, 2)


def numpy_pair_tables(g, ph, pairs):
    """Independent counting: bincount of class*9 + 3 gX + gY."""
    out = np.empty((len(pairs), 2, 9), dtype=np.int64)
    for t, (x, y) in enumerate(pairs):
        idx = ph.astype(np.int64) * 9 + 3 * g[x].astype(np.int64) + g[y]
        out[t] = np.bincount(idx, minlength=18).reshape(2, 9)
    return out


def exact_pair_k2(table):
    num = 1
    for c in range(9):
        r0, r1 = int(table[0][c]), int(table[1][c])
        num *= math.factorial(r0 + r1 + 1) // (math.factorial(r0) * math.factorial(r1))
    return math.log(num)


def check_pair_tables_bruteforce(o):
    for (m, n, n1, seed) in [(7, 53, 20, 41), (5, 130, 129, 42)]:
        g, ph = tiny_data(m, n, n1, seed)
        pairs = all_pairs(m)
        assert np.array_equal(o.pair_tables(g, ph, pairs), numpy_pair_tables(g, ph, pairs))
        rev = pairs[:, ::-1]                                # order matters: cell = 3 gX + gY
        assert np.array_equal(o.pair_tables(g, ph, rev), numpy_pair_tables(g, ph, rev))


def check_pair_scan_bruteforce(o):
    for (m, n, n1, seed, k) in [(12, 90, 40, 43, 9), (9, 33, 11, 44, 36), (20, 257, 128, 45, 50)]:
        g, ph = tiny_data(m, n, n1, seed)
        pairs = all_pairs(m)
        s = np.array([exact_pair_k2(t) for t in numpy_pair_tables(g, ph, pairs)])
        tr, sc, _ = o.scan_pairs_topk(g, ph, k)
        assert np.allclose(sc, np.sort(s)[:k], rtol=1e-13)
        # order: K2 ascending, then (i, j); the oracle's own FP64 values decide exact ties
        full_t, full_s, _ = o.scan_pairs_topk(g, ph, len(pairs))
        order = np.lexsort((full_t[:, 1], full_t[:, 0], full_s))
        assert np.array_equal(order, np.arange(len(pairs)))
        assert np.array_equal(tr, full_t[:k]) and np.array_equal(sc, full_s[:k])
        assert {tuple(p) for p in full_t} == {tuple(p) for p in pairs}


def check_pair_vs_triplet(o, seed=46):
    # a monomorphic third SNP reduces a triplet's 27-cell table to the pair's 9 cells (the
    # other 18 are empty and add exactly 0.0), so its K2 is the pair's, bit for bit
    g, ph = tiny_data(8, 150, 70, seed)
    g[7] = 0
    pt, ps, _ = o.scan_pairs_topk(g[:7], ph, 21)
    trip = np.concatenate([pt, np.full((len(pt), 1), 7, dtype=np.int32)], axis=1)
    assert np.array_equal(o.scores(g, ph, trip), ps)


def check_pair_ties_and_degenerate(o):
    g, ph = tiny_data(10, 200, 90, 47)
    g[8] = g[2]          # pairs (2, x), (8, x) with x on the same side of both: equal tables
    tr, sc, _ = o.scan_pairs_topk(g, ph, 45)
    pos = {tuple(p): r for r, p in enumerate(tr)}
    for x in (0, 1, 9):
        a, b = tuple(sorted((2, x))), tuple(sorted((8, x)))
        assert a in pos and b in pos          # 45 = every pair of 10 SNPs
        assert sc[pos[a]] == sc[pos[b]]
        assert (pos[a] < pos[b]) == (a < b)
    g2, ph2 = tiny_data(2, 40, 15, 48)                    # M = 2: the only pair
    tr, sc, _ = o.scan_pairs_topk(g2, ph2, 1)
    assert tr.tolist() == [[0, 1]]
    assert math.isclose(sc[0], exact_pair_k2(numpy_pair_tables(g2, ph2, [[0, 1]])[0]), rel_tol=1e-13)


# ---------------------------------------------------------------- any order (Eq. 1, k SNPs)
def all_sets(m, order):
    return np.array(list(itertools.combinations(range(m), order)), dtype=np.int32).reshape(-1, order)


def numpy_order_tables(g, ph, sets):
    """Independent counting: bincount of class*3^k + base-3 digits of the genotypes, the
    first SNP most significant."""
    order = sets.shape[1]
    nc = 3 ** order
    out = np.empty((len(sets), 2, nc), dtype=np.int64)
    for t, x in enumerate(sets):
        cell = np.zeros(g.shape[1], dtype=np.int64)
        for snp in x:
            cell = 3 * cell + g[snp].astype(np.int64)
        out[t] = np.bincount(ph.astype(np.int64) * nc + cell, minlength=2 * nc).reshape(2, nc)
    return out


def exact_k2_cells(table):
    """log of prod_cells (r+1)! / (r0! r1!) over any number of cells, with big integers."""
    num = 1
    for r0, r1 in zip(table[0], table[1]):
        r0, r1 = int(r0), int(r1)
        num *= math.factorial(r0 + r1 + 1) // (math.factorial(r0) * math.factorial(r1))
    return math.log(num)


def check_order_tables_bruteforce(o):
    for (m, n, n1, seed, order) in [(7, 61, 25, 51, 4), (6, 130, 129, 52, 4), (6, 40, 17, 53, 5),
                                    (5, 33, 10, 54, 1), (6, 97, 40, 55, 3), (8, 77, 30, 65, 6),
                                    (7, 200, 199, 66, 5)]:
        g, ph = tiny_data(m, n, n1, seed)
        sets = all_sets(m, order)
        want = numpy_order_tables(g, ph, sets)
        assert np.array_equal(o.tables_order(g, ph, sets), want)
        rev = np.ascontiguousarray(sets[:, ::-1])           # roles matter: first SNP = top digit
        assert np.array_equal(o.tables_order(g, ph, rev), numpy_order_tables(g, ph, rev))


def check_order_k2_bigint(o):
    g, ph = tiny_data(7, 90, 41, 56)
    tabs = numpy_order_tables(g, ph, all_sets(7, 4))[:20]
    got = o.k2_cells(tabs)
    want = np.array([exact_k2_cells(t) for t in tabs])
    assert np.allclose(got, want, rtol=1e-13)


def check_order_marginals(o):
    # summing an order-4 table over the last SNP's digit gives the table of the first three
    # SNPs, and over the first SNP's digit the table of the last three
    g, ph = tiny_data(8, 150, 66, 57)
    sets = all_sets(8, 4)
    t4 = o.tables_order(g, ph, sets).reshape(len(sets), 2, 3, 3, 3, 3)
    assert np.array_equal(t4.sum(axis=5).reshape(len(sets), 2, 27),
                          o.tables_order(g, ph, np.ascontiguousarray(sets[:, :3])))
    assert np.array_equal(t4.sum(axis=2).reshape(len(sets), 2, 27),
                          o.tables_order(g, ph, np.ascontiguousarray(sets[:, 1:])))
    n1 = int(ph.sum())
    assert np.all(t4.sum(axis=(2, 3, 4, 5)) == np.array([150 - n1, n1]))


def check_order_matches_lower_orders(o):
    # order 3 and order 2 of the generic functions are the triplet and pair functions exactly
    g, ph = tiny_data(10, 120, 50, 58)
    trip = all_triplets(10)
    assert np.array_equal(o.tables_order(g, ph, trip), o.tables(g, ph, trip))
    tr3, sc3, _ = o.scan_topk(g, ph, 25)
    x3, s3, _ = o.scan_order_topk(g, ph, 3, 25)
    assert np.array_equal(x3, tr3) and np.array_equal(s3, sc3)
    pr, ps, _ = o.scan_pairs_topk(g, ph, 30)
    x2, s2, _ = o.scan_order_topk(g, ph, 2, 30)
    assert np.array_equal(x2, pr) and np.array_equal(s2, ps)


def check_order_monomorphic(o):
    # a monomorphic fourth SNP puts each triplet cell's counts at cell 3 c (the other 54 cells
    # are empty and add exactly 0.0), so the 4-SNP K2 equals the triplet K2 bit for bit
    g, ph = tiny_data(9, 170, 80, 59)
    g[8] = 0
    trip = all_triplets(8)
    quads = np.concatenate([trip, np.full((len(trip), 1), 8, dtype=np.int32)], axis=1)
    assert np.array_equal(o.k2_cells(o.tables_order(g, ph, quads)), o.scores(g, ph, trip))


def check_order_scan_bruteforce(o):
    for (m, n, n1, seed, k) in [(9, 70, 33, 60, 12), (8, 129, 64, 61, 70), (6, 31, 31, 62, 15),
                                (7, 45, 20, 64, 35)]:                    # the last: every set
        g, ph = tiny_data(m, n, n1, seed)
        sets = all_sets(m, 4)
        s = np.array([exact_k2_cells(t) for t in numpy_order_tables(g, ph, sets)])
        s_oracle = o.k2_cells(o.tables_order(g, ph, sets))
        assert np.allclose(s_oracle, s, rtol=1e-13)
        rank = np.lexsort((sets[:, 3], sets[:, 2], sets[:, 1], sets[:, 0], s_oracle))
        x, sc, _ = o.scan_order_topk(g, ph, 4, k)
        assert np.array_equal(x, sets[rank[:k]])
        assert np.array_equal(sc, s_oracle[rank[:k]])


def check_order5_6_scan_bruteforce(o):
    # orders 5 and 6: big-integer K2 of every set, ranked by (K2, indices), against the scan
    for (m, n, n1, seed, order, k) in [(8, 90, 41, 67, 5, 20), (7, 60, 31, 68, 5, 21),
                                       (8, 130, 64, 69, 6, 28), (7, 45, 0, 70, 6, 7)]:
        g, ph = tiny_data(m, n, n1, seed)
        sets = all_sets(m, order)
        s = np.array([exact_k2_cells(t) for t in numpy_order_tables(g, ph, sets)])
        s_oracle = o.k2_cells(o.tables_order(g, ph, sets))
        assert np.allclose(s_oracle, s, rtol=1e-13)
        rank = np.lexsort(tuple(sets[:, t] for t in range(order - 1, -1, -1)) + (s_oracle,))
        x, sc, _ = o.scan_order_topk(g, ph, order, k)
        assert np.array_equal(x, sets[rank[:k]])
        assert np.array_equal(sc, s_oracle[rank[:k]])


def check_order5_6_marginals_and_monomorphic(o):
    # summing an order-5 (order-6) table over the last SNP's digit gives the order-4 (order-5)
    # table of the other SNPs; a monomorphic last SNP leaves the lower-order K2 bit for bit
    g, ph = tiny_data(9, 140, 60, 71)
    for order in (5, 6):
        sets = all_sets(8, order)
        t = o.tables_order(g, ph, sets).reshape((len(sets), 2) + (3,) * order)
        low = o.tables_order(g, ph, np.ascontiguousarray(sets[:, :order - 1]))
        assert np.array_equal(t.sum(axis=order + 1).reshape(len(sets), 2, -1), low)
    g[8] = 0
    for order in (5, 6):
        lower = all_sets(8, order - 1)
        sets = np.concatenate([lower, np.full((len(lower), 1), 8, dtype=np.int32)], axis=1)
        assert np.array_equal(o.k2_cells(o.tables_order(g, ph, sets)),
                              o.k2_cells(o.tables_order(g, ph, lower)))


def check_order_ties(o):
    # a duplicated SNP column gives 4-SNP sets with identical tables: equal K2, ordered by
    # their indices
    # (the copy sits in the same, last, role in both sets, so the cells line up one to one)
    g, ph = tiny_data(9, 200, 95, 63)
    g[8] = g[7]
    x, sc, _ = o.scan_order_topk(g, ph, 4, 126)            # every 4-SNP set of 9
    pos = {tuple(q): r for r, q in enumerate(x)}
    for rest in itertools.combinations(range(7), 3):
        a, b = rest + (7,), rest + (8,)
        assert a in pos and b in pos
        assert sc[pos[a]] == sc[pos[b]]
        assert pos[a] < pos[b]


ALL_CHECKS = [check_lf, check_hand_values, check_k2_bigint, check_tables_bruteforce,
              check_invariants, check_symmetries, check_monomorphic, check_degenerate,
              check_scan_bruteforce, check_ties, check_planted_recovery,
              check_pair_tables_bruteforce, check_pair_scan_bruteforce, check_pair_vs_triplet,
              check_pair_ties_and_degenerate, check_order_tables_bruteforce, check_order_k2_bigint,
              check_order_marginals, check_order_matches_lower_orders, check_order_monomorphic,
              check_order_scan_bruteforce, check_order5_6_scan_bruteforce,
              check_order5_6_marginals_and_monomorphic, check_order_ties]
