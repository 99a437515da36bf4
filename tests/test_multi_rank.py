"""Multi-rank host logic on CPU (gloo, world size 2): the pair-range sharding used by
`bench.py --gpus N` covers every triplet exactly once with balanced work, and merging the
ranks' per-slice top-k by (K2, i, j, k) reproduces the full scan.  Per-slice answers come
from the oracle here (no GPU)."""
import itertools
import os

import numpy as np
import pytest

import bench
import oracle
import oracle_pins as pins


def slice_topk(g, ph, pb, pe, k):
    m = g.shape[0]
    trip = np.array([t for t in itertools.combinations(range(m), 3)
                     if pb <= t[1] * (t[1] - 1) // 2 + t[0] < pe], dtype=np.int32).reshape(-1, 3)
    if len(trip) == 0:
        return []
    s = oracle.scores(g, ph, trip)
    rows = sorted((float(a), *map(int, b)) for a, b in zip(s, trip))
    return rows[:k]


@pytest.mark.parametrize("m,world", [(9, 2), (40, 2), (57, 3), (200, 8)])
def test_shards_partition_triplets(m, world):
    ranges = [bench.shard_pairs(m, world, r) for r in range(world)]
    assert ranges[0][0] == 0 and ranges[-1][1] == m * (m - 1) // 2
    for (a, b), (c, d) in zip(ranges[:-1], ranges[1:]):
        assert b == c and a <= b
    per = []
    for a, b in ranges:
        t = 0
        for p in range(a, b):
            j = int((1 + (1 + 8 * p) ** 0.5) / 2)
            while j * (j - 1) // 2 > p:
                j -= 1
            while (j + 1) * j // 2 <= p:
                j += 1
            t += m - 1 - j
        per.append(t)
    assert sum(per) == m * (m - 1) * (m - 2) // 6
    if m >= 57:
        assert max(per) - min(per) <= m  # balanced to within one pair's triplets


def _rank(rank, world, port, m, n, k, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g, ph = pins.tiny_data(m, n, n // 2, seed=42)
    pb, pe = bench.shard_pairs(m, world, rank)
    rows = slice_topk(g, ph, pb, pe, k)
    gathered = [None] * world
    dist.all_gather_object(gathered, rows)
    if rank == 0:
        merged = bench.merge_topk([r for part in gathered for r in part], k)
        out.put(merged)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_merge_equals_full_scan():
    import socket

    import torch.multiprocessing as mp
    m, n, k, world = 24, 150, 6, 2
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, m, n, k, q)) for r in range(world)]
    for p in procs:
        p.start()
    merged = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    g, ph = pins.tiny_data(m, n, n // 2, seed=42)
    tr, sc, _ = oracle.scan_topk(g, ph, k)
    assert [r[1:] for r in merged] == [tuple(map(int, t)) for t in tr]
    assert np.array_equal(np.array([r[0] for r in merged]), sc)
