"""The library's device-memory cache (needs an sm_103 GPU): handles created and destroyed one
after another take their buffers from blocks earlier handles released.  Results must not depend
on it: a sequence of data sets of different shapes, scanned with fresh handles (every later
handle reusing blocks, some of them larger than it needs), gives the oracle's answers, and the
same sequence in a process with the cache off (EPI3_CACHE_MB=0) gives identical bytes."""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
import oracle_pins as pins
import paper_2201_10956_gb300 as epi

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SHAPES = [(60, 900, 400), (33, 2000, 700), (75, 600, 300), (40, 3000, 1500), (60, 900, 400),
          (90, 257, 0)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_10956_gb300 import build as B
    B.build()
    epi.load()


def run_sequence():
    out = []
    for t, (m, n, n1) in enumerate(SHAPES):
        g, ph = pins.tiny_data(m, n, n1, seed=950 + t)
        for path in ("mma4c", "popc8"):
            with epi.Handle(g, ph) as h:
                h.set_option("path", path)
                tr, sc = h.scan(7)
            out.append((tr, sc))
    return out


def test_reused_blocks_give_the_oracle_answers():
    got = run_sequence()
    for t, (m, n, n1) in enumerate(SHAPES):
        g, ph = pins.tiny_data(m, n, n1, seed=950 + t)
        otr, osc, _ = oracle.scan_topk(g, ph, 7)
        for tr, sc in got[2 * t:2 * t + 2]:
            assert np.array_equal(tr, otr) and np.array_equal(sc, osc)


def test_cache_off_gives_identical_results(tmp_path):
    code = (
        "import sys, numpy as np\n"
        f"sys.path[:0] = [{ROOT!r}, {os.path.join(ROOT, 'tests')!r}]\n"
        "import test_gpu_memcache as t\n"
        "import paper_2201_10956_gb300 as epi\n"
        "epi.load()\n"
        "res = t.run_sequence()\n"
        f"np.savez({str(tmp_path / 'off.npz')!r}, *[a for r in res for a in r])\n")
    env = dict(os.environ, EPI3_CACHE_MB="0")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    off = np.load(tmp_path / "off.npz")
    on = [a for res in run_sequence() for a in res]
    assert len(off.files) == len(on)
    for q, a in enumerate(on):
        assert np.array_equal(off[f"arr_{q}"], a)
