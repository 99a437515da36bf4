"""The scan-path tuner: whatever it picks, the answer is the oracle's.

Path "auto" times every form that serves the shape on a slice of the pairs and keeps the
fastest per (M / 64, N / 1024) bucket; the batch measures its tensor launch's form on the first
scan.  These tests force each choice (through the tuning cache file, the "autotune" option and
EPI3_BATCH_FORM) and compare every result with the oracle."""
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


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2201_10956_gb300 import build as B
    B.build()


def _oracle_equal(g, ph, tr, sc, k):
    otr, osc, _ = oracle.scan_topk(g, ph, k)
    assert np.array_equal(tr, otr)
    assert np.array_equal(sc, osc)


def test_auto_picks_a_serving_form_and_matches_oracle():
    g, ph = pins.tiny_data(150, 2500, 1100, seed=31)
    with epi.Handle(g, ph) as h:
        tr, sc = h.scan(8)
        assert h.stats()["path"] in (epi.PATH_POPC8, epi.PATH_MMA4C, epi.PATH_MMA4)
        _oracle_equal(g, ph, tr, sc, 8)
        tr2, sc2 = h.scan(8)  # tuned: no new measurement, same answer
        assert np.array_equal(tr, tr2) and np.array_equal(sc, sc2)


def test_autotune_off_takes_the_compacted_form():
    g, ph = pins.tiny_data(90, 1800, 700, seed=32)
    with epi.Handle(g, ph) as h:
        h.set_option("autotune", "0")
        tr, sc = h.scan(6)
        assert h.stats()["path"] == epi.PATH_MMA4C
        _oracle_equal(g, ph, tr, sc, 6)


@pytest.mark.parametrize("name,code", [("mma4", epi.PATH_MMA4), ("mma4c", epi.PATH_MMA4C)])
def test_explicit_tensor_path_tunes_only_its_form(name, code):
    g, ph = pins.tiny_data(70, 2100, 1000, seed=33)
    with epi.Handle(g, ph) as h:
        h.set_option("path", name)
        tr, sc = h.scan(5)
        st = h.stats()
        assert st["path"] == code and st["form"] in (1, 2)
        _oracle_equal(g, ph, tr, sc, 5)
        for form, want in (("plain", 1), ("split", 2)):
            h.set_option("mma_form", form)
            tr2, sc2 = h.scan(5)
            assert h.stats()["form"] == want
            assert np.array_equal(tr2, tr) and np.array_equal(sc2, sc)


_CHILD = r'''
import sys
sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
import numpy as np
import oracle_pins as pins
import paper_2201_10956_gb300 as epi
g, ph = pins.tiny_data(200, 3100, 1400, seed=34)
with epi.Handle(g, ph) as h:
    tr, sc = h.scan(6)
    np.save({out!r}, np.concatenate([tr.astype(np.float64).ravel(), sc]))
    print(h.stats()["path"], h.stats()["form"])
'''


def _child(cache, out):
    env = dict(os.environ, EPI3_TUNE_CACHE=str(cache))
    code = _CHILD.format(root=ROOT, tests=os.path.join(ROOT, "tests"), out=str(out))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    path, form = (int(x) for x in r.stdout.split()[-2:])
    return path, form, np.load(out)


def test_tune_cache_forces_each_choice(tmp_path):
    cache = tmp_path / "tune.tsv"
    out = tmp_path / "res.npy"
    path0, _, res0 = _child(cache, out)  # measures, and appends its bucket's line
    lines = [l.split("\t") for l in cache.read_text().splitlines() if l.strip()]
    mine = [l for l in lines if len(l) == 7 and l[6] == "1"]
    assert mine and int(mine[-1][4]) == path0
    g, ph = pins.tiny_data(200, 3100, 1400, seed=34)
    otr, osc, _ = oracle.scan_topk(g, ph, 6)
    ref = np.concatenate([otr.astype(np.float64).ravel(), osc])
    assert np.array_equal(res0, ref)
    for path, form in ((epi.PATH_POPC8, 0), (epi.PATH_MMA4C, 1), (epi.PATH_MMA4C, 2),
                       (epi.PATH_MMA4, 1), (epi.PATH_MMA4, 2)):
        row = list(mine[-1])
        row[4], row[5] = str(path), str(form)
        cache.write_text("\t".join(row) + "\n")
        got_path, got_form, res = _child(cache, out)
        assert (got_path, got_form) == (path, form)
        assert np.array_equal(res, ref), (path, form)


@pytest.mark.parametrize("form", [None, "plain", "split"])
def test_batch_form_measured_or_forced(monkeypatch, form):
    monkeypatch.setenv("EPI3_BATCH_PATH", "mma")
    if form:
        monkeypatch.setenv("EPI3_BATCH_FORM", form)
    data = [pins.tiny_data(int(m), int(n), int(n) // 3, seed=40 + c)
            for c, (m, n) in enumerate([(30, 500), (64, 1200), (45, 900)])]
    with epi.Batch(data) as b:
        forms = b.forms()
        assert np.all(forms == ({"plain": 1, "split": 2}[form] if form else -1))
        for rep in range(2):
            tr, sc = b.scan(5)
            for c, (g, ph) in enumerate(data):
                _oracle_equal(g, ph, tr[c], sc[c], 5)
        forms = b.forms()
        assert np.all(forms == forms[0]) and forms[0] in (1, 2)
        if form:
            assert forms[0] == {"plain": 1, "split": 2}[form]
