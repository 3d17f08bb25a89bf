"""Autotuner table logic without a GPU: signatures, choice of the fastest
candidate, ties, caching and the JSON round trip."""
import json
import types

from paper_2211_00645_gb300.tune import Tuner, candidates, signature


def _items(*shapes, geo=(35.0, 0.3, 0.1)):
    out = []
    for (n, r, c) in shapes:
        p = types.SimpleNamespace(nscan=n, nrows=r, ncols=c, theta_deg=geo[0], step=geo[1], pixel=geo[2])
        out.append({"plan": p})
    return out


def test_signature_classes():
    a = _items((100, 256, 512), (150, 256, 1024))
    b = _items((110, 256, 512), (140, 256, 1024))           # same order of magnitude
    c = _items((400, 1024, 2048), (150, 256, 1024))
    d = _items((100, 256, 512), (150, 256, 1024), geo=(45.0, 0.2, 0.115))
    assert signature(a, 152) == signature(b, 152)
    assert signature(a, 152) != signature(c, 152)
    assert signature(a, 152) != signature(d, 152)
    assert signature(a, 152) != signature(a, 148)


def test_tune_picks_fastest_and_caches(tmp_path):
    calls = []

    def timer(k, c):
        calls.append((k, c))
        return 100.0 + abs(k - 64) + 10 * abs(c - 3)

    path = str(tmp_path / "tune.json")
    t = Tuner(path)
    items = _items((100, 256, 512))
    e = t.tune(items, timer=timer, sm_count=152)
    assert (e["kchunk"], e["ctas_per_sm"]) == (64, 3)
    assert len(calls) == len(candidates())
    assert t.best(items, 152) == (64, 3)
    calls.clear()
    t.tune(items, timer=timer, sm_count=152)                  # cached: no timing
    assert not calls
    t2 = Tuner(path)                                           # JSON round trip
    assert t2.best(items, 152) == (64, 3)
    with open(path) as f:
        assert signature(items, 152) in json.load(f)
    assert t2.best(_items((400, 1024, 2048)), 152) is None


def test_ties_break_to_the_smaller_candidate():
    t = Tuner()
    e = t.record("x", {(128, 4): 10.0, (32, 2): 10.0, (64, 3): 11.0})
    assert (e["kchunk"], e["ctas_per_sm"]) == (32, 2)
