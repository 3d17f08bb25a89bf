"""Autotuner table logic without a GPU: signatures, the kernel shapes that
apply to a batch, choice of the fastest candidate, ties, caching and the
JSON round trip."""
import json
import types

from paper_2211_00645_gb300.tune import (FAST_J8X4, GEN_J8X4, PER_J16X2, PER_J32X2, Tuner, candidates, shapes_for,
                                         signature)


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


def test_shapes_for_items():
    """Periodic shapes only when every fast-kernel item shares one family;
    items with z-sum or arg-max outputs do not count (the general kernel
    takes them whatever the shape)."""
    paths = {"per13": (2, 1, 3), "per14": (2, 1, 4), "per12": (2, 1, 2), "fast": (1, 0, 0), "gen": (0, 0, 0)}

    def items(*kinds, zsum=()):
        return [{"plan": k, **({"zsum": 1} if i in zsum else {})} for i, k in enumerate(kinds)]

    def f(its):
        return shapes_for(its, path_of=lambda p: paths[p])

    both = (PER_J32X2, PER_J16X2, FAST_J8X4, GEN_J8X4)
    assert f(items("per13", "per13", "gen")) == both
    assert f(items("per13", "per14")) == (FAST_J8X4, GEN_J8X4)
    assert f(items("per13", "fast")) == (FAST_J8X4, GEN_J8X4)
    assert f(items("per13", "fast", zsum=(1,))) == both
    assert f(items("gen")) == (FAST_J8X4, GEN_J8X4)
    assert f(items("per12", "per12")) == (PER_J32X2, FAST_J8X4, GEN_J8X4)   # no 16-column runs for 1/2


def test_candidates_per_shape():
    c = candidates((16, 64), (2, 3, 4), (PER_J32X2, GEN_J8X4))
    assert c == [(PER_J32X2, 16, 2), (PER_J32X2, 16, 3), (PER_J32X2, 16, 4), (PER_J32X2, 64, 2),
                 (PER_J32X2, 64, 3), (PER_J32X2, 64, 4), (GEN_J8X4, 16, 2)]


def test_tune_picks_fastest_and_caches(tmp_path):
    calls = []

    def timer(sh, k, c):
        calls.append((sh, k, c))
        return 100.0 + abs(k - 64) + 10 * abs(c - 3) + (0 if sh == PER_J16X2 else 5)

    path = str(tmp_path / "tune.json")
    t = Tuner(path)
    items = _items((100, 256, 512))
    shapes = (PER_J32X2, PER_J16X2, FAST_J8X4, GEN_J8X4)
    e = t.tune(items, timer=timer, sm_count=152, shapes=shapes)
    assert (e["shape"], e["kchunk"], e["ctas_per_sm"]) == ("per_j16x2", 64, 3)
    assert len(calls) == len(candidates(shapes=shapes)) == 3 * 15 + 1
    assert "gen_j8x4/16x2" in e["candidates"] and "per_j32x2/64x3" in e["candidates"]
    assert t.best(items, 152) == (PER_J16X2, 64, 3)
    calls.clear()
    t.tune(items, timer=timer, sm_count=152, shapes=shapes)   # cached: no timing
    assert not calls
    t2 = Tuner(path)                                           # JSON round trip
    assert t2.best(items, 152) == (PER_J16X2, 64, 3)
    with open(path) as f:
        assert signature(items, 152) in json.load(f)
    assert t2.best(_items((400, 1024, 2048)), 152) is None


def test_ties_break_to_the_smaller_candidate():
    t = Tuner()
    e = t.record("x", {(FAST_J8X4, 128, 4): 10.0, (FAST_J8X4, 32, 2): 10.0, (PER_J32X2, 16, 2): 10.0,
                       (FAST_J8X4, 64, 3): 11.0})
    assert (e["shape"], e["kchunk"], e["ctas_per_sm"]) == ("fast_j8x4", 32, 2)
