"""Host logic of the single-tree walk's autotuner (no GPU): it times every walk
shape, keeps the fastest, caches the choice per GPU name and size class, and
answers a repeated call from the cache without timing again."""
import json

from paper_1902_08083_gb300 import autotune


class _FakeTree:
    def __init__(self, n_gas, n_src):
        self.n_gas, self.n_src = n_gas, n_src


def _timer(costs, calls):
    def t(tree, theta, tau_ref, sink_idx, shape, repeats):
        calls.append(shape)
        return costs[shape]
    return t


def test_tune_walk_picks_fastest_and_caches(tmp_path, monkeypatch):
    monkeypatch.setattr(autotune, "_device_name", lambda: "fake GPU")
    costs = {(3, 0): 5.0, (2, 0): 7.0, (1, 32): 4.5, (1, 64): 6.0, (1, 128): 9.0}
    calls = []
    cache = str(tmp_path / "tune.json")
    tree = _FakeTree(1 << 20, 1 << 12)
    r = autotune.tune_walk(tree, 0.6, 0.1, cache_path=cache, timer=_timer(costs, calls))
    assert (r["walk_variant"], r["sinks_per_warp"]) == (1, 32) and r["ms"] == 4.5
    assert not r["cached"] and sorted(calls) == sorted(autotune.WALK_SHAPES)
    assert set(r["table"]) == {f"v{v}_{s}" for v, s in autotune.WALK_SHAPES}
    stored = json.load(open(cache))
    assert list(stored) == ["fake GPU|walk_sinks2^20_src2^12"]
    # the same size class comes from the cache, without timing
    calls.clear()
    again = autotune.tune_walk(_FakeTree((1 << 20) + 5, 5000), 0.6, 0.1, cache_path=cache,
                               timer=_timer(costs, calls))
    assert again["cached"] and calls == [] and again["walk_variant"] == 1
    # another size class is timed again
    autotune.tune_walk(_FakeTree(1 << 16, 1 << 12), 0.6, 0.1, cache_path=cache,
                       timer=_timer(costs, calls))
    assert len(calls) == len(autotune.WALK_SHAPES) and len(json.load(open(cache))) == 2


def test_tune_walk_without_cache(tmp_path, monkeypatch):
    monkeypatch.setattr(autotune, "_device_name", lambda: "fake GPU")
    costs = {s: 1.0 + i for i, s in enumerate(autotune.WALK_SHAPES)}
    cache = tmp_path / "none.json"
    r = autotune.tune_walk(_FakeTree(1000, 10), 0.6, 0.1, cache_path=str(cache),
                           use_cache=False, timer=_timer(costs, []))
    assert (r["walk_variant"], r["sinks_per_warp"]) == autotune.WALK_SHAPES[0]
    assert not cache.exists()
