"""Autotuner logic (no GPU): candidates are measured, the fastest wins, a
failing candidate is skipped, and the winner is cached per key."""
import json

import pytest

from paper_1705_06965_b300 import autotune


def test_grid_is_the_product():
    g = autotune.grid(a=(1, 2), b=("x", "y", "z"))
    assert len(g) == 6 and {"a": 2, "b": "z"} in g


def test_tune_picks_fastest_and_caches(tmp_path, monkeypatch):
    monkeypatch.setattr(autotune, "_machine_key", lambda: "testbox")
    cache = str(tmp_path / "c.json")
    t = autotune.Autotuner(cache)
    calls = []

    def run(cfg):
        calls.append(cfg["k"])
        if cfg["k"] == 3:
            raise RuntimeError("cannot run here")
        return abs(cfg["k"] - 2) + 0.5

    best, table = t.tune(t.key("w", n=1), autotune.grid(k=(0, 1, 2, 3)), run, repeats=2)
    assert best == {"k": 2}
    assert len(calls) == 7                     # 3 candidates x 2 repeats + 1 failure
    assert any(len(r) == 3 for r in table)     # the failed candidate is recorded
    saved = json.load(open(cache))
    assert saved[t.key("w", n=1)]["best"] == {"k": 2}
    # a second tuner reads the cache and does not measure again
    t2 = autotune.Autotuner(cache)
    best2, _ = t2.tune(t2.key("w", n=1), autotune.grid(k=(0, 1)), lambda c: pytest.fail("measured"))
    assert best2 == {"k": 2}
    assert t2.lookup(t2.key("w", n=2)) is None


def test_no_candidate_runs(tmp_path, monkeypatch):
    monkeypatch.setattr(autotune, "_machine_key", lambda: "testbox")
    t = autotune.Autotuner(str(tmp_path / "c.json"))

    def bad(cfg):
        raise RuntimeError("no")

    with pytest.raises(RuntimeError):
        t.tune(t.key("x"), [{"a": 1}], bad)
