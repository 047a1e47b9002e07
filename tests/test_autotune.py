"""Autotuner logic (CPU): candidate validity, selection and the cache."""
import pytest

from paper_2009_13349_gb300 import autotune as A


def test_candidates_are_valid_and_distinct():
    c = A.candidates(152)
    assert len(c) == len({tuple(sorted(x.items())) for x in c})
    for t in c:
        assert A.validate(t) == t


def test_tune_picks_fastest_and_caches(tmp_path):
    costs = {}
    cands = A.candidates(4)
    for i, t in enumerate(cands):
        costs[tuple(sorted(t.items()))] = 10.0 - (i == 5) * 9.0 + 0.01 * i
    calls = []

    def measure(t):
        calls.append(t)
        return costs[tuple(sorted(t.items()))]

    path = str(tmp_path / "tuning.json")
    best, timings = A.get_or_tune("GPU-X", "wl", measure, cands, reps=2, path=path)
    assert best == cands[5]
    assert len(calls) == 2 * len(cands)
    best2, timings2 = A.get_or_tune("GPU-X", "wl", measure, cands, reps=2, path=path)
    assert best2 == best and timings2 is None and len(calls) == 2 * len(cands)
    assert A.load("GPU-Y", "wl", path) is None


def test_validate_rejects_bad_shapes():
    with pytest.raises(ValueError):
        A.validate({"deep_threads": 384})
    with pytest.raises(ValueError):
        A.validate({"small_cap": 8})
