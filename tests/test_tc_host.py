"""Host logic of the T_c bracket (paper_1911_12954_gb300.tc), without a GPU: the crossing
search on a temperature grid and the narrowing of the interval round by round."""

import pytest


def test_tc_crossing_logic():
    """Host logic of the T_c bracket: the first adjacent pair where X falls through 1.5."""
    from paper_1911_12954_gb300.tc import crossing
    assert crossing([6.0, 6.5, 7.0], [2.0, 1.9, 1.0]) == 1
    assert crossing([6.0, 6.5, 7.0], [2.0, 1.5, 1.0]) == 0
    assert crossing([6.0, 6.5, 7.0], [1.2, 1.1, 1.0]) is None
    with pytest.raises(ValueError):
        crossing([6.0, 5.0], [2.0, 1.0])
    with pytest.raises(ValueError):
        crossing([6.0], [2.0])


def test_tc_bracket_rounds_narrow_the_interval(monkeypatch):
    """bracket_tc with X replaced by a step at 6.6503 (no GPU): each round keeps the
    sub-interval that holds the step and divides the width by batch - 1."""
    import numpy as np

    import paper_1911_12954_gb300.tc as tc
    calls = []

    def fake_sweep(temps, *a, **k):
        calls.append(np.array(temps))
        return np.where(np.asarray(temps) < 6.6503, 2.0, 1.0)

    monkeypatch.setattr(tc, "x_sweep", fake_sweep)
    lo, hi, hist = tc.bracket_tc(8, 6.6, 6.7, batch=5, rounds=3)
    assert lo < 6.6503 <= hi
    assert hi - lo == pytest.approx(0.1 / 4 ** 3, rel=1e-9)
    assert len(calls) == 3 and all(len(c) == 5 for c in calls)


def test_largest_jump():
    """The adjacent pair with the largest change, signed; argument checks."""
    from paper_1911_12954_gb300.tc import largest_jump
    i, d = largest_jump([1.0, 2.0, 3.0, 4.0], [-1.00, -1.01, -0.95, -0.949])
    assert i == 1 and d == pytest.approx(0.06)
    with pytest.raises(ValueError):
        largest_jump([2.0, 1.0], [0.0, 1.0])
