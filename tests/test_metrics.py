"""Hit-classification metrics (Sec. 3, "Hit classification metrics") on hand-built label arrays whose
efficiency and purity follow from the definitions by counting."""
import numpy as np
import pytest

from paper_1911_09340_gb300 import metrics as M


def _turns():
    # 10 hits of turn 0, 6 of turn 1, 4 of turn 2, 3 noise hits
    return np.array([0] * 10 + [1] * 6 + [2] * 4 + [-1] * 3)


def test_perfect_stage():
    t = _turns()
    m = M.stage_metrics(t == 1, t)
    assert (m.turn, m.efficiency, m.purity) == (1, 1.0, 1.0)
    assert (m.n_classified, m.n_largest, m.n_turn_hits) == (6, 6, 6)


def test_mixed_stage_counts():
    t = _turns()
    cls = np.zeros(t.size, bool)
    cls[:7] = True            # 7 of the 10 turn-0 hits
    cls[10:12] = True         # 2 turn-1 hits
    cls[-2:] = True           # 2 noise hits
    m = M.stage_metrics(cls, t)
    assert m.turn == 0
    assert m.efficiency == pytest.approx(7 / 10)
    assert m.purity == pytest.approx(7 / 11)


def test_noise_is_never_the_represented_turn_but_lowers_purity():
    t = _turns()
    cls = np.zeros(t.size, bool)
    cls[-3:] = True           # all noise
    cls[16] = True            # one turn-2 hit
    m = M.stage_metrics(cls, t)
    assert m.turn == 2 and m.efficiency == pytest.approx(1 / 4) and m.purity == pytest.approx(1 / 4)
    only_noise = np.zeros(t.size, bool)
    only_noise[-3:] = True
    m = M.stage_metrics(only_noise, t)
    assert m.turn is None and m.efficiency == 0.0 and m.purity == 0.0 and m.n_classified == 3


def test_tie_goes_to_the_lower_turn_and_empty_stage():
    t = _turns()
    cls = np.zeros(t.size, bool)
    cls[[0, 1, 10, 11]] = True     # two of turn 0, two of turn 1
    m = M.stage_metrics(cls, t)
    assert m.turn == 0 and m.efficiency == pytest.approx(2 / 10) and m.purity == pytest.approx(0.5)
    m = M.stage_metrics(np.zeros(t.size, bool), t)
    assert m.turn is None and m.n_classified == 0


def test_event_metrics_and_average():
    t = _turns()
    stages = [t == 0, t == 1, np.zeros(t.size, bool)]
    ms = M.event_metrics(stages, t)
    assert [m.turn for m in ms] == [0, 1, None]
    avg = M.average(ms)
    assert avg["efficiency"] == pytest.approx(2 / 3) and avg["purity"] == pytest.approx(2 / 3)
    with pytest.raises(ValueError):
        M.stage_metrics(np.zeros(3, bool), t)
