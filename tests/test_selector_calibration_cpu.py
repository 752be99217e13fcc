"""The learned selector's calibration walk (selector.choose_calibration), on
the CPU with a stand-in for the GPU measurement: looser per-pair budgets and
higher separation caps do less work and make larger errors."""
import math

from paper_2012_06925_gb300 import selector as S


def fake_measure(table):
    calls = []

    def measure(cap, le):
        calls.append((cap, le))
        return table[(cap, le)]
    return measure, calls


def grid_table(caps, budgets, err, work):
    return {(c, le): (err(c, le), work(c, le)) for c in caps for le in budgets}


CAPS = (0.8, 0.9)
BUDGETS = (-5.0, -6.0, -7.0)


def test_walk_stops_at_the_first_budget_meeting_the_target_and_takes_the_least_work():
    # error grows with the cap and the budget; work falls with both
    t = grid_table(CAPS, BUDGETS, err=lambda c, le: 10 ** le * (2.0 if c > 0.85 else 1.0),
                   work=lambda c, le: 1000 + 100 * le - 50 * c)
    measure, calls = fake_measure(t)
    le, cap, table, grid = S.choose_calibration(measure, CAPS, BUDGETS, target=2e-6)
    # cap 0.8: -5 gives 1e-5 (too large), -6 gives 1e-6 (meets) -> stop
    # cap 0.9: -5 gives 2e-5, -6 gives 2e-6 (meets) -> stop
    assert calls == [(0.8, -5.0), (0.8, -6.0), (0.9, -5.0), (0.9, -6.0)]
    assert (cap, le) == (0.9, -6.0)            # less work than (0.8, -6.0)
    assert table == [(-5.0, 2e-5, t[(0.9, -5.0)][1]), (-6.0, 2e-6, t[(0.9, -6.0)][1])]
    assert len(grid) == 4


def test_nothing_meets_the_target():
    t = grid_table(CAPS, BUDGETS, err=lambda c, le: 1.0, work=lambda c, le: 1.0)
    measure, calls = fake_measure(t)
    le, cap, table, grid = S.choose_calibration(measure, CAPS, BUDGETS, target=1e-6)
    assert (cap, le) == (0.8, -7.0)            # the tightest settings
    assert len(calls) == len(CAPS) * len(BUDGETS)
    assert all(math.isfinite(e) for _, _, e, _ in grid)
