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


def test_initial_weights_have_the_abi_length_and_layout():
    """init_params packs W1 b1 W2 b2 W3 b3 W4 b4 as the C ABI reads them: its
    length is bldtt_selector_param_count, the biases start at zero and the
    weights have He scale sqrt(2 / fan_in)."""
    import numpy as np
    import __graft_entry__
    from paper_2012_06925_gb300 import binding as B
    __graft_entry__.build()
    lib = B.load_library()
    for m in (1, 3, 6):
        p = S.init_params(m, np.random.default_rng(m))
        assert p.dtype == np.float32 and p.size == lib.bldtt_selector_param_count(m)
        w1 = p[:64 * 6]
        b1 = p[64 * 6:64 * 7]
        w2 = p[64 * 7:64 * 7 + 64 * 64]
        assert not b1.any()
        assert abs(w1.std() - math.sqrt(2 / 6)) < 0.1 and abs(w2.std() - math.sqrt(2 / 64)) < 0.02
        assert not p[-3 * m:].any()                     # output biases


def test_feature_box_contains_the_bf16_rounded_features():
    """The selector rounds each feature to float, then to bfloat16, before its
    box test; the box of the training features must still contain them."""
    import numpy as np
    import torch
    rng = np.random.default_rng(5)
    X = np.column_stack([rng.uniform(0.2, 1.4, 5000), rng.uniform(0.2, 1.4, 5000),
                         rng.uniform(0.0, 0.5, 5000), rng.uniform(0.0, 0.5, 5000),
                         rng.uniform(0.1, 0.95, 5000), rng.uniform(0.0, 0.9, 5000)])
    lo, hi = S.feature_box(X)
    xb = torch.from_numpy(X.astype(np.float32)).to(torch.bfloat16).float().numpy()
    assert np.all(xb >= lo) and np.all(xb <= hi)
    lo2, hi2 = S.feature_box(X, pad=0.1)
    assert np.all(lo2 <= lo - 0.1 + 1e-6) and np.all(hi2 >= hi + 0.1 - 1e-6)
