"""The ambiguity-aware comparison used by the grid and NC parity tests, on synthetic data (no GPU):
it must accept a result that takes the other decision inside an ambiguous part, and reject one
that differs outside every part or matches neither decision inside one."""
import numpy as np
import pytest

import ambiguity


def test_periodic_labels_join_across_the_borders():
    m = np.zeros((6, 8), dtype=bool)
    m[0, 3] = m[5, 3] = True        # joined through the top/bottom wrap
    m[2, 0] = m[2, 7] = True        # joined through the left/right wrap
    m[3, 4] = True                  # alone
    lab, n = ambiguity.periodic_labels(m)
    assert n == 3
    assert lab[0, 3] == lab[5, 3] and lab[2, 0] == lab[2, 7] and lab[3, 4] not in (lab[0, 3], lab[2, 0])


def test_reach_mask_wraps():
    m = ambiguity.reach_mask([(0, 0)], 10, 12, 2)
    assert m[0, 0] and m[9, 0] and m[0, 11] and m[8, 0] and not m[7, 0] and not m[5, 5]


def _setup():
    rng = np.random.default_rng(0)
    base = rng.normal(size=(1, 40, 50))
    bump = np.zeros_like(base)
    bump[0, 10:13, 20:23] = 0.5          # what reversing decision "a" (at (11, 21)) changes
    amb = [(0, 11, 21, "a")]

    def evaluate(keys):
        return base + (bump if "a" in keys else 0.0)
    return base, bump, amb, evaluate


def test_accepts_either_decision_inside_and_exact_match_outside():
    base, bump, amb, evaluate = _setup()
    ambiguity.check(base, base, amb, evaluate, 4, 1e-6, n_decisions=10 ** 6)
    s = ambiguity.check(base + bump, base, amb, evaluate, 4, 1e-6, n_decisions=10 ** 6)
    assert s["parts"] == 1 and s["parts_verified"] == 1


def test_rejects_errors_outside_and_results_matching_neither_decision():
    base, bump, amb, evaluate = _setup()
    bad = base.copy()
    bad[0, 30, 40] += 1e-3
    with pytest.raises(AssertionError):
        ambiguity.check(bad, base, amb, evaluate, 4, 1e-6, n_decisions=10 ** 6)
    bad = base + 0.5 * bump
    with pytest.raises(AssertionError):
        ambiguity.check(bad, base, amb, evaluate, 4, 1e-6, n_decisions=10 ** 6)


def test_rejects_too_many_ambiguous_decisions():
    base, bump, amb, evaluate = _setup()
    many = [(0, y, x, (y, x)) for y in range(40) for x in range(0, 50, 10)]
    with pytest.raises(AssertionError):
        ambiguity.check(base, base, many, evaluate, 1, 1e-6, n_decisions=1000)
