"""The sample schedule of the online training (Sec. 5.8): the oracle's plan
against the rules of the paper on hand-worked budgets and as invariants, and
the C library's mpg_training_plan (host code, no GPU) against the oracle's."""
import math

import pytest

from oracle import oracle as O


@pytest.mark.parametrize("total,expect", [
    (64, ([1, 2, 4, 12], 45)),   # budget 19: 1, 2, 4 (7 < 9.5), 8 -> 15 >= 9.5: continue to 19
    (16, ([1, 3], 12)),          # budget 4: 1 (< 2), 2 -> 3 >= 2: continue to 4
    (32, ([1, 2, 6], 23)),       # budget 9: 1, 2 (3 < 4.5), 4 -> 7: continue to 9
    (100, ([1, 2, 4, 23], 70)),  # budget 30: 1, 2, 4 (7 < 15), 8 -> 15 = 15 is not less: continue to 30
    (3, ([], 3)),                # budget 0: no training
])
def test_plan_on_hand_worked_budgets(total, expect):
    assert O.training_plan(total) == expect


@pytest.mark.parametrize("first", [1, 2, 4])
def test_plan_invariants(first):
    for total in range(0, 1500):
        it, render = O.training_plan(total, first)
        budget = math.floor(0.3 * total)
        assert sum(it) + render == total and sum(it) == budget
        # every iteration but the last doubles the one before; the last starts
        # doubled (or cut at the budget) and was begun with less than half used
        for j in range(1, len(it) - 1):
            assert it[j] == first << j
        if len(it) >= 1:
            used_before = sum(it[:-1])
            assert len(it) == 1 or 2 * used_before < budget
            assert it[-1] >= min(first << (len(it) - 1), budget - used_before)


def test_library_plan_matches_oracle():
    from paper_2311_12818_gb300 import mpg
    for first in (1, 2, 3):
        for frac in (0.3, 0.5, 0.25):
            for total in range(0, 600):
                assert mpg.mpg_training_plan(total, first, frac) == O.training_plan(total, first, frac)
