"""The serving loop's division of a wave's work budget (mm_serve_plan), on the host:
bounds, no starvation, shortest remaining work first for the priority share, plain
processor sharing at share 0, the minimum wave size, and argument validation."""
import numpy as np
import pytest

import paper_1005_5198_gb300 as mm


@pytest.fixture(scope="module", autouse=True)
def built():
    mm.build()


def _random_case(rng):
    n = int(rng.integers(1, 40))
    left = rng.integers(0, 5000, n).astype(np.uint64)
    cost = np.exp(rng.uniform(np.log(1e5), np.log(1e9), n))
    budget = float(np.exp(rng.uniform(np.log(1e8), np.log(1e12))))
    return left, cost, budget


def test_takes_are_bounded_and_every_map_with_work_moves():
    rng = np.random.default_rng(11)
    for _ in range(300):
        left, cost, budget = _random_case(rng)
        share = float(rng.choice([0.0, 0.3, 0.8, 1.0]))
        take = mm.mm_serve_plan(left, cost, budget, share, int(rng.integers(0, 3000)))
        assert np.all(take <= left)
        assert np.all(take[left > 0] >= 1)
        assert np.all(take[left == 0] == 0)


def test_share_zero_is_even_processor_sharing():
    rng = np.random.default_rng(12)
    for _ in range(200):
        left, cost, budget = _random_case(rng)
        take = mm.mm_serve_plan(left, cost, budget, 0.0, 0)
        even = np.maximum(1.0, np.floor(budget / len(left) / cost))
        np.testing.assert_array_equal(take, np.minimum(left, even.astype(np.uint64)))


def test_priority_share_goes_to_the_least_remaining_work_first():
    rng = np.random.default_rng(13)
    for _ in range(300):
        left, cost, budget = _random_case(rng)
        share = float(rng.choice([0.5, 0.8, 1.0]))
        take = mm.mm_serve_plan(left, cost, budget, share, 0)
        even = np.maximum(1.0, np.floor((1.0 - share) * budget / len(left) / cost)).astype(np.uint64)
        extra = take.astype(np.int64) - np.minimum(left, even).astype(np.int64)   # items beyond the even part
        work = left.astype(np.float64) * cost
        got = np.flatnonzero(extra > 0)
        for b in got:
            # every map with strictly less remaining work than one that got priority items is finished
            smaller = work < work[b]
            assert np.all(take[smaller] == left[smaller])
        # the priority share is spent unless every map is finished
        if np.any(take < left):
            assert float((take.astype(np.float64) * cost).sum()) >= share * budget * (1 - 1e-12)


def test_least_remaining_map_finishes_first_in_a_worked_case():
    # three maps of 10, 100 and 1000 unit-cost items; budget 100, share 0.8:
    # 80 priority units finish the first map (10) and give 70 to the second;
    # the even 20 units add floor(20 / 3) = 6 items to every map
    take = mm.mm_serve_plan([10, 100, 1000], [1.0, 1.0, 1.0], 100.0, 0.8, 0)
    np.testing.assert_array_equal(take, [10, 76, 6])
    np.testing.assert_array_equal(mm.mm_serve_plan([10, 100, 1000], [1.0, 1.0, 1.0], 100.0, 0.0, 0), [10, 33, 33])


def test_budget_grows_until_the_wave_is_large_enough():
    rng = np.random.default_rng(14)
    for _ in range(200):
        left, cost, budget = _random_case(rng)
        min_items = int(rng.integers(0, 20000))
        take = mm.mm_serve_plan(left, cost, budget, 0.8, min_items)
        assert int(take.sum()) >= min(min_items, int(left.sum()))


@pytest.mark.parametrize("args", [
    ([1], [0.0], 10.0, 0.5), ([1], [1.0], 0.0, 0.5), ([1], [1.0], 10.0, -0.1), ([1], [1.0], 10.0, 1.5),
    ([1], [float("nan")], 10.0, 0.5), ([1], [1.0], float("nan"), 0.5)])
def test_bad_arguments_rejected(args):
    with pytest.raises(mm.MMError):
        mm.mm_serve_plan(*args)


def test_no_maps_is_an_empty_plan():
    assert len(mm.mm_serve_plan(np.zeros(0, np.uint64), np.zeros(0), 10.0, 0.8, 100)) == 0
