"""The serving scheduler's admission policy, replayed on the host with a simulated executor
(ewald_server_simulate runs the same policy function as the scheduler thread; no GPU):
first fit in arrival order, admission on the idle slot that holds the most memory, idle
slots' memory reclaimed when a request does not fit, a bounded number of admissions past a
waiting head, and the held total never above the budget."""
import numpy as np
import pytest

from paper_1708_01135_gb300 import ewald as E


def _sim(slots, budget, fp, ta, du):
    try:
        E.lib()
    except RuntimeError as e:   # not built in this checkout
        pytest.skip(str(e))
    return E.simulate_admission(slots, budget, fp, ta, du)


def test_everything_fits_admits_in_arrival_order_as_slots_free():
    order, t, peak = _sim(3, 1000, [10] * 6, [0.0] * 6, [5.0, 1.0, 1.0, 1.0, 1.0, 1.0])
    assert list(order) == [0, 1, 2, 3, 4, 5]
    assert list(t) == [0.0, 0.0, 0.0, 1.0, 1.0, 2.0]
    assert peak == 30


def test_first_fit_passes_a_request_that_does_not_fit():
    # r1 does not fit beside r0 (6 + 6 > 10) and waits for r0; r2 (3) fits and goes first
    order, t, peak = _sim(2, 10, [6, 6, 3], [0.0, 0.0, 0.0], [10.0, 1.0, 1.0])
    assert list(order) == [0, 2, 1]
    assert list(t) == [0.0, 10.0, 0.0]
    assert peak == 9


def test_idle_slots_give_back_memory_to_fit_a_large_request():
    # after r0 and r1 finish their slots still hold 8 and 2; r2 (9) takes the larger idle
    # slot and the other one is reclaimed
    order, t, peak = _sim(2, 10, [8, 2, 9], [0.0, 0.0, 2.0], [1.0, 1.0, 1.0])
    assert list(order) == [0, 1, 2]
    assert t[2] == 2.0
    assert peak == 10


def test_a_waiting_head_is_passed_over_a_bounded_number_of_times():
    # r0 (6) runs for long; the head r1 (6) cannot fit beside it; 70 small requests arrive
    # behind it and one slot runs them one after another: 64 pass the head, the rest wait
    # until the head has run
    n_small = 70
    fp = [6, 6] + [1] * n_small
    ta = [0.0] * (2 + n_small)
    du = [1000.0, 1.0] + [1.0] * n_small
    order, t, peak = _sim(2, 10, fp, ta, du)
    pos = {int(r): k for k, r in enumerate(order)}
    smalls = list(range(2, 2 + n_small))
    before = [r for r in smalls if pos[r] < pos[1]]
    assert len(before) == 64
    assert t[1] == 1000.0
    assert all(t[r] >= 1000.0 for r in smalls if r not in before)
    assert peak <= 10


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_random_streams_respect_the_budget_and_admit_everything(seed):
    rng = np.random.default_rng(seed)
    n = 300
    budget = 1000
    fp = rng.integers(1, budget + 1, size=n)
    ta = np.cumsum(rng.exponential(0.3, size=n))
    du = rng.exponential(1.0, size=n)
    order, t, peak = _sim(4, budget, fp, ta, du)
    assert sorted(order) == list(range(n))
    assert peak <= budget
    assert np.all(t >= ta)
    # replay: at every admission the running requests' footprints fit the budget
    for k, i in enumerate(order):
        running = [j for j in order[:k] if t[j] <= t[i] < t[j] + du[j]]
        assert sum(fp[j] for j in running) + fp[i] <= budget
        assert len(running) < 4


def test_bad_arguments_are_rejected():
    try:
        E.lib()
    except RuntimeError as e:
        pytest.skip(str(e))
    with pytest.raises(E.EwaldError):
        E.simulate_admission(0, 10, [1], [0.0], [1.0])
    with pytest.raises(E.EwaldError):
        E.simulate_admission(1, 10, [11], [0.0], [1.0])          # above the budget
    with pytest.raises(E.EwaldError):
        E.simulate_admission(1, 10, [1, 1], [1.0, 0.0], [1.0, 1.0])   # arrivals out of order
