"""Pins of the load-balancing model (CPU only): the speed-up bound of Sec. 3
against explicit per-process loads, and the longest-first queue against
Graham's bound and the perfect balance."""
import numpy as np
import pytest

from oracle import schedule

# Sec. 3 configurations: (theta, x); the heavy problems are 20 % of all problems
SEC3_CASES = {"C1": (1.0, 0.2), "C2": (0.8, 0.25), "C3": (0.4, 0.5), "C4": (0.2, 1.0)}


@pytest.mark.parametrize("name", list(SEC3_CASES))
@pytest.mark.parametrize("xi", [2.0, 10.0, 50.0])
def test_chi_max_is_max_over_mean_load(name, xi):
    theta, x = SEC3_CASES[name]
    costs = schedule.benchmark_loads(80, 200, theta, x, xi)
    loads = costs.sum(axis=1)
    assert x * theta == pytest.approx(0.2)
    assert schedule.chi_max(theta, xi, x) == pytest.approx(loads.max() / loads.mean(), rel=1e-12)


def test_printed_denominator_agrees_only_for_theta_one():
    """The printed form (theta xi + 1/x - 1) / (1/x) is the mean load for C1
    (theta = 1) and differs from it for C2 and C3."""
    xi = 10.0
    for name, (theta, x) in SEC3_CASES.items():
        printed = (theta * xi + (1.0 - theta)) / ((theta * xi + (1.0 / x - 1.0)) / (1.0 / x))
        mine = schedule.chi_max(theta, xi, x)
        if theta == 1.0:
            assert printed == pytest.approx(mine, rel=1e-12)
        elif name in ("C2", "C3"):
            assert abs(printed - mine) > 1e-3


def test_balanced_configuration_has_no_speedup():
    """C4 spreads the heavy problems evenly: chi_max = 1 and the queue cannot
    beat the unbalanced run (the paper's chi_su ~ 1 for C4)."""
    theta, x = SEC3_CASES["C4"]
    for xi in (2.0, 10.0, 50.0):
        assert schedule.chi_max(theta, xi, x) == pytest.approx(1.0, rel=1e-12)
        costs = schedule.benchmark_loads(40, 200, theta, x, xi)
        assert schedule.unbalanced_makespan(costs) / schedule.lpt_makespan(costs, 40) == pytest.approx(1.0, abs=1e-12)


@pytest.mark.parametrize("name", ["C1", "C2", "C3"])
def test_longest_first_queue_reaches_the_bound(name):
    """With many problems per worker the longest-first queue lands on the mean
    load, so its speed-up over the unbalanced run is chi_max (within 1 %)."""
    theta, x = SEC3_CASES[name]
    xi = 10.0
    costs = schedule.benchmark_loads(40, 200, theta, x, xi)
    chi = schedule.unbalanced_makespan(costs) / schedule.lpt_makespan(costs, 40)
    assert chi == pytest.approx(schedule.chi_max(theta, xi, x), rel=0.01)


def test_lpt_within_grahams_bound_on_random_jobs():
    """Longest-first is never below the lower bound max(mean load, largest
    job), and against the true optimum (brute force over every assignment of
    7 jobs) it stays within Graham's (4/3 - 1/(3m))."""
    rng = np.random.default_rng(0)
    for m in (2, 3, 5, 16):
        for _ in range(50):
            jobs = rng.lognormal(0.0, 1.5, size=int(rng.integers(m, 6 * m)))
            lower = max(jobs.sum() / m, jobs.max())
            assert schedule.lpt_makespan(jobs, m) >= lower * (1 - 1e-12)
    import itertools
    for m in (2, 3):
        for _ in range(20):
            jobs = rng.integers(1, 20, size=7).astype(float)
            best = min(max(np.bincount(a, weights=jobs, minlength=m)) for a in itertools.product(range(m), repeat=7))
            span = schedule.lpt_makespan(jobs, m)
            assert best <= span <= (4.0 / 3.0 - 1.0 / (3 * m)) * best + 1e-9


# ---------------------------------------------------------------- Algorithm 1
def test_algorithm1_worked_example():
    """Three processes holding 1, 2 and 6 unit problems: mean 3. The first
    pair (receiver 0, sender 2) moves min(3 - 1, 6 - 3) = 2 problems and fills
    the receiver; the next (receiver 1, sender 2) moves 1; all end at 3."""
    costs = [np.ones(1), np.ones(2), np.ones(6)]
    ops, mean = schedule.balance_operations(costs)
    assert mean == 3.0
    assert [(s, r, k) for s, r, k, _ in ops] == [(2, 0, 2), (2, 1, 1)]
    np.testing.assert_array_equal(schedule.balanced_loads(costs, ops), [3.0, 3.0, 3.0])


def test_algorithm1_drops_transfers_below_one_percent_of_the_mean():
    """Loads 99.5, 100.5 (mean 100): the transfer of 0.5 < 0.01 * 100 is not
    executed; loads 90, 110 move 10 = 20 problems of 0.5."""
    small = [np.full(199, 0.5), np.full(201, 0.5)]
    ops, mean = schedule.balance_operations(small)
    assert ops == [] and mean == 100.0
    big = [np.full(180, 0.5), np.full(220, 0.5)]
    ops, _ = schedule.balance_operations(big)
    assert [(s, r, k) for s, r, k, _ in ops] == [(1, 0, 20)]


@pytest.mark.parametrize("name", list(SEC3_CASES))
def test_algorithm1_lands_every_process_near_the_mean(name):
    """After the operations every process carries the mean load to within the
    dropped transfers (< 1 % of the mean each) plus one problem's cost; no
    process both sends and receives; problems are conserved."""
    theta, x = SEC3_CASES[name]
    xi = 10.0
    costs = list(schedule.benchmark_loads(80, 200, theta, x, xi))
    ops, mean = schedule.balance_operations(costs)
    loads = schedule.balanced_loads(costs, ops)
    assert loads.sum() == pytest.approx(sum(c.sum() for c in costs), rel=1e-12)
    senders, receivers = {s for s, *_ in ops}, {r for _, r, *_ in ops}
    assert not senders & receivers
    assert np.abs(loads - mean).max() <= 0.01 * mean + xi
    if name == "C4":
        assert ops == []          # already balanced: nothing is communicated (Sec. 3)


@pytest.mark.parametrize("name", ["C1", "C2", "C3"])
def test_algorithm1_speedup_approaches_the_bound_with_more_problems(name):
    """The Sec. 3 sweep: chi_su of the model rises towards chi_max as the
    problems per process grow (the paper's explanation: with few problems one
    problem more or less over- or undershoots the target), and with 1000 per
    process it is within 2 % of chi_max; the process count does not matter."""
    theta, x = SEC3_CASES[name]
    xi = 10.0
    bound = schedule.chi_max(theta, xi, x)
    sweep = [schedule.chi_su_model(80, nprob, theta, x, xi) for nprob in (40, 200, 1000)]
    assert all(c <= bound * (1 + 1e-12) for c in sweep)
    assert sweep[0] < sweep[-1]
    assert sweep[-1] == pytest.approx(bound, rel=0.02)
    for nproc in (20, 160, 640):
        assert schedule.chi_su_model(nproc, 1000, theta, x, xi) == pytest.approx(bound, rel=0.02)
    assert schedule.chi_su_model(80, 200, 0.2, 1.0, xi) == 1.0
