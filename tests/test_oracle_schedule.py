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
