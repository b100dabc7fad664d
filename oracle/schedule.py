"""CPU model of the load-balancing arithmetic (test infrastructure only).

TEST INFRASTRUCTURE ONLY: tests/ import this; the CUDA path never does.

Sec. 3 of the paper benchmarks the balancer on pseudo-problems: every
process holds the same number of problems, a fraction theta of them "heavy"
(cost xi relative to a light problem) on a fraction x of the processes, the
heavy problems being 20 % of all problems (x * theta = 0.2). Without
balancing a step lasts as long as the most loaded process; a perfect balance
makes every process carry the mean load. The speed-up bound is their ratio.
The paper's printed denominator, (theta xi + 1/x - 1) / (1/x), equals the
mean load x theta xi + 1 - x theta only when theta = 1; the reading used here
is the ratio of the maximum to the mean load (the two agree for the paper's
C1, theta = 1).

On one GPU the balancer becomes a device queue pulled longest-first by
persistent teams, i.e. Graham's LPT list schedule (R. L. Graham, SIAM J. Appl.
Math. 17(2), 1969): each job in descending cost goes to the least loaded
worker, which finishes within (4/3 - 1/(3m)) of the optimal makespan.
"""
from __future__ import annotations

import heapq

import numpy as np


def chi_max(theta: float, xi: float, x: float) -> float:
    """Maximum speed-up of Sec. 3: most loaded process / mean process load,
    per problem: (theta xi + 1 - theta) / (x theta xi + 1 - x theta)."""
    return (theta * xi + 1.0 - theta) / (x * theta * xi + 1.0 - x * theta)


def benchmark_loads(nproc: int, nprob: int, theta: float, x: float, xi: float) -> np.ndarray:
    """Per-problem costs, one row per process, for a Sec. 3 configuration: the
    first round(x * nproc) processes hold round(theta * nprob) heavy problems
    (cost xi), everything else is light (cost 1)."""
    costs = np.ones((nproc, nprob))
    nh = int(round(x * nproc))
    kh = int(round(theta * nprob))
    costs[:nh, :kh] = xi
    return costs


def unbalanced_makespan(costs: np.ndarray) -> float:
    """Every process solves its own problems: the slowest one sets the time."""
    return float(costs.sum(axis=1).max())


def lpt_makespan(costs, workers: int) -> float:
    """Longest-processing-time-first list schedule: jobs in descending cost,
    each to the currently least loaded worker; returns the largest load."""
    loads = [0.0] * workers
    heapq.heapify(loads)
    for c in sorted(np.ravel(costs), reverse=True):
        heapq.heappush(loads, heapq.heappop(loads) + float(c))
    return max(loads)
