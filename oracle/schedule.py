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


# ---------------------------------------------------------------------------
# Algorithm 1 of the paper (stage 2 of the balancer): pair the least loaded
# process (a receiver) with the most loaded one (a sender), move the load
# min(mean - L_receiver, L_sender - mean) between them as a number of
# problems whose cost adds up to it, and advance past whichever of the two
# reached the mean. Transfers below 0.01 of the mean load are dropped.
# Readings where the paper is silent: the sender gives away problems from
# the end of its list (those it would solve last), as many as bring their
# cost sum closest to the load to move; "|L_i - mean| ~ 0" is a relative
# tolerance of 1e-12; a dropped transfer still updates the bookkeeping.
# ---------------------------------------------------------------------------

def balance_operations(costs, threshold: float = 0.01):
    """costs: one sequence of per-problem costs (t_cpu of the previous step)
    per process. Returns (operations, mean load): operations is a list of
    (sender, receiver, number of problems, moved cost)."""
    loads = np.array([float(np.sum(c)) for c in costs])
    nproc = loads.size
    mean = loads.sum() / nproc
    order = np.argsort(loads, kind="stable")     # ranks by ascending load
    L = loads[order].copy()
    remaining = [list(np.asarray(c, dtype=float)) for c in costs]
    ops = []
    i, j = 0, nproc - 1
    while i < j:
        dL = min(mean - L[i], L[j] - mean)
        receiver, sender = int(order[i]), int(order[j])
        if dL >= threshold * mean and dL > 0:
            pool = remaining[sender]
            tail = np.cumsum(pool[::-1])          # cost of sending the last 1, 2, ... problems
            k = int(np.argmin(np.abs(tail - dL))) + 1 if tail.size else 0
            if k > 0:
                moved = float(tail[k - 1])
                del pool[len(pool) - k:]
                ops.append((sender, receiver, k, moved))
        L[i] += dL
        L[j] -= dL
        if abs(L[i] - mean) <= 1e-12 * mean:
            i += 1
        else:
            j -= 1
    return ops, mean


def balanced_loads(costs, ops) -> np.ndarray:
    """Per-process load after the operations (a process solves what it kept
    and what it received)."""
    loads = np.array([float(np.sum(c)) for c in costs])
    for s, r, k, moved in ops:
        loads[s] -= moved
        loads[r] += moved
    return loads


def chi_su_model(nproc: int, nprob: int, theta: float, x: float, xi: float) -> float:
    """Speed-up of Algorithm 1 on a Sec. 3 configuration (communication not
    counted): slowest process without balancing over slowest process after
    the operations."""
    costs = benchmark_loads(nproc, nprob, theta, x, xi)
    ops, _ = balance_operations(list(costs))
    return unbalanced_makespan(costs) / float(balanced_loads(list(costs), ops).max())
