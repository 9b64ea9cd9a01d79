"""Oracle for SKIM's adaptive error estimation (Section 4.3.2, Eq. chernoff).

TEST INFRASTRUCTURE ONLY: the test suite is the only caller.  Plain numpy and
Python in FP64, following the section's steps in order.

Per SKIM iteration the selection records Delta (the exact marginal coverage
of the chosen seed, in node-instance pairs), tau (the threshold rank at which
its sketch filled, read as tau * 2^-64) and k' (the largest sketch size among
the other nodes without that rank; -1 when the ranks ran out and the choice
came from exact counts).

1. The discrepancy of the iteration is the gap between the true largest
   marginal coverage and Delta.  For a gap of d = Delta * eps, Eq. chernoff
   with Z = k', mu = tau * Delta * (1 + eps) and nu = 1 - k' / mu bounds the
   chance that the true maximum hid behind a sketch of at most k' entries:
   P[D > d] <= (exp(-nu) / (1 - nu) ** (1 - nu)) ** mu   (1 when nu <= 0).
2. Reading: D is replaced by a variable that dominates it on the grid
   {0, h, 2h, ...} with `bins` cells -- value (i + 1) h with probability
   B(i h) - B((i + 1) h), value 0 with 1 - B(0) -- and everything past the
   last cell goes to one overflow cell that stands for "unbounded".
3. The distribution of the sum over iterations is the convolution of the
   per-iteration distributions (the section's last step).
4. For a confidence c the bound is the smallest grid value b with
   P[sum > b] <= 1 - c.
"""
from __future__ import annotations

import math

import numpy as np


def chernoff_tail(kprime: int, mu: float) -> float:
    """Eq. chernoff with Z = k' and nu = 1 - k'/mu (1 where nu <= 0)."""
    if mu <= kprime:
        return 1.0
    nu = 1.0 - kprime / mu
    base = math.exp(-nu) / (1.0 - nu) ** (1.0 - nu)
    return base ** mu


def iteration_pmf(delta: int, tau: int, kprime: int, step: float, bins: int) -> tuple[np.ndarray, float]:
    """Step 2: cells 0..bins-1 and the overflow mass of one iteration."""
    pmf = np.zeros(bins)
    if kprime < 0:  # exact selection: no discrepancy
        pmf[0] = 1.0
        return pmf, 0.0
    t = math.ldexp(float(tau), -64)

    def B(d):
        return chernoff_tail(kprime, t * (delta + d))

    pmf[0] = 1.0 - B(0.0)
    for i in range(1, bins):
        pmf[i] = B((i - 1) * step) - B(i * step)
    return pmf, B((bins - 1) * step)


def discrepancy_ccdf(delta, tau, kprime, step: float, bins: int) -> np.ndarray:
    """Step 3: bins + 1 values, P[sum > i h] for i < bins and the overflow."""
    total = np.zeros(bins)
    total[0] = 1.0
    ovf = 0.0
    for d, t, kp in zip(delta, tau, kprime):
        q, qovf = iteration_pmf(int(d), int(t), int(kp), step, bins)
        full = np.convolve(total, q)
        ovf = ovf + qovf - ovf * qovf + float(full[bins:].sum())
        total = full[:bins]
    ccdf = np.empty(bins + 1)
    for i in range(bins):
        ccdf[i] = float(total[i + 1:].sum()) + ovf
    ccdf[bins] = ovf
    return ccdf


def discrepancy_bound(delta, tau, kprime, step: float, bins: int, conf) -> list[float]:
    """Step 4: the bound (pairs) for each confidence level, inf if none."""
    ccdf = discrepancy_ccdf(delta, tau, kprime, step, bins)
    out = []
    for c in conf:
        hit = [i for i in range(bins) if ccdf[i] <= 1.0 - c]
        out.append(hit[0] * step if hit else math.inf)
    return out
