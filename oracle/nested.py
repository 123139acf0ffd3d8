"""Plain FP64 reference of the nested-sampling evidence bookkeeping.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): the independent
reference the library's absorb/finalize kernels are checked against.  Only
the test-suite may use it.

Nested sampling (Sect. 3.2, after Skilling 2004) turns the evidence integral
Z = int L dpi into a one-dimensional sum over the prior mass X.  With N live
points, the i-th point to leave the live set (the lowest likelihood L*_i)
has expected prior mass X_i = exp(-i / N) enclosed by its contour, and the
weight of its shell is w_i = X_{i-1} - X_i (X_0 = 1).  Then

    Z ~ sum_i L*_i w_i  +  X_n * (1/N) sum_live L_j          (live remainder)
    H ~ sum_i (L*_i w_i / Z) ln(L*_i / Z)                      (information)

Everything is kept in logarithms and summed with log-sum-exp in double
precision, one dead point at a time, in the order the points leave.
"""
from __future__ import annotations

import math
from typing import List, Tuple

import numpy as np


def log_shell_weight(i: int, n_live: int) -> float:
    """ln w_i = ln(X_{i-1} - X_i) with X_i = exp(-i/N), i = 1, 2, ..."""
    return -(i - 1) / n_live + math.log(-math.expm1(-1.0 / n_live))


def log_add(a: float, b: float) -> float:
    """ln(e^a + e^b) without overflow; -inf is the empty sum."""
    if a == -math.inf:
        return b
    if b == -math.inf:
        return a
    m = max(a, b)
    return m + math.log(math.exp(a - m) + math.exp(b - m))


class State:
    """Running sums of one nested-sampling run."""

    def __init__(self):
        self.n_dead = 0
        self.log_z = -math.inf
        self.info = 0.0
        self.n_seen = 0

    def add(self, lnl: float, log_w: float) -> None:
        """Fold one point of likelihood e^lnl and prior weight e^log_w into ln Z and H
        (Skilling's running update: H = sum_k p_k ln L_k - ln Z with p_k = L_k w_k / Z)."""
        lw = lnl + log_w
        z_new = log_add(self.log_z, lw)
        h = 0.0
        if lw > -math.inf:
            h += math.exp(lw - z_new) * lnl
        if self.log_z > -math.inf:
            h += math.exp(self.log_z - z_new) * (self.info + self.log_z)
        self.info = h - z_new
        self.log_z = z_new


def argmin_first(v: np.ndarray) -> int:
    """Index of the smallest value, the lowest index among equal ones; a NaN counts
    as +inf (it is never the worst point)."""
    key = [math.inf if math.isnan(x) else float(x) for x in v]
    best = 0
    for j in range(1, len(key)):
        if key[j] < key[best]:
            best = j
    return best


def absorb(live_lnl: np.ndarray, live_theta: np.ndarray, cand_lnl: np.ndarray, cand_theta: np.ndarray,
           state: State, dead: List[Tuple[float, float, np.ndarray]], dead_cap: int) -> None:
    """Use the candidates in order: a candidate whose likelihood exceeds the current
    minimum of the live set replaces that point, which becomes the next dead point
    (weight w_i, i = n_dead + 1); other candidates are skipped.  Stops early when
    dead_cap dead points exist.  Modifies live_*, state and dead in place."""
    n = len(live_lnl)
    worst = argmin_first(live_lnl)
    for c in range(len(cand_lnl)):
        if state.n_dead >= dead_cap:
            return
        state.n_seen += 1
        if not (cand_lnl[c] > live_lnl[worst]):
            continue
        i = state.n_dead + 1
        log_w = log_shell_weight(i, n)
        dead.append((float(live_lnl[worst]), log_w, live_theta[worst].copy()))
        state.add(float(live_lnl[worst]), log_w)
        live_lnl[worst] = cand_lnl[c]
        live_theta[worst] = cand_theta[c]
        state.n_dead = i
        worst = argmin_first(live_lnl)


def finalize(live_lnl: np.ndarray, state: State) -> Tuple[float, float]:
    """Add the live points, each with weight X_n / N, in index order; returns (ln Z, H)."""
    n = len(live_lnl)
    s = State()
    s.log_z, s.info = state.log_z, state.info
    log_w = -state.n_dead / n - math.log(n)
    for j in range(n):
        s.add(float(live_lnl[j]), log_w)
    return s.log_z, s.info
