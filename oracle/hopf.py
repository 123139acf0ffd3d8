"""The exact Hopf function q(tau) of Milne's problem, by solving its integral
equation (test infrastructure, like the rest of ``oracle/``).

Milne's profile (Sect. 2.5, after Mihalas 1978) is
    T^4(tau_R) = 3/4 Tbar_eff^4 [tau_R + q(tau_R)],
the radiative-equilibrium solution of a gray, semi-infinite atmosphere.  With
the source function S = tau + q (up to a constant factor), radiative
equilibrium S = Lambda[S] and Lambda[t] = tau + E3(tau)/2 give the Fredholm
equation of the second kind

    q(tau) = E3(tau)/2 + Lambda[q](tau),   Lambda[f](tau) = 1/2 int_0^inf E1(|t - tau|) f(t) dt.

It is solved here by product integration: q piecewise linear on a grid
(logarithmic near the surface, uniform at depth, q constant beyond the last
node), the E1 kernel integrated exactly against each hat function through
the antiderivatives of E1 and t E1 (E2, E3), and the linear system solved
directly.  The error falls as h^2, so two nested grids are combined by
Richardson extrapolation.  scipy's exponential integrals and numpy's dense
solver are the library primitives used.
"""
from __future__ import annotations

import functools

import numpy as np
from scipy.special import expn


def _en(n: int, x):
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    z = x == 0.0
    out[z] = 1.0 / (n - 1)
    out[~z] = expn(n, x[~z])
    return out


def _grid(m_near: int, m_deep: int, t_deep: float) -> np.ndarray:
    return np.concatenate([[0.0], np.geomspace(1e-9, 1.0, m_near), np.linspace(1.0, t_deep, m_deep)[1:]])


def solve_on(t: np.ndarray) -> np.ndarray:
    """q at the nodes t (t[0] = 0, ascending) from the discretised integral equation."""
    x = t[:, None]
    a, c = t[None, :-1], t[None, 1:]
    h = c - a

    def e1_int(s):        # antiderivative in s of E1(|s - x|)
        d = s - x
        return np.sign(d) * (1.0 - _en(2, np.abs(d)))

    def te1_int(s):       # antiderivative in s of (s - x) E1(|s - x|)
        d = np.abs(s - x)
        return -(d * _en(2, d) + _en(3, d))

    i0 = e1_int(c) - e1_int(a)
    i1 = te1_int(c) - te1_int(a)
    w_left = ((c - x) * i0 - i1) / h          # weight of q at the interval's left node
    w_right = (i1 + (x - a) * i0) / h         # ... and at its right node
    lam = np.zeros((len(t), len(t)))
    lam[:, :-1] += 0.5 * w_left
    lam[:, 1:] += 0.5 * w_right
    lam[:, -1] += 0.5 * _en(2, t[-1] - t)     # q held at its last value beyond the grid
    return np.linalg.solve(np.eye(len(t)) - lam, 0.5 * _en(3, t))


@functools.lru_cache(maxsize=None)
def hopf_table():
    """(tau, q) on the fine grid, Richardson-extrapolated from two nested grids."""
    coarse = _grid(201, 401, 40.0)
    fine = _grid(401, 801, 40.0)
    q_c = solve_on(coarse)
    q_f = solve_on(fine)
    # the O(h^2) error is smooth: move the fine solution by a third of its difference
    # from the coarse one (interpolated onto the fine nodes)
    q = q_f + (q_f - np.interp(fine, coarse, q_c)) / 3.0
    return fine, q


def hopf(tau):
    """q(tau) by linear interpolation in the table (constant beyond its ends)."""
    t, q = hopf_table()
    return np.interp(tau, t, q)
