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
directly.  The nodal error of three nested grids (each halving the steps of
the last) falls as h^2 and then as h^3, so two Richardson steps at the
coarsest grid's nodes (nodes of all three) remove both terms.  Between nodes a
grid's solution is carried by the integral equation itself (Nystrom's
interpolation: the right-hand side evaluated at any tau), but that value's
error has a part that oscillates with the position inside the cell, which
Richardson cannot remove; so the finest grid's Nystrom values are kept and
only the smooth correction (extrapolated minus finest, at the coarse nodes) is
interpolated onto them, on each side of tau = 1 separately, where the grid
changes from logarithmic to uniform.  The result is tabulated on the finest
grid and its midpoints and read by cubic Lagrange interpolation through the
four nearest nodes.  scipy's exponential integrals and numpy's dense solver
are the library primitives used.
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


def lambda_rows(t: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Rows of the discretised Lambda operator: Lambda[q](x_i) = sum_j rows[i, j] q(t_j)
    for q piecewise linear on the nodes t (t[0] = 0, ascending) and constant beyond t[-1]."""
    x = np.asarray(x, dtype=np.float64)[:, None]
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
    lam = np.zeros((x.shape[0], len(t)))
    lam[:, :-1] += 0.5 * w_left
    lam[:, 1:] += 0.5 * w_right
    lam[:, -1] += 0.5 * _en(2, t[-1] - x[:, 0])   # q held at its last value beyond the grid
    return lam


def solve_on(t: np.ndarray) -> np.ndarray:
    """q at the nodes t (t[0] = 0, ascending) from the discretised integral equation."""
    return np.linalg.solve(np.eye(len(t)) - lambda_rows(t, t), 0.5 * _en(3, t))


def nystrom(t: np.ndarray, q: np.ndarray, x) -> np.ndarray:
    """The solution q (on the nodes t) carried to the points x by the integral equation."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    return 0.5 * _en(3, x) + lambda_rows(t, x) @ q


def _cubic(t: np.ndarray, q: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Cubic Lagrange interpolation of (t, q) at x through the four nearest nodes
    (the stencil slides inward at the ends)."""
    k = np.clip(np.searchsorted(t, x) - 2, 0, len(t) - 4)   # first of the four nodes
    out = np.zeros_like(x)
    for a in range(4):
        la = np.ones_like(x)
        for b in range(4):
            if b != a:
                la *= (x - t[k + b]) / (t[k + a] - t[k + b])
        out += la * q[k + a]
    return out


@functools.lru_cache(maxsize=None)
def hopf_table():
    """(tau, q) on the finest of three nested grids and its midpoints."""
    grids = [_grid(m + 1, 2 * m + 1, 40.0) for m in (200, 400, 800)]
    sols = [solve_on(g) for g in grids]
    coarse, fine = grids[0], grids[-1]
    # the coarse nodes in the two finer grids (nested: every coarse node is one)
    i_mid, i_fine = np.searchsorted(grids[1], coarse), np.searchsorted(fine, coarse)
    assert np.allclose(grids[1][i_mid], coarse, rtol=1e-13, atol=0.0)
    assert np.allclose(fine[i_fine], coarse, rtol=1e-13, atol=0.0)
    v0, v1, v2 = sols[0], sols[1][i_mid], sols[2][i_fine]
    r_coarse = v1 + (v1 - v0) / 3.0          # h^2 term removed (steps h, h/2)
    r_fine = v2 + (v2 - v1) / 3.0            # ... (steps h/2, h/4)
    correction = r_fine + (r_fine - r_coarse) / 7.0 - v2     # then the h^3 term
    tab = np.sort(np.concatenate([fine, 0.5 * (fine[:-1] + fine[1:])]))
    q = nystrom(fine, sols[2], tab)
    upper = tab <= 1.0
    c_up, c_deep = coarse <= 1.0, coarse >= 1.0
    q[upper] += _cubic(coarse[c_up], correction[c_up], tab[upper])
    q[~upper] += _cubic(coarse[c_deep], correction[c_deep], tab[~upper])
    return tab, q


def hopf(tau):
    """q(tau): cubic Lagrange interpolation in the table (constant beyond its ends)."""
    t, q = hopf_table()
    x = np.asarray(tau, dtype=np.float64)
    xf = np.atleast_1d(x)
    out = np.where(xf <= t[0], q[0], np.where(xf >= t[-1], q[-1], _cubic(t, q, xf)))
    return out if x.ndim else float(out[0])
