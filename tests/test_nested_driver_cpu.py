"""The nested-sampling driver's host logic (proposal box, termination) on the
CPU: the same NestedSampler runs with a backend built on the oracle's
bookkeeping and an analytic likelihood, and must find the closed-form
evidence of a Gaussian within its own error estimate."""
import math

import numpy as np

from oracle import nested as N
from paper_1910_01070_b300 import hr2
from paper_1910_01070_b300.nested import NestedSampler


class OracleBackend:
    def __init__(self, loglike, n_live, dead_cap=10 ** 6):
        self.loglike, self.n_live, self.cap = loglike, n_live, dead_cap
        self.state, self.dead = N.State(), []

    def init_live(self, theta):
        self.live_theta = theta.copy()
        self.live_lnl = self.loglike(theta)

    def live_theta_host(self):
        return self.live_theta

    def step(self, cand):
        N.absorb(self.live_lnl, self.live_theta, self.loglike(cand), cand, self.state, self.dead, self.cap)
        s = self.state
        return {"n_dead": s.n_dead, "n_seen": s.n_seen, "log_z": s.log_z, "info": s.info,
                "log_x": -s.n_dead / self.n_live, "lnl_min": float(np.min(self.live_lnl)),
                "lnl_max": float(np.max(self.live_lnl))}

    def finalize(self):
        return N.finalize(self.live_lnl, self.state)


def test_driver_finds_the_gaussian_evidence():
    d, sd = 3, 0.05
    c = np.array([0.4, 0.55, 0.5])
    free = slice(3, 3 + d)

    def loglike(th):
        return -np.sum((th[:, free] - c) ** 2, axis=1) / (2 * sd * sd)

    lo = np.zeros(hr2.HR2_NPARAM)
    hi = np.zeros(hr2.HR2_NPARAM)
    hi[free] = 1.0
    be = OracleBackend(loglike, 200)
    res = NestedSampler(be, lo, hi, batch=256, seed=3).run(dlogz=0.01, max_rounds=400)
    ref = 0.5 * d * math.log(2 * math.pi * sd * sd)
    assert abs(res["log_z"] - ref) < 4 * res["log_z_err"], (res, ref)
    dead = np.array([x[0] for x in be.dead])
    assert np.all(np.diff(dead) >= 0)              # dead points leave in increasing likelihood
    assert 0 < res["acceptance"] <= 1
