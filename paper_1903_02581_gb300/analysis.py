"""Analysis of bunching-probability sweeps with the paper's 1D scattering
model (Eq. bunching, from Eqs. rtqpc and bunchingket).

For two identical packets of width sigma, delayed by Delta, at a QPC whose
energy selectivity has the geometric parameter a, the model gives

    P_b(Delta) = 1/2 - 1/2 (sigma^2 / Sigma^2) exp(-Delta^2 / (4 Sigma^2)),
    Sigma^2    = sigma^2 + a^2 / (8 gamma),   gamma = 4 ln 2.

The paper fits this form to its simulated P_b, and with effective
(sigma_eff, a_eff) to the interacting case.  These helpers evaluate and fit
it; they run on the host on outputs of the library and are not part of the
propagation.
"""

from __future__ import annotations

import math

import numpy as np

GAMMA = 4.0 * math.log(2.0)


def bunching_1d(delta, sigma: float, a: float, gamma: float = GAMMA):
    """Eq. bunching: the bunching probability of the 1D model."""
    s2 = sigma * sigma + a * a / (8.0 * gamma)
    d = np.asarray(delta, dtype=np.float64)
    return 0.5 - 0.5 * (sigma * sigma / s2) * np.exp(-d * d / (4.0 * s2))


def fit_bunching_1d(delta, p_b, sigma0: float = 1.0, a0: float = 1.0, gamma: float = GAMMA):
    """Least-squares fit of (sigma, a) in Eq. bunching to a sweep of P_b over
    the delay (at least three points).  Returns (sigma, a), both >= 0."""
    from scipy.optimize import least_squares

    d = np.asarray(delta, dtype=np.float64)
    p = np.asarray(p_b, dtype=np.float64)
    if d.shape != p.shape or d.size < 3:
        raise ValueError("need matching delay and P_b arrays of at least three points")

    def resid(q):
        return bunching_1d(d, abs(q[0]), abs(q[1]), gamma) - p

    r = least_squares(resid, x0=[sigma0, a0], xtol=1e-15, ftol=1e-15, gtol=1e-15)
    return abs(float(r.x[0])), abs(float(r.x[1]))
