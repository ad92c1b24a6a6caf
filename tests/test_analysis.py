"""The 1D scattering model of Eq. bunching and its fit (host analysis, no GPU)."""

import math

import numpy as np

from paper_1903_02581_gb300 import analysis as AN


def test_closed_form_limits():
    # no energy selectivity (a = 0): perfect antibunching at zero delay
    assert abs(AN.bunching_1d(0.0, 2.0, 0.0)) <= 1e-15
    # large delay: the packets no longer overlap, P_b -> 1/2
    assert abs(AN.bunching_1d(1e3, 2.0, 3.0) - 0.5) <= 1e-15
    # plane-wave limit: sigma -> infinity gives P_b(0) -> 0
    assert AN.bunching_1d(0.0, 1e4, 3.0) < 1e-6
    # zero delay: 1/2 - 1/2 sigma^2 / (sigma^2 + a^2 / (8 gamma)), gamma = 4 ln 2
    s, a = 1.5, 2.5
    ref = 0.5 - 0.5 * s * s / (s * s + a * a / (32.0 * math.log(2.0)))
    assert abs(AN.bunching_1d(0.0, s, a) - ref) <= 1e-15


def test_fit_recovers_parameters():
    d = np.linspace(-8, 8, 33)
    p = AN.bunching_1d(d, 1.7, 4.2)
    s, a = AN.fit_bunching_1d(d, p, sigma0=1.0, a0=1.0)
    assert abs(s - 1.7) <= 1e-8 and abs(a - 4.2) <= 1e-7
