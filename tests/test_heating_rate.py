"""The thermalization-rate extraction of Sec. IV, Gamma = 1/(t_2 - t_1) with
E(t_k) = E(0) e^-k, and the fit Gamma = exp(a omega + b), against curves
whose crossing times are known in closed form (host only)."""
import math

import numpy as np
import pytest

from paper_2111_08044_gb300 import paper_model as pm


def _grid(t_max, points):
    # the run's sampling: t = 0, then log-spaced times
    return np.concatenate([[0.0], np.logspace(-1, math.log10(t_max), points)])


@pytest.mark.parametrize("gamma", [0.3, 0.02, 1e-3])
def test_exponential_decay_gives_its_rate(gamma):
    """E(t) = E(0) exp(-Gamma t) crosses E(0) e^-k at t_k = k / Gamma."""
    t = _grid(20.0 / gamma, 2000)
    e = -0.515 * np.exp(-gamma * t)
    t1 = pm.crossing_time(t, e / e[0], 1)
    t2 = pm.crossing_time(t, e / e[0], 2)
    assert abs(t1 - 1.0 / gamma) < 2e-3 / gamma
    assert abs(t2 - 2.0 / gamma) < 2e-3 / gamma
    assert abs(pm.heating_rate(t, e) / gamma - 1.0) < 5e-3


def test_plateau_then_decay():
    """A fast early drop to a plateau at 0.9 E(0), then exp(-Gamma t): the
    crossings are those of the slow part, t_k = (k + ln 0.9) / Gamma, and
    their difference is 1 / Gamma whatever the plateau."""
    gamma = 0.01
    t = _grid(1e4, 4000)
    e = -0.5 * (0.9 + 0.1 * np.exp(-5.0 * t)) * np.exp(-gamma * t)
    t1 = pm.crossing_time(t, e / e[0], 1)
    assert abs(t1 - (1.0 + math.log(0.9)) / gamma) < 0.5
    assert abs(pm.heating_rate(t, e) / gamma - 1.0) < 5e-3


def test_curve_that_never_heats_has_no_rate():
    t = _grid(1e4, 200)
    e = -0.5 * (0.7 + 0.3 * np.exp(-t))  # settles at 0.7 E(0) > e^-1 E(0)
    assert pm.crossing_time(t, e / e[0], 1) is None
    assert pm.heating_rate(t, e) is None


def test_linear_interpolation_from_t_zero():
    """A crossing between t = 0 and the first log-spaced sample is taken on
    a linear scale (log 0 does not exist)."""
    t = np.array([0.0, 1.0, 10.0])
    r = np.array([1.0, 0.2, 0.1])
    level = math.exp(-1)
    assert abs(pm.crossing_time(t, r, 1) - (1.0 - level) / 0.8) < 1e-12


def test_fit_recovers_the_exponent():
    omegas = np.array([5.0, 5.5, 6.0, 6.5, 7.0])
    a, b = -2.48, 10.9  # the paper's fitted values, used here only as a shape
    rates = np.exp(a * omegas + b)
    fa, fb = pm.fit_rates(omegas, rates)
    assert abs(fa - a) < 1e-10 and abs(fb - b) < 1e-9
