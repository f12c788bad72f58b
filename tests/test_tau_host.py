"""Host logic of the tau sweep (Section 4, Tables 1-2): the parabolic
minimiser and the (min rho)^(1 - eps) window, on synthetic rho(tau) curves
with known answers (no GPU)."""
import math

import numpy as np

from paper_1911_05888_gb300 import tau as T


def test_parabolic_min_recovers_vertex_of_log_parabola():
    t0 = 0.073
    taus = 0.1 * 2.0 ** (np.arange(-8, 9) / 4)
    rhos = np.exp(-2.0 + 0.7 * (np.log(taus) - math.log(t0)) ** 2)
    assert abs(T.parabolic_min(taus, rhos) / t0 - 1) <= 1e-9


def test_window_of_log_parabola():
    # log rho = c + a (log t - log t0)^2, threshold (1 - eps) c  ->  |log t - log t0| = sqrt(-eps c / a)
    t0, a, c = 0.1, 0.5, -2.5
    taus = t0 * 2.0 ** (np.arange(-40, 41) / 20)
    rhos = np.exp(c + a * (np.log(taus) - math.log(t0)) ** 2)
    lo, hi = T.window(taus, rhos)
    half = math.sqrt(-T.EPS * c / a)
    assert abs(math.log(lo) - (math.log(t0) - half)) <= 2e-3
    assert abs(math.log(hi) - (math.log(t0) + half)) <= 2e-3


def test_window_open_end_and_edge_minimum():
    taus = np.array([0.01, 0.02, 0.04, 0.08])
    rhos = np.array([0.10, 0.101, 0.3, 0.6])
    lo, hi = T.window(taus, rhos)
    assert lo is None and 0.02 < hi < 0.04
    assert T.parabolic_min(taus, rhos) == 0.01
