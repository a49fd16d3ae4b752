"""Pins for the SIRT oracle: convergence to the true density on a consistent,
overdetermined system, monotone decrease of the R-weighted residual, and
invariance of an exact solution."""
import numpy as np

import oracle
from oracle import sirt as osirt
from paper_2608_16960_gb300 import synth


def _problem():
    e = synth.grid_edges(2, 2, 3, r_min=2.0, r_max=6.0)
    s, d = synth.random_rays(400, 5, start_radius=20.0, aim_radius=6.0)
    s, d = s.T.astype(np.float64), d.T.astype(np.float64)
    x_true = synth.uniform_volume(e.shape, 6).astype(np.float64) + 0.5
    y = oracle.forward(e, s, d, x_true)
    return e, s, d, x_true, y


def test_sirt_converges_to_truth_on_consistent_system():
    e, s, d, x_true, y = _problem()
    x = osirt.sirt(e, s, d, y, np.zeros(e.shape), 400)
    assert np.max(np.abs(x - x_true)) < 1e-6 * np.max(x_true)


def test_sirt_weighted_residual_decreases_and_solution_is_fixed_point():
    e, s, d, x_true, y = _problem()
    R, C = osirt.weights(e, s, d)
    assert np.all(R > 0) or np.all(R >= 0)
    x = np.zeros(e.shape)
    prev = np.inf
    for _ in range(10):
        x = osirt.sirt(e, s, d, y, x, 1, weights_rc=(R, C))
        res = np.sum(R * (y - oracle.forward(e, s, d, x)) ** 2)
        assert res <= prev * (1 + 1e-12)
        prev = res
    x1 = osirt.sirt(e, s, d, y, x_true, 1, weights_rc=(R, C))
    assert np.max(np.abs(x1 - x_true)) < 1e-12


def test_sirt_nonneg_clamp():
    e, s, d, x_true, y = _problem()
    x = osirt.sirt(e, s, d, y - 5.0, np.zeros(e.shape), 5, nonneg=True)
    assert np.all(x >= 0)
