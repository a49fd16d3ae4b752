"""Pins for the dynamic-object oracle (Sec. 4.4: a 4D object seen by a
collection of sequential views, one volume per view).

A shrinking uniform ball gives closed-form chords per view; scaling each
volume by its own factor scales exactly that view's block (a mix-up of views
and volumes fails it); the FP64 adjoint identity pins the adjoint's layout.
"""
import math

import numpy as np

import oracle
from paper_2608_16960_gb300 import synth


def views(n, H=8, W=8, radius=20.0):
    ang = np.linspace(0.0, 2 * math.pi, n, endpoint=False)
    pos = np.stack([radius * np.cos(ang), radius * np.sin(ang), 3.0 * np.sin(2 * ang)], 1)
    return oracle.cone_rays(pos, H, W, 25.0)


def test_shrinking_ball_chords():
    """Volume k is 1 inside r < R_k (shell edges at every R_k): view k sees
    the chord 2 sqrt(R_k^2 - b^2) of its own ball."""
    e = synth.grid_edges(4, 3, 6, r_min=0.0, r_max=4.0, log_r=False)
    R = [4.0, 3.0, 2.0, 1.0]
    rho = np.stack([(np.arange(4) < Rk).astype(np.float64)[:, None, None] * np.ones(e.shape) for Rk in R])
    st, di = views(4)
    y = oracle.forward_dynamic(e, st, di, rho, 4)
    n = di / np.linalg.norm(di, axis=1, keepdims=True)
    b = np.linalg.norm(np.cross(st, n), axis=1).reshape(4, -1)
    for k, Rk in enumerate(R):
        ref = 2.0 * np.sqrt(np.maximum(Rk * Rk - b[k] ** 2, 0.0))
        assert np.max(np.abs(y[k] - ref)) < 1e-12


def test_each_view_sees_its_own_volume():
    e = synth.grid_edges(6, 5, 8)
    base = synth.SplitMix64(2).uniform(6 * 5 * 8, 0.1, 1.0).reshape(e.shape)
    c = np.array([1.0, 2.0, 5.0, 0.5, 3.0])
    st, di = views(5)
    y = oracle.forward_dynamic(e, st, di, c[:, None, None, None] * base, 5)
    static = oracle.forward(e, st, di, base).reshape(5, -1)
    assert np.allclose(y, c[:, None] * static, rtol=1e-13, atol=0.0)
    assert np.any(static > 0)


def test_dynamic_adjoint_identity():
    e = synth.grid_edges(5, 4, 7)
    g = synth.SplitMix64(9)
    rho = g.uniform(3 * 5 * 4 * 7, -1.0, 1.0).reshape((3,) + e.shape)
    st, di = views(3)
    yv = g.uniform(3 * 64, -1.0, 1.0).reshape(3, 64)
    lhs = np.sum(oracle.forward_dynamic(e, st, di, rho, 3) * yv)
    rhs = np.sum(rho * oracle.adjoint_dynamic(e, st, di, yv, 3))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))
