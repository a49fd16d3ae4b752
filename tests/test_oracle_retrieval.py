"""Pins for the retrieval oracle (Sec. 6, Eq. 9-10).

A polar detector looking at the centre of a uniform ball sees, in radial bin
i, the chord at impact parameter D sin(theta_i), whatever the azimuthal bin;
the image orientation is pinned on a hand-checked view. The per-shell model
is checked on closed forms of the degree-0 and degree-1 harmonics and its
adjoint identity, the radial regulariser on a coefficient field linear in
the shell index, and the whole objective's gradient by finite differences.
"""
import math

import numpy as np

import oracle
from oracle import retrieval as orr
from paper_2608_16960_gb300 import synth


def test_polar_detector_chords_of_a_ball():
    """Camera at distance D looking at the centre of a uniform unit-density
    ball of radius R: bin (i, j) integrates 2 sqrt(R^2 - (D sin theta_i)^2)
    with theta_i = (i + 1/2) / n_rad * fov / 2."""
    R, D, fov = 10.0, 40.0, 30.0
    e = synth.grid_edges(12, 9, 16, r_min=0.0, r_max=R, log_r=False)
    st, di = orr.polar_rays([D, 0.0, 0.0], [0.0, 0.0, 0.0], [0.0, 0.0, 1.0], 8, 6, fov)
    y = oracle.forward(e, st, di, np.ones(e.shape)).reshape(8, 6)
    th = (np.arange(8) + 0.5) / 8 * math.radians(fov) / 2
    ref = 2.0 * np.sqrt(np.maximum(R * R - (D * np.sin(th)) ** 2, 0.0))
    assert np.max(np.abs(y - ref[:, None])) < 1e-11
    assert np.allclose(np.linalg.norm(di, axis=1), 1.0)


def test_polar_detector_orientation():
    """From +x looking at the origin with +z up, the image's right axis is +y
    (right = look x up): the azimuth psi near 0 leans to +y, near pi/2 to +z."""
    st, di = orr.polar_rays([50.0, 0.0, 0.0], [0.0, 0.0, 0.0], [0.0, 0.0, 1.0], 3, 4, 20.0)
    d = di.reshape(3, 4, 3)
    assert np.all(d[..., 0] < 0)                  # all look back toward the origin
    assert np.all(d[:, 0, 1] > 0) and np.all(d[:, 0, 2] > 0)   # psi = pi/4: +y and +z
    assert np.all(d[:, 1, 1] < 0) and np.all(d[:, 1, 2] > 0)   # psi = 3pi/4: -y, +z
    assert np.all(d[:, 3, 1] > 0) and np.all(d[:, 3, 2] < 0)   # psi = 7pi/4: +y, -z


def test_shell_model_closed_forms_and_adjoint():
    e = synth.grid_edges(5, 7, 9)
    L = 2
    nq = (L + 1) ** 2
    a = np.array([1.0, 0.5, 0.25, 0.125, 0.0625])
    c = np.zeros((5, nq))
    c[:, 0] = a                       # degree 0: a_r / (2 sqrt(pi)), constant on each shell
    rho = orr.shell_render(e, c, L)
    assert np.allclose(rho, (a / (2 * math.sqrt(math.pi)))[:, None, None] * np.ones(e.shape), rtol=1e-14)
    c = np.zeros((5, nq))
    c[2, 2] = 1.0                     # (1, 0) on shell 2 only: sqrt(3 / 4 pi) cos(theta)
    rho = orr.shell_render(e, c, L)
    tc = 0.5 * (e.theta[1:] + e.theta[:-1])
    assert np.allclose(rho[2], math.sqrt(3 / (4 * math.pi)) * np.cos(tc)[:, None] * np.ones((7, 9)), rtol=1e-13)
    assert np.all(rho[[0, 1, 3, 4]] == 0)
    g = synth.SplitMix64(4)
    c, r = g.uniform(5 * nq, -1, 1).reshape(5, nq), g.uniform(5 * 7 * 9, -1, 1).reshape(e.shape)
    assert abs(np.sum(orr.shell_render(e, c, L) * r) - np.sum(c * orr.shell_render_adjoint(e, r, L))) < 1e-12


def test_tikhonov_linear_field():
    """c[r] = alpha r + beta: every difference is alpha, so the term is
    lambda alpha^2 (N_r - 1) per coefficient; the gradient vanishes inside
    and is -/+ 2 lambda alpha at the first / last shell."""
    alpha, beta, lam = np.array([0.5, -2.0, 1.5]), np.array([1.0, 0.0, 3.0]), 0.7
    c = np.arange(6)[:, None] * alpha + beta
    val, g = orr.tikhonov(c, lam)
    assert abs(val - lam * 5 * np.sum(alpha ** 2)) < 1e-12
    assert np.allclose(g[1:-1], 0.0) and np.allclose(g[0], -2 * lam * alpha) and np.allclose(g[-1], 2 * lam * alpha)


def test_objective_gradient_by_finite_differences():
    e = synth.grid_edges(3, 4, 6, r_min=2.0, r_max=9.0)
    L, lam = 1, 0.3
    g = synth.SplitMix64(12)
    st, di = orr.polar_rays([[30.0, 4.0, 2.0], [-5.0, 28.0, -3.0]], [[0.0, 0.0, 0.0]] * 2, [[0.0, 0.0, 1.0]] * 2,
                            3, 4, 40.0)
    w = g.uniform(st.shape[0], 0.5, 1.5)
    y = g.uniform(st.shape[0], 0.0, 2.0)
    c = g.uniform(3 * 4, 0.0, 1.0).reshape(3, 4)
    val, grad = orr.objective(e, st, di, w, y, c, L, lam)
    h = 1e-6
    for idx in np.ndindex(c.shape):
        cp, cm = c.copy(), c.copy()
        cp[idx] += h
        cm[idx] -= h
        fd = (orr.objective(e, st, di, w, y, cp, L, lam)[0] - orr.objective(e, st, di, w, y, cm, L, lam)[0]) / (2 * h)
        assert abs(fd - grad[idx]) < 1e-6 * max(1.0, abs(fd)), (idx, fd, grad[idx])
