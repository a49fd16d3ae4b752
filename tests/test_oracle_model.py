"""Pins for the model and Adam oracles: spherical-harmonic orthonormality by
quadrature and low-degree closed forms, B-spline partition of unity and
support, Adam closed forms, and the render adjoint identity."""
import math

import numpy as np

from oracle import shbs
from paper_2608_16960_gb300 import synth


def test_real_sh_orthonormal_by_quadrature():
    L = 8
    xg, wg = np.polynomial.legendre.leggauss(24)  # exact for the polynomial part in cos(theta)
    nphi = 40
    ph = 2 * math.pi * np.arange(nphi) / nphi
    T, P = np.meshgrid(np.arccos(xg), ph, indexing="ij")
    W = np.repeat(wg[:, None], nphi, axis=1) * (2 * math.pi / nphi)
    Y = shbs.real_sh(L, T.ravel(), P.ravel())
    G = Y.T @ (Y * W.ravel()[:, None])
    assert np.max(np.abs(G - np.eye((L + 1) ** 2))) < 1e-12


def test_real_sh_low_degree_closed_forms():
    rng = synth.SplitMix64(3)
    th, ph = rng.uniform(20, 0, math.pi), rng.uniform(20, 0, 2 * math.pi)
    Y = shbs.real_sh(2, th, ph)
    c1 = math.sqrt(3 / (4 * math.pi))
    assert np.allclose(Y[:, 0], 0.5 / math.sqrt(math.pi))
    assert np.allclose(Y[:, 2], c1 * np.cos(th))                 # (1, 0): z
    assert np.allclose(Y[:, 3], c1 * np.sin(th) * np.cos(ph))    # (1, 1): x
    assert np.allclose(Y[:, 1], c1 * np.sin(th) * np.sin(ph))    # (1,-1): y
    assert np.allclose(Y[:, 6], math.sqrt(5 / (16 * math.pi)) * (3 * np.cos(th) ** 2 - 1))  # (2, 0)


def test_bspline_partition_of_unity_and_support():
    r = np.linspace(3.0, 25.0, 301)
    B = shbs.bspline_matrix(r, 3.0, 25.0, 20)
    assert B.shape == (301, 20)
    assert np.allclose(B.sum(axis=1), 1.0) and np.all(B >= -1e-15)
    assert np.all(np.count_nonzero(B > 1e-14, axis=1) <= 4)      # cubic: at most 4 non-zero
    assert abs(B[0, 0] - 1.0) < 1e-12 and abs(B[-1, -1] - 1.0) < 1e-12  # clamped ends


def test_adam_closed_forms():
    p0 = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    # first step: bias-corrected moments are g and g^2, so p1 = p0 - lr g / (|g| + eps)
    p1 = shbs.adam(p0, [g], lr=0.1, eps=1e-8)
    assert np.allclose(p1, p0 - 0.1 * g / (np.abs(g) + 1e-8), atol=1e-15)
    # constant gradient: every step moves by the same amount
    p5 = shbs.adam(p0, [g] * 5, lr=0.1, eps=1e-8)
    assert np.allclose(p5, p0 - 5 * 0.1 * g / (np.abs(g) + 1e-8), atol=1e-12)


def test_render_adjoint_identity():
    e = synth.grid_edges(10, 6, 8)
    rng = synth.SplitMix64(4)
    c = rng.normal(20 * 9).reshape(20, 9)
    g = rng.normal(int(np.prod(e.shape))).reshape(e.shape)
    tables = shbs.model_tables(e, 20, 2)
    lhs = np.sum(shbs.render(e, c, 20, 2, tables) * g)
    rhs = np.sum(c * shbs.render_adjoint(e, g, 20, 2, tables))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
