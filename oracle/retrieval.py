"""FP64 oracle of the exospheric retrieval pieces (Sec. 6, Eq. 9-10).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import this module.

  * polar-binned detector (Sec. 6: images binned to 100 radial x 50 azimuthal
    polar pixels with an equivalent field of view): the pixel (i, j) looks at
    angle theta_i = (i + 1/2) / n_rad * fov / 2 from the boresight, at
    azimuth psi_j = 2 pi (j + 1/2) / n_az around it;
  * per-shell spherical-harmonic model M(c) (Eq. 10):
    rho[ir, ie, ia] = sum_q c[ir, q] H_q(theta_ie, phi_ia), with the real
    orthonormal harmonics of oracle.shbs at the voxel centres;
  * radial Tikhonov term lambda ||D_r c||^2 (Eq. 10), D_r the first
    difference between neighbouring shells of each coefficient;
  * Eq. 9's known factor (g / 4 pi) phi(n) as a per-ray weight w: the model
    radiance is w * F rho, the data term sum (w F rho - y)^2.
"""
from __future__ import annotations

import math

import numpy as np

from . import adjoint as _adjoint
from . import forward as _forward
from .shbs import centres, real_sh


def _basis(pos, look_at, up):
    """Boresight and two image axes (right-handed: right = look x up)."""
    look = np.asarray(look_at, float) - np.asarray(pos, float)
    look /= np.linalg.norm(look)
    right = np.cross(look, np.asarray(up, float))
    right /= np.linalg.norm(right)
    return look, right, np.cross(right, look)


def polar_rays(pos, look_at, up, n_rad, n_az, fov_deg):
    """(V * n_rad * n_az, 3) starts and unit directions, row-major
    (view, radial bin, azimuthal bin)."""
    pos = np.asarray(pos, float).reshape(-1, 3)
    look_at = np.asarray(look_at, float).reshape(-1, 3)
    up = np.asarray(up, float).reshape(-1, 3)
    half = 0.5 * math.radians(fov_deg)
    th = (np.arange(n_rad) + 0.5) / n_rad * half
    ps = 2.0 * math.pi * (np.arange(n_az) + 0.5) / n_az
    starts, dirs = [], []
    for v in range(pos.shape[0]):
        look, right, upv = _basis(pos[v], look_at[v], up[v])
        T, P = np.meshgrid(th, ps, indexing="ij")
        d = (np.cos(T)[..., None] * look + np.sin(T)[..., None] * (np.cos(P)[..., None] * right
                                                                   + np.sin(P)[..., None] * upv))
        dirs.append(d.reshape(-1, 3))
        starts.append(np.broadcast_to(pos[v], (n_rad * n_az, 3)))
    return np.concatenate(starts), np.concatenate(dirs)


def shell_tables(edges, L):
    """H (N_e N_a, (L+1)^2): the harmonics at the voxel centres."""
    _, tc, pc = centres(edges)
    T, P = np.meshgrid(tc, pc, indexing="ij")
    return real_sh(L, T.ravel(), P.ravel())


def shell_render(edges, c, L, H=None):
    """M(c) of Eq. 10: one harmonic series per shell."""
    H = shell_tables(edges, L) if H is None else H
    return (np.asarray(c, float) @ H.T).reshape(edges.shape)


def shell_render_adjoint(edges, g, L, H=None):
    H = shell_tables(edges, L) if H is None else H
    return np.asarray(g, float).reshape(edges.shape[0], -1) @ H


def tikhonov(c, lam):
    """lambda ||D_r c||^2 and its gradient, D_r c = c[1:] - c[:-1]."""
    c = np.asarray(c, float)
    d = c[1:] - c[:-1]
    g = np.zeros_like(c)
    g[1:] += 2.0 * lam * d
    g[:-1] -= 2.0 * lam * d
    return lam * float(np.sum(d * d)), g


def weighted_residual(yhat, w, y):
    """sum (w yhat - y)^2 and its gradient with respect to yhat."""
    r = np.asarray(w, float) * np.asarray(yhat, float) - np.asarray(y, float)
    return float(np.sum(r * r)), 2.0 * np.asarray(w, float) * r


def objective(edges, starts, dirs, w, y, c, L, lam):
    """Eq. 10's objective ||y - w F M(c)||^2 + lambda ||D_r c||^2 and its
    gradient with respect to c (chain rule through M, F and the weight)."""
    H = shell_tables(edges, L)
    rho = shell_render(edges, c, L, H)
    yhat = _forward(edges, starts, dirs, rho)
    data, gy = weighted_residual(yhat, w, y)
    reg, gr = tikhonov(c, lam)
    g = shell_render_adjoint(edges, _adjoint(edges, starts, dirs, gy), L, H) + gr
    return data + reg, g
