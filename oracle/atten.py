"""FP64 oracle of the attenuated projector (Sec. 9.3, Eq. 14-18).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import this module. The
product path never calls it and shares no code with it.

Model (Eq. 16-17): the radiance of a line of sight x + n l, l in [0, inf), is

    y = sum_i (e^{-tau_1} rho)[v_i] e^{-tau_2,i} dl_i,
    tau_2,i = sum_{j <= i} (sigma rho)[v_j] dl_j          (Eq. 18, inclusive)

over the ray's segments (v_i, dl_i) in order of increasing l, and
tau_1 = F_1(sigma rho) (Eq. 14, 17): F_1 traces one ray per voxel from its
centroid toward the sun (Fig. 16b).

Readings (the paper leaves these open):
  * the segments that Eq. 17-18 sum over are the maximal runs of the ray in
    one voxel: pieces that touch end to start in the same voxel are one
    segment (a traversal may cut a voxel's run at points that are no grid
    boundary, e.g. the closest approach to the origin; with the inclusive
    running sum such a cut would change y). Pieces of one voxel separated by
    a stretch outside the grid (the inner hole, outside a wedge) stay apart;
  * the centroid of a voxel is the point at the arithmetic midpoints of its r,
    theta and phi edges;
  * the sun is given as a direction vector; F_1's rays run from the centroids
    along it to infinity, through the same grid;
  * Eq. 18 is read as printed: a segment's own optical depth attenuates it.

The gradient functions differentiate these sums term by term, with the
suffix sums of the per-segment contributions written out explicitly.
"""
from __future__ import annotations

import numpy as np

from . import adjoint as _adjoint
from . import forward as _forward
from . import ray_pieces as _ray_pieces


def centroids(edges) -> np.ndarray:
    """(N_r N_e N_a, 3) Cartesian centroids in flat voxel order (r, theta,
    phi midpoints; Sec. 2.2's spherical coordinates)."""
    r, t, p = (np.asarray(e, dtype=np.float64) for e in (edges.r, edges.theta, edges.phi))
    rc, tc, pc = 0.5 * (r[1:] + r[:-1]), 0.5 * (t[1:] + t[:-1]), 0.5 * (p[1:] + p[:-1])
    R, T, P = np.meshgrid(rc, tc, pc, indexing="ij")
    return np.stack([R * np.sin(T) * np.cos(P), R * np.sin(T) * np.sin(P), R * np.cos(T)], -1).reshape(-1, 3)


def sunward_rays(edges, sun):
    """F_1's rays (Fig. 16b): one per voxel, from its centroid along the unit
    sun direction. Returns (V, 3) starts and directions."""
    s = np.asarray(sun, dtype=np.float64)
    s = s / np.linalg.norm(s)
    st = centroids(edges)
    return st, np.broadcast_to(s, st.shape).copy()


def optical_depth(edges, rho, sigma, starts, dirs) -> np.ndarray:
    """tau_1 = F_1(sigma rho) (Eq. 14 discretised as in Eq. 17): the plain
    projector applied to sigma * rho over the sunward rays, one value per voxel."""
    b = np.asarray(sigma, np.float64) * np.asarray(rho, np.float64)
    return _forward(edges, starts, dirs, b).reshape(edges.shape)


def optical_depth_backward(edges, rho, sigma, starts, dirs, g_tau1):
    """Gradients of <g_tau1, F_1(sigma rho)> with respect to rho and sigma:
    sigma F_1^T g and rho F_1^T g."""
    g = _adjoint(edges, starts, dirs, np.asarray(g_tau1, np.float64).reshape(-1))
    return np.asarray(sigma, np.float64) * g, np.asarray(rho, np.float64) * g


def segments(edges, x, n):
    """Segments of one ray in order: the definition's pieces with touching
    pieces of the same voxel joined (voxel, length)."""
    v, l0, ln = _ray_pieces(edges, x, n)
    vs, ls = [], []
    for k in range(len(v)):
        if vs and v[k] == vs[-1] and l0[k] == l0[k - 1] + ln[k - 1]:
            ls[-1] += ln[k]
        else:
            vs.append(v[k])
            ls.append(ln[k])
    return np.asarray(vs, dtype=np.int64), np.asarray(ls, dtype=np.float64)


def _ray_terms(edges, x, n, rho, sigma, tau1):
    """Per-segment quantities of one ray: voxels, lengths, a = e^{-tau_1} rho
    and b = sigma rho at the voxels, tau_2 (Eq. 18) and the contributions c_i."""
    v, dl = segments(edges, x, n)
    a = (np.exp(-tau1) * rho).reshape(-1)[v]
    b = (sigma * rho).reshape(-1)[v]
    tau2 = np.cumsum(b * dl)
    c = a * np.exp(-tau2) * dl
    return v, dl, a, b, tau2, c


def forward(edges, starts, dirs, rho, sigma, tau1) -> np.ndarray:
    """Attenuated y (Eq. 16-18) for rays given as (n, 3) starts and
    directions; rho, sigma, tau1 are volumes (N_r, N_e, N_a)."""
    rho, sigma, tau1 = (np.asarray(z, np.float64).reshape(edges.shape) for z in (rho, sigma, tau1))
    starts, dirs = np.asarray(starts).reshape(-1, 3), np.asarray(dirs).reshape(-1, 3)
    y = np.zeros(starts.shape[0])
    for i in range(starts.shape[0]):
        *_, c = _ray_terms(edges, starts[i], dirs[i], rho, sigma, tau1)
        y[i] = c.sum()
    return y


def backward(edges, starts, dirs, rho, sigma, tau1, gy):
    """Gradients of sum_k gy_k y_k (y of `forward`) with respect to rho, sigma
    and tau1. Per ray, with S_i = sum_{k >= i} c_k:
      d y / d a(v_i) = e^{-tau_2,i} dl_i,   d y / d b(v_i) = -dl_i S_i,
    and a = e^{-tau_1} rho, b = sigma rho."""
    rho, sigma, tau1 = (np.asarray(z, np.float64).reshape(edges.shape) for z in (rho, sigma, tau1))
    starts, dirs = np.asarray(starts).reshape(-1, 3), np.asarray(dirs).reshape(-1, 3)
    V = rho.size
    ga, gb = np.zeros(V), np.zeros(V)
    for i in range(starts.shape[0]):
        if gy[i] == 0.0:
            continue
        v, dl, a, b, tau2, c = _ray_terms(edges, starts[i], dirs[i], rho, sigma, tau1)
        S = np.cumsum(c[::-1])[::-1]
        np.add.at(ga, v, gy[i] * np.exp(-tau2) * dl)
        np.add.at(gb, v, -gy[i] * dl * S)
    e1 = np.exp(-tau1).reshape(-1)
    r, s = rho.reshape(-1), sigma.reshape(-1)
    g_rho = e1 * ga + s * gb
    g_sigma = r * gb
    g_tau1 = -r * e1 * ga
    return g_rho.reshape(edges.shape), g_sigma.reshape(edges.shape), g_tau1.reshape(edges.shape)
