"""Seeded synthetic inputs for the spherical-grid projector.

This module only *makes inputs*: grid boundary locations, phantom densities,
detector positions and free-form rays. It holds none of the projector's
arithmetic (no ray/boundary intersection, no ordering, no voxel lookup), so
both the CUDA path and the FP64 oracle can be fed from it without sharing
any of the method.

Randomness comes from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), implemented here from its
published definition so that the same seed gives the same numbers on every
machine and numpy version.

Workload shapes follow the paper: grids spanning 3-25 planetary radii with
log-spaced radial shells (Sec. 6), uniform polar and azimuthal bins
(Sec. 4.1), detectors at orbit distance looking at the origin (Sec. 4.2-4.3),
and the grid/detector sizes of Table 3.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


class SplitMix64:
    """Counter-based SplitMix64 stream: output i = mix(seed + (i+1)*golden)."""

    def __init__(self, seed: int):
        self.state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
        self.count = 0

    def next_u64(self, n: int) -> np.ndarray:
        idx = np.arange(self.count + 1, self.count + n + 1, dtype=np.uint64)
        self.count += n
        with np.errstate(over="ignore"):
            z = self.state + idx * _GOLDEN
            z = (z ^ (z >> np.uint64(30))) * _M1
            z = (z ^ (z >> np.uint64(27))) * _M2
            z = z ^ (z >> np.uint64(31))
        return z

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        u = (self.next_u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u

    def normal(self, n: int) -> np.ndarray:
        # Box-Muller on two uniform streams; 1-u keeps the log argument in (0, 1].
        u1 = 1.0 - self.uniform(n)
        u2 = self.uniform(n)
        return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)

    def integers(self, lo: int, hi: int, n: int) -> np.ndarray:
        """Uniform integers in [lo, hi] inclusive."""
        return lo + np.floor(self.uniform(n) * (hi - lo + 1)).astype(np.int64)

    def unit_vectors(self, n: int) -> np.ndarray:
        z = self.uniform(n, -1.0, 1.0)
        ph = self.uniform(n, 0.0, 2.0 * math.pi)
        s = np.sqrt(np.maximum(0.0, 1.0 - z * z))
        return np.stack([s * np.cos(ph), s * np.sin(ph), z], axis=1)


@dataclass
class GridEdges:
    r: np.ndarray      # (N_r+1,) radial boundaries, increasing
    theta: np.ndarray  # (N_e+1,) polar boundaries in [0, pi], increasing
    phi: np.ndarray    # (N_a+1,) azimuthal boundaries, increasing, span <= 2 pi

    @property
    def shape(self):
        return (len(self.r) - 1, len(self.theta) - 1, len(self.phi) - 1)


def grid_edges(nr: int, ne: int, na: int, r_min: float = 3.0, r_max: float = 25.0,
               log_r: bool = True, theta=(0.0, math.pi), phi=(0.0, 2.0 * math.pi)) -> GridEdges:
    """Boundary locations: log-spaced shells (Sec. 6 uses 3-25 Re) and uniform angles."""
    k = np.arange(nr + 1, dtype=np.float64)
    if log_r and r_min > 0:
        r = r_min * (r_max / r_min) ** (k / nr)
        r[0], r[-1] = r_min, r_max
    else:
        r = r_min + (r_max - r_min) * k / nr
    th = theta[0] + (theta[1] - theta[0]) * np.arange(ne + 1, dtype=np.float64) / ne
    ph = phi[0] + (phi[1] - phi[0]) * np.arange(na + 1, dtype=np.float64) / na
    th[-1] = theta[1]
    ph[-1] = phi[1]
    return GridEdges(r, th, ph)


def voxel_centres(edges: GridEdges):
    """Cartesian coordinates of voxel centres, taken at the arithmetic midpoint of
    each pair of boundaries. Returns (x, y, z, r) arrays of shape (N_r, N_e, N_a)."""
    rc = 0.5 * (edges.r[:-1] + edges.r[1:])
    tc = 0.5 * (edges.theta[:-1] + edges.theta[1:])
    pc = 0.5 * (edges.phi[:-1] + edges.phi[1:])
    R, T, P = np.meshgrid(rc, tc, pc, indexing="ij")
    return R * np.sin(T) * np.cos(P), R * np.sin(T) * np.sin(P), R * np.cos(T), R


def blob_params(seed: int, n_blobs: int = 5, scale_height: float = 4.0, sigma=(1.0, 3.0), amp=(0.1, 1.0),
                centre_r=(4.0, 20.0)) -> np.ndarray:
    """Phantom parameters: row 0 = (scale height, 0, 0, 0, 0), then one row per
    blob (centre x, y, z, amplitude, sigma). float64 (1 + n_blobs, 5)."""
    rng = SplitMix64(seed)
    dirs = rng.unit_vectors(n_blobs)
    radii = rng.uniform(n_blobs, *centre_r)
    amps = rng.uniform(n_blobs, *amp)
    sig = rng.uniform(n_blobs, *sigma)
    out = np.zeros((1 + n_blobs, 5))
    out[0, 0] = scale_height
    out[1:, :3] = dirs * radii[:, None]
    out[1:, 3] = amps
    out[1:, 4] = sig
    return out


def render_phantom(edges: GridEdges, params: np.ndarray) -> np.ndarray:
    """exp(-r/H) + sum_j A_j exp(-|p - c_j|^2 / (2 s_j^2)) at the voxel centres."""
    x, y, z, r = voxel_centres(edges)
    rho = np.exp(-r / params[0, 0])
    for c0, c1, c2, A, s in params[1:]:
        d2 = (x - c0) ** 2 + (y - c1) ** 2 + (z - c2) ** 2
        rho = rho + A * np.exp(-d2 / (2.0 * s * s))
    return rho.astype(np.float32)


def blob_phantom(edges: GridEdges, seed: int, n_blobs: int = 5, scale_height: float = 4.0,
                 sigma=(1.0, 3.0), amp=(0.1, 1.0), centre_r=(4.0, 20.0)) -> np.ndarray:
    """exp(-r/H) background plus seeded isotropic Gaussian blobs, float32, C-order
    (N_r, N_e, N_a)."""
    return render_phantom(edges, blob_params(seed, n_blobs, scale_height, sigma, amp, centre_r))


def training_params(seed: int) -> np.ndarray:
    """Phantom family of the learned warm start: 1-8 blobs on exp(-r/H), H in U(2,6)."""
    rng = SplitMix64(seed ^ 0x5A5A5A5A)
    nb = int(rng.integers(1, 8, 1)[0])
    h = float(rng.uniform(1, 2.0, 6.0)[0])
    return blob_params(seed, n_blobs=nb, scale_height=h)


def training_phantom(edges: GridEdges, seed: int) -> np.ndarray:
    return render_phantom(edges, training_params(seed))


def circular_orbit(n_views: int, radius: float = 60.0, incline_deg: float = 0.0,
                   phase: float = 0.0) -> np.ndarray:
    """(n_views, 3) detector positions evenly spaced on a circle of given radius,
    tilted by incline_deg about the x axis."""
    w = phase + 2.0 * math.pi * np.arange(n_views) / n_views
    p = np.stack([radius * np.cos(w), radius * np.sin(w), np.zeros(n_views)], axis=1)
    a = math.radians(incline_deg)
    rot = np.array([[1, 0, 0], [0, math.cos(a), -math.sin(a)], [0, math.sin(a), math.cos(a)]])
    return p @ rot.T


def random_positions(n_views: int, seed: int, radius: float = 60.0) -> np.ndarray:
    """(n_views, 3) detector positions at isotropic random directions."""
    return SplitMix64(seed).unit_vectors(n_views) * radius


def random_rays(n: int, seed: int, start_radius: float = 60.0, aim_radius: float = 25.0):
    """Free-form rays: starts on a sphere of start_radius, each aimed at a random
    point inside the ball of aim_radius (some miss the grid, as in a real
    detector's corners). Directions are left unnormalised (scaled by a random
    factor) as in the paper's custom-ray example. Returns float32 (3, n) SoA
    arrays (starts, dirs)."""
    rng = SplitMix64(seed)
    starts = rng.unit_vectors(n) * start_radius
    aim = rng.unit_vectors(n) * (aim_radius * rng.uniform(n) ** (1.0 / 3.0))[:, None]
    dirs = (aim - starts) * rng.uniform(n, 0.5, 2.0)[:, None]
    return (np.ascontiguousarray(starts.T.astype(np.float32)),
            np.ascontiguousarray(dirs.T.astype(np.float32)))


def interior_rays(n: int, seed: int, radius: float = 20.0):
    """Free-form rays whose starts lie inside the grid (start-inside support)."""
    rng = SplitMix64(seed)
    starts = rng.unit_vectors(n) * (radius * rng.uniform(n) ** (1.0 / 3.0))[:, None]
    dirs = rng.unit_vectors(n)
    return (np.ascontiguousarray(starts.T.astype(np.float32)),
            np.ascontiguousarray(dirs.T.astype(np.float32)))


def uniform_volume(shape, seed: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    return SplitMix64(seed).uniform(int(np.prod(shape)), lo, hi).reshape(shape).astype(np.float32)
