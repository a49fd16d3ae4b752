"""Synthetic workloads of the projector benchmarks and parity tests.

Shapes follow the paper's use cases: grids from 3 to 25 planetary radii with
log-spaced shells (Sec. 6), detectors at orbit distance 60 looking at the
origin (Sec. 4.2-4.3), Table 3 grid/detector sizes. All densities and
orientations are seeded (synth.SplitMix64). Only shapes and seeds live here.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import synth


@dataclass
class ViewSet:
    kind: str                 # "cone" or "parallel"
    pos: np.ndarray           # (n_views, 3)
    shape: tuple              # (H, W)
    fov_deg: float = 30.0     # cone: full field of view
    size: float = 50.0        # parallel: detector extent

    @property
    def n_rays(self):
        return self.pos.shape[0] * self.shape[0] * self.shape[1]


@dataclass
class Workload:
    name: str
    edges: synth.GridEdges
    rho: np.ndarray
    views: list = field(default_factory=list)

    @property
    def n_rays(self):
        return sum(v.n_rays for v in self.views)

    def describe(self):
        nr, ne, na = self.edges.shape
        parts = [f"{v.pos.shape[0]}x{v.kind}{v.shape[0]}x{v.shape[1]}" for v in self.views]
        return f"{self.name}: grid {nr}x{ne}x{na}, " + " + ".join(parts)


def tiny() -> Workload:
    """Plain projector, tiny: 20 x 15 x 30 grid, one 64 x 64 cone view at 60, 30 deg."""
    e = synth.grid_edges(20, 15, 30)
    rho = synth.blob_phantom(e, seed=1, n_blobs=5, scale_height=4.0)
    return Workload("tiny", e, rho, [ViewSet("cone", np.array([[60.0, 0.0, 0.0]]), (64, 64), 30.0)])


def paper_scale() -> Workload:
    """Paper-like scale: 100 x 60 x 120 grid; 32 cone views of 256^2 on a circular
    orbit of radius 60 (30 deg) plus 32 parallel views of 256^2 at random
    orientations (detector 50 x 50)."""
    e = synth.grid_edges(100, 60, 120)
    rho = synth.blob_phantom(e, seed=2, n_blobs=5, scale_height=4.0)
    cone = ViewSet("cone", synth.circular_orbit(32, 60.0), (256, 256), 30.0)
    par = ViewSet("parallel", synth.random_positions(32, seed=3, radius=60.0), (256, 256), size=50.0)
    return Workload("paper_scale", e, rho, [cone, par])


def table3(row: int) -> Workload:
    """Table 3 shapes: 1x256^2 on (100,100,100), 1x512^2 on (50,50,50), 30x64^2 on (50,50,50)."""
    shapes = [((100, 100, 100), 1, 256), ((50, 50, 50), 1, 512), ((50, 50, 50), 30, 64)]
    (nr, ne, na), nv, det = shapes[row]
    e = synth.grid_edges(nr, ne, na)
    rho = synth.blob_phantom(e, seed=10 + row)
    pos = synth.circular_orbit(nv, 60.0)
    return Workload(f"table3_{row}", e, rho, [ViewSet("cone", pos, (det, det), 30.0)])


@dataclass
class Instance:
    edges: synth.GridEdges
    rho: np.ndarray
    view: ViewSet


def batched(n: int = 64, seed: int = 6, fov_deg: float = 50.0):
    """Uneven independent reconstructions: N_r in 20-120, N_e in 20-90, N_a in
    40-180, 4-96 cone views of 64^2-512^2 on orbits of radius 60 at seeded
    inclinations, seeded blob densities."""
    rng = synth.SplitMix64(seed)
    nr, ne, na = rng.integers(20, 120, n), rng.integers(20, 90, n), rng.integers(40, 180, n)
    nv, det = rng.integers(4, 96, n), rng.integers(64, 512, n)
    incl = rng.uniform(n, 0.0, 60.0)
    out = []
    for i in range(n):
        e = synth.grid_edges(int(nr[i]), int(ne[i]), int(na[i]))
        rho = synth.blob_phantom(e, seed=10_000 + i)
        pos = synth.circular_orbit(int(nv[i]), 60.0, incline_deg=float(incl[i]), phase=0.1 * i)
        out.append(Instance(e, rho, ViewSet("cone", pos, (int(det[i]), int(det[i])), fov_deg)))
    return out


@dataclass
class Differentiation:
    edges: synth.GridEdges
    view: ViewSet
    n_basis: int
    L: int
    coeffs: np.ndarray     # true model coefficients (n_basis, (L+1)^2)
    noise_seed: int
    noise_frac: float


def differentiation(shape=(128, 64, 128), n_views=64, det=512, n_basis=20, L=8) -> Differentiation:
    """SH (L <= 8) x 20 radial cubic B-splines rendered on a 128 x 64 x 128 grid;
    64 cone views of 512^2 (50 deg) from an orbit of radius 60 inclined 30 deg;
    Gaussian noise of 1% of the peak. True coefficients: an exp(-r/4) radial
    profile in the l = 0 term (its B-spline coefficients at the knot averages),
    seeded higher-degree terms of 20% relative size, decaying with l."""
    e = synth.grid_edges(*shape)
    rng = synth.SplitMix64(4)
    nq = (L + 1) ** 2
    k = 3
    n_int = n_basis - k - 1
    knots = np.concatenate([[3.0] * (k + 1), 3.0 + 22.0 * np.arange(1, n_int + 1) / (n_int + 1), [25.0] * (k + 1)])
    greville = np.array([knots[j + 1:j + k + 1].mean() for j in range(n_basis)])
    c = np.zeros((n_basis, nq))
    c[:, 0] = np.exp(-greville / 4.0) * 2.0 * np.sqrt(np.pi)
    ell = np.floor(np.sqrt(np.arange(nq))).astype(int)
    c[:, 1:] = 0.2 * c[:, :1] * rng.normal(n_basis * (nq - 1)).reshape(n_basis, nq - 1) / (ell[1:] + 1.0)
    pos = synth.circular_orbit(n_views, 60.0, incline_deg=30.0, phase=float(synth.SplitMix64(5).uniform(1)[0]))
    return Differentiation(e, ViewSet("cone", pos, (det, det), 50.0), n_basis, L, c.astype(np.float32), 44, 0.01)


class Exosphere:
    edges: synth.GridEdges
    pos: np.ndarray        # (n_views, 3) spacecraft positions
    shape: tuple           # (n_rad, n_az) polar bins
    fov_deg: float
    L: int
    coeffs: np.ndarray     # true per-shell coefficients (N_r, (L+1)^2)
    weights: np.ndarray    # (n_views, n_rad, n_az): Eq. 9's (g / 4 pi) phi(n)
    snr_db: float
    noise_seed: int
    threshold: float       # density above which the retrieval error is scored


def exosphere(shape=(50, 45, 90), n_views=10, bins=(100, 50), fov_deg=18.0, L=3) -> Exosphere:
    """Synthetic stand-in for the Sec. 6 experiment (the [33] model and the
    Carruthers ephemeris are not available): a hydrogen exosphere from 3 to
    25 Earth radii (log-spaced shells) with density 10 (3 / r)^3 in units of
    1000 atoms/cm^3, times (1 + 0.3 sin(t) cos(p) + 0.1 P_2(cos t)) (a
    day-night and a polar asymmetry, exact in degree <= 2); 10 views spread
    evenly over a circle of radius 60 around the sun-Earth line at 235 Earth
    radii (within 15 deg of the line, a stand-in for the unavailable
    ephemeris), looking at the Earth, +z up, 18 deg field of view
    polar-binned to 100 x 50; the
    known factor (g / 4 pi) phi(n) with g / 4 pi = 1 and a Rayleigh-like
    phase function 3/4 (1 + cos^2 T), T the angle between the pixel's nominal
    line of sight and the sun direction +x; 45 dB additive white Gaussian
    noise; errors scored where the density exceeds 25 atoms/cm^3."""
    e = synth.grid_edges(*shape)
    nq = (L + 1) ** 2
    rc = 0.5 * (e.r[1:] + e.r[:-1])
    n = 10.0 * (3.0 / rc) ** 3
    c = np.zeros((shape[0], nq))
    c[:, 0] = n * 2.0 * np.sqrt(np.pi)                       # 1 = 2 sqrt(pi) Y_00
    c[:, 3] = 0.3 * n * np.sqrt(4.0 * np.pi / 3.0)           # sin t cos p = sqrt(4 pi / 3) Y_11
    c[:, 6] = 0.1 * n * np.sqrt(4.0 * np.pi / 5.0)           # P_2(cos t) = sqrt(4 pi / 5) Y_20
    ang = 2.0 * np.pi * np.arange(n_views) / n_views
    pos = np.stack([np.full(n_views, 235.0), 60.0 * np.cos(ang), 60.0 * np.sin(ang)], 1)
    half = 0.5 * np.radians(fov_deg)
    th = (np.arange(bins[0]) + 0.5) / bins[0] * half
    ps = 2.0 * np.pi * (np.arange(bins[1]) + 0.5) / bins[1]
    w = np.zeros((n_views,) + tuple(bins))
    for v in range(n_views):
        look = -pos[v] / np.linalg.norm(pos[v])
        right = np.cross(look, [0.0, 0.0, 1.0])
        right /= np.linalg.norm(right)
        up = np.cross(right, look)
        T, P = np.meshgrid(th, ps, indexing="ij")
        d = np.cos(T)[..., None] * look + np.sin(T)[..., None] * (np.cos(P)[..., None] * right
                                                                  + np.sin(P)[..., None] * up)
        cos_t = d[..., 0]  # sun along +x
        w[v] = 0.75 * (1.0 + cos_t ** 2)
    ex = Exosphere()
    ex.edges, ex.pos, ex.shape, ex.fov_deg, ex.L = e, pos, tuple(bins), fov_deg, L
    ex.coeffs = c.astype(np.float32)
    ex.weights = w.astype(np.float32)
    ex.snr_db, ex.noise_seed, ex.threshold = 45.0, 61, 0.025
    return ex
