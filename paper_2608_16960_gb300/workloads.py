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
