"""Parity at the sizes of every workload configuration, in the launch
configuration the library picks by default: the forward sampled against the
FP64 oracle (per ray, with the tolerance rule of tests/_util.py, and
normwise), the adjoint of sparse rays against the oracle's exact volume (per
voxel 1e-4 relative plus the crossing-position term of grazing_allowance in
tests/_util.py, and normwise 1e-4), and the adjoint identity
<F x, y> = <x, F^T y>.

Configurations: the differentiation grid 128 x 64 x 128 with 512^2 cone views
(50 deg); the largest instances of the uneven batched set, by voxels
(114 x 59 x 155, 93 views of 326^2) and by rays (94 views of 463^2, 20 M
rays); the three Table 3 shapes; the warm-start grid 64 x 48 x 96 with 48
cone views of 256^2. The GPU projects every view of a configuration; the
oracle checks rays of three of them (first, middle, last)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2608_16960_gb300 import synth, workloads
from paper_2608_16960_gb300.projector import Geometry, Grid, tsp_adjoint, tsp_device_status, tsp_forward

from _util import grazing_allowance, sparse_adjoint_parity

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _check(edges, rho, pos, shape, fov, n_fwd=1500, n_adj=600, seed=0, what=""):
    grid = Grid.from_edges(edges)
    geom = Geometry.cone(pos, shape, fov)
    nv, H, W = len(pos), shape[0], shape[1]
    views = sorted({0, nv // 2, nv - 1})
    st, di = oracle.cone_rays(np.asarray(pos)[views], H, W, fov)
    per = H * W

    # forward: every k-th ray of the checked views
    y = tsp_forward(grid, geom, torch.tensor(rho, device=DEV)).cpu().numpy().reshape(nv, per)
    assert np.all(np.isfinite(y)) and np.all(y >= 0)
    k = max(1, (len(views) * per) // n_fwd)
    idx = np.arange(k // 2, len(views) * per, k)
    got = y[views].reshape(-1)[idx]
    ref = oracle.forward(edges, st[idx], di[idx], rho)
    big = np.max(np.abs(ref))
    err = np.abs(got - ref)
    assert np.all(err <= 1e-4 * np.maximum(np.abs(ref), 1e-2 * big)), (what, err.max(), big)
    assert np.linalg.norm(got - ref) <= 1e-4 * np.linalg.norm(ref), what

    # adjoint of sparse rays: y non-zero on every k-th ray of the checked views
    k = max(1, (len(views) * per) // n_adj)
    idx = np.arange(k // 3, len(views) * per, k)
    vals = synth.SplitMix64(seed).uniform(len(idx), 0.5, 1.5)
    yv = np.zeros((nv, per), np.float32)
    sub = np.zeros(len(views) * per, np.float32)
    sub[idx] = vals
    yv[views] = sub.reshape(len(views), per)
    out = tsp_adjoint(grid, geom, torch.tensor(yv.reshape(geom.det_shape), device=DEV)).cpu().numpy()
    ref = oracle.adjoint(edges, st[idx], di[idx], sub[idx].astype(np.float64))
    allow, gmax = grazing_allowance(edges, st[idx], di[idx], sub[idx])
    sparse_adjoint_parity(out, ref, allow, gmax, what=f"sparse adjoint {what}")

    # adjoint identity over every view
    x = torch.tensor(synth.uniform_volume(grid.shape, seed + 1), device=DEV)
    yu = torch.tensor(synth.uniform_volume(geom.det_shape, seed + 2), device=DEV)
    lhs = torch.dot(tsp_forward(grid, geom, x).double().ravel(), yu.double().ravel()).item()
    rhs = torch.dot(x.double().ravel(), tsp_adjoint(grid, geom, yu).double().ravel()).item()
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs), (what, lhs, rhs)
    assert tsp_device_status() == 0


def test_differentiation_config():
    d = workloads.differentiation()
    pos = d.view.pos[[0, 21, 42, 63]]
    _check(d.edges, synth.blob_phantom(d.edges, seed=81), pos, d.view.shape, d.view.fov_deg, seed=810,
           what="128x64x128, 512^2")


@pytest.fixture(scope="module")
def batched_extremes():
    inst = workloads.batched()
    by_vox = max(inst, key=lambda i: int(np.prod(i.edges.shape)))
    by_rays = max(inst, key=lambda i: i.view.n_rays)
    return [by_vox, by_rays]


@pytest.mark.parametrize("which", [0, 1])
def test_batched_largest_instances(batched_extremes, which):
    it = batched_extremes[which]
    v = it.view
    _check(it.edges, it.rho, v.pos, v.shape, v.fov_deg, seed=820 + which,
           what=f"batched {it.edges.shape}, {len(v.pos)} x {v.shape}")


@pytest.mark.parametrize("row", [0, 1, 2])
def test_table3_shapes(row):
    wl = workloads.table3(row)
    v = wl.views[0]
    _check(wl.edges, wl.rho, v.pos, v.shape, v.fov_deg, seed=830 + row, what=f"table3 row {row}")


def test_warm_start_config():
    e = synth.grid_edges(64, 48, 96)
    pos = synth.circular_orbit(48, 60.0, incline_deg=20.0)
    _check(e, synth.training_phantom(e, 77), pos, (256, 256), 50.0, seed=840, what="64x48x96, 48 x 256^2")
