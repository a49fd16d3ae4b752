"""Autotuner and batched persistent / graph-captured SIRT, through the C ABI.

Each instance of a batch must equal the single-instance tsp_sirt (same
traversal; only float32 atomic summation order differs), graph replay must be
idempotent, and the autotuner's cached choice must be what default calls use.
"""
import math

import numpy as np
import pytest
import torch

from paper_2608_16960_gb300 import synth, workloads
from paper_2608_16960_gb300._lib import TspError
from paper_2608_16960_gb300.projector import (Batch, Geometry, Grid, tsp_autotune, tsp_autotune_clear,
                                              tsp_device_status, tsp_forward, tsp_sirt)

from _util import parity

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _instances():
    """Uneven instances: cone, parallel and free-form geometries, wedge and full grids."""
    out = []
    specs = [((12, 9, 20), "cone", 5, (40, 48)), ((20, 14, 30), "parallel", 3, (33, 37)),
             ((8, 6, 10), "cone", 9, (24, 24)), ((16, 12, 24), "rays", 0, (2000,)),
             ((24, 10, 40), "cone", 2, (64, 50))]
    for i, (shape, kind, nv, det) in enumerate(specs):
        if i == 2:
            e = synth.grid_edges(*shape, theta=(0.3, 2.5), phi=(0.5, 4.0))
        else:
            e = synth.grid_edges(*shape)
        grid = Grid.from_edges(e)
        if kind == "cone":
            geom = Geometry.cone(synth.circular_orbit(nv, 60.0, incline_deg=10.0 * i), det, 50.0)
        elif kind == "parallel":
            geom = Geometry.parallel(synth.random_positions(nv, 200 + i), det, 50.0)
        else:
            s, d = synth.random_rays(det[0], 300 + i)
            geom = Geometry.rays(torch.tensor(s, device=DEV), torch.tensor(d, device=DEV))
        truth = torch.tensor(synth.training_phantom(e, 500 + i), device=DEV)
        y = tsp_forward(grid, geom, truth).contiguous()
        out.append((grid, geom, y))
    return out


def test_autotune_caches_and_default_calls_use_it():
    tsp_autotune_clear()
    wl = workloads.tiny()
    grid = Grid.from_edges(wl.edges)
    v = wl.views[0]
    geom = Geometry.cone(v.pos, v.shape, v.fov_deg)
    f, a = tsp_autotune(grid, geom)
    assert f[0] in (64, 128, 256, 512) and f[1] in (4, 8, 16, 32) and a[2] in (0, 1)
    rho = torch.tensor(wl.rho, device=DEV)
    # default call (tuned) and explicit call give bit-identical forward results
    assert torch.equal(tsp_forward(grid, geom, rho), tsp_forward(grid, geom, rho, launch=f))
    assert tsp_device_status() == 0


@pytest.mark.parametrize("nonneg", [False, True])
def test_batch_matches_single_instance_sirt(nonneg):
    inst = _instances()
    xs = [torch.zeros(g.shape, device=DEV) for g, _, _ in inst]
    b = Batch([(g, geo, y, x) for (g, geo, y), x in zip(inst, xs)])
    b.sirt(4, nonneg=nonneg)
    torch.cuda.synchronize()
    for i, (g, geo, y) in enumerate(inst):
        ref = torch.zeros(g.shape, device=DEV)
        tsp_sirt(g, geo, y, ref, 4, nonneg=nonneg)
        parity(xs[i].cpu().numpy(), ref.cpu().numpy(), what=f"batch instance {i}")
    assert tsp_device_status() == 0


def test_batch_graph_replay_is_idempotent_and_matches_direct():
    inst = _instances()
    xs = [torch.zeros(g.shape, device=DEV) for g, _, _ in inst]
    b = Batch([(g, geo, y, x) for (g, geo, y), x in zip(inst, xs)])
    b.capture(6)
    b.launch()
    torch.cuda.synchronize()
    first = [x.clone() for x in xs]
    for x in xs:
        x.zero_()
    b.launch()
    torch.cuda.synchronize()
    for a, c in zip(first, xs):
        assert torch.allclose(a, c, rtol=1e-5, atol=1e-7)
    for x in xs:
        x.zero_()
    b.sirt(6)
    torch.cuda.synchronize()
    for a, c in zip(first, xs):
        assert torch.allclose(a, c, rtol=1e-5, atol=1e-7)
    r, v, blk = b.info()
    assert r == sum(geo.n_rays for _, geo, _ in inst) and v == sum(g.voxels for g, _, _ in inst)


def test_batch_launch_without_capture_is_rejected():
    inst = _instances()[:2]
    xs = [torch.zeros(g.shape, device=DEV) for g, _, _ in inst]
    b = Batch([(g, geo, y, x) for (g, geo, y), x in zip(inst, xs)])
    with pytest.raises(TspError):
        b.launch()
