"""CUDA SIRT (tsp_sirt) against the FP64 oracle's SIRT, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
from oracle import sirt as osirt
from paper_2608_16960_gb300 import synth, workloads
from paper_2608_16960_gb300.projector import Geometry, Grid, sirt_workspace, tsp_device_status, tsp_forward, tsp_sirt

from _util import oracle_rays, parity, pinned_scatter

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module")
def tiny():
    wl = workloads.tiny()
    grid = Grid.from_edges(wl.edges)
    v = wl.views[0]
    geom = Geometry.cone(v.pos, v.shape, v.fov_deg)
    st, di = oracle_rays(v)
    y = oracle.forward(wl.edges, st, di, wl.rho)
    return wl, grid, geom, st, di, y


@pytest.mark.parametrize("n_iter,nonneg", [(1, False), (5, False), (5, True)])
def test_sirt_matches_oracle(tiny, n_iter, nonneg):
    wl, grid, geom, st, di, y = tiny
    x = torch.zeros(grid.shape, device=DEV)
    yt = torch.tensor(y.astype(np.float32).reshape(geom.det_shape), device=DEV)
    tsp_sirt(grid, geom, yt, x, n_iter, nonneg=nonneg)
    ref = osirt.sirt(wl.edges, st, di, y.astype(np.float32), np.zeros(wl.edges.shape), n_iter, nonneg=nonneg)
    parity(x.cpu().numpy(), ref, what=f"sirt {n_iter}")
    assert tsp_device_status() == 0


def test_sirt_aggregated_scatter_matches_oracle(tiny):
    """SIRT with the adjoint's neighbouring lanes combined before the atomic add."""
    wl, grid, geom, st, di, y = tiny
    x = torch.zeros(grid.shape, device=DEV)
    yt = torch.tensor(y.astype(np.float32).reshape(geom.det_shape), device=DEV)
    with pinned_scatter([(grid, geom)], 1):
        tsp_sirt(grid, geom, yt, x, 5)
    ref = osirt.sirt(wl.edges, st, di, y.astype(np.float32), np.zeros(wl.edges.shape), 5)
    parity(x.cpu().numpy(), ref, what="sirt, aggregated scatter")
    assert tsp_device_status() == 0


def test_sirt_reuse_weights_continues(tiny):
    wl, grid, geom, st, di, y = tiny
    yt = torch.tensor(y.astype(np.float32).reshape(geom.det_shape), device=DEV)
    ws = sirt_workspace(grid, geom)
    a = torch.zeros(grid.shape, device=DEV)
    tsp_sirt(grid, geom, yt, a, 3, workspace=ws)
    tsp_sirt(grid, geom, yt, a, 2, workspace=ws, reuse_weights=True)
    b = torch.zeros(grid.shape, device=DEV)
    tsp_sirt(grid, geom, yt, b, 5)
    assert torch.allclose(a, b, rtol=1e-5, atol=1e-6)


def test_sirt_reduces_residual_multiview():
    e = synth.grid_edges(16, 12, 24)
    truth = synth.training_phantom(e, 1234)
    grid = Grid.from_edges(e)
    geom = Geometry.cone(synth.circular_orbit(12, 60.0, incline_deg=20.0), (48, 48), 50.0)
    xt = torch.tensor(truth, device=DEV)
    y = tsp_forward(grid, geom, xt)
    x = torch.zeros_like(xt)
    ws = sirt_workspace(grid, geom)
    res = []
    for k in range(4):
        tsp_sirt(grid, geom, y, x, 5, workspace=ws, reuse_weights=k > 0)
        res.append(torch.linalg.norm(tsp_forward(grid, geom, x) - y).item())
    assert all(b < a for a, b in zip(res, res[1:])), res
    assert res[-1] < 0.5 * torch.linalg.norm(y).item()


def test_sirt_rejects_bad_arguments(tiny):
    wl, grid, geom, st, di, y = tiny
    from paper_2608_16960_gb300._lib import TspError
    x = torch.zeros(grid.shape, device=DEV)
    yt = torch.zeros(geom.det_shape, device=DEV)
    small = torch.empty(16, dtype=torch.uint8, device=DEV)
    with pytest.raises(TspError):
        tsp_sirt(grid, geom, yt, x, 1, workspace=small)
    with pytest.raises(TspError):
        tsp_sirt(grid, geom, yt, x, -1)
