"""Dynamic objects (Sec. 4.4) on the GPU against the FP64 oracle, through
the C ABI: view k of a collection sees volume k. Tolerances as the static
projector's (tests/_util.parity); the adjoint within 2e-4 normwise."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2608_16960_gb300 import synth, workloads
from paper_2608_16960_gb300.projector import (Geometry, Grid, Operator, tsp_adjoint_dynamic, tsp_device_status,
                                              tsp_forward, tsp_forward_dynamic)

from _util import oracle_rays, parity, pinned_scatter

pytestmark = pytest.mark.gpu
DEV = "cuda"
NV, H, W = 6, 32, 32


@pytest.fixture(scope="module")
def case():
    wl = workloads.tiny()
    grid = Grid.from_edges(wl.edges)
    ang = np.linspace(0.0, 2 * math.pi, NV, endpoint=False)
    pos = np.stack([60 * np.cos(ang), 60 * np.sin(ang), 8 * np.sin(3 * ang)], 1)
    geom = Geometry.cone(pos, (H, W), 30.0)
    st, di = oracle.cone_rays(pos, H, W, 30.0)
    g = synth.SplitMix64(21)
    # a drifting object: the phantom scaled and perturbed per view
    rho = np.stack([wl.rho * (0.5 + 0.25 * k) + 0.05 * g.uniform(wl.rho.size, 0.0, 1.0).reshape(wl.rho.shape)
                    for k in range(NV)]).astype(np.float32)
    return wl, grid, geom, st, di, rho


def test_forward_parity(case):
    wl, grid, geom, st, di, rho = case
    y = tsp_forward_dynamic(grid, geom, torch.tensor(rho, device=DEV)).cpu().numpy()
    ref = oracle.forward_dynamic(wl.edges, st, di, rho, NV)
    for k in range(NV):
        parity(y[k], ref[k], what=f"dynamic view {k}")
    assert tsp_device_status() == 0


@pytest.mark.parametrize("strategy", [0, 1], ids=["atomic", "warp-aggregated"])
def test_adjoint_parity_and_identity(case, strategy):
    wl, grid, geom, st, di, rho = case
    yv = synth.uniform_volume((NV, H, W), 3).astype(np.float32)
    with pinned_scatter([(grid, geom)], strategy):
        g = tsp_adjoint_dynamic(grid, geom, torch.tensor(yv, device=DEV)).cpu().numpy()
    ref = oracle.adjoint_dynamic(wl.edges, st, di, yv, NV)
    assert np.linalg.norm(g - ref) <= 2e-4 * np.linalg.norm(ref)
    y = tsp_forward_dynamic(grid, geom, torch.tensor(rho, device=DEV)).cpu().numpy().astype(np.float64)
    lhs, rhs = np.sum(y * yv), np.sum(rho.astype(np.float64) * g)
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def test_constant_object_is_static(case):
    """The same volume for every view: the dynamic projection equals F."""
    wl, grid, geom, st, di, rho = case
    r = torch.tensor(rho[0], device=DEV)
    y = tsp_forward_dynamic(grid, geom, r.expand(NV, *r.shape).contiguous())
    assert torch.equal(y, tsp_forward(grid, geom, r))


def test_operator_dynamic_autograd(case):
    wl, grid, geom, st, di, rho = case
    op = Operator(grid, geom, dynamic=True)
    r = torch.tensor(rho, device=DEV, requires_grad=True)
    yv = torch.tensor(synth.uniform_volume((NV, H, W), 8).astype(np.float32), device=DEV)
    (op(r) * yv).sum().backward()
    assert torch.equal(r.grad, op.T(yv)) or torch.allclose(r.grad, op.T(yv), rtol=1e-5, atol=1e-6)
    with pytest.raises(ValueError):
        tsp_forward_dynamic(grid, geom, r.detach()[:NV - 1].contiguous())  # one volume per view


def test_paper_scale_sampled():
    """The bench's dynamic leg: each 32-view set of the 100 x 60 x 120
    workload seen as 32 time steps of a drifting object; every 1021st ray."""
    wl = workloads.paper_scale()
    grid = Grid.from_edges(wl.edges)
    for v in wl.views:
        g = Geometry.cone(v.pos, v.shape, v.fov_deg) if v.kind == "cone" else Geometry.parallel(v.pos, v.shape, v.size)
        nv = g.det_shape[0]
        scale = 0.5 + np.arange(nv) / nv
        rho = (scale[:, None, None, None] * wl.rho[None]).astype(np.float32)
        y = tsp_forward_dynamic(grid, g, torch.tensor(rho, device=DEV)).cpu().numpy().reshape(nv, -1)
        st, di = oracle_rays(v)
        per = st.shape[0] // nv
        for k in range(0, nv, 7):
            idx = np.arange(k * per, (k + 1) * per, 1021)
            ref = oracle.forward(wl.edges, st[idx], di[idx], rho[k])
            parity(y[k][idx - k * per], ref, what=f"{v.kind} view {k}")
    assert tsp_device_status() == 0


def test_dynamic_over_polar_views():
    """Polar-binned views (Sec. 6) keep their view structure: view k of a
    polar geometry sees volume k."""
    from oracle import retrieval as orr
    e = synth.grid_edges(8, 6, 12)
    grid = Grid.from_edges(e)
    pos = np.array([[70.0, 5.0, 3.0], [60.0, -25.0, 15.0], [20.0, 65.0, -10.0]])
    geom = Geometry.polar(pos, (10, 6), 40.0)
    rho = np.stack([synth.blob_phantom(e, seed=800 + k) for k in range(3)]).astype(np.float32)
    y = tsp_forward_dynamic(grid, geom, torch.tensor(rho, device=DEV)).cpu().numpy()
    st, di = orr.polar_rays(pos, np.zeros((3, 3)), [[0.0, 0.0, 1.0]] * 3, 10, 6, 40.0)
    ref = oracle.forward_dynamic(e, st, di, rho, 3)
    for k in range(3):
        parity(y[k].reshape(-1), ref[k], what=f"polar dynamic view {k}")
