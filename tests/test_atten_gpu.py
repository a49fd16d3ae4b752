"""Attenuated projection (Sec. 9.3, Eq. 14-18) on the GPU against the FP64
oracle (oracle/atten.py), through the C ABI.

Tolerances: values (y, tau_1) follow the projector's parity rule (tests/_util:
per ray 1e-4 relative with a floor of 1e-2 of the largest value); gradients,
sums of float32 atomics over many rays, within 2e-4 normwise and 1e-3 of the
largest entry elementwise.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import atten
from paper_2608_16960_gb300 import synth, workloads
from paper_2608_16960_gb300.projector import (AttenuatedOperator, Geometry, Grid, atten_backward, atten_forward,
                                              optical_depth, optical_depth_adjoint, sunward_geometry, sunward_rays,
                                              tsp_device_status, tsp_forward)

from _util import oracle_rays, parity, pinned_scatter

pytestmark = pytest.mark.gpu
DEV = "cuda"
SUN = (0.61, -0.42, 0.67)


def grad_parity(g, ref, what, rel=2e-4, elem=1e-3):
    g, ref = np.asarray(g, np.float64).reshape(-1), np.asarray(ref, np.float64).reshape(-1)
    nrm = np.linalg.norm(ref)
    assert nrm > 0, what
    assert np.linalg.norm(g - ref) <= rel * nrm, (what, np.linalg.norm(g - ref) / nrm)
    assert np.max(np.abs(g - ref)) <= elem * np.max(np.abs(ref)), what


@pytest.fixture(scope="module")
def case():
    wl = workloads.tiny()
    grid = Grid.from_edges(wl.edges)
    v = wl.views[0]
    geom = Geometry.cone(v.pos, v.shape, v.fov_deg) if v.kind == "cone" else Geometry.parallel(v.pos, v.shape, v.size)
    st, di = oracle_rays(v)
    rho = wl.rho.astype(np.float32)
    # cross-section of order 1/(typical rho x path): optical depths of order one
    sigma = (0.2 + 0.3 * synth.uniform_volume(wl.edges.shape, 77)).astype(np.float32)
    sun = sunward_geometry(grid, SUN)
    return wl, grid, geom, st, di, rho, sigma, sun


def test_sunward_rays_are_centroids(case):
    wl, grid, geom, st, di, rho, sigma, sun = case
    s, d = (t.cpu().numpy().T.astype(np.float64) for t in sunward_rays(grid, SUN))
    ref_s, ref_d = atten.sunward_rays(wl.edges, SUN)
    assert np.max(np.abs(s - ref_s)) <= 4e-7 * np.max(np.abs(ref_s))
    assert np.max(np.abs(d - ref_d)) <= 2e-7


def test_optical_depth_parity(case):
    wl, grid, geom, st, di, rho, sigma, sun = case
    tau = optical_depth(grid, sun, torch.tensor(rho, device=DEV), torch.tensor(sigma, device=DEV)).cpu().numpy()
    s, d = atten.sunward_rays(wl.edges, SUN)  # the oracle's own FP64 rays
    ref = atten.optical_depth(wl.edges, rho, sigma, s, d)
    parity(tau, ref, what="tau_1")
    assert tsp_device_status() == 0


def test_forward_parity(case):
    wl, grid, geom, st, di, rho, sigma, sun = case
    tau1 = (0.5 * synth.uniform_volume(wl.edges.shape, 5)).astype(np.float32)
    y = atten_forward(grid, geom, *(torch.tensor(a, device=DEV) for a in (rho, sigma, tau1))).cpu().numpy()
    ref = atten.forward(wl.edges, st, di, rho, sigma, tau1)
    parity(y, ref, what="attenuated y")
    plain = oracle.forward(wl.edges, st, di, rho)
    assert np.linalg.norm(ref - plain) > 0.05 * np.linalg.norm(plain)  # the attenuation is not negligible


def test_no_absorption_is_the_plain_projector(case):
    wl, grid, geom, st, di, rho, sigma, sun = case
    r = torch.tensor(rho, device=DEV)
    z = torch.zeros_like(r)
    y = atten_forward(grid, geom, r, z, z).cpu().numpy()
    y0 = tsp_forward(grid, geom, r).cpu().numpy()
    assert np.max(np.abs(y - y0)) <= 1e-6 * np.max(np.abs(y0))


@pytest.mark.parametrize("strategy", [0, 1], ids=["atomic", "warp-aggregated"])
def test_backward_parity(case, strategy):
    wl, grid, geom, st, di, rho, sigma, sun = case
    tau1 = (0.5 * synth.uniform_volume(wl.edges.shape, 5)).astype(np.float32)
    gy = synth.SplitMix64(12).uniform(st.shape[0], -1.0, 1.0).astype(np.float32)
    t = [torch.tensor(a, device=DEV) for a in (rho, sigma, tau1)]
    y = atten_forward(grid, geom, *t)
    with pinned_scatter([(grid, geom)], strategy):
        g = atten_backward(grid, geom, *t, y, torch.tensor(gy, device=DEV).view_as(y))
    ref = atten.backward(wl.edges, st, di, rho, sigma, tau1, gy.astype(np.float64))
    for name, a, b in zip(("g_rho", "g_sigma", "g_tau1"), g, ref):
        grad_parity(a.cpu().numpy(), b, name)
    assert tsp_device_status() == 0


@pytest.mark.parametrize("strategy", [0, 1], ids=["atomic", "warp-aggregated"])
def test_optical_depth_adjoint_parity(case, strategy):
    wl, grid, geom, st, di, rho, sigma, sun = case
    gt = synth.uniform_volume(wl.edges.shape, 19).astype(np.float32) - 0.5
    with pinned_scatter([(grid, sun)], strategy):
        g_rho, g_sig = optical_depth_adjoint(grid, sun, torch.tensor(rho, device=DEV),
                                             torch.tensor(sigma, device=DEV), torch.tensor(gt, device=DEV))
    s, d = atten.sunward_rays(wl.edges, SUN)  # the oracle's own FP64 rays
    r_rho, r_sig = atten.optical_depth_backward(wl.edges, rho, sigma, s, d, gt)
    grad_parity(g_rho.cpu().numpy(), r_rho, "g_rho (tau_1)")
    grad_parity(g_sig.cpu().numpy(), r_sig, "g_sigma (tau_1)")


def test_operator_autograd_chain(case):
    """AttenuatedOperator: y(rho, sigma) with tau_1 = F_1(sigma rho); torch
    autograd through both hand-written backwards equals the oracle's chain."""
    wl, grid, geom, st, di, rho, sigma, sun = case
    op = AttenuatedOperator(grid, geom, SUN)
    r = torch.tensor(rho, device=DEV, requires_grad=True)
    q = torch.tensor(sigma, device=DEV, requires_grad=True)
    y = op(r, q)
    gy = synth.SplitMix64(4).uniform(st.shape[0], -1.0, 1.0)
    (y.reshape(-1) * torch.tensor(gy, device=DEV, dtype=torch.float32)).sum().backward()
    s, d = atten.sunward_rays(wl.edges, SUN)  # the oracle's own FP64 rays
    tau1 = atten.optical_depth(wl.edges, rho, sigma, s, d)
    parity(y.detach().cpu().numpy(), atten.forward(wl.edges, st, di, rho, sigma, tau1), what="operator y")
    g_rho, g_sig, g_tau = atten.backward(wl.edges, st, di, rho, sigma, tau1, gy)
    c_rho, c_sig = atten.optical_depth_backward(wl.edges, rho, sigma, s, d, g_tau)
    grad_parity(r.grad.cpu().numpy(), g_rho + c_rho, "d/d rho")
    grad_parity(q.grad.cpu().numpy(), g_sig + c_sig, "d/d sigma")


def test_batched_matches_single(case):
    wl, grid, geom, st, di, rho, sigma, sun = case
    r = torch.stack([torch.tensor(rho, device=DEV), 0.5 * torch.tensor(rho, device=DEV)])
    q = torch.tensor(sigma, device=DEV).expand(2, *sigma.shape).contiguous()
    t = optical_depth(grid, sun, r, q)
    y = atten_forward(grid, geom, r, q, t)
    for b in range(2):
        tb = optical_depth(grid, sun, r[b].contiguous(), q[b].contiguous())
        assert torch.equal(tb, t[b])
        assert torch.equal(atten_forward(grid, geom, r[b].contiguous(), q[b].contiguous(), tb), y[b])


def test_bad_sunward_geometry_is_rejected(case):
    wl, grid, geom, st, di, rho, sigma, sun = case
    r = torch.tensor(rho, device=DEV)
    with pytest.raises(Exception):
        optical_depth(grid, geom, r, r)  # the cone view has no ray per voxel


def test_paper_scale_sampled():
    """The bench's workload (100 x 60 x 120 grid, 32 cone + 32 parallel views
    of 256^2), default launch: tau_1 on every 97th voxel and the attenuated y
    on every 1021st ray of each view set against the oracle (whose tau_1 is
    its own, over all voxels)."""
    wl = workloads.paper_scale()
    grid = Grid.from_edges(wl.edges)
    rho = wl.rho.astype(np.float32)
    sigma = (0.2 + 0.3 * synth.uniform_volume(wl.edges.shape, 77)).astype(np.float32)
    sun = sunward_geometry(grid, SUN)
    r, q = torch.tensor(rho, device=DEV), torch.tensor(sigma, device=DEV)
    tau = optical_depth(grid, sun, r, q)
    s, d = atten.sunward_rays(wl.edges, SUN)
    ref_tau = atten.optical_depth(wl.edges, rho, sigma, s, d)
    iv = np.arange(0, grid.voxels, 97)
    parity(tau.cpu().numpy().reshape(-1)[iv], ref_tau.reshape(-1)[iv], what="paper-scale tau_1")
    for v in wl.views:
        g = Geometry.cone(v.pos, v.shape, v.fov_deg) if v.kind == "cone" else Geometry.parallel(v.pos, v.shape, v.size)
        y = atten_forward(grid, g, r, q, tau).cpu().numpy().reshape(-1)
        st, di = oracle_rays(v)
        idx = np.arange(0, v.n_rays, 1021)
        ref = atten.forward(wl.edges, st[idx], di[idx], rho, sigma, ref_tau)
        big = np.max(np.abs(ref))
        err = np.abs(y[idx] - ref)
        assert np.all(err <= 1e-4 * np.maximum(np.abs(ref), 1e-2 * big)), (v.kind, err.max())
        assert np.all(np.isfinite(y)) and np.all(y >= 0)
    assert tsp_device_status() == 0


def test_wedge_grid_and_rays_starting_inside():
    """A wedge (theta in [0.5, 2.6], phi in [0.3, 2.5]) and free-form rays,
    some starting inside the grid: rays leave and re-enter the wedge, so
    runs of one voxel are split by gaps; y and the gradients against the
    oracle."""
    e = synth.GridEdges(np.geomspace(3.0, 25.0, 9), np.linspace(0.5, 2.6, 7), np.linspace(0.3, 2.5, 10))
    grid = Grid.from_edges(e)
    g = synth.SplitMix64(71)
    n = 600
    s_out, d_out = synth.random_rays(n // 2, 5, start_radius=60.0, aim_radius=25.0)
    s_in = (g.uniform(3 * (n // 2), -15.0, 15.0).reshape(3, n // 2)).astype(np.float32)
    d_in = g.unit_vectors(n // 2).T.astype(np.float32)
    st = np.concatenate([s_out, s_in], 1).astype(np.float32)
    di = np.concatenate([d_out, d_in], 1).astype(np.float32)
    geom = Geometry.rays(torch.tensor(st, device=DEV), torch.tensor(di, device=DEV))
    rho = (0.2 + synth.uniform_volume(e.shape, 2)).astype(np.float32)
    sigma = (0.2 + 0.3 * synth.uniform_volume(e.shape, 3)).astype(np.float32)
    tau1 = (0.5 * synth.uniform_volume(e.shape, 4)).astype(np.float32)
    t = [torch.tensor(a, device=DEV) for a in (rho, sigma, tau1)]
    y = atten_forward(grid, geom, *t)
    st64, di64 = st.T.astype(np.float64), di.T.astype(np.float64)
    parity(y.cpu().numpy(), atten.forward(e, st64, di64, rho, sigma, tau1), what="wedge attenuated y")
    gy = g.uniform(n, -1.0, 1.0).astype(np.float32)
    grads = atten_backward(grid, geom, *t, y, torch.tensor(gy, device=DEV))
    refs = atten.backward(e, st64, di64, rho, sigma, tau1, gy.astype(np.float64))
    for name, a, b in zip(("g_rho", "g_sigma", "g_tau1"), grads, refs):
        grad_parity(a.cpu().numpy(), b, "wedge " + name)
    assert tsp_device_status() == 0


def test_invalid_arguments_are_rejected(case):
    wl, grid, geom, st, di, rho, sigma, sun = case
    r = torch.tensor(rho, device=DEV)
    with pytest.raises(ValueError):
        atten_forward(grid, geom, r, r[:-1].contiguous(), r)  # sigma of the wrong shape
    with pytest.raises(Exception):
        sunward_geometry(grid, (0.0, 0.0, 0.0))  # no sun direction
