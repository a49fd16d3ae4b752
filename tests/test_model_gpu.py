"""Parametric model (SH x radial B-splines), loss and Adam kernels, and the
differentiation pattern: d/dc ||y - F M(c)||^2 through the autograd functions
whose backwards are the hand-written adjoint kernels, checked by finite
differences of the FP64 oracle's loss."""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import shbs as oshbs
from paper_2608_16960_gb300 import synth
from paper_2608_16960_gb300.model import Adam, SHBSpline, squared_error
from paper_2608_16960_gb300.projector import Geometry, Grid, Operator, tsp_device_status

from _util import parity

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module")
def small():
    e = synth.grid_edges(24, 12, 24)
    model = SHBSpline(e, n_basis_r=8, L=4)
    return e, model


def test_tables_match_scipy(small):
    e, model = small
    B, Yt = model.tables()
    Bo, Yo = oshbs.model_tables(e, 8, 4)
    assert np.max(np.abs(B - Bo)) < 2e-7
    assert np.max(np.abs(Yt.T - Yo)) < 1e-6


def test_render_and_adjoint_match_oracle(small):
    e, model = small
    rng = synth.SplitMix64(11)
    c = rng.normal(8 * 25).reshape(8, 25).astype(np.float32)
    rho = model.render(torch.tensor(c, device=DEV)).cpu().numpy()
    parity(rho, oshbs.render(e, c, 8, 4), what="render")
    g = rng.normal(int(np.prod(e.shape))).reshape(e.shape).astype(np.float32)
    ct = torch.tensor(c, device=DEV, requires_grad=True)
    model.render(ct).backward(torch.tensor(g, device=DEV))
    ref = oshbs.render_adjoint(e, g, 8, 4)
    assert np.linalg.norm(ct.grad.cpu().numpy() - ref) <= 1e-5 * np.linalg.norm(ref)


def test_adam_kernel_matches_oracle():
    rng = synth.SplitMix64(12)
    p0 = rng.normal(1000).astype(np.float32)
    grads = [rng.normal(1000).astype(np.float32) for _ in range(7)]
    p = torch.tensor(p0, device=DEV)
    opt = Adam([p], lr=3e-2, weight_decay=1e-2)
    for g in grads:
        p.grad = torch.tensor(g, device=DEV)
        opt.step()
    ref = oshbs.adam(p0, grads, lr=3e-2, weight_decay=1e-2)
    assert np.allclose(p.cpu().numpy(), ref, rtol=1e-5, atol=1e-6)


def test_squared_error_kernel():
    rng = synth.SplitMix64(13)
    a, b = rng.normal(100003).astype(np.float32), rng.normal(100003).astype(np.float32)
    ta = torch.tensor(a, device=DEV, requires_grad=True)
    loss = squared_error(ta, torch.tensor(b, device=DEV))
    loss.backward()
    ref = np.sum((a.astype(np.float64) - b) ** 2)
    assert abs(loss.item() - ref) <= 1e-6 * ref
    assert np.allclose(ta.grad.cpu().numpy(), 2 * (a - b), rtol=1e-6, atol=1e-6)


def _problem(e):
    pos = synth.circular_orbit(4, 60.0, incline_deg=30.0)
    geom = Geometry.cone(pos, (48, 48), 50.0)
    st, di = oracle.cone_rays(pos, 48, 48, 50.0)
    return geom, st, di


def test_gradient_matches_finite_differences_of_oracle_loss(small):
    e, model = small
    geom, st, di = _problem(e)
    grid = Grid.from_edges(e)
    op = Operator(grid, geom)
    rng = synth.SplitMix64(14)
    c_true = rng.normal(8 * 25).reshape(8, 25) * 0.3
    c_true[:, 0] += 2.0
    tables = oshbs.model_tables(e, 8, 4)
    y = oracle.forward(e, st, di, oshbs.render(e, c_true, 8, 4, tables))
    c0 = (c_true + rng.normal(8 * 25).reshape(8, 25) * 0.2).astype(np.float32)
    c = torch.tensor(c0, device=DEV, requires_grad=True)
    loss = squared_error(op(model.render(c)), torch.tensor(y.reshape(geom.det_shape), device=DEV, dtype=torch.float32))
    loss.backward()
    grad = c.grad.cpu().numpy().astype(np.float64)

    def L(cc):
        return float(np.sum((oracle.forward(e, st, di, oshbs.render(e, cc, 8, 4, tables)) - y) ** 2))

    idx = rng.integers(0, 8 * 25 - 1, 32)
    h = 1e-3
    c64 = c0.astype(np.float64)
    for f in idx:
        j, q = divmod(int(f), 25)
        cp, cm = c64.copy(), c64.copy()
        cp[j, q] += h
        cm[j, q] -= h
        fd = (L(cp) - L(cm)) / (2 * h)
        assert abs(fd - grad[j, q]) <= 2e-3 * abs(fd) + 1e-4 * np.abs(grad).max(), (j, q, fd, grad[j, q])
    assert tsp_device_status() == 0


def test_adam_reconstruction_reduces_loss(small):
    e, model = small
    geom, st, di = _problem(e)
    grid = Grid.from_edges(e)
    op = Operator(grid, geom)
    rng = synth.SplitMix64(15)
    c_true = rng.normal(8 * 25).reshape(8, 25) * 0.2
    c_true[:, 0] += 1.5
    y = torch.tensor(oracle.forward(e, st, di, oshbs.render(e, c_true, 8, 4)).reshape(geom.det_shape),
                     device=DEV, dtype=torch.float32)
    c = torch.zeros((8, 25), device=DEV, requires_grad=True)
    opt = Adam([c], lr=5e-2)
    losses = []
    for _ in range(150):
        opt.zero_grad()
        loss = squared_error(op(model.render(c)), y)
        loss.backward()
        opt.step()
        losses.append(loss.item())
    assert losses[-1] < 1e-2 * losses[0]
