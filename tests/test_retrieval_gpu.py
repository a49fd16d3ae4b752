"""Exospheric retrieval pieces (Sec. 6, Eq. 9-10) on the GPU against the FP64
oracle (oracle/retrieval.py), through the C ABI: polar-binned views, the
per-shell harmonic model, the radial regulariser, the weighted data term,
the whole objective's gradient (also at the bench's size) and a noise-free
retrieval that converges. Line integrals use the projector's parity rule;
reductions and gradients agree to 1e-4 (model) / 2e-4 (objective) normwise.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import retrieval as orr
from paper_2608_16960_gb300 import synth, workloads
from paper_2608_16960_gb300.model import ShellSH, TikhonovRadialFn, WeightedSquaredErrorFn
from paper_2608_16960_gb300.projector import Geometry, Grid, tsp_device_status, tsp_forward
from paper_2608_16960_gb300.retrieval import Retrieval

from _util import parity

pytestmark = pytest.mark.gpu
DEV = "cuda"


def small():
    e = synth.grid_edges(6, 5, 12, r_min=3.0, r_max=25.0)
    pos = np.array([[80.0, 10.0, 5.0], [70.0, -30.0, 20.0]])
    return e, pos, (12, 8), 40.0


def test_polar_geometry_parity():
    e, pos, bins, fov = small()
    grid = Grid.from_edges(e)
    geom = Geometry.polar(pos, bins, fov)
    assert geom.det_shape == (2,) + bins
    rho = synth.uniform_volume(e.shape, 5).astype(np.float32)
    y = tsp_forward(grid, geom, torch.tensor(rho, device=DEV)).cpu().numpy()
    st, di = orr.polar_rays(pos, np.zeros((2, 3)), [[0.0, 0.0, 1.0]] * 2, *bins, fov)
    parity(y, oracle.forward(e, st, di, rho), what="polar views")
    assert tsp_device_status() == 0


def test_shell_model_render_and_adjoint():
    e, *_ = small()
    L = 3
    m = ShellSH(e, L)
    g = synth.SplitMix64(3)
    c = g.uniform(6 * 16, -1.0, 1.0).reshape(6, 16).astype(np.float32)
    ct = torch.tensor(c, device=DEV, requires_grad=True)
    rho = m.render(ct)
    ref = orr.shell_render(e, c, L)
    assert np.linalg.norm(rho.detach().cpu().numpy() - ref) <= 1e-5 * np.linalg.norm(ref)
    gr = g.uniform(int(np.prod(e.shape)), -1.0, 1.0).reshape(e.shape).astype(np.float32)
    (rho * torch.tensor(gr, device=DEV)).sum().backward()
    ref_g = orr.shell_render_adjoint(e, gr, L)
    assert np.linalg.norm(ct.grad.cpu().numpy() - ref_g) <= 1e-5 * np.linalg.norm(ref_g)


def test_regulariser_and_weighted_data_term():
    g = synth.SplitMix64(7)
    c = g.uniform(8 * 16, -2.0, 2.0).reshape(8, 16).astype(np.float32)
    ct = torch.tensor(c, device=DEV, requires_grad=True)
    val = TikhonovRadialFn.apply(ct, 0.35)
    val.backward()
    rv, rg = orr.tikhonov(c.astype(np.float64), 0.35)
    assert abs(float(val) - rv) <= 1e-6 * rv
    assert np.allclose(ct.grad.cpu().numpy(), rg, rtol=1e-5, atol=1e-5)
    n = 5000
    yhat, w, y = (g.uniform(n, a, b).astype(np.float32) for a, b in ((0, 3), (0.5, 1.5), (0, 3)))
    yt = torch.tensor(yhat, device=DEV, requires_grad=True)
    loss = WeightedSquaredErrorFn.apply(yt, torch.tensor(w, device=DEV), torch.tensor(y, device=DEV))
    loss.backward()
    rl, rgy = orr.weighted_residual(yhat, w, y)
    assert abs(float(loss) - rl) <= 1e-6 * rl
    assert np.allclose(yt.grad.cpu().numpy(), rgy, rtol=1e-5, atol=1e-5)


def _objective_case(e, pos, bins, fov, L, lam, seed):
    g = synth.SplitMix64(seed)
    nq = (L + 1) ** 2
    st, di = orr.polar_rays(pos, np.zeros_like(pos), [[0.0, 0.0, 1.0]] * len(pos), *bins, fov)
    w = g.uniform(st.shape[0], 0.5, 1.5)
    c_true = g.uniform(e.shape[0] * nq, 0.0, 1.0).reshape(e.shape[0], nq)
    y = w * oracle.forward(e, st, di, orr.shell_render(e, c_true, L)) + 0.01 * g.normal(st.shape[0])
    return st, di, w, y


def test_objective_gradient_matches_oracle():
    e, pos, bins, fov = small()
    L, lam = 3, 0.2
    st, di, w, y = _objective_case(e, pos, bins, fov, L, lam, 9)
    c = synth.SplitMix64(10).uniform(6 * 16, 0.0, 1.0).reshape(6, 16).astype(np.float32)
    ref_val, ref_g = orr.objective(e, st, di, w, y.astype(np.float32), c, L, lam)
    grid, geom, m = Grid.from_edges(e), Geometry.polar(pos, bins, fov), ShellSH(e, L)
    r = Retrieval(grid, geom, m, torch.tensor(w, dtype=torch.float32, device=DEV),
                  torch.tensor(y, dtype=torch.float32, device=DEV), lam)
    ct = torch.tensor(c, device=DEV, requires_grad=True)
    val = r.loss(ct)
    val.backward()
    assert abs(float(val) - ref_val) <= 2e-4 * ref_val
    assert np.linalg.norm(ct.grad.cpu().numpy() - ref_g) <= 2e-4 * np.linalg.norm(ref_g)


def test_full_size_objective_gradient():
    """The bench's exosphere (50 x 45 x 90 grid, 10 polar views of 100 x 50),
    at a point away from the truth."""
    ex = workloads.exosphere()
    e = ex.edges
    st, di = orr.polar_rays(ex.pos, np.zeros_like(ex.pos), [[0.0, 0.0, 1.0]] * len(ex.pos), *ex.shape, ex.fov_deg)
    w = ex.weights.reshape(-1).astype(np.float64)
    y = w * oracle.forward(e, st, di, orr.shell_render(e, ex.coeffs, ex.L))
    c = (0.8 * ex.coeffs).astype(np.float32)
    ref_val, ref_g = orr.objective(e, st, di, w, y.astype(np.float32), c, ex.L, 1e-3)
    grid, geom, m = Grid.from_edges(e), Geometry.polar(ex.pos, ex.shape, ex.fov_deg), ShellSH(e, ex.L)
    r = Retrieval(grid, geom, m, torch.tensor(ex.weights, device=DEV), torch.tensor(y, dtype=torch.float32, device=DEV),
                  1e-3)
    ct = torch.tensor(c, device=DEV, requires_grad=True)
    val = r.loss(ct)
    val.backward()
    # the residual is a fifth of y here: float32 line integrals weigh ~5x on it
    assert abs(float(val) - ref_val) <= 5e-4 * ref_val
    assert np.linalg.norm(ct.grad.cpu().numpy() - ref_g) <= 5e-4 * np.linalg.norm(ref_g)


def test_noise_free_retrieval_converges():
    """Data generated in the model space without noise: Adam brings the
    coefficients to the truth (the model and regulariser are consistent)."""
    e, pos, bins, fov = small()
    pos = np.array([[80.0, 10.0, 5.0], [70.0, -30.0, 20.0], [10.0, 75.0, -15.0], [-60.0, 20.0, 40.0]])
    L, lam = 1, 1e-4
    nq = (L + 1) ** 2
    g = synth.SplitMix64(33)
    c_true = np.zeros((6, nq))
    c_true[:, 0] = 2.0 * np.exp(-np.arange(6) / 3.0)
    c_true[:, 1:] = 0.2 * c_true[:, :1] * g.uniform(6 * (nq - 1), -1.0, 1.0).reshape(6, nq - 1)
    st, di = orr.polar_rays(pos, np.zeros_like(pos), [[0.0, 0.0, 1.0]] * 4, *bins, fov)
    w = np.ones(st.shape[0])
    y = oracle.forward(e, st, di, orr.shell_render(e, c_true, L))
    grid, geom, m = Grid.from_edges(e), Geometry.polar(pos, bins, fov), ShellSH(e, L)
    r = Retrieval(grid, geom, m, torch.tensor(w, dtype=torch.float32, device=DEV),
                  torch.tensor(y, dtype=torch.float32, device=DEV), lam)
    c, first, last = r.run(1500, 0.05)
    err = np.linalg.norm(c.cpu().numpy() - c_true) / np.linalg.norm(c_true)
    assert float(last) < 1e-3 * float(first)
    assert err < 0.05, err


def test_cgls_reaches_the_regularised_optimum():
    """CGLS on Eq. 10 (small problem, noise, lambda > 0) against the exact
    minimiser from the oracle's dense normal equations."""
    e, pos, bins, fov = small()
    L, lam = 1, 0.05
    nq = (L + 1) ** 2
    st, di, w, y = _objective_case(e, pos, bins, fov, L, lam, 14)
    H = orr.shell_tables(e, L)
    A = np.zeros((st.shape[0], 6 * nq))
    for j in range(6 * nq):
        cj = np.zeros(6 * nq)
        cj[j] = 1.0
        A[:, j] = w * oracle.forward(e, st, di, orr.shell_render(e, cj.reshape(6, nq), L, H))
    D = np.zeros((5 * nq, 6 * nq))
    for k in range(5 * nq):
        D[k, k], D[k, k + nq] = -1.0, 1.0
    yf = y.astype(np.float32).astype(np.float64)
    c_opt = np.linalg.solve(A.T @ A + lam * D.T @ D, A.T @ yf)
    grid, geom, m = Grid.from_edges(e), Geometry.polar(pos, bins, fov), ShellSH(e, L)
    r = Retrieval(grid, geom, m, torch.tensor(w, dtype=torch.float32, device=DEV),
                  torch.tensor(y, dtype=torch.float32, device=DEV), lam)
    c, first, last = r.cgls(60)
    assert np.linalg.norm(c.cpu().numpy().reshape(-1) - c_opt) <= 2e-3 * np.linalg.norm(c_opt)
    opt_val = np.sum((A @ c_opt - yf) ** 2) + lam * np.sum((D @ c_opt) ** 2)
    assert abs(last - opt_val) <= 1e-3 * opt_val and last < first
