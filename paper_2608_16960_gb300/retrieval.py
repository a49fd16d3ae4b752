"""Tomographic retrieval of an exosphere (Sec. 6, Eq. 9-10) with the
library's kernels:

    c_hat = argmin_c || y - w F M(c) ||^2 + lambda || D_r c ||^2

M the per-shell spherical-harmonic model (ShellSH), F the projector over
polar-binned views, w Eq. 9's known per-ray factor (g / 4 pi) phi(n), D_r the
first difference between shells. The objective is quadratic in c, so
`cgls` solves it by conjugate gradients on the normal equations (CGLS: per
iteration one application of w F M and one of its transpose, the
regulariser, three dot products and four vector updates, all library
kernels; the host reads two scalars per iteration). `run` is the
differentiable path instead: Adam (tsp_adam) with a cosine step size on
losses chained by torch autograd.
"""
from __future__ import annotations

import ctypes
import math

import torch

from . import _lib
from ._lib import check
from .model import Adam, ShellSH, TikhonovRadialFn, WeightedSquaredErrorFn
from .projector import Operator, _stream, tsp_adjoint, tsp_forward


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


class Retrieval:
    def __init__(self, grid, geom, model: ShellSH, w: torch.Tensor, y: torch.Tensor, lam: float):
        self.op = Operator(grid, geom)
        self.model, self.w, self.y, self.lam = model, w.reshape(-1), y.reshape(-1), lam

    def loss(self, c: torch.Tensor):
        yhat = self.op(self.model.render(c)).reshape(-1)
        return WeightedSquaredErrorFn.apply(yhat, self.w, self.y) + TikhonovRadialFn.apply(c, self.lam)

    def run(self, steps: int, lr: float, c0: torch.Tensor | None = None):
        """Adam for `steps` steps with step size lr * (0.02 + 0.98 (1 + cos(pi s / steps)) / 2).
        Returns the coefficients and the first and last loss."""
        c = (torch.zeros(self.model.coeff_shape, device=self.y.device) if c0 is None else c0.clone())
        c.requires_grad_(True)
        opt = Adam([c], lr=lr)
        first = last = None
        for s in range(steps):
            opt.lr = lr * (0.02 + 0.98 * 0.5 * (1.0 + math.cos(math.pi * s / steps)))
            opt.zero_grad()
            loss = self.loss(c)
            loss.backward()
            opt.step()
            if s == 0:
                first = loss.detach()
            last = loss.detach()
        return c.detach(), first, last

    # ---- CGLS on [w F M; sqrt(lambda) D_r] c = [y; 0] ----
    def _A(self, c, out):
        """out = w * F M c (ray vector)."""
        L, st = _lib.load(), _stream(c)
        rho = torch.empty(self.model.shape, device=c.device)
        check(L.tsp_shbs_render(self.model.handle, _p(c), _p(rho), st), "tsp_shbs_render")
        y = tsp_forward(self.op.grid, self.op.geom, rho).reshape(-1)
        check(L.tsp_vec_mul(_p(self.w), _p(y), _p(out), out.numel(), st), "tsp_vec_mul")

    def _At(self, r, out):
        """out = M^T F^T (w * r) (coefficients)."""
        L, st = _lib.load(), _stream(r)
        wr = torch.empty_like(r)
        check(L.tsp_vec_mul(_p(self.w), _p(r), _p(wr), r.numel(), st), "tsp_vec_mul")
        g = tsp_adjoint(self.op.grid, self.op.geom, wr.reshape(self.op.geom.det_shape))
        check(L.tsp_shbs_render_adjoint(self.model.handle, _p(g), _p(out), st), "tsp_shbs_render_adjoint")

    def cgls(self, iters: int):
        """Minimise Eq. 10's objective from c = 0 by CGLS; returns the
        coefficients and the objective before and after."""
        L = _lib.load()
        y = self.y.contiguous()
        st = _stream(y)
        nr, nq = self.model.coeff_shape
        nc = nr * nq
        x = torch.zeros(self.model.coeff_shape, device=y.device)
        r = y.clone()
        s = torch.empty_like(x)
        q = torch.empty_like(y)
        gtik = torch.empty_like(x)
        acc = torch.zeros(4, dtype=torch.float64, device=y.device)
        accp = lambda i: ctypes.c_void_p(acc.data_ptr() + 8 * i)

        def residual_grad():  # s = A^T r - lambda D^T D x
            self._At(r, s)
            gtik.zero_()
            check(L.tsp_tikhonov_radial(_p(x), nr, nq, float(self.lam), _p(gtik), accp(3), st), "tsp_tikhonov_radial")
            check(L.tsp_vec_axpby(-0.5, _p(gtik), 1.0, _p(s), nc, st), "tsp_vec_axpby")

        acc.zero_()
        check(L.tsp_vec_dot(_p(r), _p(r), r.numel(), accp(0), st), "tsp_vec_dot")
        first = float(acc[0])
        residual_grad()
        p = s.clone()
        acc.zero_()
        check(L.tsp_vec_dot(_p(s), _p(s), nc, accp(0), st), "tsp_vec_dot")
        gamma = float(acc[0])
        for _ in range(iters):
            if gamma <= 0.0:
                break
            self._A(p, q)
            acc.zero_()
            check(L.tsp_vec_dot(_p(q), _p(q), q.numel(), accp(0), st), "tsp_vec_dot")
            check(L.tsp_tikhonov_radial(_p(p), nr, nq, float(self.lam), None, accp(1), st), "tsp_tikhonov_radial")
            den = float(acc[0] + acc[1])
            if den <= 0.0:
                break
            alpha = gamma / den
            check(L.tsp_vec_axpby(alpha, _p(p), 1.0, _p(x), nc, st), "tsp_vec_axpby")
            check(L.tsp_vec_axpby(-alpha, _p(q), 1.0, _p(r), r.numel(), st), "tsp_vec_axpby")
            residual_grad()
            acc.zero_()
            check(L.tsp_vec_dot(_p(s), _p(s), nc, accp(0), st), "tsp_vec_dot")
            g_new = float(acc[0])
            check(L.tsp_vec_axpby(1.0, _p(s), g_new / gamma, _p(p), nc, st), "tsp_vec_axpby")
            gamma = g_new
        acc.zero_()
        check(L.tsp_vec_dot(_p(r), _p(r), r.numel(), accp(0), st), "tsp_vec_dot")
        check(L.tsp_tikhonov_radial(_p(x), nr, nq, float(self.lam), None, accp(1), st), "tsp_tikhonov_radial")
        return x, first, float(acc[0] + acc[1])
