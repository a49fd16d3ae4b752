"""Parametric density model and optimisation pieces for reconstructions that
differentiate through the projector (Sec. 4.5 Eq. 6-7, Listing 7-8; Sec. 6).

SHBSpline: rho = B(r) c Y(theta, phi)^T with radial cubic B-splines and real
spherical harmonics, rendered and back-propagated by library kernels
(tsp_shbs_*). SquaredError: sum (yhat - y)^2 with its gradient from
tsp_sq_residual. Adam: tsp_adam. Torch only chains them (autograd plumbing)
and holds the memory.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib, synth
from ._lib import check
from .projector import _require_cuda, _stream


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class SHBSpline:
    """n_basis_r radial cubic B-splines x real spherical harmonics of degree <= L
    on a grid's voxel centres (arithmetic midpoints of the edges)."""

    def __init__(self, edges, n_basis_r: int = 20, L: int = 8):
        L_ = _lib.load()
        rc = np.ascontiguousarray(0.5 * (edges.r[:-1] + edges.r[1:]), dtype=np.float64)
        tc = np.ascontiguousarray(0.5 * (edges.theta[:-1] + edges.theta[1:]), dtype=np.float64)
        pc = np.ascontiguousarray(0.5 * (edges.phi[:-1] + edges.phi[1:]), dtype=np.float64)
        h = ctypes.c_void_p()
        check(L_.tsp_shbs_create(n_basis_r, L, _dp(rc), len(rc), _dp(tc), len(tc), _dp(pc), len(pc),
                                 float(edges.r[0]), float(edges.r[-1]), ctypes.byref(h)), "tsp_shbs_create")
        self.handle = h
        self.n_basis_r, self.L = n_basis_r, L
        self.nq = (L + 1) ** 2
        self.shape = (len(rc), len(tc), len(pc))
        self.coeff_shape = (n_basis_r, self.nq)

    def tables(self):
        B = np.zeros((self.shape[0], self.n_basis_r), np.float32)
        Yt = np.zeros((self.nq, self.shape[1] * self.shape[2]), np.float32)
        check(_lib.load().tsp_shbs_tables(self.handle, ctypes.c_void_p(B.ctypes.data), ctypes.c_void_p(Yt.ctypes.data)),
              "tsp_shbs_tables")
        return B, Yt

    def render(self, coeffs: torch.Tensor) -> torch.Tensor:
        return ShbsRenderFn.apply(coeffs, self)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            try:
                _lib.load(build_if_missing=False).tsp_shbs_destroy(h)
            except Exception:
                pass
            self.handle = None


class ShellSH(SHBSpline):
    """Eq. 10's model: one real spherical-harmonic series of degree <= L per
    shell, rho[ir] = sum_q c[ir][q] Y_q at the voxel centres (the SHBSpline
    handle with the identity as radial basis; coefficients (N_r, (L+1)^2))."""

    def __init__(self, edges, L: int = 3):
        L_ = _lib.load()
        tc = np.ascontiguousarray(0.5 * (edges.theta[:-1] + edges.theta[1:]), dtype=np.float64)
        pc = np.ascontiguousarray(0.5 * (edges.phi[:-1] + edges.phi[1:]), dtype=np.float64)
        nr = len(edges.r) - 1
        h = ctypes.c_void_p()
        check(L_.tsp_shbs_create_shells(L, nr, _dp(tc), len(tc), _dp(pc), len(pc), ctypes.byref(h)),
              "tsp_shbs_create_shells")
        self.handle = h
        self.n_basis_r, self.L = nr, L
        self.nq = (L + 1) ** 2
        self.shape = (nr, len(tc), len(pc))
        self.coeff_shape = (nr, self.nq)


class ShbsRenderFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, coeffs, model):
        _require_cuda(coeffs, "coeffs")
        if tuple(coeffs.shape) != model.coeff_shape:
            raise ValueError(f"coeffs must have shape {model.coeff_shape}")
        ctx.model = model
        rho = torch.empty(model.shape, device=coeffs.device)
        check(_lib.load().tsp_shbs_render(model.handle, ctypes.c_void_p(coeffs.data_ptr()),
                                          ctypes.c_void_p(rho.data_ptr()), _stream(coeffs)), "tsp_shbs_render")
        return rho

    @staticmethod
    def backward(ctx, g):
        g = g.contiguous()
        gc = torch.empty(ctx.model.coeff_shape, device=g.device)
        check(_lib.load().tsp_shbs_render_adjoint(ctx.model.handle, ctypes.c_void_p(g.data_ptr()),
                                                  ctypes.c_void_p(gc.data_ptr()), _stream(g)), "tsp_shbs_render_adjoint")
        return gc, None


class SquaredErrorFn(torch.autograd.Function):
    """sum (yhat - y)^2 (Eq. 6) with the gradient 2 (yhat - y) from one kernel."""

    @staticmethod
    def forward(ctx, yhat, y):
        yhat, y = yhat.contiguous(), y.contiguous()
        _require_cuda(yhat, "yhat")
        grad = torch.empty_like(yhat)
        loss = torch.zeros((), dtype=torch.float64, device=yhat.device)
        check(_lib.load().tsp_sq_residual(ctypes.c_void_p(yhat.data_ptr()), ctypes.c_void_p(y.data_ptr()), yhat.numel(),
                                          ctypes.c_void_p(grad.data_ptr()), ctypes.c_void_p(loss.data_ptr()),
                                          _stream(yhat)), "tsp_sq_residual")
        ctx.save_for_backward(grad)
        return loss

    @staticmethod
    def backward(ctx, gl):
        (grad,) = ctx.saved_tensors
        return grad * gl.to(grad.dtype), None


def squared_error(yhat, y):
    return SquaredErrorFn.apply(yhat, y)


class WeightedSquaredErrorFn(torch.autograd.Function):
    """Eq. 10's data term with Eq. 9's per-ray factor: sum (w yhat - y)^2,
    the gradient 2 w (w yhat - y) from one kernel (tsp_sq_residual_weighted)."""

    @staticmethod
    def forward(ctx, yhat, w, y):
        yhat, w, y = yhat.contiguous(), w.contiguous(), y.contiguous()
        _require_cuda(yhat, "yhat")
        grad = torch.empty_like(yhat)
        loss = torch.zeros((), dtype=torch.float64, device=yhat.device)
        check(_lib.load().tsp_sq_residual_weighted(ctypes.c_void_p(yhat.data_ptr()), ctypes.c_void_p(w.data_ptr()),
                                                   ctypes.c_void_p(y.data_ptr()), yhat.numel(),
                                                   ctypes.c_void_p(grad.data_ptr()), ctypes.c_void_p(loss.data_ptr()),
                                                   _stream(yhat)), "tsp_sq_residual_weighted")
        ctx.save_for_backward(grad)
        return loss

    @staticmethod
    def backward(ctx, gl):
        (grad,) = ctx.saved_tensors
        return grad * gl.to(grad.dtype), None, None


class TikhonovRadialFn(torch.autograd.Function):
    """Eq. 10's regulariser lambda ||D_r c||^2 (tsp_tikhonov_radial)."""

    @staticmethod
    def forward(ctx, c, lam):
        c = c.contiguous()
        _require_cuda(c, "c")
        grad = torch.zeros_like(c)
        loss = torch.zeros((), dtype=torch.float64, device=c.device)
        check(_lib.load().tsp_tikhonov_radial(ctypes.c_void_p(c.data_ptr()), c.shape[0], c.shape[1], float(lam),
                                              ctypes.c_void_p(grad.data_ptr()), ctypes.c_void_p(loss.data_ptr()),
                                              _stream(c)), "tsp_tikhonov_radial")
        ctx.save_for_backward(grad)
        return loss

    @staticmethod
    def backward(ctx, gl):
        (grad,) = ctx.saved_tensors
        return grad * gl.to(grad.dtype), None


class Adam:
    """Adam over a list of float32 CUDA parameters, stepped by tsp_adam."""

    def __init__(self, params, lr=1e-3, betas=(0.9, 0.999), eps=1e-8, weight_decay=0.0):
        self.params = list(params)
        self.lr, self.betas, self.eps, self.wd = lr, betas, eps, weight_decay
        self.m = [torch.zeros_like(p) for p in self.params]
        self.v = [torch.zeros_like(p) for p in self.params]
        self.t = 0

    def zero_grad(self):
        for p in self.params:
            p.grad = None

    def step(self):
        self.t += 1
        L = _lib.load()
        for p, m, v in zip(self.params, self.m, self.v):
            if p.grad is None:
                continue
            g = p.grad.contiguous()
            check(L.tsp_adam(ctypes.c_void_p(p.data_ptr()), ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(m.data_ptr()),
                             ctypes.c_void_p(v.data_ptr()), p.numel(), self.lr, self.betas[0], self.betas[1], self.eps,
                             self.wd, self.t, _stream(p)), "tsp_adam")


class WarmStartNet:
    """Residual 3D convolutional network on the spherical grid (tsp_net_*):
    bfloat16 weights/activations, float32 accumulation, trained by the
    library's own forward, backward and Adam kernels."""

    def __init__(self, shape, max_batch: int):
        L_ = _lib.load()
        h = ctypes.c_void_p()
        check(L_.tsp_net_create(shape[0], shape[1], shape[2], max_batch, ctypes.byref(h)), "tsp_net_create")
        self.handle = h
        self.shape = tuple(shape)
        self.max_batch = max_batch
        n = ctypes.c_size_t()
        check(L_.tsp_net_num_params(h, ctypes.byref(n)), "tsp_net_num_params")
        self.n_params = n.value
        self.version = 0  # bumped whenever the parameters change (set_params, adam)

    @staticmethod
    def layout():
        """(offset, shape) of each weight and bias in the flat parameter vector."""
        shapes = [(27, 32, 1), (32,)] + [(27, 32, 32), (32,)] * 4 + [(27, 1, 32), (1,)]
        out, off = [], 0
        for sh in shapes:
            out.append((off, sh))
            off += int(np.prod(sh))
        return out

    def init_params(self, seed: int = 0):
        """Seeded He initialisation (normal, std sqrt(2 / fan_in), fan_in = 27 x
        input channels), scaled by 1/2 in the four residual layers and by 1/10
        in the output layer so that the untrained network stays close to its
        input; biases zero. Draws from synth.SplitMix64."""
        rng = synth.SplitMix64(seed)
        flat = np.zeros(self.n_params, np.float32)
        layers = self.layout()
        for k in range(6):
            off, sh = layers[2 * k]
            std = np.sqrt(2.0 / (27 * sh[2])) * (0.1 if k == 5 else (0.5 if k > 0 else 1.0))
            flat[off:off + int(np.prod(sh))] = (std * rng.normal(int(np.prod(sh)))).astype(np.float32)
        self.set_params(flat)

    def set_params(self, flat: np.ndarray):
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        check(_lib.load().tsp_net_set_params(self.handle, ctypes.c_void_p(flat.ctypes.data), flat.size),
              "tsp_net_set_params")
        self.version += 1

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.n_params, np.float32)
        check(_lib.load().tsp_net_get_params(self.handle, ctypes.c_void_p(out.ctypes.data), out.size),
              "tsp_net_get_params")
        return out

    def get_state(self) -> dict:
        """Training state for a checkpoint: params, Adam moments m and v, step."""
        f = [np.zeros(self.n_params, np.float32) for _ in range(3)]
        step = ctypes.c_int()
        vp = lambda a: ctypes.c_void_p(a.ctypes.data)
        check(_lib.load().tsp_net_get_state(self.handle, vp(f[0]), vp(f[1]), vp(f[2]), self.n_params,
                                            ctypes.byref(step)), "tsp_net_get_state")
        return {"params": f[0], "m": f[1], "v": f[2], "adam_step": step.value}

    def set_state(self, state: dict):
        """Restore a state from get_state: training continues bit for bit."""
        f = [np.ascontiguousarray(state[k], dtype=np.float32) for k in ("params", "m", "v")]
        vp = lambda a: ctypes.c_void_p(a.ctypes.data)
        check(_lib.load().tsp_net_set_state(self.handle, vp(f[0]), vp(f[1]), vp(f[2]), f[0].size,
                                            int(state["adam_step"])), "tsp_net_set_state")
        self.version += 1

    def get_grads(self) -> np.ndarray:
        out = np.zeros(self.n_params, np.float32)
        check(_lib.load().tsp_net_get_grads(self.handle, ctypes.c_void_p(out.ctypes.data), out.size),
              "tsp_net_get_grads")
        return out

    def forward(self, a: torch.Tensor) -> torch.Tensor:
        _require_cuda(a, "a")
        B = a.shape[0]
        out = torch.empty_like(a)
        check(_lib.load().tsp_net_forward(self.handle, ctypes.c_void_p(a.data_ptr()), B, ctypes.c_void_p(out.data_ptr()),
                                          _stream(a)), "tsp_net_forward")
        return out

    def loss_grad(self, a: torch.Tensor, target: torch.Tensor) -> float:
        _require_cuda(a, "a")
        _require_cuda(target, "target")
        loss = ctypes.c_double()
        check(_lib.load().tsp_net_loss_grad(self.handle, ctypes.c_void_p(a.data_ptr()),
                                            ctypes.c_void_p(target.data_ptr()), a.shape[0], ctypes.byref(loss),
                                            _stream(a)), "tsp_net_loss_grad")
        return loss.value

    def adam(self, lr=1e-3, betas=(0.9, 0.999), eps=1e-8, weight_decay=0.0):
        check(_lib.load().tsp_net_adam(self.handle, lr, betas[0], betas[1], eps, weight_decay,
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)), "tsp_net_adam")
        self.version += 1

    def activation(self, layer: int, batch: int) -> np.ndarray:
        nv = batch * int(np.prod(self.shape))
        if layer < 5:
            raw = np.zeros(nv * 32, np.uint16)
            check(_lib.load().tsp_net_activation(self.handle, layer, batch, ctypes.c_void_p(raw.ctypes.data)),
                  "tsp_net_activation")
            return (raw.astype(np.uint32) << 16).view(np.float32).reshape(batch, *self.shape, 32)
        out = np.zeros(nv, np.float32)
        check(_lib.load().tsp_net_activation(self.handle, 5, batch, ctypes.c_void_p(out.ctypes.data)),
              "tsp_net_activation")
        return out.reshape(batch, *self.shape)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            try:
                _lib.load(build_if_missing=False).tsp_net_destroy(h)
            except Exception:
                pass
            self.handle = None
