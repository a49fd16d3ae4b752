"""FP64 oracle of the learned warm-start network (test infrastructure only).

Network (a small residual 3D convolutional network on the spherical grid;
3x3x3 kernels, zero padding in r and theta, periodic in phi):
    h1 = relu(conv(a; w1) + b1)                    1 -> 32 channels
    h_k = h_{k-1} + relu(conv(h_{k-1}; wk) + bk)   k = 2..5, 32 -> 32
    out = a + conv(h5; w6) + b6                    32 -> 1 (global residual)
Weights and the stored activations a, h_k are bfloat16 (round to nearest
even), every sum is accumulated in float64 here (float32 on the GPU), the
loss is the mean squared error against the target density.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import lib

C = 32
N_LAYERS = 6


def bf16(x):
    """Round float32 values to bfloat16 (nearest, ties to even); returns float32."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def _f(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def _g(a, exact):
    """float32 operand (default) or float64 operand (exact mode) for the C oracle."""
    if exact:
        a = np.ascontiguousarray(a, dtype=np.float64)
        return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    return _f(a)


def _d(shape):
    out = np.zeros(shape, dtype=np.float64)
    return out, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def conv_fwd(x, w, b, circ=True, exact=False):
    """x (B, Nr, Ne, Na, Ci); w (27, Co, Ci); b (Co,) -> float64 (B, Nr, Ne, Na, Co)."""
    B, Nr, Ne, Na, Ci = x.shape
    Co = w.shape[1]
    xa, xp = _g(x, exact)
    wa, wp = _g(w, exact)
    ba, bp = _g(b, exact)
    y, yp = _d((B, Nr, Ne, Na, Co))
    fn = lib().oracle_conv3d_fwd_f64 if exact else lib().oracle_conv3d_fwd
    fn(B, Ci, Co, Nr, Ne, Na, int(circ), xp, wp, bp, yp)
    return y


def conv_dgrad(gy, w, circ=True, exact=False):
    B, Nr, Ne, Na, Co = gy.shape
    Ci = w.shape[2]
    ga, gp = _g(gy, exact)
    wa, wp = _g(w, exact)
    gx, gxp = _d((B, Nr, Ne, Na, Ci))
    fn = lib().oracle_conv3d_dgrad_f64 if exact else lib().oracle_conv3d_dgrad
    fn(B, Ci, Co, Nr, Ne, Na, int(circ), gp, wp, gxp)
    return gx


def conv_wgrad(x, gy, circ=True, exact=False):
    B, Nr, Ne, Na, Ci = x.shape
    Co = gy.shape[-1]
    xa, xp = _g(x, exact)
    ga, gp = _g(gy, exact)
    gw, gwp = _d((27, Co, Ci))
    gb, gbp = _d((Co,))
    fn = lib().oracle_conv3d_wgrad_f64 if exact else lib().oracle_conv3d_wgrad
    fn(B, Ci, Co, Nr, Ne, Na, int(circ), xp, gp, gwp, gbp)
    return gw, gb


def init_params(seed: int):
    """He-style initialisation, seeded (SplitMix64 via the synthetic-input module's
    generator is not used here: plain numpy Generator on a fixed seed)."""
    rng = np.random.default_rng(seed)
    ps = []
    shapes = [(27, C, 1)] + [(27, C, C)] * 4 + [(27, 1, C)]
    for i, sh in enumerate(shapes):
        fan_in = 27 * sh[2]
        w = rng.normal(0, np.sqrt(2.0 / fan_in), sh).astype(np.float32)
        if i in (1, 2, 3, 4):
            w *= 0.5
        if i == 5:
            w *= 0.1
        ps.append((w, np.zeros(sh[1], np.float32)))
    return ps


def forward(params, a, keep=False, exact=False):
    """a (B, Nr, Ne, Na) input; returns out (B, Nr, Ne, Na) and, if keep, the
    bf16 activations and pre-activation signs needed for the backward pass.
    exact=True skips every bfloat16 rounding (used to pin the backward pass by
    finite differences; the conv oracle still takes float32 operands)."""
    rnd = (lambda v: np.asarray(v, np.float64)) if exact else (lambda v: bf16(np.asarray(v, np.float32)))
    a16 = rnd(a)[..., None]
    ws = [rnd(w) for w, _ in params]
    z1 = conv_fwd(a16, ws[0], params[0][1], exact=exact)
    h = [rnd(np.maximum(z1, 0.0))]
    masks = [z1 > 0]
    for k in range(1, 5):
        z = conv_fwd(h[-1], ws[k], params[k][1], exact=exact)
        masks.append(z > 0)
        h.append(rnd(h[-1].astype(np.float64) + np.maximum(z, 0.0)))
    out = a16[..., 0].astype(np.float64) + conv_fwd(h[-1], ws[5], params[5][1], exact=exact)[..., 0]
    if keep:
        return out, (a16, ws, h, masks)
    return out


def loss_and_grads(params, a, target, exact=False, keep=False):
    """MSE loss and float64 gradients (dw, db) per layer. The gradients of the
    four 32 -> 32 layers' pre-activations are rounded to bfloat16 before their
    weight and input gradients are formed (tensor-core operands on the GPU).
    With keep=True also returns, per layer, the two operands of its weight
    gradient (layer input, output gradient), as the sums used them."""
    rnd = (lambda v: np.asarray(v, np.float64)) if exact else (lambda v: bf16(np.asarray(v, np.float32)))
    f32 = (lambda v: np.asarray(v, np.float64)) if exact else (lambda v: np.asarray(v, np.float32))
    out, (a16, ws, h, masks) = forward(params, a, keep=True, exact=exact)
    n = out.size
    diff = out - np.asarray(target, np.float64)
    loss = float(np.mean(diff ** 2))
    g_out = (2.0 / n) * diff
    grads = [None] * 6
    operands = [None] * 6
    g6 = f32(g_out[..., None])
    grads[5] = conv_wgrad(h[4], g6, exact=exact)
    operands[5] = (h[4], g6)
    g_h = conv_dgrad(g6, ws[5], exact=exact)
    for k in range(4, 0, -1):
        g_z = rnd(np.where(masks[k], g_h, 0.0))
        grads[k] = conv_wgrad(h[k - 1], g_z, exact=exact)
        operands[k] = (h[k - 1], g_z)
        g_h = g_h + conv_dgrad(g_z, ws[k], exact=exact)
    g_z1 = f32(np.where(masks[0], g_h, 0.0))
    grads[0] = conv_wgrad(a16, g_z1, exact=exact)
    operands[0] = (a16, g_z1)
    if keep:
        return loss, grads, operands
    return loss, grads
