"""Pins for the convolution and network oracles: delta and shift kernels
(closed forms, including the periodic azimuth), adjoint identities of dgrad
and wgrad, roll equivariance in phi, bfloat16 rounding, and finite
differences of the network loss."""
import numpy as np

from oracle import net
from paper_2608_16960_gb300 import synth


def _x(shape, seed):
    return synth.SplitMix64(seed).normal(int(np.prod(shape))).reshape(shape).astype(np.float32)


def _eye_kernel(tap, c):
    w = np.zeros((27, c, c), np.float32)
    w[tap] = np.eye(c)
    return w


def test_delta_kernel_is_identity():
    x = _x((2, 3, 4, 6, 5), 1)
    y = net.conv_fwd(x, _eye_kernel(13, 5), np.zeros(5, np.float32))
    assert np.array_equal(y, x.astype(np.float64))


def test_shift_kernels_periodic_phi_zero_r_theta():
    x = _x((1, 3, 4, 6, 2), 2)
    zero = np.zeros(2, np.float32)
    # tap (0, 0, +1) reads a+1: periodic in phi
    y = net.conv_fwd(x, _eye_kernel(13 + 1, 2), zero)
    assert np.array_equal(y, np.roll(x, -1, axis=3).astype(np.float64))
    # tap (+1, 0, 0) reads r+1: zero beyond the last shell
    y = net.conv_fwd(x, _eye_kernel(13 + 9, 2), zero)
    ref = np.zeros_like(x)
    ref[:, :-1] = x[:, 1:]
    assert np.array_equal(y, ref.astype(np.float64))
    # tap (0, -1, 0) reads e-1: zero before the first cone
    y = net.conv_fwd(x, _eye_kernel(13 - 3, 2), zero)
    ref = np.zeros_like(x)
    ref[:, :, 1:] = x[:, :, :-1]
    assert np.array_equal(y, ref.astype(np.float64))


def test_adjoint_identities():
    x = _x((2, 3, 4, 5, 4), 3)
    g = _x((2, 3, 4, 5, 6), 4)
    w = _x((27, 6, 4), 5)
    y = net.conv_fwd(x, w, np.zeros(6, np.float32))
    lhs = np.sum(y * g)
    assert abs(lhs - np.sum(x * net.conv_dgrad(g, w))) <= 1e-10 * abs(lhs)
    gw, gb = net.conv_wgrad(x, g)
    assert abs(lhs - np.sum(w * gw)) <= 1e-10 * abs(lhs)
    assert np.allclose(gb, g.sum(axis=(0, 1, 2, 3)))


def test_roll_equivariance_in_phi():
    x = _x((1, 3, 3, 7, 3), 6)
    w = _x((27, 2, 3), 7)
    b = np.zeros(2, np.float32)
    y = net.conv_fwd(x, w, b)
    yr = net.conv_fwd(np.roll(x, 2, axis=3), w, b)
    assert np.allclose(yr, np.roll(y, 2, axis=3), atol=1e-12)


def test_bf16_rounding():
    v = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, 3.14159, -2.5e-3, 0.0], np.float32)
    r = net.bf16(v)
    assert r[0] == 1.0 and r[1] == 1.0  # exact tie rounds to even
    assert r[2] == np.float32(1.0 + 2 ** -7)
    assert abs(r[3] - 3.14159) <= 2 ** -8 * 3.14159
    assert np.all((r.view(np.uint32) & 0xFFFF) == 0)


def test_network_gradients_match_finite_differences():
    """Exact (float64, no bfloat16) mode; h small enough not to cross a ReLU kink."""
    rng = synth.SplitMix64(8)
    params = net.init_params(3)
    params = [(w.astype(np.float64), 0.05 * rng.normal(len(b))) for w, b in params]
    a = np.abs(_x((1, 3, 3, 6), 9)).astype(np.float64)
    t = np.abs(_x((1, 3, 3, 6), 10)).astype(np.float64)
    loss, grads = net.loss_and_grads(params, a, t, exact=True)
    h = 1e-5

    def fd(layer, which, idx):
        pp = [(w.copy(), b.copy()) for w, b in params]
        pm = [(w.copy(), b.copy()) for w, b in params]
        pp[layer][which][idx] += h
        pm[layer][which][idx] -= h
        return (net.loss_and_grads(pp, a, t, exact=True)[0] - net.loss_and_grads(pm, a, t, exact=True)[0]) / (2 * h)

    picks = [(0, 0, (4, 3, 0)), (1, 0, (13, 5, 7)), (2, 1, (4,)), (4, 0, (26, 1, 30)), (5, 0, (13, 0, 11)),
             (5, 1, (0,))]
    nonzero = 0
    for layer, which, idx in picks:
        g = grads[layer][which][idx]
        f = fd(layer, which, idx)
        assert abs(f - g) <= 1e-6 * abs(g) + 1e-12, (layer, which, idx, f, g)
        nonzero += abs(g) > 0
    assert nonzero >= 5
