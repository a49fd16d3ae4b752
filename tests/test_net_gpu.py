"""Warm-start network kernels (implicit-GEMM BF16 tensor-core convolutions and
CUDA-core end layers) against the network oracle, which rounds weights and
stored activations to bfloat16 at the same points and accumulates in float64.

Tolerances follow from that arithmetic: the GPU accumulates in float32, so a
pre-rounding value within ~1e-6 of a bfloat16 rounding boundary can land one
bfloat16 ulp (2^-8 relative) away; activations must agree to one ulp and such
flips must be rare (a flip feeds the next layer, hence two ulps); outputs and gradients (sums over many voxels) agree
normwise to 1e-2.
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle import net as onet
from paper_2608_16960_gb300 import _lib, synth
from paper_2608_16960_gb300.model import WarmStartNet

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _params(seed):
    ps = onet.init_params(seed)
    rng = synth.SplitMix64(seed + 100)
    return [(w, (0.05 * rng.normal(len(b))).astype(np.float32)) for w, b in ps]


def _flat(params):
    return np.concatenate([np.concatenate([w.ravel(), b.ravel()]) for w, b in params]).astype(np.float32)


def _unflat(flat):
    out = []
    for (off_w, sh_w), (off_b, sh_b) in zip(WarmStartNet.layout()[0::2], WarmStartNet.layout()[1::2]):
        out.append((flat[off_w:off_w + int(np.prod(sh_w))].reshape(sh_w), flat[off_b:off_b + int(np.prod(sh_b))]))
    return out


# Grid shapes covering every tensor-core tile plan: azimuth 32..128 take 4
# tiles of 128 positions per CTA, 160 takes 2, 192 takes 1; several CTAs per
# shell and a last CTA whose tiles run past the shell's end.
SHAPES = [(4, 5, 64), (3, 9, 96), (3, 20, 32), (2, 4, 160), (2, 3, 192)]


def _case(shape):
    B = 2
    params = _params(1)
    rng = synth.SplitMix64(2)
    a = np.abs(rng.normal(B * int(np.prod(shape)))).reshape(B, *shape).astype(np.float32)
    t = np.abs(rng.normal(B * int(np.prod(shape)))).reshape(B, *shape).astype(np.float32)
    net = WarmStartNet(shape, max_batch=B)
    net.set_params(_flat(params))
    return shape, B, params, a, t, net


@pytest.fixture(scope="module")
def case():
    return _case(SHAPES[0])


@pytest.fixture(scope="module", params=SHAPES, ids=lambda s: "x".join(map(str, s)))
def shaped(request):
    return _case(request.param)


def test_param_layout_roundtrip(case):
    shape, B, params, a, t, net = case
    assert net.n_params == sum(w.size + b.size for w, b in params)
    assert np.array_equal(net.get_params(), _flat(params))


def test_forward_matches_oracle(shaped):
    shape, B, params, a, t, net = shaped
    out = net.forward(torch.tensor(a, device=DEV)).cpu().numpy()
    ref, (a16, ws, h, masks) = onet.forward(params, a, keep=True)
    for k in range(5):
        hg = net.activation(k, B)
        diff = np.abs(hg - h[k])
        ulp2 = np.maximum(np.abs(h[k]), 1e-30) * 2.0 ** -6  # two bfloat16 ulps
        far = np.mean(diff > ulp2 + 1e-6)
        nrm = np.linalg.norm(diff) / np.linalg.norm(h[k])
        print(f"h{k + 1}: differing {np.mean(diff > 0):.4f}, beyond 2 ulps {far:.2e}, normwise {nrm:.2e}")
        assert nrm <= 5e-3 and far <= 1e-3, (k, nrm, far)
    assert np.linalg.norm(out - ref) <= 1e-2 * np.linalg.norm(ref)


def test_gradients_match_oracle(shaped):
    shape, B, params, a, t, net = shaped
    loss = net.loss_grad(torch.tensor(a, device=DEV), torch.tensor(t, device=DEV))
    ref_loss, grads = onet.loss_and_grads(params, a, t)
    assert abs(loss - ref_loss) <= 1e-2 * ref_loss
    g = _unflat(net.get_grads())
    for k in range(6):
        for which in range(2):
            gg, rr = g[k][which].astype(np.float64), np.asarray(grads[k][which], np.float64)
            assert np.linalg.norm(gg - rr) <= 2e-2 * np.linalg.norm(rr) + 1e-9, (k, which)


def test_gradients_are_deterministic(shaped):
    """Every weight and bias gradient comes from per-CTA partial sums added in
    a fixed order (no atomics): repeated calls agree bit for bit."""
    shape, B, params, a, t, net = shaped
    at, tt = torch.tensor(a, device=DEV), torch.tensor(t, device=DEV)
    net.loss_grad(at, tt)
    g1 = _unflat(net.get_grads())
    net.loss_grad(at, tt)
    g2 = _unflat(net.get_grads())
    for k in range(6):
        assert np.array_equal(g1[k][1], g2[k][1]), k
        assert np.array_equal(g1[k][0], g2[k][0]), k


def test_training_steps_reduce_loss(case):
    """A learnable target (an affine map of the input) is approached by Adam."""
    shape, B, params, a, t, net = case
    at = torch.tensor(a, device=DEV)
    tt = 0.5 * at + 0.3
    net.set_params(_flat(params))
    losses = []
    for _ in range(60):
        losses.append(net.loss_grad(at, tt))
        net.adam(lr=1e-3)
    assert losses[-1] < 0.5 * losses[0], losses[::10]
    net.set_params(_flat(params))


def test_bounded_wait_runs_out_and_the_next_call_matches_the_oracle(case):
    """Failure detection without a fault: tsp_debug_tc_stall makes the next
    tensor-core convolution's loader issue no shell copy and limits its waits
    to 2e5 cycles (about 0.1 ms). The MMA warp's first wait for a shell then
    runs out; the kernel sets the timeout bit, releases its tensor memory and
    returns with nothing in flight, and tsp_device_status reports TSP_ETIMEOUT.
    The next forward pass (which allocates the tensor memory again on every
    multiprocessor) must run normally and match the oracle."""
    shape, B, params, a, t, net = case
    L = _lib.load()
    net.set_params(_flat(params))
    at = torch.tensor(a, device=DEV)
    torch.cuda.synchronize()
    assert L.tsp_debug_tc_stall(200000) == 0
    net.forward(at)
    code = ctypes.c_int(0)
    st = L.tsp_device_status(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), ctypes.byref(code))
    assert st == 5, (st, L.tsp_last_error())  # TSP_ETIMEOUT
    assert code.value & 0x100, code.value      # TSP_DEVERR_WAIT_TIMEOUT
    assert b"bounded wait" in L.tsp_last_error()
    out = net.forward(at).cpu().numpy()
    ref = onet.forward(params, a)
    assert np.linalg.norm(out - ref) <= 1e-2 * np.linalg.norm(ref)
    code = ctypes.c_int(0)
    assert L.tsp_device_status(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), ctypes.byref(code)) == 0
    assert code.value == 0



@pytest.fixture(scope="module")
def c5_case():
    """The warm-start workload's grid (64 x 48 x 96), batch 2, with the oracle's
    forward pass and gradients (float64 sums; several seconds of CPU time)."""
    shape, B = (64, 48, 96), 2
    params = _params(3)
    rng = synth.SplitMix64(4)
    a = np.abs(rng.normal(B * int(np.prod(shape)))).reshape(B, *shape).astype(np.float32)
    t = np.abs(rng.normal(B * int(np.prod(shape)))).reshape(B, *shape).astype(np.float32)
    net = WarmStartNet(shape, max_batch=B)
    net.set_params(_flat(params))
    out = net.forward(torch.tensor(a, device=DEV)).cpu().numpy()
    acts = [net.activation(k, B) for k in range(5)]
    loss = net.loss_grad(torch.tensor(a, device=DEV), torch.tensor(t, device=DEV))
    grads = _unflat(net.get_grads())
    ref, (a16, ws, h, masks) = onet.forward(params, a, keep=True)
    ref_loss, ref_grads, operands = onet.loss_and_grads(params, a, t, keep=True)
    return shape, B, params, a, t, out, acts, loss, grads, ref, a16, ws, h, operands, ref_loss, ref_grads


def test_c5_shape_outputs_and_activations_elementwise(c5_case):
    """4096 sampled output positions element by element: |out - ref| within
    2^-7 of S = sum |w6| |h5| over the output's receptive inputs (two bfloat16
    ulps of every input of the output layer) plus float32 rounding; the five
    activations at the same positions by the two-ulp rule of the smaller
    shapes."""
    shape, B, params, a, t, out, acts, loss, grads, ref, a16, ws, h, operands, ref_loss, ref_grads = c5_case
    S = onet.conv_fwd(np.abs(h[4]), np.abs(ws[5]), np.zeros(1, np.float32))[..., 0]
    idx = synth.SplitMix64(5).integers(0, out.size - 1, 4096)
    o, r, sv = out.reshape(-1)[idx], ref.reshape(-1)[idx], S.reshape(-1)[idx]
    bound = 2.0 ** -7 * sv + 2.0 ** -20 * (np.abs(r) + sv)
    err = np.abs(o - r)
    print(f"c5 outputs: worst err / bound {np.max(err / bound):.3f}, median {np.median(err / bound):.3e}")
    assert np.all(err <= bound), (np.flatnonzero(err > bound)[:5], np.max(err / bound))
    vox = idx  # flat (b, r, e, a) positions
    for k in range(5):
        hg = acts[k].reshape(-1, 32)[vox]
        hr = np.asarray(h[k]).reshape(-1, 32)[vox]
        diff = np.abs(hg - hr)
        far = np.mean(diff > np.maximum(np.abs(hr), 1e-30) * 2.0 ** -6 + 1e-6)
        print(f"c5 h{k + 1}: beyond 2 ulps {far:.2e}")
        assert far <= 1e-3, (k, far)


def test_c5_shape_gradients_elementwise(c5_case):
    """Every weight and bias gradient entry of all six layers element by
    element: |g - ref| within 2^-6 of the entry's absolute sum G =
    sum_v |gz[v]| |h[v + d]| over the oracle's own operands (bfloat16
    operands: a term whose two factors each sit up to two ulps, 2^-7, from
    the oracle's moves by up to 2^-6 of its magnitude), plus 1e-4 of the
    largest entry of the layer. The loss within 1e-3."""
    shape, B, params, a, t, out, acts, loss, grads, ref, a16, ws, h, operands, ref_loss, ref_grads = c5_case
    assert abs(loss - ref_loss) <= 1e-3 * ref_loss
    for k in range(6):
        x_in, g_z = operands[k]
        mags = onet.conv_wgrad(np.abs(np.asarray(x_in, np.float32)), np.abs(np.asarray(g_z, np.float32)))
        for which in range(2):
            gg = grads[k][which].astype(np.float64).reshape(-1)
            rr = np.asarray(ref_grads[k][which], np.float64).reshape(-1)
            G = np.asarray(mags[which], np.float64).reshape(-1)
            bound = 2.0 ** -6 * G + 1e-4 * np.max(np.abs(rr))
            err = np.abs(gg - rr)
            print(f"c5 layer {k + 1} {'wb'[which]}: {err.size} entries, worst err / bound {np.max(err / bound):.3f}, "
                  f"median {np.median(err / bound):.2e}, worst err / G {np.max(err[G > 0] / G[G > 0]):.2e}")
            assert np.all(err <= bound), (k, which, np.max(err / bound))
