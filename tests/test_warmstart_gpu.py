"""Learned warm-start pipeline: phantom and noise kernels against their host
definitions, the network input against the FP64 oracle, and a small training
run in which the trained network improves on its own input (the SIRT-weighted
back-projection)."""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import sirt as osirt
from paper_2608_16960_gb300 import _lib, synth
from paper_2608_16960_gb300.warmstart import WarmStart, _p, _st

from _util import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ws():
    e = synth.grid_edges(12, 10, 32)
    pos = synth.circular_orbit(12, 60.0, incline_deg=35.0)
    return WarmStart(e, pos, 32, 50.0, max_batch=4)


def test_phantoms_match_host_renderer(ws):
    seeds = [7, 8, 9]
    rho = ws.phantoms(seeds).cpu().numpy()
    for i, s in enumerate(seeds):
        ref = synth.render_phantom(ws.edges, synth.training_params(s)).astype(np.float64)
        assert np.max(np.abs(rho[i] - ref)) <= 1e-5 * np.max(ref)


def test_noise_matches_host_stream(ws):
    n = 10007
    y = torch.tensor(np.linspace(0.0, 2.0, 2 * n, dtype=np.float32).reshape(2, n), device="cuda")
    seeds = torch.tensor(np.array([123, 456], dtype=np.uint64).view(np.int64), device="cuda")
    ymax = torch.empty(2, device="cuda")
    y0 = y.clone()
    assert _lib.load().tsp_add_noise(_p(y), n, 2, _p(seeds), 0.01, _p(ymax), _st()) == 0
    assert np.allclose(ymax.cpu().numpy(), [y0[0].max().item(), y0[1].max().item()])
    for b, s in enumerate((123, 456)):
        z = synth.SplitMix64(s).normal(n)
        got = (y[b] - y0[b]).cpu().numpy().astype(np.float64) / (0.01 * ymax[b].item())
        assert np.max(np.abs(got - z)) < 2e-4


def test_net_input_matches_oracle(ws):
    """Measurements come from the oracle's own projection of the host-rendered phantom."""
    st, di = oracle.cone_rays(synth.circular_orbit(12, 60.0, incline_deg=35.0), 32, 32, 50.0)
    rho = synth.render_phantom(ws.edges, synth.training_params(11))
    y = oracle.forward(ws.edges, st, di, rho)
    a, scale = ws.net_input(torch.tensor(y.astype(np.float32).reshape((1,) + ws.geom.det_shape), device="cuda"))
    R, C = osirt.weights(ws.edges, st, di)
    ref = C * oracle.adjoint(ws.edges, st, di, R * y.astype(np.float32).astype(np.float64))
    parity(a[0].cpu().numpy() * scale[0].item(), ref, what="network input")
    assert abs(scale[0].item() - ref.max()) <= 1e-4 * ref.max()


def test_network_starts_initialised(ws):
    """A fresh warm-start network has seeded non-zero weights (an all-zero
    ReLU network has no gradient in its inner layers and cannot train)."""
    p = ws.net.get_params()
    for k, (off, sh) in enumerate(ws.net.layout()[0::2]):
        w = p[off:off + int(np.prod(sh))]
        assert np.std(w) > 0, k
        assert abs(np.std(w) / np.sqrt(2.0 / (27 * sh[2])) - (1.0 if k == 0 else (0.1 if k == 5 else 0.5))) < 0.1, k


def test_training_improves_on_the_input(ws):
    losses = ws.train(n_samples=320, batch=4, lr=2e-3, seed0=1000)
    assert np.mean(losses[-20:]) < np.mean(losses[:20])  # fresh phantoms every batch: a noisy but falling loss
    gains = []
    for s in (900001, 900002, 900003):
        rho = ws.phantoms([s])
        y = ws.measure(rho, [s])
        a, scale = ws.net_input(y)
        base = ws.rel_error(torch.clamp(a[0] * scale[0], min=0.0), rho[0])
        warm = ws.rel_error(ws.warm_start(y[0]), rho[0])
        gains.append(base - warm)
    assert np.mean(gains) > 0, gains


def test_captured_warm_start_equals_the_launches():
    """The warm start replayed as a captured CUDA graph gives the eager
    launches' result bit for bit, and is captured again after the weights
    change (one training step). From stored segment lists every sum of the
    pipeline has a fixed order, so the two must agree exactly."""
    e = synth.grid_edges(12, 10, 32)
    w = WarmStart(e, synth.circular_orbit(12, 60.0, incline_deg=35.0), 32, 50.0, max_batch=4, use_lists=True)
    rho = w.phantoms([4242])
    y = w.measure(rho, [4242])[0]
    a = w.warm_start(y)
    assert torch.equal(a, w._warm_start_launches(y))
    assert torch.equal(w.warm_start(y), a)  # replay with the same input
    y2 = w.measure(w.phantoms([4243]), [4243])[0]
    assert torch.equal(w.warm_start(y2), w._warm_start_launches(y2))  # new input, same graph
    w.train(4, batch=4, lr=1e-3, seed0=77)
    b = w.warm_start(y)
    assert torch.equal(b, w._warm_start_launches(y))  # new weights: captured again
    assert not torch.equal(b, a)  # (a stale graph would repeat a)


def test_captured_warm_start_on_the_fly(ws):
    """The same with the on-the-fly back-projection, whose atomic adds sum in
    a varying order: two eager runs of the pipeline differ by a few float32
    ulps in the network's input, which the bf16 activations can round apart
    (measured up to 3.5e-4 of the largest output between two eager runs after
    a training step). Graph and launches agree to 2e-3 of the largest value."""
    close = lambda u, v: float((u - v).abs().max()) <= 2e-3 * float(v.abs().max())
    rho = ws.phantoms([4242])
    y = ws.measure(rho, [4242])[0]
    a = ws.warm_start(y)
    assert close(a, ws._warm_start_launches(y))
    ws.train(4, batch=4, lr=1e-3, seed0=77)
    assert close(ws.warm_start(y), ws._warm_start_launches(y))


def test_list_weights_match_traversal_weights_and_repeat():
    """R = 1/(F 1) and C = 1/(F^T 1) from the stored lists: equal to the
    traversal's weights up to float32 summation order, identical over two
    builds of the lists (fixed-order sums, no atomics)."""
    from paper_2608_16960_gb300.projector import Segments
    e = synth.grid_edges(12, 10, 32)
    w = WarmStart(e, synth.circular_orbit(12, 60.0, incline_deg=35.0), 32, 50.0, max_batch=4)
    R0 = torch.empty(w.geom.n_rays, device="cuda")
    C0 = torch.empty(w.shape, device="cuda")
    _lib.check(_lib.load().tsp_sirt_weights(w.grid.handle, w.geom.handle, _p(R0), _p(C0), _st()), "tsp_sirt_weights")
    R1, C1 = Segments(w.grid, w.geom).sirt_weights()
    R2, C2 = Segments(w.grid, w.geom).sirt_weights()
    assert torch.equal(R1, R2) and torch.equal(C1, C2)
    assert torch.equal(R1 > 0, R0 > 0) and torch.equal(C1 > 0, C0 > 0)
    assert torch.allclose(R1, R0, rtol=2e-6, atol=0.0) and torch.allclose(C1, C0, rtol=2e-6, atol=0.0)


def test_training_from_lists_repeats_bit_for_bit():
    """Two warm starts built from scratch on stored lists train to identical
    losses and weights: phantoms, noise, the network input (list weights and
    list back-projection) and every gradient are fixed-order computations."""
    e = synth.grid_edges(12, 10, 32)
    pos = synth.circular_orbit(12, 60.0, incline_deg=35.0)
    runs = []
    for _ in range(2):
        w = WarmStart(e, pos, 32, 50.0, max_batch=4, use_lists=True)
        losses = w.train(24, batch=4, lr=2e-3, seed0=500)
        y = w.measure(w.phantoms([77]), [77])[0]
        runs.append((losses, w.warm_start(y).cpu()))
    assert runs[0][0] == runs[1][0]
    assert torch.equal(runs[0][1], runs[1][1])


def test_checkpoint_resume_continues_bit_for_bit():
    """A training run split at a checkpoint (network, Adam moments and step
    count saved to disk, restored into a fresh warm start) takes the same
    steps as an uninterrupted run: identical losses and final weights."""
    e = synth.grid_edges(12, 10, 32)
    pos = synth.circular_orbit(12, 60.0, incline_deg=35.0)
    kw = dict(batch=4, lr=2e-3, seed0=600)
    whole = WarmStart(e, pos, 32, 50.0, max_batch=4, use_lists=True)
    l_whole = whole.train(40, **kw)
    first = WarmStart(e, pos, 32, 50.0, max_batch=4, use_lists=True)
    l_a = first.train(40, stop_step=4, **kw)
    import os
    scratch = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build")
    os.makedirs(scratch, exist_ok=True)
    path = os.path.join(scratch, f"ws_checkpoint_{os.getpid()}.npz")
    first.save_checkpoint(path, next_step=4)
    second = WarmStart(e, pos, 32, 50.0, max_batch=4, use_lists=True)
    start = second.load_checkpoint(path)
    assert start == 4
    l_b = second.train(40, start_step=start, **kw)
    assert l_a + l_b == l_whole
    sw, s2 = whole.net.get_state(), second.net.get_state()
    assert sw["adam_step"] == s2["adam_step"] == 10
    for k in ("params", "m", "v"):
        assert np.array_equal(sw[k], s2[k]), k
    with pytest.raises(ValueError, match="checkpoint for grid"):
        WarmStart(synth.grid_edges(8, 10, 32), pos, 32, 50.0, max_batch=4).load_checkpoint(path)
    os.remove(path)
