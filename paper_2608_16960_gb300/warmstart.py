"""Learned warm start for SIRT: training data from this projector, a small
residual 3D convolutional network (tsp_net_*), and the warm-vs-cold
reconstruction comparison.

Every numerical step runs in the library: phantoms (tsp_phantoms), projection
(tsp_forward), noise (tsp_add_noise), the normalised back-projection
a = C * F^T(R * y) (tsp_sirt_weights, tsp_mul_bcast, tsp_adjoint,
tsp_scale_batch), the network and its training (tsp_net_*), SIRT (tsp_sirt).
Torch holds the buffers and computes the reported error metrics.
"""
from __future__ import annotations

import ctypes
import math
import time

import numpy as np
import torch

from . import _lib, synth
from ._lib import check
from .model import WarmStartNet
from .projector import Geometry, Grid, Segments, sirt_workspace, tsp_adjoint, tsp_forward, tsp_sirt

MAX_BLOBS = 8


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _st():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class WarmStart:
    def __init__(self, edges, pos, det, fov_deg, max_batch=8, noise_frac=0.01, use_lists=False):
        self.edges = edges
        self.grid = Grid.from_edges(edges)
        self.geom = Geometry.cone(pos, (det, det), fov_deg)
        self.shape = self.grid.shape
        self.V = self.grid.voxels
        self.noise_frac = noise_frac
        self.max_batch = max_batch
        self.net = WarmStartNet(self.shape, max_batch)
        self.net.init_params(seed=7)
        self._graphs = {}  # (measurement shape, weights version) -> captured warm start
        # SIRT projections: stored segment lists (steps 1-3 once) or on-the-fly traversal
        self.segs = Segments(self.grid, self.geom) if use_lists else None
        self.ws = self.segs.sirt_workspace() if use_lists else sirt_workspace(self.grid, self.geom)
        # weights R = 1/(F 1), C = 1/(F^T 1); from the lists they sum in a fixed
        # order, so the network's input, and training, repeat bit for bit
        if use_lists:
            self.R, self.C = self.segs.sirt_weights()
        else:
            self.R = torch.empty(self.geom.n_rays, device="cuda")
            self.C = torch.empty(self.shape, device="cuda")
            check(_lib.load().tsp_sirt_weights(self.grid.handle, self.geom.handle, _p(self.R), _p(self.C), _st()),
                  "tsp_sirt_weights")
        self.mask = self.C > 0  # voxels some ray crosses

    # ---- data -------------------------------------------------------------
    def phantoms(self, seeds):
        rows = 1 + MAX_BLOBS
        P = np.zeros((len(seeds), rows, 5), np.float32)
        for i, s in enumerate(seeds):
            prm = synth.training_params(int(s))
            P[i, :len(prm)] = prm
            P[i, len(prm):, 4] = 1.0  # unused rows: amplitude 0, unit width
        Pd = torch.tensor(P, device="cuda")
        rho = torch.empty((len(seeds),) + self.shape, device="cuda")
        check(_lib.load().tsp_phantoms(self.grid.handle, _p(Pd), rows, len(seeds), _p(rho), _st()), "tsp_phantoms")
        return rho

    def measure(self, rho, seeds):
        """Noisy measurements y = F rho + noise (1% of each sample's peak)."""
        y = tsp_forward(self.grid, self.geom, rho.contiguous())
        s = torch.tensor(np.asarray(seeds, dtype=np.uint64).view(np.int64), device="cuda")
        ymax = torch.empty(len(seeds), device="cuda")
        check(_lib.load().tsp_add_noise(_p(y), self.geom.n_rays, len(seeds), _p(s), self.noise_frac, _p(ymax), _st()),
              "tsp_add_noise")
        return y

    def net_input(self, y):
        """a = C * F^T(R * y), each sample divided by its maximum; returns (a, scale)."""
        L = _lib.load()
        B = y.shape[0]
        yr = y.clone()
        check(L.tsp_mul_bcast(_p(yr), _p(self.R), self.geom.n_rays, B, _st()), "tsp_mul_bcast")
        a = self.segs.adjoint(yr) if self.segs is not None else tsp_adjoint(self.grid, self.geom, yr)
        check(L.tsp_mul_bcast(_p(a), _p(self.C), self.V, B, _st()), "tsp_mul_bcast")
        scale = torch.empty(B, device="cuda")
        check(L.tsp_batch_max(_p(a), self.V, B, _p(scale), _st()), "tsp_batch_max")
        check(L.tsp_scale_batch(_p(a), _p(scale), self.V, B, 1, _st()), "tsp_scale_batch")
        return a, scale

    def batch(self, seeds):
        rho = self.phantoms(seeds)
        y = self.measure(rho, seeds)
        a, scale = self.net_input(y)
        t = rho.clone()
        check(_lib.load().tsp_scale_batch(_p(t), _p(scale), self.V, len(seeds), 1, _st()), "tsp_scale_batch")
        return a, t, y, rho, scale

    # ---- training -----------------------------------------------------------
    def train(self, n_samples, batch=8, lr=1e-3, seed0=1000, log_every=0, cosine=True, start_step=0,
              stop_step=None):
        """Adam on fresh phantoms, `batch` per step; with cosine=True the step
        size decays from lr to lr / 20 along a half cosine over the whole run.
        Steps start_step .. stop_step - 1 of the run are taken (a run split at
        a checkpoint takes the same steps, on the same phantoms, with the same
        step sizes as an uninterrupted one)."""
        losses = []
        steps = (n_samples + batch - 1) // batch
        for s in range(start_step, steps if stop_step is None else min(stop_step, steps)):
            seeds = [seed0 + s * batch + i for i in range(batch)]
            a, t, _, _, _ = self.batch(seeds)
            losses.append(self.net.loss_grad(a, t))
            f = 0.05 + 0.95 * 0.5 * (1.0 + math.cos(math.pi * s / max(1, steps))) if cosine else 1.0
            self.net.adam(lr=lr * f)
            if log_every and s % log_every == 0:
                print(f"step {s}/{steps} loss {losses[-1]:.4e}", flush=True)
        return losses

    # ---- checkpoint / resume ----------------------------------------------------
    def save_checkpoint(self, path, next_step):
        """Network parameters, Adam state and the next training step to `path` (.npz)."""
        st = self.net.get_state()
        np.savez(path, params=st["params"], m=st["m"], v=st["v"], adam_step=np.int64(st["adam_step"]),
                 next_step=np.int64(next_step), shape=np.array(self.shape, np.int64))

    def load_checkpoint(self, path):
        """Restore a checkpoint of save_checkpoint; returns the step to resume at."""
        with np.load(path) as z:
            if tuple(int(x) for x in z["shape"]) != self.shape:
                raise ValueError(f"checkpoint for grid {tuple(z['shape'])}, this warm start has {self.shape}")
            self.net.set_state({"params": z["params"], "m": z["m"], "v": z["v"], "adam_step": int(z["adam_step"])})
            return int(z["next_step"])

    # ---- reconstruction -------------------------------------------------------
    def rel_error(self, x, truth):
        m = self.mask
        return float(torch.linalg.norm((x - truth)[m]) / torch.linalg.norm(truth[m]))

    def _warm_start_launches(self, y):
        a, scale = self.net_input(y[None])
        out = self.net.forward(a)
        check(_lib.load().tsp_scale_batch(_p(out), _p(scale), self.V, 1, 0, _st()), "tsp_scale_batch")
        return torch.clamp(out[0], min=0.0)

    def warm_start(self, y):
        """rho0 = net(a) * scale (clamped at 0). The input back-projection, the
        network and the rescaling (about twenty short launches) are captured
        once per measurement shape as a CUDA graph on a static input buffer and
        replayed; the graphs are dropped whenever the weights change."""
        key = (tuple(y.shape), self.net.version)
        g = self._graphs.get(key)
        if g is None:
            self._graphs.clear()
            static_y = y.detach().clone()
            side = torch.cuda.Stream()
            side.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(side):  # first run outside the capture: lazy set-up, weight copies
                self._warm_start_launches(static_y)
            torch.cuda.current_stream().wait_stream(side)
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph):
                out = self._warm_start_launches(static_y)
            g = self._graphs[key] = (graph, static_y, out)
        graph, static_y, out = g
        static_y.copy_(y)
        graph.replay()
        return out.clone()

    def sirt(self, y, x, n_iter, reuse_weights):
        """n_iter non-negative SIRT updates of x in place (weights kept in self.ws)."""
        if self.segs is not None:
            return self.segs.sirt(y.contiguous(), x, n_iter, nonneg=True, workspace=self.ws, reuse_weights=reuse_weights)
        return tsp_sirt(self.grid, self.geom, y.contiguous(), x, n_iter, nonneg=True, workspace=self.ws,
                        reuse_weights=reuse_weights)

    def sirt_curve(self, y, truth, x0, n_iter, every=1):
        """Errors after 0, every, 2*every, ... SIRT iterations from x0 and the time per iteration."""
        x = x0.clone()
        errs = [self.rel_error(x, truth)]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        first = True
        done = 0
        while done < n_iter:
            k = min(every, n_iter - done)
            self.sirt(y, x, k, reuse_weights=not first)
            first = False
            done += k
            errs.append(self.rel_error(x, truth))
        torch.cuda.synchronize()
        return x, errs, (time.perf_counter() - t0) / max(1, n_iter)
