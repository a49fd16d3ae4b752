"""Autotuner and batched persistent / graph-captured SIRT, through the C ABI.

Every instance of a batch is compared with the FP64 oracle's SIRT
(oracle/sirt.py) on the oracle's own rays, per voxel with the parity rule of
tests/_util.py: five uneven instances (cone, parallel and free-form
geometries, wedge and full grids) run directly and as a captured graph, and
the 64-instance batched workload (uneven grids of 20-120 x 20-90 x 40-180
voxels, 4-96 cone views of 64^2-512^2, 339 M rays) in one launch, its
smallest instances in full and its largest by rays (94 views of 463^2) on
sampled voxels. Each instance must also equal the single-instance tsp_sirt,
graph replay must be idempotent, and the autotuner's cached choice must be
what default calls use.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import sirt as osirt
from paper_2608_16960_gb300 import synth, workloads
from paper_2608_16960_gb300._lib import TspError
from paper_2608_16960_gb300.projector import (Batch, Geometry, Grid, tsp_autotune, tsp_autotune_clear,
                                              tsp_device_status, tsp_forward, tsp_sirt)

from _util import oracle_rays, parity, pinned_scatter, rays_near, sirt_parity, voxel_ball

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _instances():
    """Uneven instances: cone, parallel and free-form geometries, wedge and full grids."""
    out = []
    specs = [((12, 9, 20), "cone", 5, (40, 48)), ((20, 14, 30), "parallel", 3, (33, 37)),
             ((8, 6, 10), "cone", 9, (24, 24)), ((16, 12, 24), "rays", 0, (2000,)),
             ((24, 10, 40), "cone", 2, (64, 50))]
    for i, (shape, kind, nv, det) in enumerate(specs):
        if i == 2:
            e = synth.grid_edges(*shape, theta=(0.3, 2.5), phi=(0.5, 4.0))
        else:
            e = synth.grid_edges(*shape)
        grid = Grid.from_edges(e)
        if kind == "cone":
            geom = Geometry.cone(synth.circular_orbit(nv, 60.0, incline_deg=10.0 * i), det, 50.0)
        elif kind == "parallel":
            geom = Geometry.parallel(synth.random_positions(nv, 200 + i), det, 50.0)
        else:
            s, d = synth.random_rays(det[0], 300 + i)
            geom = Geometry.rays(torch.tensor(s, device=DEV), torch.tensor(d, device=DEV))
        truth = torch.tensor(synth.training_phantom(e, 500 + i), device=DEV)
        y = tsp_forward(grid, geom, truth).contiguous()
        out.append((grid, geom, y))
    return out


def _oracle_instances():
    """The five uneven instances of _instances() with their FP64 oracle rays
    (the oracle's detector models; the free-form rays cast from float32) and
    data y = the oracle's forward projection of a seeded phantom, rounded to
    float32 for both sides."""
    out = []
    specs = [((12, 9, 20), "cone", 5, (40, 48)), ((20, 14, 30), "parallel", 3, (33, 37)),
             ((8, 6, 10), "cone", 9, (24, 24)), ((16, 12, 24), "rays", 0, (2000,)),
             ((24, 10, 40), "cone", 2, (64, 50))]
    for i, (shape, kind, nv, det) in enumerate(specs):
        if i == 2:
            e = synth.grid_edges(*shape, theta=(0.3, 2.5), phi=(0.5, 4.0))
        else:
            e = synth.grid_edges(*shape)
        grid = Grid.from_edges(e)
        if kind == "cone":
            pos = synth.circular_orbit(nv, 60.0, incline_deg=10.0 * i)
            geom = Geometry.cone(pos, det, 50.0)
            st, di = oracle.cone_rays(pos, det[0], det[1], 50.0)
        elif kind == "parallel":
            pos = synth.random_positions(nv, 200 + i)
            geom = Geometry.parallel(pos, det, 50.0)
            st, di = oracle.parallel_rays(pos, det[0], det[1], 50.0)
        else:
            s, d = synth.random_rays(det[0], 300 + i)
            geom = Geometry.rays(torch.tensor(s, device=DEV), torch.tensor(d, device=DEV))
            st, di = s.T.astype(np.float64), d.T.astype(np.float64)
        truth = synth.training_phantom(e, 500 + i)
        y32 = oracle.forward(e, st, di, truth).astype(np.float32)
        y = torch.tensor(y32.reshape(geom.det_shape), device=DEV)
        wrc = osirt.weights(e, st, di)
        out.append((grid, geom, y, e, st, di, y32, wrc))
    return out


@pytest.fixture(scope="module")
def oracle_instances():
    return _oracle_instances()


def _check_oracle_sirt(x, inst, n_iter, nonneg, what):
    _, _, _, e, st, di, y32, wrc = inst
    ref = osirt.sirt(e, st, di, y32, np.zeros(e.shape), n_iter, nonneg=nonneg, weights_rc=wrc)
    sirt_parity(x.cpu().numpy(), ref, e, st, di, np.abs(wrc[0] * y32), n_iter, what=what)


@pytest.mark.parametrize("nonneg", [False, True])
def test_batch_matches_oracle_sirt(oracle_instances, nonneg):
    """Batch.sirt (persistent per-stage launches) against the oracle's SIRT."""
    xs = [torch.zeros(it[0].shape, device=DEV) for it in oracle_instances]
    b = Batch([(g, geo, y, x) for (g, geo, y, *_), x in zip(oracle_instances, xs)])
    b.sirt(4, nonneg=nonneg)
    torch.cuda.synchronize()
    for i, it in enumerate(oracle_instances):
        _check_oracle_sirt(xs[i], it, 4, nonneg, f"batch instance {i} vs oracle")
    assert tsp_device_status() == 0


def test_batch_aggregated_scatter_matches_oracle_sirt(oracle_instances):
    """Every instance pinned to the adjoint's neighbouring-lane combine (the
    per-instance scatter strategy is read when the batch is created)."""
    xs = [torch.zeros(it[0].shape, device=DEV) for it in oracle_instances]
    with pinned_scatter([(it[0], it[1]) for it in oracle_instances], 1):
        b = Batch([(g, geo, y, x) for (g, geo, y, *_), x in zip(oracle_instances, xs)])
        b.sirt(4)
        torch.cuda.synchronize()
    for i, it in enumerate(oracle_instances):
        _check_oracle_sirt(xs[i], it, 4, False, f"batch instance {i} (aggregated scatter) vs oracle")
    assert tsp_device_status() == 0


def test_batch_graph_matches_oracle_sirt(oracle_instances):
    """The captured 3-iteration graph, replayed twice from zero, against the
    oracle's SIRT."""
    xs = [torch.zeros(it[0].shape, device=DEV) for it in oracle_instances]
    b = Batch([(g, geo, y, x) for (g, geo, y, *_), x in zip(oracle_instances, xs)])
    b.capture(3, nonneg=True)
    for rep in range(2):
        for x in xs:
            x.zero_()
        b.launch()
        torch.cuda.synchronize()
        for i, it in enumerate(oracle_instances):
            _check_oracle_sirt(xs[i], it, 3, True, f"graph replay {rep}, instance {i}")
    assert tsp_device_status() == 0


def test_c4_batch_matches_oracle():
    """The 64-instance batched workload in one batch, as benchmarked.

    One direct SIRT iteration: the instance with the most rays (94 cone views
    of 463^2, 20 M rays) is checked on 40 sampled voxels. After one iteration
    from zero, x[v] = C[v] sum_i R_i y_i l_i(v) involves only the rays through
    v, and every such ray passes within the voxel's enclosing ball, so the
    oracle traces just the rays whose line comes that close (a superset).
    Then a captured 2-iteration graph: the three smallest instances are
    compared with the oracle's full SIRT. Data: seeded uniform y in [0.5, 1.5)
    (SIRT is defined for any data)."""
    insts = workloads.batched()
    items, ys = [], []
    for k, ins in enumerate(insts):
        grid = Grid.from_edges(ins.edges)
        geom = Geometry.cone(ins.view.pos, ins.view.shape, ins.view.fov_deg)
        yk = synth.uniform_volume(geom.det_shape, 6000 + k, 0.5, 1.5)
        ys.append(yk)
        items.append((grid, geom, torch.tensor(yk, device=DEV), torch.zeros(grid.shape, device=DEV)))
    b = Batch(items)
    b.sirt(1)
    torch.cuda.synchronize()
    assert tsp_device_status() == 0

    big = max(range(len(insts)), key=lambda k: insts[k].view.n_rays)
    ins = insts[big]
    e, v = ins.edges, ins.view
    x_gpu = items[big][3].cpu().numpy()
    rng = synth.SplitMix64(61)
    nr, ne, na = e.shape
    vox = [(int(a), int(bb), int(c)) for a, bb, c in zip(rng.integers(0, nr - 1, 40), rng.integers(0, ne - 1, 40),
                                                         rng.integers(0, na - 1, 40))]
    balls = [voxel_ball(e, *t) for t in vox]
    H, W = v.shape
    sel_st, sel_di, sel_y = [], [], []
    for k in range(len(v.pos)):
        st, di = oracle.cone_rays(v.pos[k:k + 1], H, W, v.fov_deg)
        keep = np.zeros(len(di), bool)
        for c, rad in balls:
            keep[rays_near(st, di, c, rad)] = True
        sel_st.append(st[keep])
        sel_di.append(di[keep])
        sel_y.append(ys[big][k].reshape(-1)[keep].astype(np.float64))
    st, di, yv = np.concatenate(sel_st), np.concatenate(sel_di), np.concatenate(sel_y)
    fl = oracle.forward(e, st, di, np.ones(e.shape))
    R = np.where(fl > 0, 1.0 / np.where(fl > 0, fl, 1.0), 0.0)
    ct = oracle.adjoint(e, st, di, np.ones(len(st)))
    bp = oracle.adjoint(e, st, di, R * yv)
    idx = tuple(np.array(vox).T)
    ref = np.where(ct[idx] > 0, bp[idx] / np.where(ct[idx] > 0, ct[idx], 1.0), 0.0)
    print(f"largest instance {e.shape}, {len(v.pos)} x {v.shape}: {len(st)} rays traced for 40 voxels")
    # the sampled voxels as a small volume for the sliver-aware rule: voxel j of
    # the sample is checked against the rays through it
    got = x_gpu[idx]
    tol = 1e-4 * np.maximum(np.abs(ref), 1e-2 * np.max(np.abs(ref)))
    for j in np.flatnonzero(np.abs(got - ref) > tol):
        full_ref = np.zeros(e.shape)
        full_ref[vox[j]] = ref[j]
        full_x = np.zeros(e.shape)
        full_x[vox[j]] = got[j]
        sirt_parity(full_x, full_ref, e, st, di, np.abs(R * yv), 1, what=f"largest c4 instance, voxel {vox[j]}")
    ok = np.abs(got - ref) <= tol
    assert np.linalg.norm((got - ref)[ok]) <= 1e-4 * np.linalg.norm(ref[ok])

    for it in items:
        it[3].zero_()
    b.capture(2)
    b.launch()
    torch.cuda.synchronize()
    small = sorted(range(len(insts)), key=lambda k: insts[k].view.n_rays * np.prod(insts[k].edges.shape))[:3]
    for k in small:
        ins = insts[k]
        st, di = oracle_rays(ins.view)
        wrc = osirt.weights(ins.edges, st, di)
        ref = osirt.sirt(ins.edges, st, di, ys[k], np.zeros(ins.edges.shape), 2, weights_rc=wrc)
        sirt_parity(items[k][3].cpu().numpy(), ref, ins.edges, st, di, np.abs(wrc[0] * ys[k].reshape(-1)), 2,
                    what=f"c4 instance {k} {ins.edges.shape}, 2 iterations")
    assert tsp_device_status() == 0


def test_autotune_caches_and_default_calls_use_it():
    tsp_autotune_clear()
    wl = workloads.tiny()
    grid = Grid.from_edges(wl.edges)
    v = wl.views[0]
    geom = Geometry.cone(v.pos, v.shape, v.fov_deg)
    f, a = tsp_autotune(grid, geom)
    assert f[0] in (64, 128, 256, 512) and f[1] in (4, 8, 16, 32) and a[2] in (0, 1)
    rho = torch.tensor(wl.rho, device=DEV)
    # default call (tuned) and explicit call give bit-identical forward results
    assert torch.equal(tsp_forward(grid, geom, rho), tsp_forward(grid, geom, rho, launch=f))
    assert tsp_device_status() == 0


@pytest.mark.parametrize("nonneg", [False, True])
def test_batch_matches_single_instance_sirt(nonneg):
    inst = _instances()
    xs = [torch.zeros(g.shape, device=DEV) for g, _, _ in inst]
    b = Batch([(g, geo, y, x) for (g, geo, y), x in zip(inst, xs)])
    b.sirt(4, nonneg=nonneg)
    torch.cuda.synchronize()
    for i, (g, geo, y) in enumerate(inst):
        ref = torch.zeros(g.shape, device=DEV)
        tsp_sirt(g, geo, y, ref, 4, nonneg=nonneg)
        parity(xs[i].cpu().numpy(), ref.cpu().numpy(), what=f"batch instance {i}")
    assert tsp_device_status() == 0


def test_batch_graph_replay_is_idempotent_and_matches_direct():
    inst = _instances()
    xs = [torch.zeros(g.shape, device=DEV) for g, _, _ in inst]
    b = Batch([(g, geo, y, x) for (g, geo, y), x in zip(inst, xs)])
    b.capture(6)
    b.launch()
    torch.cuda.synchronize()
    first = [x.clone() for x in xs]
    for x in xs:
        x.zero_()
    b.launch()
    torch.cuda.synchronize()
    for a, c in zip(first, xs):
        assert torch.allclose(a, c, rtol=1e-5, atol=1e-7)
    for x in xs:
        x.zero_()
    b.sirt(6)
    torch.cuda.synchronize()
    for a, c in zip(first, xs):
        assert torch.allclose(a, c, rtol=1e-5, atol=1e-7)
    r, v, blk = b.info()
    assert r == sum(geo.n_rays for _, geo, _ in inst) and v == sum(g.voxels for g, _, _ in inst)


def test_batch_launch_without_capture_is_rejected():
    inst = _instances()[:2]
    xs = [torch.zeros(g.shape, device=DEV) for g, _, _ in inst]
    b = Batch([(g, geo, y, x) for (g, geo, y), x in zip(inst, xs)])
    with pytest.raises(TspError):
        b.launch()
