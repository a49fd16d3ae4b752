"""Stored segment lists (Sec. 3 steps 1-3 kept, step 4 repeated): the lists
against the oracle's per-ray segments, and forward / adjoint from the lists
against the FP64 oracle and against the on-the-fly traversal, through the C ABI.

Tolerances as for the traversal (tests/_util.py): the lists hold exactly the
segments the traversal walks, so list and traversal results differ only by
float32 summation order (checked at 2e-6 relative)."""
from collections import defaultdict

import numpy as np
import pytest
import torch

import oracle
from paper_2608_16960_gb300 import synth, workloads
from paper_2608_16960_gb300._lib import TspError
from paper_2608_16960_gb300.projector import (Geometry, Grid, Operator, Segments, tsp_adjoint, tsp_count_segments,
                                              tsp_device_status, tsp_forward)

from _util import oracle_rays, parity

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _merge(v, l):
    """Merge consecutive pieces in the same voxel (a virtual azimuth plane
    splits a segment without changing its voxel)."""
    mv, ml = [], []
    for a, b in zip(v.tolist(), l.tolist()):
        if mv and mv[-1] == a:
            ml[-1] += b
        else:
            mv.append(a)
            ml.append(b)
    return mv, np.array(ml)


def test_lists_match_oracle_segments():
    """Identical float32 rays on both sides; voxel order along each ray must
    match the oracle's definition (Eq. 4) wherever no crossing is within
    float32 reach of another, and per-voxel lengths agree everywhere."""
    e = synth.grid_edges(20, 15, 30)
    grid = Grid.from_edges(e)
    s32, d32 = synth.random_rays(3000, 61)
    geom = Geometry.rays(torch.tensor(s32, device=DEV), torch.tensor(d32, device=DEV))
    seg = Segments(grid, geom, transpose=True)
    off, vox, ln = seg.export()
    counts = tsp_count_segments(grid, geom).cpu().numpy()
    assert np.array_equal(np.diff(off), counts)
    assert off[0] == 0 and off[-1] == len(vox) == seg.info()[1]
    S, D = s32.T.astype(np.float64), d32.T.astype(np.float64)
    exact = close = 0
    for i in range(S.shape[0]):
        ov, ol = oracle.ray_segments(e, S[i], D[i])
        gv, gl = vox[off[i]:off[i + 1]].astype(np.int64), ln[off[i]:off[i + 1]].astype(np.float64)
        chord = max(ol.sum(), 1e-30)
        assert abs(gl.sum() - ol.sum()) <= 1e-4 * chord + 1e-6, i
        mo, mlo = _merge(ov, ol)
        mg, mlg = _merge(gv, gl)
        if mo == mg:
            exact += 1
            assert np.max(np.abs(mlo - mlg), initial=0.0) <= 1e-3 * chord + 1e-5, i
        else:
            # a differing sequence may only come from near-coincident crossings:
            # per voxel the lengths still agree up to the tiny pieces involved
            ro, rg = defaultdict(float), defaultdict(float)
            for a, b in zip(ov.tolist(), ol.tolist()):
                ro[a] += b
            for a, b in zip(gv.tolist(), gl.tolist()):
                rg[a] += b
            worst = max(abs(ro[k] - rg[k]) for k in set(ro) | set(rg))
            assert worst <= 1e-3 * chord, (i, worst, chord)
            close += 1
    assert exact >= 0.995 * S.shape[0], (exact, close)
    assert tsp_device_status() == 0


def _cone(e, pos, shape, fov):
    return Geometry.cone(pos, shape, fov), oracle.cone_rays(pos, shape[0], shape[1], fov)


@pytest.mark.parametrize("transpose", [True, False])
def test_forward_adjoint_parity_ragged(transpose):
    e = synth.grid_edges(25, 18, 33)
    grid = Grid.from_edges(e)
    pos = synth.circular_orbit(5, 60.0, incline_deg=30.0)
    geom, (st, di) = _cone(e, pos, (45, 29), (50.0, 40.0))
    seg = Segments(grid, geom, transpose=transpose)
    rho = synth.blob_phantom(e, 6)
    y = seg.forward(torch.tensor(rho, device=DEV)).cpu().numpy()
    parity(y, oracle.forward(e, st, di, rho), group=45 * 29, what="segments forward")
    yv = synth.uniform_volume(geom.det_shape, 62)
    g = seg.adjoint(torch.tensor(yv, device=DEV)).cpu().numpy()
    parity(g, oracle.adjoint(e, st, di, yv.reshape(-1)), what="segments adjoint")
    assert tsp_device_status() == 0


def test_lists_equal_traversal_up_to_summation_order():
    wl = workloads.tiny()
    grid = Grid.from_edges(wl.edges)
    v = wl.views[0]
    geom = Geometry.cone(v.pos, v.shape, v.fov_deg)
    seg_t = Segments(grid, geom, transpose=True)
    seg_s = Segments(grid, geom, transpose=False)
    B = 11  # more than one chunk of 8, ragged last chunk
    vols = torch.tensor(np.stack([synth.uniform_volume(grid.shape, 120 + b) for b in range(B)]), device=DEV)
    yl = seg_t.forward(vols)
    yt = tsp_forward(grid, geom, vols)
    assert torch.allclose(yl, yt, rtol=2e-6, atol=1e-7 * yt.abs().max().item())
    assert torch.equal(seg_s.forward(vols), yl)
    assert torch.equal(seg_t.forward(vols), yl)  # reproducible: no atomics, fixed order
    assert torch.equal(seg_t.adjoint(ys0 := torch.ones(geom.det_shape, device=DEV)), seg_t.adjoint(ys0))
    ys = torch.tensor(np.stack([synth.uniform_volume(geom.det_shape, 140 + b) for b in range(B)]), device=DEV)
    gt = tsp_adjoint(grid, geom, ys)
    for seg in (seg_t, seg_s):
        gl = seg.adjoint(ys)
        assert torch.allclose(gl, gt, rtol=2e-6, atol=1e-6 * gt.abs().max().item())
    # accumulate adds to what is there
    base = torch.ones_like(gt)
    acc = seg_t.adjoint(ys, out=base.clone(), accumulate=True)
    assert torch.allclose(acc, gt + 1.0, rtol=2e-6, atol=2e-6 * gt.abs().max().item())
    acc = seg_s.adjoint(ys, out=base.clone(), accumulate=True)
    assert torch.allclose(acc, gt + 1.0, rtol=2e-6, atol=2e-6 * gt.abs().max().item())


def test_adjoint_identity_lists():
    wl = workloads.tiny()
    grid = Grid.from_edges(wl.edges)
    geom = Geometry.parallel(synth.random_positions(3, 41), (37, 53), 50.0)
    seg = Segments(grid, geom)
    x = torch.tensor(synth.uniform_volume(grid.shape, 42), device=DEV)
    yv = torch.tensor(synth.uniform_volume(geom.det_shape, 43), device=DEV)
    lhs = torch.dot(seg.forward(x).double().ravel(), yv.double().ravel()).item()
    rhs = torch.dot(x.double().ravel(), seg.adjoint(yv).double().ravel()).item()
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs), (lhs, rhs)


def test_empty_lists():
    """Every ray misses the grid: no segments, zero results."""
    e = synth.grid_edges(10, 8, 12)
    grid = Grid.from_edges(e)
    s = np.array([[100.0, 100.0], [0.0, 1.0], [0.0, 0.0]], np.float32)
    d = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]], np.float32)
    geom = Geometry.rays(torch.tensor(s, device=DEV), torch.tensor(d, device=DEV))
    for tr in (True, False):
        seg = Segments(grid, geom, transpose=tr)
        assert seg.info()[:2] == (2, 0)
        y = seg.forward(torch.ones(grid.shape, device=DEV))
        assert torch.equal(y, torch.zeros_like(y))
        g = seg.adjoint(torch.ones(2, device=DEV))
        assert torch.equal(g, torch.zeros_like(g))


@pytest.fixture(scope="module")
def paper_scale():
    wl = workloads.paper_scale()
    return wl, Grid.from_edges(wl.edges)


def test_paper_scale_lists(paper_scale):
    """Full 100x60x120 grid, 32 cone + 32 parallel views of 256^2: lists built
    with the voxel-major transpose; forward sampled against the oracle, dense
    adjoint of two whole views per voxel against the oracle, and the full
    adjoint against the traversal's."""
    wl, grid = paper_scale
    rho = torch.tensor(wl.rho, device=DEV)
    for v in wl.views:
        g = Geometry.cone(v.pos, v.shape, v.fov_deg) if v.kind == "cone" else Geometry.parallel(v.pos, v.shape, v.size)
        seg = Segments(grid, g, transpose=True)
        n_rays, n_segs, nbytes = seg.info()
        assert n_segs == int(tsp_count_segments(grid, g).sum().item())
        lo = 16 * n_segs + 8 * (n_rays + 1) + 8 * (grid.voxels + 1)
        # plus per direction: 4 B per non-empty row, 17 B per 256-entry tile
        assert lo < nbytes <= lo + 4 * (n_rays + grid.voxels) + 2 * 17 * (n_segs // 256 + 2) + 64
        y = seg.forward(rho).cpu().numpy().reshape(-1)
        st, di = oracle_rays(v)
        idx = np.arange(0, v.n_rays, 257)
        y_ref = oracle.forward(wl.edges, st[idx], di[idx], wl.rho)
        big = np.max(np.abs(y_ref))
        assert np.all(np.abs(y[idx] - y_ref) <= 1e-4 * np.maximum(np.abs(y_ref), 1e-2 * big))
        yv = torch.tensor(synth.uniform_volume(g.det_shape, 74), device=DEV)
        ga = seg.adjoint(yv)
        gt = tsp_adjoint(grid, g, yv)
        assert torch.allclose(ga, gt, rtol=1e-5, atol=1e-6 * gt.abs().max().item())
        del seg
        # dense per-voxel check of the first two views against the oracle
        sub = type(v)(v.kind, v.pos[:2], v.shape, v.fov_deg, v.size)
        g2 = Geometry.cone(sub.pos, sub.shape, sub.fov_deg) if v.kind == "cone" else \
            Geometry.parallel(sub.pos, sub.shape, sub.size)
        seg2 = Segments(grid, g2, transpose=True)
        y2 = synth.uniform_volume(g2.det_shape, 73)
        out = seg2.adjoint(torch.tensor(y2, device=DEV)).cpu().numpy()
        st2, di2 = oracle_rays(sub)
        parity(out, oracle.adjoint(wl.edges, st2, di2, y2.reshape(-1).astype(np.float64)),
               what=f"dense list adjoint {v.kind}")
    assert tsp_device_status() == 0


@pytest.mark.parametrize("n_iter,nonneg", [(1, False), (5, True)])
def test_list_sirt_matches_oracle(n_iter, nonneg):
    from oracle import sirt as osirt
    wl = workloads.tiny()
    grid = Grid.from_edges(wl.edges)
    v = wl.views[0]
    geom = Geometry.cone(v.pos, v.shape, v.fov_deg)
    st, di = oracle_rays(v)
    y = oracle.forward(wl.edges, st, di, wl.rho)
    seg = Segments(grid, geom)
    x = torch.zeros(grid.shape, device=DEV)
    seg.sirt(torch.tensor(y.astype(np.float32).reshape(geom.det_shape), device=DEV), x, n_iter, nonneg=nonneg)
    ref = osirt.sirt(wl.edges, st, di, y.astype(np.float32), np.zeros(wl.edges.shape), n_iter, nonneg=nonneg)
    parity(x.cpu().numpy(), ref, what=f"list sirt {n_iter}")
    assert tsp_device_status() == 0


def test_list_sirt_follows_traversal_sirt_and_is_reproducible():
    from paper_2608_16960_gb300.projector import sirt_workspace, tsp_sirt
    e = synth.grid_edges(16, 12, 24)
    grid = Grid.from_edges(e)
    geom = Geometry.cone(synth.circular_orbit(12, 60.0, incline_deg=20.0), (48, 48), 50.0)
    y = tsp_forward(grid, geom, torch.tensor(synth.training_phantom(e, 1234), device=DEV))
    seg = Segments(grid, geom)
    a = torch.zeros(grid.shape, device=DEV)
    ws = seg.sirt_workspace()
    seg.sirt(y, a, 6, nonneg=True, workspace=ws)
    seg.sirt(y, a, 4, nonneg=True, workspace=ws, reuse_weights=True)
    b = torch.zeros(grid.shape, device=DEV)
    seg.sirt(y, b, 10, nonneg=True)
    assert torch.equal(a, b)  # no atomics: the same lists give the same iterates
    c = torch.zeros(grid.shape, device=DEV)
    tsp_sirt(grid, geom, y, c, 10, nonneg=True, workspace=sirt_workspace(grid, geom))
    assert torch.allclose(a, c, rtol=1e-4, atol=1e-4 * c.abs().max().item())


def test_chunked_sirt_matches_oracle_and_respects_the_budget():
    """Four independent reconstructions with a list budget below their total:
    the lists are built in several chunks, each item's iterates follow the
    oracle's SIRT, and no more than the budget (plus one item) is held."""
    from oracle import sirt as osirt
    from paper_2608_16960_gb300.projector import sirt_chunked
    items, refs = [], []
    for k in range(4):
        e = synth.grid_edges(8 + 2 * k, 6 + k, 12 + 4 * k)
        pos = synth.circular_orbit(3 + k, 60.0, incline_deg=10.0 * k, phase=0.3 * k)
        grid = Grid.from_edges(e)
        geom = Geometry.cone(pos, (24, 24), 40.0)
        st, di = oracle.cone_rays(pos, 24, 24, 40.0)
        rho = synth.blob_phantom(e, seed=500 + k)
        y = oracle.forward(e, st, di, rho).astype(np.float32)
        items.append((grid, geom, torch.tensor(y.reshape(geom.det_shape), device=DEV), torch.zeros(grid.shape, device=DEV)))
        refs.append(osirt.sirt(e, st, di, y, np.zeros(e.shape), 4, nonneg=True))
    sizes = [Segments(g, m).info()[2] for g, m, _, _ in items]
    budget = int(sum(sizes) * 0.45)
    chunks, peak = sirt_chunked(items, 4, nonneg=True, budget_bytes=budget)
    assert chunks >= 2 and peak <= budget + max(sizes)
    for (grid, geom, y, x), ref in zip(items, refs):
        parity(x.cpu().numpy(), ref, what="chunked sirt")
    assert tsp_device_status() == 0


@pytest.mark.parametrize("shape", [(6, 5, 8), (25, 18, 33), (60, 40, 80)])
def test_transpose_is_the_stable_voxel_sort(shape):
    """The voxel-major lists are exactly the ray-major entries sorted by voxel
    with ties kept in ray-major order (bit-exact: integer and byte work), on
    grids of 240, 14850 and 192000 voxels (one, two and three radix passes);
    two builds give identical lists and bit-identical adjoints."""
    e = synth.grid_edges(*shape)
    grid = Grid.from_edges(e)
    geom = Geometry.cone(synth.circular_orbit(4, 60.0, incline_deg=25.0), (61, 47), 45.0)
    a = Segments(grid, geom, transpose=True)
    off, vox, ln = a.export()
    ray = np.repeat(np.arange(len(off) - 1, dtype=np.uint32), np.diff(off))
    order = np.argsort(vox, kind="stable")
    toff, tray, tln = a.export_transposed()
    assert np.array_equal(toff, np.concatenate([[0], np.cumsum(np.bincount(vox, minlength=grid.voxels))]))
    assert np.array_equal(tray, ray[order])
    assert np.array_equal(tln.view(np.uint32), ln[order].view(np.uint32))
    b = Segments(grid, geom, transpose=True)
    boff, bray, bln = b.export_transposed()
    assert np.array_equal(boff, toff) and np.array_equal(bray, tray) and np.array_equal(bln.view(np.uint32), tln.view(np.uint32))
    ys = torch.tensor(np.stack([synth.uniform_volume(geom.det_shape, 300 + k) for k in range(3)]), device=DEV)
    ga, gb = a.adjoint(ys), b.adjoint(ys)
    assert torch.equal(ga, gb)
    gt = tsp_adjoint(grid, geom, ys)
    assert torch.allclose(ga, gt, rtol=2e-6, atol=1e-6 * gt.abs().max().item())
    assert tsp_device_status() == 0


def test_transposed_export_needs_the_transpose():
    e = synth.grid_edges(6, 5, 8)
    grid = Grid.from_edges(e)
    geom = Geometry.cone(synth.circular_orbit(1, 60.0), (16, 16), 45.0)
    with pytest.raises(TspError, match="without the transpose"):
        Segments(grid, geom, transpose=False).export_transposed()


def _alloc_count():
    import ctypes
    from paper_2608_16960_gb300._lib import check, load
    n = ctypes.c_int64()
    check(load().tsp_debug_allocation_count(ctypes.byref(n)), "tsp_debug_allocation_count")
    return n.value


def test_build_out_of_memory_at_every_allocation_is_reported_and_recovered():
    """The failure is made on the host (the allocation hook returns
    out-of-memory without touching the device): whichever allocation of the
    build fails, the build returns TSP_ENOMEM, frees what it holds, and the
    next build succeeds with the same results."""
    from paper_2608_16960_gb300._lib import load
    e = synth.grid_edges(10, 8, 12)
    grid = Grid.from_edges(e)
    geom = Geometry.cone(synth.circular_orbit(2, 60.0), (24, 24), 40.0)
    rho = torch.tensor(synth.blob_phantom(e, 5), device=DEV)
    n0 = _alloc_count()
    ref = Segments(grid, geom, transpose=True)
    n_build = _alloc_count() - n0
    assert n_build >= 10
    y_ref = ref.forward(rho)
    free0 = torch.cuda.mem_get_info()[0]
    L = load()
    try:
        for k in range(n_build):
            assert L.tsp_debug_fail_allocation(k) == 0
            with pytest.raises(TspError) as ei:
                Segments(grid, geom, transpose=True)
            assert ei.value.status == 3, (k, str(ei.value))  # TSP_ENOMEM
            assert torch.equal(Segments(grid, geom, transpose=True).forward(rho), y_ref)
    finally:
        L.tsp_debug_fail_allocation(-1)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free0 - (64 << 20)  # nothing of the failed builds is held
    assert tsp_device_status() == 0


def test_chunked_sirt_finishes_the_chunk_and_retries_after_out_of_memory():
    """An out-of-memory failure while building the third item's lists: the
    chunked driver runs the two items it holds, frees their lists and builds
    the third again; every item ends bit-identical to the run without the
    failure, in one more chunk."""
    from paper_2608_16960_gb300._lib import load
    from paper_2608_16960_gb300.projector import sirt_chunked
    items = []
    for k in range(4):
        e = synth.grid_edges(8 + 2 * k, 6 + k, 12 + 4 * k)
        grid = Grid.from_edges(e)
        geom = Geometry.cone(synth.circular_orbit(3 + k, 60.0, incline_deg=10.0 * k), (24, 24), 40.0)
        y = tsp_forward(grid, geom, torch.tensor(synth.blob_phantom(e, seed=700 + k), device=DEV))
        items.append((grid, geom, y))
    per_item = []
    for grid, geom, _ in items:
        n0 = _alloc_count()
        Segments(grid, geom, transpose=True)
        per_item.append(_alloc_count() - n0)
    runs = []
    L = load()
    for fail_at in (None, per_item[0] + per_item[1] + 2):
        xs = [(g, m, y, torch.zeros(g.shape, device=DEV)) for g, m, y in items]
        try:
            if fail_at is not None:
                assert L.tsp_debug_fail_allocation(fail_at) == 0
            chunks, _ = sirt_chunked(xs, 5, nonneg=True, budget_bytes=1 << 40)
        finally:
            L.tsp_debug_fail_allocation(-1)
        runs.append((chunks, [x for _, _, _, x in xs]))
    assert runs[0][0] == 1 and runs[1][0] == 2
    for a, b in zip(runs[0][1], runs[1][1]):
        assert torch.equal(a, b)
    assert tsp_device_status() == 0


def test_operator_over_lists_differentiates_like_the_oracle():
    """Operator(grid, geom, segments=...) takes F and F^T from the stored
    lists: the forward matches the oracle's and the gradient of
    <F rho, w> is the oracle's F^T w (per voxel 1e-4 with the floor)."""
    wl = workloads.tiny()
    grid = Grid.from_edges(wl.edges)
    v = wl.views[0]
    geom = Geometry.cone(v.pos, v.shape, v.fov_deg)
    segs = Segments(grid, geom, transpose=True)
    op = Operator(grid, geom, segments=segs)
    rho = torch.tensor(wl.rho, device=DEV, requires_grad=True)
    y = op(rho)
    w = torch.tensor(synth.uniform_volume(geom.det_shape, 17), device=DEV)
    (y * w).sum().backward()
    st, di = oracle_rays(v)
    parity(y.detach().cpu().numpy(), oracle.forward(wl.edges, st, di, wl.rho), what="list operator forward")
    parity(rho.grad.cpu().numpy(), oracle.adjoint(wl.edges, st, di, w.cpu().numpy().reshape(-1).astype(np.float64)),
           what="list operator gradient")
    assert torch.equal(op.T(w), segs.adjoint(w))
    with pytest.raises(ValueError):
        Operator(grid, Geometry.cone(v.pos, v.shape, v.fov_deg), segments=segs)
    assert tsp_device_status() == 0
