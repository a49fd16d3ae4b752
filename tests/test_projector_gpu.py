"""CUDA projector F / F^T against the FP64 oracle, through the C ABI.

Tolerance (float32 kernels vs FP64 definition): per ray |y - y_ref| <= 1e-4 *
max(|y_ref|, 1e-2 * max_view |y_ref|) and normwise <= 1e-4; adjoint identity
<F x, y> = <x, F^T y> within 1e-5 relative (tests/_util.py).
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2608_16960_gb300 import synth, workloads
from paper_2608_16960_gb300.projector import Geometry, Grid, Operator, tsp_adjoint, tsp_device_status, tsp_forward

from _util import grazing_allowance, oracle_rays, parity, sparse_adjoint_parity

pytestmark = pytest.mark.gpu
DEV = "cuda"


def gpu_geoms(wl):
    out = []
    for v in wl.views:
        if v.kind == "cone":
            out.append(Geometry.cone(v.pos, v.shape, v.fov_deg))
        else:
            out.append(Geometry.parallel(v.pos, v.shape, v.size))
    return out


def rays_geom(starts, dirs):
    s = torch.tensor(np.ascontiguousarray(starts, dtype=np.float32), device=DEV)
    d = torch.tensor(np.ascontiguousarray(dirs, dtype=np.float32), device=DEV)
    return Geometry.rays(s, d), s.cpu().numpy().astype(np.float64), d.cpu().numpy().astype(np.float64)


@pytest.fixture(scope="module")
def tiny():
    wl = workloads.tiny()
    grid = Grid.from_edges(wl.edges)
    geom = gpu_geoms(wl)[0]
    st, di = oracle_rays(wl.views[0])
    return wl, grid, geom, st, di


def test_tiny_forward_parity(tiny):
    wl, grid, geom, st, di = tiny
    rho = torch.tensor(wl.rho, device=DEV)
    y = tsp_forward(grid, geom, rho).cpu().numpy()
    y_ref = oracle.forward(wl.edges, st, di, wl.rho)
    parity(y, y_ref, group=64 * 64, what="tiny forward")
    assert tsp_device_status() == 0


def test_tiny_adjoint_parity(tiny):
    wl, grid, geom, st, di = tiny
    yv = synth.uniform_volume((1, 64, 64), 31)
    g = tsp_adjoint(grid, geom, torch.tensor(yv, device=DEV)).cpu().numpy()
    g_ref = oracle.adjoint(wl.edges, st, di, yv.reshape(-1))
    parity(g, g_ref, what="tiny adjoint")


def test_adjoint_identity_tiny_and_mixed(tiny):
    wl, grid, geom, st, di = tiny
    for geo in [geom, Geometry.parallel(synth.random_positions(3, 41), (37, 53), 50.0)]:
        x = torch.tensor(synth.uniform_volume(grid.shape, 42), device=DEV)
        yv = torch.tensor(synth.uniform_volume(geo.det_shape, 43), device=DEV)
        fx = tsp_forward(grid, geo, x)
        fty = tsp_adjoint(grid, geo, yv)
        lhs = float(np.dot(fx.cpu().numpy().ravel().astype(np.float64), yv.cpu().numpy().ravel()))
        rhs = float(np.dot(x.cpu().numpy().ravel().astype(np.float64), fty.cpu().numpy().ravel()))
        assert abs(lhs - rhs) <= 1e-5 * abs(lhs), (lhs, rhs)


def test_parallel_ragged_parity():
    e = synth.grid_edges(30, 20, 40)
    rho = synth.blob_phantom(e, 5)
    grid = Grid.from_edges(e)
    pos = synth.random_positions(3, 44)
    geom = Geometry.parallel(pos, (37, 53), 50.0)
    y = tsp_forward(grid, geom, torch.tensor(rho, device=DEV)).cpu().numpy()
    st, di = oracle.parallel_rays(pos, 37, 53, 50.0)
    parity(y, oracle.forward(e, st, di, rho), group=37 * 53, what="parallel ragged")


def test_cone_ragged_multiview_parity():
    e = synth.grid_edges(25, 18, 33)
    rho = synth.blob_phantom(e, 6)
    grid = Grid.from_edges(e)
    pos = synth.circular_orbit(5, 60.0, incline_deg=30.0)
    geom = Geometry.cone(pos, (45, 29), (50.0, 40.0))
    y = tsp_forward(grid, geom, torch.tensor(rho, device=DEV)).cpu().numpy()
    st, di = oracle.cone_rays(pos, 45, 29, (50.0, 40.0))
    parity(y, oracle.forward(e, st, di, rho), group=45 * 29, what="cone ragged")


@pytest.mark.parametrize("grid_kind", ["log", "wedge_fig3", "fig4", "offset_phi", "na1", "na2", "na3", "polar_cap",
                                       "nonuniform", "ball"])
def test_free_form_rays_parity(grid_kind):
    """Identical float32 rays on both sides: isolates the traversal error."""
    rng = synth.SplitMix64(50)
    if grid_kind == "log":
        e = synth.grid_edges(20, 15, 30)
    elif grid_kind == "wedge_fig3":
        e = synth.grid_edges(2, 2, 2, r_min=5.0, r_max=20.0, theta=(0.8, 1.6), phi=(0.2, 0.9))
    elif grid_kind == "fig4":
        e = synth.grid_edges(1, 2, 7, r_min=10.0, r_max=20.0, theta=(0.6, 2.2), phi=(0.0, 1.75 * math.pi))
    elif grid_kind == "offset_phi":
        e = synth.grid_edges(8, 6, 9, phi=(1.0, 1.0 + 2 * math.pi))
    elif grid_kind == "na1":
        e = synth.grid_edges(6, 5, 1)
    elif grid_kind == "na2":
        e = synth.grid_edges(6, 5, 2)
    elif grid_kind == "na3":
        e = synth.grid_edges(6, 5, 3, phi=(0.0, 5.0))
    elif grid_kind == "polar_cap":
        e = synth.grid_edges(6, 4, 8, theta=(0.0, 0.7))
    elif grid_kind == "nonuniform":
        r = np.concatenate([[3.0], np.sort(rng.uniform(10, 3.5, 24.5)), [25.0]])
        th = np.concatenate([[0.0], np.sort(rng.uniform(7, 0.05, 3.1)), [math.pi]])
        ph = np.concatenate([[-0.4], np.sort(rng.uniform(9, -0.3, 5.8)), [-0.4 + 2 * math.pi]])
        e = synth.GridEdges(r, th, ph)
    else:  # the unit-sphere test of Fig. 11 scaled to radius 25, from r = 0
        e = synth.grid_edges(50, 50, 50, r_min=0.0, r_max=25.0, log_r=False)
    rho = synth.uniform_volume(e.shape, 51) + 0.25
    s1, d1 = synth.random_rays(3000, 52)
    s2, d2 = synth.interior_rays(1000, 53, radius=24.0)
    geom, s, d = rays_geom(np.concatenate([s1, s2], 1), np.concatenate([d1, d2], 1))
    grid = Grid.from_edges(e)
    y = tsp_forward(grid, geom, torch.tensor(rho, device=DEV)).cpu().numpy()
    y_ref = oracle.forward(e, s.T, d.T, rho)
    parity(y, y_ref, what=f"free-form {grid_kind}")
    assert tsp_device_status() == 0


def _nudged(e, rho, x, n, nudges, eps=1e-6):
    """Oracle values for a ray lying in a boundary surface, moved off it to every
    side: each nudge is a (start offset, direction offset) pair of unit vectors."""
    out = []
    for dx, dn in nudges:
        for sx in (1, -1):
            for sn in ((1, -1) if np.any(dn) else (0,)):
                xx = x + sx * eps * np.asarray(dx, float) if np.any(dx) else x
                nn = n + sn * eps * np.asarray(dn, float)
                out.append(oracle.forward(e, xx[None], nn[None], rho)[0])
    return out


def test_degenerate_rays():
    """Sec. 5.1 / Fig. 10 spirit: hand-picked line/boundary configurations."""
    e = synth.grid_edges(10, 8, 12, r_min=3.0, r_max=25.0)
    rho = synth.uniform_volume(e.shape, 60) + 0.5
    grid = Grid.from_edges(e)
    cases = {
        "parallel_to_z_offset": ([0.5, 0.3, -60.0], [0, 0, 1]),
        "parallel_to_z_far": ([12.0, -7.0, 60.0], [0, 0, -1]),
        "through_origin": ([-40.0, -30.0, 20.0], [40.0, 30.0, -20.0]),
        "crosses_phi_seam": ([20.0, -60.0, 1.0], [0, 1, 0]),
        "misses_grid": ([-60.0, 30.0, 0.0], [1, 0, 0]),
        "tangent_outer": ([-60.0, 25.0, 0.0], [1, 0, 0]),
        "tangent_inner": ([-60.0, 3.0, 1e-3], [1, 0, 0]),
        "parallel_to_cone_generator": ([-40.0, 2.0, -40.0], [1, 0, 1]),
        "through_cone_sphere_corner": ([10 * math.sin(math.pi / 4) - 30, 0.0, 10 * math.cos(math.pi / 4) - 20], [30, 0.1, 20]),
        "starts_on_sphere": ([10.0, 0.5, 0.5], [0.3, 0.5, 0.2]),
        "starts_in_inner_hole": ([1.0, 0.5, 0.2], [0.2, -0.7, 0.4]),
        "starts_at_origin": ([0.0, 0.0, 0.0], [0.3, 0.4, 0.5]),
        "near_axis_crossing": ([1e-4, -60.0, 3.0], [0, 1, 0]),
        "zero_direction": ([-60.0, 0.0, 0.0], [0, 0, 0]),
        "moving_away": ([40.0, 0.0, 0.0], [1, 0, 0]),
    }
    names = list(cases)
    xs = np.array([cases[k][0] for k in names], dtype=np.float32)
    ns = np.array([cases[k][1] for k in names], dtype=np.float32)
    geom, s, d = rays_geom(xs.T, ns.T)
    y = tsp_forward(grid, geom, torch.tensor(rho, device=DEV)).cpu().numpy()
    for i, k in enumerate(names):
        if k == "zero_direction":
            assert y[i] == 0.0
            continue
        y_ref = oracle.forward(e, s.T[i:i + 1], d.T[i:i + 1], rho)[0]
        if k in ("misses_grid", "moving_away"):
            assert y[i] == 0.0 and y_ref == 0.0, k
            continue
        tol = 1e-4 * max(abs(y_ref), 1e-2 * 25.0)
        assert abs(y[i] - y_ref) <= tol, (k, y[i], y_ref)
    # rays lying in a boundary surface: any adjacent voxel is a correct answer
    c45 = math.cos(math.pi / 4)
    on_bound = {
        "in_half_plane_phi0": ([10.0, 0.0, -60.0], [0, 0, 1], [([0, 1, 0], [0, 0, 0])]),
        "in_equatorial_plane": ([-60.0, 0.7, 0.0], [1, 0, 0], [([0, 0, 1], [0, 0, 0])]),
        "along_cone_in_half_plane": ([0.0, 0.0, 0.0], [c45, 0.0, c45],
                                     [([0, 0, 0], [c45, 0, -c45]), ([0, 0, 0], [0, 1, 0])]),
    }
    for k, (x, n, nudges) in on_bound.items():
        geom, s, d = rays_geom(np.array([x], np.float32).T, np.array([n], np.float32).T)
        yv = float(tsp_forward(grid, geom, torch.tensor(rho, device=DEV)).cpu().numpy()[0])
        cands = _nudged(e, rho, s.T[0], d.T[0], nudges)
        assert min(abs(yv - c) for c in cands) <= 1e-4 * max(cands), (k, yv, cands)
    assert tsp_device_status() == 0


@pytest.fixture(scope="module")
def paper_scale():
    wl = workloads.paper_scale()
    grid = Grid.from_edges(wl.edges)
    geoms = gpu_geoms(wl)
    return wl, grid, geoms


def test_paper_scale_forward_sampled(paper_scale):
    """Full 100x60x120 grid, 32 cone + 32 parallel views of 256^2 (4.19 M rays),
    default launch; every 257th ray checked against the oracle."""
    wl, grid, geoms = paper_scale
    rho = torch.tensor(wl.rho, device=DEV)
    for v, g in zip(wl.views, geoms):
        y = tsp_forward(grid, g, rho).cpu().numpy().reshape(-1)
        st, di = oracle_rays(v)
        idx = np.arange(0, v.n_rays, 257)
        y_ref = oracle.forward(wl.edges, st[idx], di[idx], wl.rho)
        # floor relative to the largest value of the whole view set
        big = np.max(np.abs(y_ref))
        err = np.abs(y[idx] - y_ref)
        assert np.all(err <= 1e-4 * np.maximum(np.abs(y_ref), 1e-2 * big)), (v.kind, err.max())
        assert np.linalg.norm(y[idx] - y_ref) <= 1e-4 * np.linalg.norm(y_ref)
        assert np.all(np.isfinite(y)) and np.all(y >= 0)


def test_paper_scale_adjoint_sparse_rays(paper_scale):
    """Full-size adjoint with y non-zero on every 509th ray only, so the oracle
    can compute the exact volume from those rays. Each voxel is then fed by one
    or two segments, so a segment whose end is a boundary crossed at a grazing
    angle alpha shows the float32 position error amplified by 1 / sin(alpha)
    undiluted. Per voxel the bound is 1e-4 relative plus, for each segment in
    it, |y| times 16 float32 ulps of the outer radius over sin(alpha) at each
    end (tests/_util.py: grazing_allowance); a voxel bounded by crossings at
    good angles therefore gets no more than about 5e-5 |y| absolute, and a
    wrong voxel index (an O(1) error) fails. Normwise 1e-4."""
    wl, grid, geoms = paper_scale
    for v, g in zip(wl.views, geoms):
        idx = np.arange(0, v.n_rays, 509)
        yv = np.zeros(v.n_rays, np.float32)
        yv[idx] = synth.SplitMix64(70).uniform(len(idx), 0.5, 1.5)
        out = tsp_adjoint(grid, g, torch.tensor(yv.reshape(g.det_shape), device=DEV)).cpu().numpy()
        st, di = oracle_rays(v)
        ref = oracle.adjoint(wl.edges, st[idx], di[idx], yv[idx].astype(np.float64))
        allow, gmax = grazing_allowance(wl.edges, st[idx], di[idx], yv[idx])
        sparse_adjoint_parity(out, ref, allow, gmax, what=f"sparse adjoint {v.kind}")
    assert tsp_device_status() == 0


@pytest.mark.parametrize("strategy", [0, 1], ids=["atomic", "warp-aggregated"])
def test_paper_scale_adjoint_dense_views(paper_scale, strategy):
    """Full-size grid, every ray of two whole views non-zero: per-voxel 1e-4,
    for both scatter strategies (one atomic add per segment; lanes of a warp
    that hit the same voxel combined first, Sec. 4.4's adjoint)."""
    wl, grid, geoms = paper_scale
    for v in wl.views:
        sub = type(v)(v.kind, v.pos[:2], v.shape, v.fov_deg, v.size)
        g = Geometry.cone(sub.pos, sub.shape, sub.fov_deg) if v.kind == "cone" else Geometry.parallel(sub.pos, sub.shape, sub.size)
        yv = synth.uniform_volume(g.det_shape, 73)
        out = tsp_adjoint(grid, g, torch.tensor(yv, device=DEV), launch=(128, 8, strategy)).cpu().numpy()
        st, di = oracle_rays(sub)
        ref = oracle.adjoint(wl.edges, st, di, yv.reshape(-1).astype(np.float64))
        parity(out, ref, what=f"dense adjoint {v.kind}, strategy {strategy}")
    assert tsp_device_status() == 0


def test_paper_scale_adjoint_identity(paper_scale):
    wl, grid, geoms = paper_scale
    x = torch.tensor(synth.uniform_volume(grid.shape, 71), device=DEV)
    for g in geoms:
        yv = torch.tensor(synth.uniform_volume(g.det_shape, 72), device=DEV)
        lhs = torch.dot(tsp_forward(grid, g, x).double().ravel(), yv.double().ravel()).item()
        rhs = torch.dot(x.double().ravel(), tsp_adjoint(grid, g, yv).double().ravel()).item()
        assert abs(lhs - rhs) <= 1e-5 * abs(lhs), (lhs, rhs)


def test_forward_into_a_caller_buffer(tiny):
    wl, grid, geom, st, di = tiny
    rho = torch.tensor(wl.rho, device=DEV)
    out = torch.full(geom.det_shape, -1.0, device=DEV)
    y = tsp_forward(grid, geom, rho, out=out)
    assert y.data_ptr() == out.data_ptr()
    assert torch.equal(out, tsp_forward(grid, geom, rho))
    with pytest.raises(ValueError):
        tsp_forward(grid, geom, rho, out=torch.empty(7, device=DEV))


def test_batched_equals_single(tiny):
    wl, grid, geom, st, di = tiny
    B = 11  # more than one chunk of 8
    vols = torch.tensor(np.stack([synth.uniform_volume(grid.shape, 80 + b) for b in range(B)]), device=DEV)
    yb = tsp_forward(grid, geom, vols)
    for b in range(B):
        assert torch.equal(yb[b], tsp_forward(grid, geom, vols[b]))
    ys = torch.tensor(np.stack([synth.uniform_volume(geom.det_shape, 90 + b) for b in range(B)]), device=DEV)
    gb = tsp_adjoint(grid, geom, ys)
    for b in range(B):
        gs = tsp_adjoint(grid, geom, ys[b])
        assert torch.allclose(gb[b], gs, rtol=1e-5, atol=1e-6)


@pytest.mark.parametrize("strategy", [0, 1], ids=["atomic", "warp-aggregated"])
def test_batched_adjoint_parity(tiny, strategy):
    """F^T of a batch of 3 and of 11 (one chunk of 8 plus 3) against the
    oracle per item, for both scatter strategies."""
    wl, grid, geom, st, di = tiny
    for B in (3, 11):
        ys = np.stack([synth.uniform_volume(geom.det_shape, 110 + b) for b in range(B)]).astype(np.float32)
        gb = tsp_adjoint(grid, geom, torch.tensor(ys, device=DEV), launch=(128, 8, strategy)).cpu().numpy()
        for b in range(B):
            ref = oracle.adjoint(wl.edges, st, di, ys[b].reshape(-1).astype(np.float64))
            parity(gb[b], ref, what=f"batched adjoint {b} of {B}, strategy {strategy}")
    assert tsp_device_status() == 0


def test_launch_variants_bit_identical_forward(tiny):
    wl, grid, geom, st, di = tiny
    rho = torch.tensor(wl.rho, device=DEV)
    base = tsp_forward(grid, geom, rho)
    for blk in (64, 128, 256, 512):
        for tw in (4, 8, 16, 32):
            assert torch.equal(tsp_forward(grid, geom, rho, launch=(blk, tw, 0)), base)
    yv = torch.tensor(synth.uniform_volume(geom.det_shape, 33), device=DEV)
    a0 = tsp_adjoint(grid, geom, yv, launch=(128, 8, 0))
    a1 = tsp_adjoint(grid, geom, yv, launch=(256, 16, 1))
    assert torch.allclose(a0, a1, rtol=1e-5, atol=1e-6)


def test_adjoint_accumulate(tiny):
    wl, grid, geom, st, di = tiny
    yv = torch.tensor(synth.uniform_volume(geom.det_shape, 34), device=DEV)
    base = torch.full(grid.shape, 2.0, device=DEV)
    out = tsp_adjoint(grid, geom, yv, out=base.clone(), accumulate=True)
    assert torch.allclose(out, base + tsp_adjoint(grid, geom, yv), rtol=1e-6, atol=1e-6)


def test_autograd_backward_is_adjoint_and_matches_fd(tiny):
    """ProjectorFn.backward equals the oracle's F^T; the gradient of
    ||y - F rho||^2 matches central finite differences of the oracle's FP64 loss."""
    wl, grid, geom, st, di = tiny
    op = Operator(grid, geom)
    y_obs = oracle.forward(wl.edges, st, di, wl.rho)
    rho0 = synth.uniform_volume(grid.shape, 35)
    rho = torch.tensor(rho0, device=DEV, requires_grad=True)
    loss = torch.sum((torch.tensor(y_obs.reshape(geom.det_shape), device=DEV, dtype=torch.float32) - op(rho)) ** 2)
    loss.backward()
    g = rho.grad.cpu().numpy().astype(np.float64)
    resid = oracle.forward(wl.edges, st, di, rho0) - y_obs
    g_ref = 2.0 * oracle.adjoint(wl.edges, st, di, resid)
    assert np.linalg.norm(g - g_ref) <= 1e-3 * np.linalg.norm(g_ref)
    rng = synth.SplitMix64(36)
    flat = rng.integers(0, grid.voxels - 1, 32)
    L = lambda r: float(np.sum((oracle.forward(wl.edges, st, di, r) - y_obs) ** 2))
    for f in flat:
        idx = np.unravel_index(int(f), grid.shape)
        if abs(g_ref[idx]) < 1e-3 * np.abs(g_ref).max():
            continue
        h = 1e-3
        rp = rho0.astype(np.float64).copy(); rp[idx] += h
        rm = rho0.astype(np.float64).copy(); rm[idx] -= h
        fd = (L(rp) - L(rm)) / (2 * h)
        assert abs(fd - g[idx]) <= 2e-3 * abs(fd) + 1e-6 * np.abs(g_ref).max(), (idx, fd, g[idx])


def test_rays_through_the_axis_in_a_half_plane():
    """Rays lying in a boundary half-plane that cross the z axis away from the
    origin; float32 rounding leaves them a few 1e-6 off the axis. Each half
    must land in a sector beside its half-plane: y matches the oracle for the
    float32 ray, or for the exact ray moved off the surface by 1e-9 (shifted
    across it, which sends the halves to opposite sides, or turned about z,
    which sends both to the same side). A walk that let rounding noise decide
    whether the half-planes are crossed left the second half in the first
    half's sector, an O(1) error."""
    e = synth.grid_edges(20, 15, 30)
    grid = Grid.from_edges(e)
    rho = synth.uniform_volume(e.shape, 6, 0.1, 1.0)
    R = float(e.r[-1])
    rng = np.random.default_rng(31)
    s64, d64, nrm = [], [], []
    for _ in range(200):
        p = e.phi[rng.integers(0, len(e.phi) - 1)]
        u = np.array([math.cos(p), math.sin(p), 0.0])
        s64.append(2 * R * u + rng.uniform(-R, R) * np.array([0.0, 0.0, 1.0]))
        d64.append(-u + np.array([0.0, 0.0, rng.uniform(-0.3, 0.3)]))
        nrm.append(np.array([-math.sin(p), math.cos(p), 0.0]))
    s64, d64, nrm = np.array(s64), np.array(d64), np.array(nrm)
    geom, st, di = rays_geom(s64.T, d64.T)
    y = tsp_forward(grid, geom, torch.tensor(rho, device=DEV)).cpu().numpy().reshape(-1)
    cands = [oracle.forward(e, st.T, di.T, rho)]
    cands += [oracle.forward(e, s64 + h * nrm, d64, rho) for h in (1e-9, -1e-9)]
    for ang in (1e-9, -1e-9):
        c, sn = math.cos(ang), math.sin(ang)
        rot = np.array([[c, -sn, 0.0], [sn, c, 0.0], [0.0, 0.0, 1.0]])
        cands.append(oracle.forward(e, s64 @ rot.T, d64 @ rot.T, rho))
    big = max(np.max(np.abs(c)) for c in cands)
    bad = [i for i in range(len(y))
           if min(abs(y[i] - c[i]) for c in cands) > 1e-4 * max(max(abs(c[i]) for c in cands), 1e-2 * big)]
    assert not bad, (bad[:5], y[bad[:5]])
    assert tsp_device_status() == 0


def test_lines_passing_just_off_the_axis():
    """The device build on lines passing 1e-7 .. 1e-3 from the z axis, from
    horizontal to within 1e-3 of vertical, starting 2 to 100 grid radii away
    (the host build's set, tests/test_host_walk.py): the parity rule, plus,
    for the few rays outside it, float32 crossing position over the sine of
    the grazing angle at each crossing (a line nearly parallel to a
    half-plane far from the axis)."""
    from _util import K_POS, U32, _crossing_gain
    e = synth.grid_edges(20, 15, 30)
    grid = Grid.from_edges(e)
    rho = synth.uniform_volume(e.shape, 6, 0.1, 1.0)
    R = float(e.r[-1])
    rng = np.random.default_rng(7)
    rays = []
    for S in (2.0, 10.0, 100.0):
        for nxy in (1.0, 0.1, 0.01, 1e-3):
            for dist in (1e-7, 1e-6, 1e-5, 1e-4, 1e-3):
                for _ in range(25):
                    a = rng.uniform(0, 2 * np.pi)
                    u = np.array([np.cos(a), np.sin(a), 0.0])
                    w = np.array([-np.sin(a), np.cos(a), 0.0])
                    n = nxy * u + np.array([0.0, 0.0, np.sqrt(1.0 - nxy * nxy) * rng.choice([-1.0, 1.0])])
                    p0 = dist * w + np.array([0.0, 0.0, rng.uniform(-0.5, 0.5) * R])
                    rays.append((p0 - S * R * n, n))
    s64 = np.array([a for a, _ in rays])
    d64 = np.array([b for _, b in rays])
    geom, st, di = rays_geom(s64.T, d64.T)
    y = tsp_forward(grid, geom, torch.tensor(rho, device=DEV)).cpu().numpy().reshape(-1)
    ref = oracle.forward(e, st.T, di.T, rho)
    big = np.max(np.abs(ref))
    err = np.abs(y - ref)
    plain = 1e-4 * np.maximum(np.abs(ref), 1e-2 * big)
    over = np.flatnonzero(err > plain)
    for i in over:
        x, d = st.T[i], di.T[i]
        n = d / np.linalg.norm(d)
        vox, l0, ln = oracle.ray_pieces(e, x, d)
        g = _crossing_gain(e, x[None, :] + np.concatenate([l0, l0 + ln])[:, None] * n[None, :], n, R)
        allow = float(rho.max()) * K_POS * U32 * R * g.sum()
        assert err[i] <= plain[i] + allow, (i, y[i], ref[i], allow)
    assert len(over) <= 0.01 * len(rays), len(over)
    assert tsp_device_status() == 0


def test_grid_whose_table_exceeds_48_kb_of_shared_memory():
    """1024 x 1024 x 512 voxels (2.1 GB volume): the grid table (51 KB) and
    the per-thread cone lists need more than the default 48 KB of dynamic
    shared memory per block, which the launch opts into. Forward on a 64 x 64
    cone view against the oracle on every 7th ray; the adjoint identity."""
    e = synth.grid_edges(1024, 1024, 512)
    grid = Grid.from_edges(e)
    rng = synth.SplitMix64(91)
    # a separable volume built from seeded 1-D profiles (keeps the host copy cheap)
    fr, fe, fa = (rng.uniform(n, 0.2, 1.0).astype(np.float32) for n in e.shape)
    rho = (fr[:, None, None] * fe[None, :, None] + fa[None, None, :]).astype(np.float32)
    geom = Geometry.cone(np.array([[60.0, 5.0, 3.0]]), (64, 64), 30.0)
    y = tsp_forward(grid, geom, torch.tensor(rho, device=DEV)).cpu().numpy().reshape(-1)
    st, di = oracle.cone_rays(np.array([[60.0, 5.0, 3.0]]), 64, 64, 30.0)
    idx = np.arange(0, len(st), 7)
    ref = oracle.forward(e, st[idx], di[idx], rho)
    parity(y[idx], ref, what="1024^3 grid forward")
    yv = torch.tensor(synth.uniform_volume(geom.det_shape, 92), device=DEV)
    x = torch.tensor(rho, device=DEV)
    lhs = torch.dot(tsp_forward(grid, geom, x).double().ravel(), yv.double().ravel()).item()
    rhs = torch.dot(x.double().ravel(), tsp_adjoint(grid, geom, yv).double().ravel()).item()
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs), (lhs, rhs)
    assert tsp_device_status() == 0
