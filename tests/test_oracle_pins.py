"""Pins for the FP64 oracle against what the paper and the geometry fix.

None of these re-types the oracle's own formulas: closed forms of the line
integral (uniform ball, shell-only densities), invariants (rotation, mirror,
linearity, positivity), brute-force quadrature with an independent point
classifier, hand-worked fixtures from Table 2 and Eq. 11-13, and agreement of
two independent derivations (definition vs the paper's steps 1-3).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2608_16960_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def impact(x, n):
    """Distance of the line x + l n from the origin (brute: min over a dense l grid
    is not needed; |x cross n| / |n| is the textbook point-line distance)."""
    n = n / np.linalg.norm(n, axis=-1, keepdims=True)
    return np.linalg.norm(np.cross(x, n), axis=-1)


def chord(r, b):
    return 2.0 * np.sqrt(np.maximum(r * r - b * b, 0.0))


def outside_rays(n, seed, radius=60.0, aim=25.0):
    s, d = synth.random_rays(n, seed, start_radius=radius, aim_radius=aim)
    return s.T.astype(np.float64), d.T.astype(np.float64)


# --------------------------------------------------------------------------
# closed forms (Sec. 5.1: the unit-sphere test; chords of balls and shells)
# --------------------------------------------------------------------------

def test_uniform_unit_ball_chord():
    """Fig. 11: a (50, 50, 50) grid of the unit ball with rho = 1 integrates to the
    chord 2 sqrt(1 - b^2)."""
    e = synth.grid_edges(50, 50, 50, r_min=0.0, r_max=1.0, log_r=False)
    s, d = outside_rays(400, 11, radius=3.0, aim=1.0)
    y = oracle.forward(e, s, d, np.ones(e.shape))
    ref = chord(1.0, impact(s, d))
    assert np.max(np.abs(y - ref)) < 1e-12


def test_shell_only_density_closed_form():
    """rho depends on the shell only: y = sum_k rho_k (C(r_{k+1}) - C(r_k)) for a
    ray starting outside the grid, whatever the angular edges are."""
    rng = synth.SplitMix64(5)
    r = np.sort(rng.uniform(9, 2.0, 20.0))
    th = np.concatenate([[0.0], np.sort(rng.uniform(6, 0.1, 3.0)), [math.pi]])
    ph = np.concatenate([[0.3], np.sort(rng.uniform(8, 0.4, 6.5)), [0.3 + 2 * math.pi]])
    e = synth.GridEdges(r, th, ph)
    rho_k = rng.uniform(8, 0.1, 2.0)
    rho = np.broadcast_to(rho_k[:, None, None], e.shape).copy()
    s, d = outside_rays(500, 12, radius=50.0, aim=20.0)
    y = oracle.forward(e, s, d, rho)
    b = impact(s, d)
    ref = sum(rho_k[k] * (chord(r[k + 1], b) - chord(r[k], b)) for k in range(len(rho_k)))
    assert np.max(np.abs(y - ref)) < 1e-10


def test_chord_sum_invariant():
    """Summed segment lengths = chord of the outer sphere minus chord of the inner."""
    e = synth.grid_edges(20, 15, 30)
    s, d = outside_rays(300, 13)
    b = impact(s, d)
    for i in range(0, 300, 7):
        vox, ln = oracle.ray_segments(e, s[i], d[i])
        assert abs(ln.sum() - (chord(25.0, b[i]) - chord(3.0, b[i]))) < 1e-10
        assert np.all(ln > 0) and np.all(vox >= 0)


def _bins(edges, v):
    return np.searchsorted(edges, v, side="right") - 1


def test_rays_through_origin():
    """b = 0: polar and azimuthal angles are constant on each half, so
    y = sum_k dr_k (rho[k, bin(-n)] + rho[k, bin(n)]). Pins the theta/phi bins
    and the flat index order (r, e, a)."""
    e = synth.grid_edges(7, 9, 11, r_min=1.0, r_max=9.0, log_r=False)
    rho = synth.uniform_volume(e.shape, 3).astype(np.float64)
    rng = synth.SplitMix64(77)
    dirs = rng.unit_vectors(40)
    L = 30.0
    for n in dirs:
        x = -L * n
        y = oracle.forward(e, x[None], n[None], rho)[0]
        ref = 0.0
        for u in (n, -n):
            th = math.acos(max(-1.0, min(1.0, u[2])))
            ph = math.atan2(u[1], u[0]) % (2 * math.pi)
            ie, ia = _bins(e.theta, th), min(_bins(e.phi, ph), e.shape[2] - 1)
            ref += sum((e.r[k + 1] - e.r[k]) * rho[k, ie, ia] for k in range(e.shape[0]))
        assert abs(y - ref) < 1e-10


# --------------------------------------------------------------------------
# invariants
# --------------------------------------------------------------------------

def _rot_z(v, a):
    c, s = math.cos(a), math.sin(a)
    out = v.copy()
    out[:, 0] = c * v[:, 0] - s * v[:, 1]
    out[:, 1] = s * v[:, 0] + c * v[:, 1]
    return out


def test_rotation_by_one_azimuth_bin_rolls_density():
    e = synth.grid_edges(10, 8, 12)
    rho = synth.uniform_volume(e.shape, 4)
    s, d = outside_rays(300, 14)
    da = 2 * math.pi / 12
    y_rot = oracle.forward(e, _rot_z(s, da), _rot_z(d, da), rho)
    y_roll = oracle.forward(e, s, d, np.roll(rho, -1, axis=2))
    assert np.max(np.abs(y_rot - y_roll)) < 1e-10


def test_z_mirror_flips_polar_index():
    e = synth.grid_edges(10, 8, 12)  # uniform theta edges are mirror-symmetric
    rho = synth.uniform_volume(e.shape, 5)
    s, d = outside_rays(300, 15)
    m = np.array([1.0, 1.0, -1.0])
    y_m = oracle.forward(e, s * m, d * m, rho)
    y_f = oracle.forward(e, s, d, rho[:, ::-1, :])
    assert np.max(np.abs(y_m - y_f)) < 1e-10


def test_linearity_and_positivity():
    e = synth.grid_edges(12, 9, 14)
    a = synth.uniform_volume(e.shape, 6).astype(np.float64)
    b = synth.uniform_volume(e.shape, 7).astype(np.float64)
    s, d = outside_rays(200, 16)
    ya, yb = oracle.forward(e, s, d, a), oracle.forward(e, s, d, b)
    yab = oracle.forward(e, s, d, 2.0 * a - 3.0 * b)
    assert np.max(np.abs(yab - (2 * ya - 3 * yb))) < 1e-10
    assert np.all(ya >= 0) and np.all(yb >= 0)
    # F 1 = in-grid path length
    ones = oracle.forward(e, s, d, np.ones(e.shape))
    bb = impact(s, d)
    assert np.max(np.abs(ones - (chord(25.0, bb) - chord(3.0, bb)))) < 1e-10


def test_adjoint_identity_fp64():
    e = synth.grid_edges(10, 8, 16)
    x = synth.uniform_volume(e.shape, 8).astype(np.float64)
    s, d = outside_rays(500, 17)
    yv = synth.SplitMix64(9).uniform(500)
    lhs = np.dot(oracle.forward(e, s, d, x), yv)
    rhs = np.sum(x * oracle.adjoint(e, s, d, yv))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


# --------------------------------------------------------------------------
# brute-force quadrature with an independent classifier
# --------------------------------------------------------------------------

def _quadrature(e, x, n, rho, h, L):
    n = n / np.linalg.norm(n)
    l = (np.arange(int(L / h)) + 0.5) * h
    p = x[None, :] + l[:, None] * n[None, :]
    r = np.linalg.norm(p, axis=1)
    th = np.arccos(np.clip(p[:, 2] / np.maximum(r, 1e-300), -1, 1))
    span = e.phi[-1] - e.phi[0]
    ph = e.phi[0] + np.mod(np.arctan2(p[:, 1], p[:, 0]) - e.phi[0], 2 * math.pi)
    ir, ie, ia = _bins(e.r, r), _bins(e.theta, th), _bins(e.phi, ph)
    if abs(span - 2 * math.pi) < 1e-9:
        ia = np.minimum(ia, e.shape[2] - 1)
    ok = (ir >= 0) & (ir < e.shape[0]) & (ie >= 0) & (ie < e.shape[1]) & (ia >= 0) & (ia < e.shape[2])
    vals = np.zeros_like(l)
    vals[ok] = rho[ir[ok], ie[ok], ia[ok]]
    return vals.sum() * h


@pytest.mark.parametrize("kind", ["full", "wedge", "fig4", "inside"])
def test_fine_step_quadrature_converges(kind):
    """Midpoint rule with step h, error <= h * (#crossings + 2) * max|rho|."""
    if kind == "full":
        e = synth.grid_edges(4, 3, 5, r_min=1.0, r_max=4.0)
        s, d = outside_rays(12, 18, radius=10.0, aim=4.0)
    elif kind == "wedge":  # Fig. 3: a grid over a small wedge
        e = synth.grid_edges(2, 2, 2, r_min=2.0, r_max=4.0, theta=(0.8, 1.6), phi=(0.2, 0.9))
        start = np.array([9.0, 3.0, 1.5])  # outside, aimed at points near (3, 1.5, 0.3) inside the wedge
        aim = np.array([3.0, 1.5, 0.3]) + 0.5 * synth.SplitMix64(19).unit_vectors(12)
        s, d = np.broadcast_to(start, aim.shape).copy(), aim - start
    elif kind == "fig4":  # Fig. 4: shape (1, 2, 7), not covering the whole sphere
        e = synth.grid_edges(1, 2, 7, r_min=1.0, r_max=2.0, theta=(0.6, 2.2), phi=(0.0, 1.75 * math.pi))
        s, d = outside_rays(12, 20, radius=6.0, aim=2.0)
    else:  # rays starting inside the grid
        e = synth.grid_edges(4, 3, 5, r_min=1.0, r_max=4.0)
        s, d = synth.interior_rays(12, 21, radius=3.5)
        s, d = s.T.astype(np.float64), d.T.astype(np.float64)
    rho = synth.uniform_volume(e.shape, 10).astype(np.float64) + 0.5
    y = oracle.forward(e, s, d, rho)
    h = 2e-4
    for i in range(len(y)):
        L = np.linalg.norm(s[i]) + 10.0
        q = _quadrature(e, s[i], d[i], rho, h, L)
        ncross = 2 * (e.shape[0] + 1) + 2 * (e.shape[1] + 1) + e.shape[2] + 1
        assert abs(q - y[i]) <= h * (ncross + 2) * rho.max(), (i, q, y[i])
    assert np.count_nonzero(y) >= len(y) // 3


# --------------------------------------------------------------------------
# two derivations agree: definition vs the paper's steps 1-3
# --------------------------------------------------------------------------

@pytest.mark.parametrize("grid", ["c1", "wedge", "offset_phi"])
def test_definition_matches_paper_steps(grid):
    if grid == "c1":
        e = synth.grid_edges(20, 15, 30)
    elif grid == "wedge":
        e = synth.grid_edges(6, 5, 7, theta=(0.4, 2.0), phi=(-0.5, 2.5))
    else:
        e = synth.grid_edges(6, 5, 7, phi=(1.0, 1.0 + 2 * math.pi))
    rho = synth.uniform_volume(e.shape, 11)
    s, d = outside_rays(1500, 22)
    si, di = synth.interior_rays(500, 23, radius=20.0)
    s = np.concatenate([s, si.T]); d = np.concatenate([d, di.T])
    y0 = oracle.forward(e, s, d, rho, method=0)
    y1 = oracle.forward(e, s, d, rho, method=1)
    assert np.max(np.abs(y0 - y1)) < 1e-10


# --------------------------------------------------------------------------
# hand-worked fixtures
# --------------------------------------------------------------------------

def test_table2_fill_and_zero():
    g = json.load(open(os.path.join(GOLD, "table2_fill_zero.json")))
    so = g["sorted"]
    lens = [float(v) for v in so["len"]]
    r, e, a, ln = oracle.fill_zero(so["r"], so["e"], so["a"], lens, g["grid_shape"])
    assert list(r) == g["filled"]["r"]
    assert list(e) == g["filled"]["e"]
    assert list(a) == g["filled"]["a"]
    assert np.allclose(ln, g["zeroed_len"])


def test_crossing_directions_eq11_13():
    g = json.load(open(os.path.join(GOLD, "crossing_direction.json")))
    for c in g["cases"]:
        assert oracle.is_negative(c["kind"], np.array(c["p"], float), np.array(c["n"], float)) == c["negative"], c


# --------------------------------------------------------------------------
# detector models (Sec. 4.2)
# --------------------------------------------------------------------------

def test_cone_rays_geometry():
    pos = np.array([[60.0, 0, 0], [0, 40.0, 30.0]])
    H, W, fov = 5, 7, 30.0
    st, di = oracle.cone_rays(pos, H, W, fov)
    assert np.allclose(st.reshape(2, H * W, 3), pos[:, None, :])
    assert np.allclose(np.linalg.norm(di, axis=1), 1.0)
    di = di.reshape(2, H, W, 3)
    for v in range(2):
        look = -pos[v] / np.linalg.norm(pos[v])
        assert np.allclose(di[v, H // 2, W // 2], look)  # odd raster: centre pixel on the axis
        # first column's centre pixel sits (1 - 1/W) of the half-angle off axis
        ang = math.degrees(math.acos(np.dot(di[v, H // 2, 0], look)))
        assert abs(ang - math.degrees(math.atan(math.tan(math.radians(15)) * (1 - 1 / W)))) < 1e-9
    # pos (60,0,0) looking at the origin with up +Z: row 0 is the top (+z), column 0 is -right (-y)
    assert di[0, 0, W // 2, 2] > 0 and di[0, H // 2, 0, 1] < 0


def test_parallel_rays_geometry():
    pos = np.array([[0.0, 0.0, 60.0], [30.0, -30.0, 10.0]])
    H, W, size = 4, 6, 50.0
    st, di = oracle.parallel_rays(pos, H, W, size)
    st, di = st.reshape(2, H * W, 3), di.reshape(2, H * W, 3)
    for v in range(2):
        look = -pos[v] / np.linalg.norm(pos[v])
        assert np.allclose(di[v], look)
        assert np.allclose((st[v] - pos[v]) @ look, 0.0)  # starts on the detector plane
        off = st[v] - pos[v]
        assert np.allclose(off.mean(axis=0), 0.0)
        ext = np.ptp(np.linalg.norm(off, axis=1))
        assert ext > 0
        corner = np.max(np.linalg.norm(off, axis=1))
        assert abs(corner - 0.5 * math.hypot(size * (1 - 1 / H), size * (1 - 1 / W))) < 1e-9
