"""The library's per-ray walk (tsp_trace.cuh over the library's boundary table,
tsp_table.h), built for the host, against the FP64 oracle on the CPU.

- Line integrals (Eq. 5) of random rays on full, wedge and hollow grids, with
  starts outside and inside, meet the parity rule of tests/_util.py.
- The degenerate families of Sec. 5.1 meet it too: rays through the origin,
  along and parallel to the axis, and grazing a sphere. Rays in the
  equatorial plane or in a half-plane match the oracle for the ray or for
  the ray moved just off that surface.
- Voxel sequences equal the oracle's (Eq. 4) wherever no two crossings lie
  within float32 reach of each other.
- Lines passing just off the z axis, from horizontal to nearly vertical,
  meet the parity rule too.

No GPU: this checks the walk's index logic wherever the driver runs the CPU
tests. Its host build rounds divisions and square roots correctly, so lengths
differ from the GPU's in the last bits; the GPU itself is checked by the
`gpu` tests."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_2608_16960_gb300 import synth

from _util import K_POS, U32, _crossing_gain, parity

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2608_16960_gb300", "csrc")
BUILD = os.path.join(HERE, "_build")
SO = os.path.join(BUILD, "libhostwalk.so")
SRCS = [os.path.join(HERE, "host_walk.cpp"), os.path.join(CSRC, "tsp_trace.cuh"), os.path.join(CSRC, "tsp_table.h"),
        os.path.join(CSRC, "tsp_internal.h"), os.path.join(ROOT, "include", "tsp.h")]
CUDA_INC = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")


def _lib():
    if shutil.which("g++") is None or not os.path.isdir(CUDA_INC):
        pytest.skip("g++ or the CUDA headers are not available")
    os.makedirs(BUILD, exist_ok=True)
    if not os.path.exists(SO) or os.path.getmtime(SO) < max(os.path.getmtime(s) for s in SRCS):
        tmp = SO + f".{os.getpid()}.tmp"
        subprocess.run(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off", "-I" + CUDA_INC,
                        "-I" + CSRC, SRCS[0], "-o", tmp], check=True)
        os.replace(tmp, SO)
    L = ctypes.CDLL(SO)
    P = ctypes.c_void_p
    L.host_walk.restype = ctypes.c_int
    L.host_walk.argtypes = [P, ctypes.c_int, P, ctypes.c_int, P, ctypes.c_int, ctypes.c_long, P, P, ctypes.c_int, P, P,
                            P]
    L.host_walk_list.restype = ctypes.c_int
    L.host_walk_list.argtypes = L.host_walk.argtypes + [ctypes.c_int]
    L.host_table.restype = ctypes.c_int
    L.host_table.argtypes = [P, ctypes.c_int, P, ctypes.c_int, P, ctypes.c_int, P, ctypes.c_int, P]
    return L


@pytest.fixture(scope="module")
def lib():
    return _lib()


def walk(lib, edges, starts, dirs, cap=1024, ccap=32):
    """Segments of rays given as float32 (n, 3) starts and directions; ccap is
    the length of the walk's cone-crossing list."""
    r, t, p = [np.ascontiguousarray(a, np.float64) for a in (edges.r, edges.theta, edges.phi)]
    x = np.ascontiguousarray(starts, np.float32)
    d = np.ascontiguousarray(dirs, np.float32)
    n = len(x)
    vox = np.zeros((n, cap), np.int32)
    ln = np.zeros((n, cap), np.float32)
    cnt = np.zeros(n, np.int32)
    bad = lib.host_walk_list(r.ctypes.data, len(r), t.ctypes.data, len(t), p.ctypes.data, len(p), n, x.ctypes.data,
                             d.ctypes.data, cap, vox.ctypes.data, ln.ctypes.data, cnt.ctypes.data, ccap)
    assert bad == 0
    assert cnt.max(initial=0) <= cap
    return vox, ln, cnt


def forward(lib, edges, starts, dirs, rho):
    vox, ln, cnt = walk(lib, edges, starts, dirs)
    flat = rho.reshape(-1).astype(np.float64)
    mask = np.arange(vox.shape[1])[None, :] < cnt[:, None]
    return np.where(mask, flat[np.where(mask, vox, 0)] * ln.astype(np.float64), 0.0).sum(axis=1)


GRIDS = {
    "paper": lambda: synth.grid_edges(100, 60, 120),
    "wedge": lambda: synth.GridEdges(np.linspace(1.0, 2.0, 11), np.linspace(0.3, 2.0, 18),
                                     np.linspace(0.2, 2.5, 21)),
    "hollow-free": lambda: synth.GridEdges(np.array([0.0, 1.0, 2.0, 5.0, 25.0]),
                                           np.array([0.0, 0.5, np.pi / 2, 2.5, np.pi]),
                                           np.linspace(-np.pi, np.pi, 4)),
    "polar-cap": lambda: synth.GridEdges(np.linspace(0.5, 3.0, 6), np.linspace(0.1, 1.2, 7),
                                         np.linspace(0.0, 2 * np.pi, 9)),
}


@pytest.mark.parametrize("name", sorted(GRIDS))
def test_forward_parity_random_rays(lib, name):
    e = GRIDS[name]()
    R = float(e.r[-1])
    rho = synth.uniform_volume(e.shape, 5, 0.1, 1.0)
    s1, d1 = synth.random_rays(1500, 11, start_radius=2.4 * R, aim_radius=R)
    s2, d2 = synth.interior_rays(500, 12, radius=0.9 * R)
    st = np.concatenate([s1.T, s2.T])
    di = np.concatenate([d1.T, d2.T])
    y = forward(lib, e, st, di, rho)
    ref = oracle.forward(e, st.astype(np.float64), di.astype(np.float64), rho)
    parity(y, ref, what=f"host walk {name}")
    assert np.linalg.norm(y - ref) <= 1e-4 * np.linalg.norm(ref)


def _close(y, candidates, big):
    return min(abs(y - c) for c in candidates) <= 1e-4 * max(max(abs(c) for c in candidates), 1e-2 * big)


def test_degenerate_rays(lib):
    """Rays through the origin, parallel to and along the axis, grazing a
    sphere: the parity rule. Rays lying in a boundary surface (the equatorial
    cone theta = pi/2, an azimuth half-plane) may be attributed to either
    neighbouring voxel: they must match the oracle for the ray itself or for
    the ray moved just off the surface (shifted to either side, or turned
    either way about the axis, which moves both halves of a ray through the
    axis to the same rotational side)."""
    e = synth.grid_edges(20, 15, 30)
    rho = synth.uniform_volume(e.shape, 6, 0.1, 1.0)
    R = float(e.r[-1])
    rng = np.random.default_rng(3)
    plain, on_surface = [], []
    for _ in range(40):
        v = rng.normal(size=3)
        v /= np.linalg.norm(v)
        plain.append((2.0 * R * v, -v))                                                  # through the origin
        off = rng.uniform(-R, R, size=2)
        plain.append((np.array([off[0], off[1], 2.0 * R]), np.array([0.0, 0.0, -1.0])))  # parallel to the axis
        k = rng.integers(1, len(e.r))
        plain.append((np.array([-2.0 * R, float(e.r[k]) * (1 - 1e-7), 0.3]), np.array([1.0, 0.0, 0.0])))  # grazing
        a = rng.uniform(0, 2 * np.pi)
        on_surface.append((np.array([2.0 * R * np.cos(a), 2.0 * R * np.sin(a), 0.0]),
                           np.array([-np.cos(a + 0.3), -np.sin(a + 0.3), 0.0]), np.array([0.0, 0.0, 1.0])))
        p = e.phi[rng.integers(0, len(e.phi) - 1)]
        u = np.array([np.cos(p), np.sin(p), 0.0])
        on_surface.append((2 * R * u + rng.uniform(-R, R) * np.array([0.0, 0.0, 1.0]), -u + np.array([0, 0, 0.1]),
                           np.array([-np.sin(p), np.cos(p), 0.0])))
    plain.append((np.array([0.0, 0.0, 2.0 * R]), np.array([0.0, 0.0, -1.0])))          # along the axis
    for _ in range(12):  # exactly through the origin (b = 0 in float-float: the start a power-of-two
        v = rng.normal(size=3).astype(np.float32)  # multiple of the direction), from outside, and from
        for sc in (-32.0, -0.25, 0.25):  # just before and just after the origin
            plain.append((np.float32(sc) * v, v))
        # exactly meeting the z axis (m_z = 0): the azimuth jumps by pi there
        a3 = (rng.uniform(-1, 1, size=3) * [2.0 * R, 2.0 * R, R]).astype(np.float32)
        plain.append((a3, np.array([-a3[0], -a3[1], rng.uniform(-R, R)], np.float32)))
    st = np.array([a for a, _ in plain], np.float32)
    di = np.array([b for _, b in plain], np.float32)
    y = forward(lib, e, st, di, rho)
    ref = oracle.forward(e, st.astype(np.float64), di.astype(np.float64), rho)
    parity(y, ref, what="host walk degenerate rays")
    st = np.array([a for a, _, _ in on_surface], np.float32)
    di = np.array([b for _, b, _ in on_surface], np.float32)
    y = forward(lib, e, st, di, rho)
    # The rays as given, and the exact surface rays they round (built in
    # float64 in the surface) moved off it by 1e-9: shifted across it, or
    # turned about z. A half-plane ray crosses the axis into the opposite
    # half-plane, and its two halves may each fall on either side: a shift
    # puts them on opposite sides, a turn on the same side.
    s64 = np.array([a for a, _, _ in on_surface])
    d64 = np.array([b for _, b, _ in on_surface])
    nrm = np.array([n for _, _, n in on_surface])
    cands = [oracle.forward(e, st.astype(np.float64), di.astype(np.float64), rho)]
    cands += [oracle.forward(e, s64 + h * nrm, d64, rho) for h in (1e-9, -1e-9)]
    for ang in (1e-9, -1e-9):
        c, sn = np.cos(ang), np.sin(ang)
        rot = np.array([[c, -sn, 0.0], [sn, c, 0.0], [0.0, 0.0, 1.0]])
        cands.append(oracle.forward(e, s64 @ rot.T, d64 @ rot.T, rho))
    big = max(np.max(np.abs(c)) for c in cands)
    bad = [i for i in range(len(y)) if not _close(y[i], [c[i] for c in cands], big)]
    assert not bad, (bad[:5], y[bad[:5]], [c[bad[:5]] for c in cands])


def _merge(v, l):
    mv, ml = [], []
    for a, b in zip(v.tolist(), l.tolist()):
        if mv and mv[-1] == a:
            ml[-1] += b
        else:
            mv.append(a)
            ml.append(b)
    return mv, np.array(ml)


def test_voxel_sequences_match_the_definition(lib):
    e = synth.grid_edges(20, 15, 30)
    s, d = synth.random_rays(1500, 21)
    st, di = s.T, d.T
    vox, ln, cnt = walk(lib, e, st, di)
    same = 0
    for i in range(len(st)):
        ov, ol = oracle.ray_segments(e, st[i].astype(np.float64), di[i].astype(np.float64))
        mo, _ = _merge(ov, ol)
        mg, _ = _merge(vox[i, :cnt[i]].astype(np.int64), ln[i, :cnt[i]].astype(np.float64))
        same += mo == mg
        assert abs(ln[i, :cnt[i]].astype(np.float64).sum() - ol.sum()) <= 1e-4 * max(ol.sum(), 1e-30) + 1e-6, i
    assert same >= 0.995 * len(st), same


def _unit(v):
    return v / np.linalg.norm(v)


def test_more_degenerate_families(lib):
    """The rest of the degenerate suite (Sec. 5.1, Fig. 10 spirit), checked
    with the parity rule: rays parallel to a cone's generator (the cone
    quadratic's leading term vanishes), through a corner where a sphere, a
    cone and a half-plane meet (three-way ties), across the azimuth seam
    phi = 0 = 2 pi, and starting exactly on a sphere or a cone. Rays tangent
    to a cone (along a circle of latitude) get the parity rule plus the
    sliver that float32 rounding of a tangent line can add or remove."""
    e = synth.grid_edges(20, 15, 30)
    rho = synth.uniform_volume(e.shape, 8, 0.1, 1.0)
    R = float(e.r[-1])
    rng = np.random.default_rng(5)
    rays = []
    for _ in range(60):
        k = rng.integers(1, len(e.theta) - 1)
        th = float(e.theta[k])
        ph = rng.uniform(0, 2 * np.pi)
        r = rng.uniform(e.r[0], R)
        p = r * np.array([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])
        t_phi = np.array([-np.sin(ph), np.cos(ph), 0.0])
        rays.append((p - 2 * R * t_phi, t_phi))                                      # tangent to the cone
        g = np.array([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])
        off = _unit(np.cross(g, rng.normal(size=3))) * rng.uniform(0.1, 0.5) * R
        rays.append((off - 2 * R * g, g))                                            # parallel to a generator
        j, m = rng.integers(1, len(e.r)), rng.integers(0, len(e.phi) - 1)
        c = e.r[j] * np.array([np.sin(th) * np.cos(e.phi[m]), np.sin(th) * np.sin(e.phi[m]), np.cos(th)])
        d = _unit(rng.normal(size=3))
        rays.append((c - 2 * R * d, d))                                              # through a corner
        x0 = rng.uniform(0.1, 0.9) * R
        rays.append((np.array([x0, -2 * R, rng.uniform(-0.3, 0.3) * R]),
                     np.array([0.0, 1.0, rng.uniform(-0.2, 0.2)])))                  # across the seam
        u = _unit(rng.normal(size=3))
        rays.append((e.r[j] * u, _unit(rng.normal(size=3))))                         # starting on a sphere
        rays.append((p, _unit(rng.normal(size=3))))                                  # starting on a cone
    st = np.array([a for a, _ in rays], np.float32)
    di = np.array([b for _, b in rays], np.float32)
    y = forward(lib, e, st, di, rho)
    ref = oracle.forward(e, st.astype(np.float64), di.astype(np.float64), rho)
    tangent = np.arange(len(rays)) % 6 == 0
    parity(y[~tangent], ref[~tangent], what="host walk: more degenerate families")
    # At exact tangency, float32 rounding puts the line up to delta ~ 8 ulps of
    # R inside or outside the cone, cutting or missing a sliver of width up to
    # 2 sqrt(2 R delta); no float32 evaluation decides which the rounded line
    # does. So the bound adds that sliver in the densest voxel.
    delta = 8 * 2.0 ** -24 * R
    sliver = 2 * np.sqrt(2 * R * delta) * float(rho.max())
    big = np.max(np.abs(ref))
    err = np.abs(y[tangent] - ref[tangent])
    assert np.all(err <= 1e-4 * np.maximum(np.abs(ref[tangent]), 1e-2 * big) + sliver), (err.max(), sliver)


def test_fig4_grid_and_single_shell(lib):
    """The (1, 2, 7) grid of Fig. 4 (one shell, two polar bins, seven
    azimuth bins: sectors wider than a quarter turn get virtual half-planes),
    full and as a wedge, on rays from outside and from inside."""
    for e in (synth.GridEdges(np.array([1.0, 2.0]), np.array([0.0, 1.2, np.pi]), np.linspace(0.0, 2 * np.pi, 8)),
              synth.GridEdges(np.array([1.0, 2.0]), np.array([0.0, 1.2, np.pi]), np.linspace(0.3, 5.0, 8))):
        rho = synth.uniform_volume(e.shape, 9, 0.1, 1.0)
        s1, d1 = synth.random_rays(800, 31, start_radius=5.0, aim_radius=2.0)
        s2, d2 = synth.interior_rays(400, 32, radius=1.9)
        st = np.concatenate([s1.T, s2.T])
        di = np.concatenate([d1.T, d2.T])
        y = forward(lib, e, st, di, rho)
        ref = oracle.forward(e, st.astype(np.float64), di.astype(np.float64), rho)
        parity(y, ref, what=f"host walk Fig. 4 grid {e.phi[0]:.1f}..{e.phi[-1]:.1f}")


def test_extreme_direction_scales(lib):
    """Free-form directions are normalised (reading 7) whatever their scale:
    directions of length 1e-20 and 1e20 (whose squared length is subnormal or
    overflows float32) and starts 1e4 grid radii away give the same line
    integrals as the oracle."""
    e = synth.grid_edges(12, 9, 16)
    R = float(e.r[-1])
    rho = synth.uniform_volume(e.shape, 3, 0.1, 1.0)
    rng = np.random.default_rng(19)
    for scale, dist in ((1e-20, 2.0), (1e20, 2.0), (1.0, 1e4)):
        rays = []
        for _ in range(200):
            v = _unit(rng.normal(size=3))
            rays.append((dist * R * v, scale * (-v + 0.3 * _unit(rng.normal(size=3)) / dist)))
        st = np.array([a for a, _ in rays], np.float32)
        di = np.array([b for _, b in rays], np.float32)
        y = forward(lib, e, st, di, rho)
        ref = oracle.forward(e, st.astype(np.float64), di.astype(np.float64), rho)
        assert np.count_nonzero(ref) > 50
        parity(y, ref, what=f"host walk, directions x {scale:g}, starts at {dist:g} R")


def test_lines_passing_just_off_the_axis(lib):
    """Lines passing 1e-7 .. 1e-3 from the z axis, from horizontal to within
    1e-3 of vertical, starting 2 to 100 grid radii away. Near the axis the
    whole azimuth sweep happens within |m_z| / |n_xy|^2 of the point t_a
    where the line's horizontal projection passes closest to the axis; the
    walk measures half-plane crossings from t_a (float-float), so these rays
    meet the parity rule. The bound adds, for each crossing, float32 position
    error over the sine of its grazing angle (tests/_util.py): a line nearly
    parallel to a half-plane far from the axis crosses it at a grazing angle,
    like a line grazing a sphere."""
    e = synth.grid_edges(20, 15, 30)
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
    st = np.array([a for a, _ in rays], np.float32)
    di = np.array([b for _, b in rays], np.float32)
    y = forward(lib, e, st, di, rho)
    s64, d64 = st.astype(np.float64), di.astype(np.float64)
    ref = oracle.forward(e, s64, d64, rho)
    big = np.max(np.abs(ref))
    err = np.abs(y - ref)
    plain = 1e-4 * np.maximum(np.abs(ref), 1e-2 * big)
    over = np.flatnonzero(err > plain)
    for i in over:  # only these need the crossing term
        n = d64[i] / np.linalg.norm(d64[i])
        vox, l0, ln = oracle.ray_pieces(e, s64[i], d64[i])
        g = _crossing_gain(e, s64[i][None, :] + np.concatenate([l0, l0 + ln])[:, None] * n[None, :], n, R)
        allow = float(rho.max()) * K_POS * U32 * R * g.sum()
        assert err[i] <= plain[i] + allow, (i, y[i], ref[i], allow, g.max())
    assert len(over) <= 0.01 * len(rays), len(over)


def test_cone_list_refills_give_the_same_segments(lib):
    """The walk produces cone crossings ahead into a list and refills it when a
    ray has more crossings than the list holds: lists of 1, 2, 3 and 7
    entries give bit-identical segments to one of 32 (paper-scale grid, rays
    with up to 50 cone crossings)."""
    e = synth.grid_edges(100, 60, 120)
    s, d = synth.random_rays(600, 41)
    st, di = s.T, d.T
    v0, l0, c0 = walk(lib, e, st, di)
    assert c0.max() > 100
    for ccap in (1, 2, 3, 7):
        v1, l1, c1 = walk(lib, e, st, di, ccap=ccap)
        assert np.array_equal(c0, c1), ccap
        m = np.arange(v0.shape[1])[None, :] < c0[:, None]
        assert np.array_equal(np.where(m, v0, 0), np.where(m, v1, 0)), ccap
        assert np.array_equal(np.where(m, l0, 0).view(np.uint32), np.where(m, l1, 0).view(np.uint32)), ccap


def _table(edges):
    L = _lib()
    r, t, p = [np.ascontiguousarray(a, np.float64) for a in (edges.r, edges.theta, edges.phi)]
    out = np.zeros(200000, np.float32)
    info = np.zeros(8, np.int32)
    n = L.host_table(r.ctypes.data, len(r), t.ctypes.data, len(t), p.ctypes.data, len(p), out.ctypes.data, len(out),
                     info.ctypes.data)
    assert 0 < n <= len(out)
    return out[:n], info


@pytest.mark.parametrize("kind", ["paper", "wedge", "virtual", "offset"])
def test_table_layout(kind):
    """The boundary table the kernels read (the layout of tsp_table.h as seen
    through TGrid): 16-byte half-plane records per direction of travel with
    the next record's index and the sector beyond, cone records between
    +-inf sentinels, (high, low) squared radii after (-inf, 0), every part
    aligned for its vector loads, every sector narrower than pi/2."""
    if kind == "paper":
        e = synth.grid_edges(100, 60, 120)
    elif kind == "wedge":
        e = synth.GridEdges(np.linspace(1.0, 2.0, 11), np.linspace(0.3, 2.0, 18), np.linspace(0.2, 2.5, 21))
    elif kind == "virtual":  # three wide sectors, split by virtual planes
        e = synth.GridEdges(np.array([0.0, 1.0, 2.0]), np.array([0.0, 1.0, np.pi]), np.linspace(0.0, 2 * np.pi, 4))
    else:
        e = synth.GridEdges(np.array([1.0, 3.0]), np.array([0.2, 1.5, 2.9]), np.linspace(-2.0, -2.0 + 2 * np.pi, 9))
    T, info = _table(e)
    words, M, pr, cr, rr, s2l, k2l, pa = (int(v) for v in info)
    Nr, Ne, Na = len(e.r) - 1, len(e.theta) - 1, len(e.phi) - 1
    bits = T.view(np.int32)
    # parts in order, contiguous, aligned for float4 / float2 loads
    assert pr == 0 and cr == 8 * M + 4 and cr % 4 == 0
    assert rr == cr + 4 * (Ne + 2) + 2 and rr % 2 == 0
    assert s2l == rr + 2 * (Nr + 1) and k2l == s2l + Ne + 1 and pa == k2l + Ne + 1 and words == pa + M
    # half-plane records: same plane in both directions, unit (cos, sin),
    # next record one plane on, sector beyond = the neighbouring sector
    ang = T[pa:pa + M].astype(np.float64)
    assert ang[0] == 0.0 and np.all(np.diff(ang) > 0) and ang[-1] < 2 * np.pi
    gaps = np.diff(np.concatenate([ang, [2 * np.pi]]))
    assert np.all(gaps < 0.5 * np.pi + 1e-6), gaps.max()
    wrap = abs((e.phi[-1] - e.phi[0]) - 2 * np.pi) <= 1e-9
    for j in range(M):
        up, dn = T[4 * j:4 * j + 4], T[4 * (M + j):4 * (M + j) + 4]
        assert up[0] == dn[0] and up[1] == dn[1]
        assert abs(float(up[0]) ** 2 + float(up[1]) ** 2 - 1.0) < 1e-6
        assert abs(np.angle(complex(up[0], up[1]) / complex(T[4 * 0], T[4 * 0 + 1])) % (2 * np.pi)
                   - ang[j] % (2 * np.pi)) < 1e-5 or abs(ang[j]) < 1e-6
        assert bits[4 * j + 3] == (j + 1) % M
        assert bits[4 * (M + j) + 3] == M + (j - 1) % M
        assert bits[4 * (M + j) + 2] == bits[4 * ((j - 1) % M) + 2]
        sec = bits[4 * j + 2]
        assert -1 <= sec < Na
    secs = bits[2:4 * M:4]
    assert set(secs.tolist()) - {-1} == set(range(Na))  # every azimuth voxel has a sector
    assert (-1 in secs.tolist()) == (not wrap)  # a wedge has its gap sector
    # cone records between +inf and -inf, (cos, sin^2, cos^2 high parts, 0)
    C = T[cr - 4:cr + 4 * (Ne + 2)].reshape(Ne + 3, 4)
    assert C[0, 0] == np.inf and C[-1, 0] == -np.inf
    th = np.clip(e.theta, 0.0, np.pi)
    assert np.array_equal(C[1:-1, 0], np.cos(th).astype(np.float32))
    assert np.all(np.diff(C[1:-1, 0]) < 0)
    s2 = C[1:-1, 1].astype(np.float64) + T[s2l:s2l + Ne + 1].astype(np.float64)
    k2 = C[1:-1, 2].astype(np.float64) + T[k2l:k2l + Ne + 1].astype(np.float64)
    assert np.allclose(s2, np.sin(th) ** 2, rtol=1e-13, atol=1e-15)
    assert np.allclose(k2, np.cos(th) ** 2, rtol=1e-13, atol=1e-15)
    assert np.all(C[:, 3] == 0.0)
    # squared radii as (high, low) pairs after (-inf, 0)
    R = T[rr - 2:rr + 2 * (Nr + 1)].reshape(Nr + 2, 2)
    assert R[0, 0] == -np.inf and R[0, 1] == 0.0
    assert np.allclose(R[1:, 0].astype(np.float64) + R[1:, 1].astype(np.float64), e.r ** 2, rtol=1e-13, atol=0)
