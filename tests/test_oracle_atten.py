"""Pins for the attenuated-projector oracle (Sec. 9.3, Eq. 14-18).

Closed forms along radial lines of a shells-only grid (lengths known from the
radii alone, so the order of the segments and the inclusive running sum of
Eq. 18 are checked without the oracle's traversal), the single-voxel optical
depth toward the sun (a ray-sphere exit distance), the reduction to the plain
projector when nothing absorbs, and central finite differences of the
gradients.
"""
import math

import numpy as np

import oracle
from oracle import atten
from paper_2608_16960_gb300 import synth


def shells(radii, n_phi=1):
    """Shells-only grid: one theta bin [0, pi], n_phi equal phi bins over [0, 2 pi]."""
    return synth.GridEdges(np.asarray(radii, np.float64), np.array([0.0, math.pi]),
                           np.linspace(0.0, 2 * math.pi, n_phi + 1))


def attenuated_sum(rho_seq, sig_seq, e1_seq, lengths):
    """Eq. 17-18 for a hand-listed sequence of segments (in ray order)."""
    tau2, y = 0.0, 0.0
    for rho, sig, e1, dl in zip(rho_seq, sig_seq, e1_seq, lengths):
        tau2 += sig * rho * dl
        y += e1 * rho * math.exp(-tau2) * dl
    return y


RADII = [1.0, 2.0, 4.0, 7.0, 11.0]
RHO = np.array([0.9, 0.5, 0.3, 0.2])
SIG = np.array([0.7, 0.4, 0.25, 0.1])
TAU1 = np.array([0.3, 0.1, 0.05, 0.0])


def test_radial_ray_from_inside_closed_form():
    """A ray from the centre outward (off every angular boundary) crosses the
    shells in order 0..3 with lengths r_{k+1} - r_k (the hole r < 1 holds no
    voxel). The attenuation is asymmetric, so the order and the inclusive sum
    are pinned."""
    e = shells(RADII)
    vol = lambda a: a.reshape(4, 1, 1)
    y = atten.forward(e, [[0.0, 0.0, 0.0]], [[0.48, 0.36, 0.8]], vol(RHO), vol(SIG), vol(TAU1))[0]
    lengths = np.diff(RADII)
    ref = attenuated_sum(RHO, SIG, np.exp(-TAU1), lengths)
    assert abs(y - ref) < 1e-13 * ref
    # an exclusive sum (segment not attenuating itself) or the reversed order differ
    excl = sum(np.exp(-TAU1[k]) * RHO[k] * np.exp(-np.sum(SIG[:k] * RHO[:k] * lengths[:k])) * lengths[k]
               for k in range(4))
    rev = attenuated_sum(RHO[::-1], SIG[::-1], np.exp(-TAU1[::-1]), lengths[::-1])
    assert abs(y - excl) > 1e-3 and abs(y - rev) > 1e-3


def test_line_past_the_hole_closed_form():
    """From outside, parallel to z at distance b = 1.5 (r_0 < b < r_1): the
    ray meets shells 3, 2, 1, 0, 1, 2, 3, with lengths from the half-chords
    sqrt(r^2 - b^2); shell 0 is crossed in one piece of length 2 sqrt(r_1^2 - b^2)."""
    b = 1.5
    e = shells(RADII)
    vol = lambda a: a.reshape(4, 1, 1)
    x0 = [b * math.cos(0.3), b * math.sin(0.3), -30.0]
    y = atten.forward(e, [x0], [[0.0, 0.0, 1.0]], vol(RHO), vol(SIG), vol(TAU1))[0]
    h = np.sqrt(np.maximum(np.asarray(RADII) ** 2 - b * b, 0.0))  # half-chord at each radius
    seq, lens = [], []
    for k in (3, 2, 1):
        seq.append(k)
        lens.append(h[k + 1] - h[k])
    seq.append(0)
    lens.append(2 * h[1])  # b > r_0: the chord stays in shell 0
    for k in (1, 2, 3):
        seq.append(k)
        lens.append(h[k + 1] - h[k])
    seq = np.array(seq)
    ref = attenuated_sum(RHO[seq], SIG[seq], np.exp(-TAU1[seq]), lens)
    assert abs(y - ref) < 1e-12 * ref


def test_line_through_the_hole_closed_form():
    """Parallel to z at b = 0.5 < r_0: shell 0 is met before and after the
    hole; the two pieces are separate segments of Eq. 17-18 (joining them
    would attenuate the first piece by the second one's optical depth)."""
    b = 0.5
    e = shells(RADII)
    vol = lambda a: a.reshape(4, 1, 1)
    x0 = [b * math.cos(1.1), b * math.sin(1.1), -30.0]
    y = atten.forward(e, [x0], [[0.0, 0.0, 1.0]], vol(RHO), vol(SIG), vol(TAU1))[0]
    h = np.sqrt(np.asarray(RADII) ** 2 - b * b)
    seq = [3, 2, 1, 0, 0, 1, 2, 3]
    lens = [h[4] - h[3], h[3] - h[2], h[2] - h[1], h[1] - h[0], h[1] - h[0], h[2] - h[1], h[3] - h[2], h[4] - h[3]]
    ref = attenuated_sum(RHO[seq], SIG[seq], np.exp(-TAU1[seq]), lens)
    assert abs(y - ref) < 1e-12 * ref
    joined = [3, 2, 1, 0, 1, 2, 3]
    lj = lens[:3] + [2 * (h[1] - h[0])] + lens[5:]
    assert abs(y - attenuated_sum(RHO[joined], SIG[joined], np.exp(-TAU1[joined]), lj)) > 1e-4


def test_no_absorption_is_the_plain_projector():
    """sigma = 0 and tau_1 = 0: Eq. 17 reduces to Eq. 5."""
    e = synth.grid_edges(6, 5, 8)
    rho = synth.SplitMix64(3).uniform(6 * 5 * 8, 0.1, 1.0).reshape(e.shape)
    s, d = synth.random_rays(200, 17, start_radius=60.0, aim_radius=25.0)
    s, d = s.T.astype(np.float64), d.T.astype(np.float64)
    y = atten.forward(e, s, d, rho, np.zeros(e.shape), np.zeros(e.shape))
    assert np.allclose(y, oracle.forward(e, s, d, rho), rtol=1e-13, atol=0.0)


def test_single_voxel_optical_depth():
    """One voxel (r in [0, R], the full sphere): its centroid is (-R/2, 0, 0)
    (midpoints r = R/2, theta = pi/2, phi = pi), and tau_1 = sigma rho t with t
    the distance from there to the sphere along the sun direction."""
    R = 5.0
    e = shells([0.0, R])
    for sun in ([0.9, 0.3, 0.2], [0.3, -0.8, 0.52], [-1.0, 0.2, 0.1]):
        st, di = atten.sunward_rays(e, sun)
        assert np.allclose(st, [[-R / 2, 0.0, 0.0]], atol=1e-15)
        p, s = st[0], di[0]
        ps = p @ s
        t = -ps + math.sqrt(ps * ps - p @ p + R * R)
        tau = atten.optical_depth(e, np.full(e.shape, 0.8), np.full(e.shape, 0.6), st, di)
        assert abs(tau.item() - 0.48 * t) < 1e-13 * t


def test_shell_optical_depth_closed_form():
    """Shells-only grid with two phi bins and densities of the shell alone,
    sun along -y. Voxel (k, 0, 0) has its centroid at (0, c_k, 0), c_k =
    (r_k + r_{k+1}) / 2: its sunward ray runs back to r_k, through the inner
    shells and the hole, then out through every shell. Voxel (k, 0, 1) sits
    at (0, -c_k, 0) and its ray runs straight out."""
    e = shells(RADII, n_phi=2)
    vol = lambda a: np.repeat(a.reshape(4, 1, 1), 2, axis=2)
    st, di = atten.sunward_rays(e, [0.0, -3.0, 0.0])
    tau = atten.optical_depth(e, vol(RHO), vol(SIG), st, di)
    r = np.asarray(RADII)
    kap = SIG * RHO
    for k in range(4):
        c = 0.5 * (r[k] + r[k + 1])
        inward = kap[k] * (c - r[k]) + sum(kap[j] * (r[j + 1] - r[j]) for j in range(k))
        outward_all = sum(kap[j] * (r[j + 1] - r[j]) for j in range(4))
        outward_own = kap[k] * (r[k + 1] - c) + sum(kap[j] * (r[j + 1] - r[j]) for j in range(k + 1, 4))
        assert abs(tau[k, 0, 0] - (inward + outward_all)) < 1e-13 * tau[k, 0, 0]
        assert abs(tau[k, 0, 1] - outward_own) < 1e-13 * tau[k, 0, 1]


def _tiny():
    e = synth.grid_edges(2, 3, 4, r_min=2.0, r_max=9.0)
    g = synth.SplitMix64(41)
    rho = g.uniform(24, 0.2, 1.0).reshape(e.shape)
    sig = g.uniform(24, 0.05, 0.3).reshape(e.shape)
    tau1 = g.uniform(24, 0.0, 0.5).reshape(e.shape)
    s, d = synth.random_rays(12, 9, start_radius=30.0, aim_radius=9.0)
    return e, rho, sig, tau1, s.T.astype(np.float64), d.T.astype(np.float64), g.uniform(12, -1.0, 1.0)


def test_backward_matches_finite_differences():
    """Central differences of sum gy y in every input entry (FP64, h = 1e-6)."""
    e, rho, sig, tau1, s, d, gy = _tiny()
    g_rho, g_sig, g_tau = atten.backward(e, s, d, rho, sig, tau1, gy)
    f = lambda r, q, t: float(gy @ atten.forward(e, s, d, r, q, t))
    h = 1e-6
    for which, grad in ((0, g_rho), (1, g_sig), (2, g_tau)):
        for idx in np.ndindex(e.shape):
            args_p = [rho.copy(), sig.copy(), tau1.copy()]
            args_m = [rho.copy(), sig.copy(), tau1.copy()]
            args_p[which][idx] += h
            args_m[which][idx] -= h
            fd = (f(*args_p) - f(*args_m)) / (2 * h)
            assert abs(fd - grad[idx]) < 1e-7 * max(1.0, abs(fd)), (which, idx, fd, grad[idx])
    assert np.any(g_sig != 0) and np.any(g_tau != 0)


def test_optical_depth_backward_matches_finite_differences():
    e, rho, sig, tau1, s, d, gy = _tiny()
    st, di = atten.sunward_rays(e, [0.4, 0.7, -0.3])
    gt = synth.SplitMix64(8).uniform(24, -1.0, 1.0).reshape(e.shape)
    g_rho, g_sig = atten.optical_depth_backward(e, rho, sig, st, di, gt)
    f = lambda r, q: float(np.sum(gt * atten.optical_depth(e, r, q, st, di)))
    h = 1e-6
    for idx in np.ndindex(e.shape):
        for which, grad in ((0, g_rho), (1, g_sig)):
            p, m = [rho.copy(), sig.copy()], [rho.copy(), sig.copy()]
            p[which][idx] += h
            m[which][idx] -= h
            fd = (f(*p) - f(*m)) / (2 * h)
            assert abs(fd - grad[idx]) < 1e-7 * max(1.0, abs(fd))
