"""FP64 CPU oracle for the spherical-grid projector (TomoSphero, Sec. 2-3).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import this package. The
product path never calls it and shares no code with it.

Each function cites the passage it follows; the C++ source holds the
arithmetic (``tsp_oracle.cpp``) and ``shbs.py`` / ``conv.py`` / ``sirt.py``
hold the oracles of the reconstruction layers.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libtsp_oracle.so")
_SRC = [os.path.join(_HERE, "tsp_oracle.cpp"), os.path.join(_HERE, "conv_oracle.cpp")]
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library with g++ (plain -O2, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    srcs = [s for s in _SRC if os.path.exists(s)]
    newest = max(os.path.getmtime(s) for s in srcs)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + f".{os.getpid()}.tmp"
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-pthread", "-o", tmp] + srcs
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            lp = ctypes.POINTER(ctypes.c_int64)
            i, i64, d = ctypes.c_int, ctypes.c_int64, ctypes.c_double
            grid = [dp, i, dp, i, dp, i]
            L.oracle_threads.restype = i
            L.oracle_ray_segments.argtypes = grid + [dp, dp, i, i, lp, dp]
            L.oracle_ray_segments.restype = i
            L.oracle_ray_pieces.argtypes = grid + [dp, dp, i, lp, dp, dp]
            L.oracle_ray_pieces.restype = i
            L.oracle_forward.argtypes = grid + [i64, dp, dp, dp, i, dp, i, i]
            L.oracle_forward.restype = i
            L.oracle_adjoint.argtypes = grid + [i64, dp, dp, dp, i, dp, i]
            L.oracle_adjoint.restype = i
            L.oracle_cone_rays.argtypes = [i, dp, dp, dp, i, i, d, d, dp, dp]
            L.oracle_parallel_rays.argtypes = [i, dp, dp, i, i, d, d, dp, dp]
            L.oracle_fill_zero.argtypes = [i, ip, ip, ip, dp, i, i, i]
            L.oracle_is_negative.argtypes = [i, dp, dp]
            L.oracle_is_negative.restype = i
            if hasattr(L, "oracle_conv3d_fwd"):
                fp = ctypes.POINTER(ctypes.c_float)
                conv = [i, i, i, i, i, i, i]
                L.oracle_conv3d_fwd.argtypes = conv + [fp, fp, fp, dp]
                L.oracle_conv3d_dgrad.argtypes = conv + [fp, fp, dp]
                L.oracle_conv3d_wgrad.argtypes = conv + [fp, fp, dp, dp]
                L.oracle_conv3d_fwd_f64.argtypes = conv + [dp, dp, dp, dp]
                L.oracle_conv3d_dgrad_f64.argtypes = conv + [dp, dp, dp]
                L.oracle_conv3d_wgrad_f64.argtypes = conv + [dp, dp, dp, dp]
            _lib = L
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _grid_args(edges):
    r, rp = _d(edges.r)
    t, tp = _d(edges.theta)
    p, pp = _d(edges.phi)
    return (r, t, p), [rp, len(r), tp, len(t), pp, len(p)]


def threads() -> int:
    return lib().oracle_threads()


def ray_segments(edges, x, n, method: int = 0, cap: int = 4096):
    """Segment list (flat voxel index, length) of one ray. method 0 = definition
    (sorted crossings, midpoint classification; Eq. 4), 1 = the paper's steps 1-3
    (Eq. 11-13 directions, sort, forward fill, zeroing; Sec. 3.2-3.3, Table 2)."""
    keep, ga = _grid_args(edges)
    xa, xp = _d(x)
    na, np_ = _d(n)
    vox = np.zeros(cap, dtype=np.int64)
    ln = np.zeros(cap, dtype=np.float64)
    cnt = lib().oracle_ray_segments(*ga, xp, np_, method, cap, vox.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                    ln.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if cnt < 0:
        raise ValueError("invalid grid")
    if cnt > cap:
        return ray_segments(edges, x, n, method, cnt)
    return vox[:cnt].copy(), ln[:cnt].copy()


def ray_pieces(edges, x, n, cap: int = 4096):
    """Pieces of one ray by the definition (Eq. 4): flat voxel index, start
    distance l0 along the normalised direction, and length."""
    keep, ga = _grid_args(edges)
    xa, xp = _d(x)
    na, np_ = _d(n)
    vox = np.zeros(cap, dtype=np.int64)
    l0 = np.zeros(cap, dtype=np.float64)
    ln = np.zeros(cap, dtype=np.float64)
    dp = ctypes.POINTER(ctypes.c_double)
    cnt = lib().oracle_ray_pieces(*ga, xp, np_, cap, vox.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                  l0.ctypes.data_as(dp), ln.ctypes.data_as(dp))
    if cnt < 0:
        raise ValueError("invalid grid")
    if cnt > cap:
        return ray_pieces(edges, x, n, cnt)
    return vox[:cnt].copy(), l0[:cnt].copy(), ln[:cnt].copy()


def forward(edges, starts, dirs, rho, method: int = 0, n_threads: int = 0):
    """y = F rho by Eq. 5 for rays given as (n, 3) starts and directions; rho is
    (N_r, N_e, N_a) or (B, N_r, N_e, N_a). Returns float64 (n,) or (B, n)."""
    keep, ga = _grid_args(edges)
    s, sp = _d(np.asarray(starts).reshape(-1, 3))
    d, dp = _d(np.asarray(dirs).reshape(-1, 3))
    shape = edges.shape
    rho = np.asarray(rho, dtype=np.float64)
    batched = rho.ndim == 4
    rb = rho.reshape(-1, *shape)
    rb, rp = _d(rb)
    n = s.shape[0]
    y = np.zeros((rb.shape[0], n), dtype=np.float64)
    rc = lib().oracle_forward(*ga, n, sp, dp, rp, rb.shape[0], y.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                              method, n_threads)
    if rc != 0:
        raise ValueError("invalid grid")
    return y if batched else y[0]


def adjoint(edges, starts, dirs, y, n_threads: int = 0):
    """F^T y: the adjoint of Eq. 5 (scatter of y * segment length; Sec. 4.4)."""
    keep, ga = _grid_args(edges)
    s, sp = _d(np.asarray(starts).reshape(-1, 3))
    d, dp = _d(np.asarray(dirs).reshape(-1, 3))
    n = s.shape[0]
    y = np.asarray(y, dtype=np.float64)
    batched = y.ndim == 2
    yb, yp = _d(y.reshape(-1, n))
    shape = edges.shape
    g = np.zeros((yb.shape[0],) + tuple(shape), dtype=np.float64)
    rc = lib().oracle_adjoint(*ga, n, sp, dp, yp, yb.shape[0], g.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                              n_threads)
    if rc != 0:
        raise ValueError("invalid grid")
    return g if batched else g[0]


def forward_dynamic(edges, starts, dirs, rho, n_views: int):
    """Dynamic object (Sec. 4.4): the rays are n_views equal consecutive
    blocks (one per view of a collection) and block k sees rho[k]. The
    definition written out: Eq. 5 per view on its own volume."""
    starts = np.asarray(starts).reshape(n_views, -1, 3)
    dirs = np.asarray(dirs).reshape(n_views, -1, 3)
    rho = np.asarray(rho, dtype=np.float64).reshape((n_views,) + tuple(edges.shape))
    return np.stack([forward(edges, starts[k], dirs[k], rho[k]) for k in range(n_views)])


def adjoint_dynamic(edges, starts, dirs, y, n_views: int):
    """Adjoint of forward_dynamic: volume k = F_k^T y[k]."""
    starts = np.asarray(starts).reshape(n_views, -1, 3)
    dirs = np.asarray(dirs).reshape(n_views, -1, 3)
    y = np.asarray(y, dtype=np.float64).reshape(n_views, -1)
    return np.stack([adjoint(edges, starts[k], dirs[k], y[k]) for k in range(n_views)])


def cone_rays(pos, H, W, fov_deg, look_at=None, up=None):
    """Cone-beam rays: pinhole at each pos, flat raster uniform in tangent space
    over the full field of view (Sec. 4.2, 4.6). Returns (V*H*W, 3) starts, dirs."""
    pos, pp = _d(np.asarray(pos).reshape(-1, 3))
    nv = pos.shape[0]
    fh, fw = (fov_deg, fov_deg) if np.isscalar(fov_deg) else fov_deg
    la = None if look_at is None else _d(np.asarray(look_at).reshape(-1, 3))
    uh = None if up is None else _d(np.asarray(up).reshape(-1, 3))
    st = np.zeros((nv * H * W, 3))
    di = np.zeros((nv * H * W, 3))
    lib().oracle_cone_rays(nv, pp, la[1] if la else None, uh[1] if uh else None, H, W, float(fh), float(fw),
                           st.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                           di.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return st, di


def parallel_rays(pos, H, W, size, up=None):
    """Parallel-beam rays on a detector plane through pos (Sec. 4.2)."""
    pos, pp = _d(np.asarray(pos).reshape(-1, 3))
    nv = pos.shape[0]
    sh, sw = (size, size) if np.isscalar(size) else size
    uh = None if up is None else _d(np.asarray(up).reshape(-1, 3))
    st = np.zeros((nv * H * W, 3))
    di = np.zeros((nv * H * W, 3))
    lib().oracle_parallel_rays(nv, pp, uh[1] if uh else None, H, W, float(sh), float(sw),
                               st.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                               di.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return st, di


def fill_zero(r, e, a, lens, shape):
    """Table 2 (b)-(c): forward fill of blank indices (None) and zeroing of rows
    with an invalid index or a non-finite length."""
    blank = -(2 ** 31)
    conv = lambda v: np.array([blank if x is None else x for x in v], dtype=np.int32)
    r, e, a = conv(r), conv(e), conv(a)
    ln = np.array(lens, dtype=np.float64)
    ip = lambda z: z.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    lib().oracle_fill_zero(len(ln), ip(r), ip(e), ip(a), ln.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                           *shape)
    return r, e, a, ln


def is_negative(kind: int, p, n) -> bool:
    """Crossing direction by Eq. 11 (kind 0, sphere), 12 (1, cone), 13 (2, half-plane)."""
    pa, pp = _d(p)
    na, np_ = _d(n)
    return bool(lib().oracle_is_negative(kind, pp, np_))
