"""Python binding of the projector: grid and geometry handles, F, F^T, and the
autograd function whose backward is the hand-written adjoint.

Argument marshalling only: shapes and pointers are checked here, every step
of the projection runs in libtsp.so (include/tsp.h). Torch provides device
memory and the current CUDA stream.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np
import torch

from . import _lib
from ._lib import check, tsp_launch


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _stream(t: torch.Tensor):
    return ctypes.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)


def _require_cuda(t: torch.Tensor, name: str):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float32:
        raise TypeError(f"{name} must be float32")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


class Grid:
    """Spherical grid (Sec. 2.2, 4.1): N_r+1 shells, N_e+1 polar cones, N_a+1 half-planes.

    Mirrors tsp_grid_create. The handle lives on the current CUDA device."""

    def __init__(self, r_edges, theta_edges, phi_edges):
        L = _lib.load()
        self.r = np.ascontiguousarray(r_edges, dtype=np.float64)
        self.theta = np.ascontiguousarray(theta_edges, dtype=np.float64)
        self.phi = np.ascontiguousarray(phi_edges, dtype=np.float64)
        h = ctypes.c_void_p()
        check(L.tsp_grid_create(_dptr(self.r), len(self.r), _dptr(self.theta), len(self.theta), _dptr(self.phi),
                                len(self.phi), ctypes.byref(h)), "tsp_grid_create")
        self.handle = h
        self.device = torch.cuda.current_device()
        self.shape = (len(self.r) - 1, len(self.theta) - 1, len(self.phi) - 1)

    @classmethod
    def from_edges(cls, edges):
        return cls(edges.r, edges.theta, edges.phi)

    @classmethod
    def uniform(cls, shape, size_r=(0.0, 1.0)):
        """Uniform grid of the given shape out to size_r (Listing 1)."""
        nr, ne, na = shape
        return cls(np.linspace(size_r[0], size_r[1], nr + 1), np.linspace(0, math.pi, ne + 1),
                   np.linspace(0, 2 * math.pi, na + 1))

    @property
    def voxels(self):
        return int(np.prod(self.shape))

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            try:
                _lib.load(build_if_missing=False).tsp_grid_destroy(h)
            except Exception:
                pass
            self.handle = None


class Geometry:
    """View geometry handle: cone (ConeRectGeom), parallel (ParallelGeom) or
    free-form rays (ViewGeom), Sec. 4.2. A collection of equal-shape views
    (Sec. 4.3) is one handle with n_views > 1."""

    def __init__(self, handle, kind, det_shape, n_rays, keep=None):
        self.handle = handle
        self.kind = kind
        self.det_shape = det_shape  # (n_views, H, W) or (n_rays,)
        self.n_rays = n_rays
        self._keep = keep
        self.device = torch.cuda.current_device()

    @classmethod
    def cone(cls, pos, shape, fov_deg, look_at=None, up=None):
        """Pinhole detector at each pos looking at look_at (default origin);
        shape (H, W) pixels; fov_deg scalar or (fov_h, fov_w), full angles."""
        L = _lib.load()
        pos = np.ascontiguousarray(np.asarray(pos, dtype=np.float64).reshape(-1, 3))
        nv = pos.shape[0]
        H, W = shape
        fh, fw = (fov_deg, fov_deg) if np.isscalar(fov_deg) else fov_deg
        la = None if look_at is None else np.ascontiguousarray(np.asarray(look_at, np.float64).reshape(nv, 3))
        uh = None if up is None else np.ascontiguousarray(np.asarray(up, np.float64).reshape(nv, 3))
        h = ctypes.c_void_p()
        check(L.tsp_geom_cone(nv, _dptr(pos), _dptr(la) if la is not None else None,
                              _dptr(uh) if uh is not None else None, H, W, float(fh), float(fw), ctypes.byref(h)),
              "tsp_geom_cone")
        return cls(h, "cone", (nv, H, W), nv * H * W)

    @classmethod
    def parallel(cls, pos, shape, size, up=None):
        L = _lib.load()
        pos = np.ascontiguousarray(np.asarray(pos, dtype=np.float64).reshape(-1, 3))
        nv = pos.shape[0]
        H, W = shape
        sh, sw = (size, size) if np.isscalar(size) else size
        uh = None if up is None else np.ascontiguousarray(np.asarray(up, np.float64).reshape(nv, 3))
        h = ctypes.c_void_p()
        check(L.tsp_geom_parallel(nv, _dptr(pos), _dptr(uh) if uh is not None else None, H, W, float(sh), float(sw),
                                  ctypes.byref(h)), "tsp_geom_parallel")
        return cls(h, "parallel", (nv, H, W), nv * H * W)

    @classmethod
    def polar(cls, pos, shape, fov_deg, look_at=None, up=None):
        """Polar-binned detectors (Sec. 6): per view n_rad x n_az polar pixels
        over the field of view fov_deg; shape = (n_rad, n_az)."""
        L = _lib.load()
        pos = np.ascontiguousarray(np.asarray(pos, dtype=np.float64).reshape(-1, 3))
        nv = pos.shape[0]
        la = None if look_at is None else np.ascontiguousarray(np.asarray(look_at, np.float64).reshape(nv, 3))
        uh = None if up is None else np.ascontiguousarray(np.asarray(up, np.float64).reshape(nv, 3))
        nr, na = shape
        h = ctypes.c_void_p()
        check(L.tsp_geom_polar(nv, _dptr(pos), _dptr(la) if la is not None else None,
                               _dptr(uh) if uh is not None else None, nr, na, float(fov_deg), ctypes.byref(h)),
              "tsp_geom_polar")
        return cls(h, "polar", (nv, nr, na), nv * nr * na)

    @classmethod
    def rays(cls, starts: torch.Tensor, dirs: torch.Tensor, copy: bool = True):
        """Free-form rays; starts and dirs are CUDA float32 (3, n) tensors."""
        L = _lib.load()
        for t, nm in ((starts, "starts"), (dirs, "dirs")):
            _require_cuda(t, nm)
            if t.dim() != 2 or t.shape[0] != 3:
                raise ValueError(f"{nm} must have shape (3, n)")
        n = starts.shape[1]
        if dirs.shape[1] != n:
            raise ValueError("starts and dirs differ in length")
        h = ctypes.c_void_p()
        check(L.tsp_geom_rays(n, ctypes.c_void_p(starts.data_ptr()), ctypes.c_void_p(dirs.data_ptr()), int(copy),
                              ctypes.byref(h)), "tsp_geom_rays")
        return cls(h, "rays", (n,), n, keep=None if copy else (starts, dirs))

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            try:
                _lib.load(build_if_missing=False).tsp_geom_destroy(h)
            except Exception:
                pass
            self.handle = None


def _launch_ptr(launch):
    if launch is None:
        return None
    if isinstance(launch, tsp_launch):
        return ctypes.byref(launch)
    return ctypes.byref(tsp_launch(*launch))


def tsp_forward(grid: Grid, geom: Geometry, rho: torch.Tensor, launch=None,
                out: torch.Tensor | None = None) -> torch.Tensor:
    """y = F rho (Eq. 5). rho: (N_r, N_e, N_a) or (B, N_r, N_e, N_a) CUDA float32.
    Returns y shaped like the detector: (B?,) + det_shape, written into `out`
    (contiguous float32 on rho's device, B x the detector's size) if given."""
    _require_cuda(rho, "rho")
    batched = rho.dim() == 4
    if tuple(rho.shape[-3:]) != grid.shape or rho.dim() not in (3, 4):
        raise ValueError(f"rho shape {tuple(rho.shape)} does not match grid {grid.shape}")
    B = rho.shape[0] if batched else 1
    if out is None:
        y = torch.empty((B,) + geom.det_shape, device=rho.device, dtype=torch.float32)
    else:
        _require_cuda(out, "out")
        if out.numel() != B * geom.n_rays or not out.is_contiguous() or out.device != rho.device:
            raise ValueError("out must be a contiguous float32 tensor of the detector's size on rho's device")
        y = out.view((B,) + geom.det_shape)
    L = _lib.load()
    check(L.tsp_forward_ex(grid.handle, geom.handle, ctypes.c_void_p(rho.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                           B, _launch_ptr(launch), _stream(rho)), "tsp_forward")
    return y if batched else y[0]


def tsp_adjoint(grid: Grid, geom: Geometry, y: torch.Tensor, out: torch.Tensor | None = None,
                accumulate: bool = False, launch=None) -> torch.Tensor:
    """F^T y (adjoint of Eq. 5). y: det_shape or (B,) + det_shape."""
    _require_cuda(y, "y")
    nd = len(geom.det_shape)
    batched = y.dim() == nd + 1
    if tuple(y.shape[-nd:]) != geom.det_shape:
        raise ValueError(f"y shape {tuple(y.shape)} does not match geometry {geom.det_shape}")
    B = y.shape[0] if batched else 1
    if out is None:
        out = torch.empty((B,) + grid.shape, device=y.device, dtype=torch.float32)
        accumulate = False
    else:
        _require_cuda(out, "out")
        if out.numel() != B * grid.voxels:
            raise ValueError("out has the wrong size")
    L = _lib.load()
    check(L.tsp_adjoint_ex(grid.handle, geom.handle, ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                           B, int(accumulate), _launch_ptr(launch), _stream(y)), "tsp_adjoint")
    if batched:
        return out.view((B,) + grid.shape)
    return out.view(grid.shape)


def sirt_workspace(grid: Grid, geom: Geometry) -> torch.Tensor:
    """Device scratch for tsp_sirt (R, C, residual, back-projection)."""
    L = _lib.load()
    n = ctypes.c_size_t()
    check(L.tsp_sirt_workspace_bytes(grid.handle, geom.handle, ctypes.byref(n)), "tsp_sirt_workspace_bytes")
    return torch.empty(n.value, dtype=torch.uint8, device=torch.device("cuda", geom.device))


def tsp_sirt(grid: Grid, geom: Geometry, y: torch.Tensor, x: torch.Tensor, n_iter: int, nonneg: bool = False,
             workspace: torch.Tensor | None = None, reuse_weights: bool = False, launch=None) -> torch.Tensor:
    """n_iter SIRT updates of x (in place) toward measurements y; returns x."""
    _require_cuda(y, "y")
    _require_cuda(x, "x")
    if tuple(x.shape[-3:]) != grid.shape or x.numel() != grid.voxels:
        raise ValueError("x must have the grid's shape")
    if y.numel() != geom.n_rays:
        raise ValueError("y must hold one value per ray")
    ws = sirt_workspace(grid, geom) if workspace is None else workspace
    if reuse_weights and workspace is None:
        raise ValueError("reuse_weights needs the workspace of an earlier call")
    flags = (_lib.TSP_SIRT_NONNEG if nonneg else 0) | (_lib.TSP_SIRT_REUSE_WEIGHTS if reuse_weights else 0)
    L = _lib.load()
    check(L.tsp_sirt(grid.handle, geom.handle, ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                     int(n_iter), flags, ctypes.c_void_p(ws.data_ptr()), ws.numel(), _launch_ptr(launch),
                     _stream(x)), "tsp_sirt")
    return x


def tsp_autotune(grid: Grid, geom: Geometry):
    """Time candidate launch knobs for this size class and cache the fastest.
    Returns ((block, tile, scatter) forward, (block, tile, scatter) adjoint)."""
    L = _lib.load()
    f, a = tsp_launch(), tsp_launch()
    check(L.tsp_autotune(grid.handle, geom.handle, ctypes.byref(f), ctypes.byref(a),
                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)), "tsp_autotune")
    as_t = lambda l: (l.block_threads, l.warp_tile_w, l.scatter)
    return as_t(f), as_t(a)


def tsp_autotune_clear():
    _lib.load().tsp_autotune_clear()


def tsp_autotune_store(grid: Grid, geom: Geometry, fwd, adj):
    """Pin (block, tile, scatter) knobs for this size class as if tuned: later
    calls without explicit knobs use them."""
    f, a = tsp_launch(*fwd), tsp_launch(*adj)
    check(_lib.load().tsp_autotune_store(grid.handle, geom.handle, ctypes.byref(f), ctypes.byref(a)),
          "tsp_autotune_store")


def tsp_count_segments(grid: Grid, geom: Geometry) -> torch.Tensor:
    """Valid segments per ray (int32, det_shape)."""
    L = _lib.load()
    counts = torch.empty(geom.det_shape, dtype=torch.int32, device=torch.device("cuda", geom.device))
    check(L.tsp_count_segments(grid.handle, geom.handle, ctypes.c_void_p(counts.data_ptr()), _stream(counts)),
          "tsp_count_segments")
    return counts


class Segments:
    """Stored segment lists of one grid and geometry (Sec. 3 steps 1-3 kept,
    step 4 repeated): forward and adjoint stream 8 bytes per segment instead
    of re-tracing. transpose=True also keeps voxel-major lists, so that the
    adjoint gathers per voxel without atomics (twice the memory)."""

    def __init__(self, grid: Grid, geom: Geometry, transpose: bool = True):
        L = _lib.load()
        self.grid, self.geom = grid, geom
        h = ctypes.c_void_p()
        st = torch.cuda.current_stream(torch.device("cuda", geom.device)).cuda_stream
        check(L.tsp_segments_build(grid.handle, geom.handle, int(transpose), ctypes.byref(h), ctypes.c_void_p(st)),
              "tsp_segments_build")
        self.handle = h

    def info(self):
        """(n_rays, n_segments, device bytes)."""
        L = _lib.load()
        a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_size_t()
        check(L.tsp_segments_info(self.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
              "tsp_segments_info")
        return a.value, b.value, c.value

    def export(self):
        """Host copies (ray_off int64, vox uint32, len float32) of the ray-major lists."""
        n_rays, n_segs, _ = self.info()
        off = np.zeros(n_rays + 1, dtype=np.int64)
        vox = np.zeros(max(n_segs, 1), dtype=np.uint32)
        ln = np.zeros(max(n_segs, 1), dtype=np.float32)
        vp = lambda a: ctypes.c_void_p(a.ctypes.data)
        check(_lib.load().tsp_segments_export(self.handle, vp(off), vp(vox), vp(ln)), "tsp_segments_export")
        return off, vox[:n_segs], ln[:n_segs]

    def export_transposed(self):
        """Host copies (vox_off int64, ray uint32, len float32) of the voxel-major lists."""
        n_rays, n_segs, _ = self.info()
        off = np.zeros(self.grid.voxels + 1, dtype=np.int64)
        ray = np.zeros(max(n_segs, 1), dtype=np.uint32)
        ln = np.zeros(max(n_segs, 1), dtype=np.float32)
        vp = lambda a: ctypes.c_void_p(a.ctypes.data)
        check(_lib.load().tsp_segments_export_transposed(self.handle, vp(off), vp(ray), vp(ln)),
              "tsp_segments_export_transposed")
        return off, ray[:n_segs], ln[:n_segs]

    def forward(self, rho: torch.Tensor) -> torch.Tensor:
        _require_cuda(rho, "rho")
        if tuple(rho.shape[-3:]) != self.grid.shape or rho.dim() not in (3, 4):
            raise ValueError(f"rho shape {tuple(rho.shape)} does not match grid {self.grid.shape}")
        rho = rho.contiguous()
        B = rho.shape[0] if rho.dim() == 4 else 1
        y = torch.empty((B,) + self.geom.det_shape, device=rho.device, dtype=torch.float32)
        check(_lib.load().tsp_segments_forward(self.handle, ctypes.c_void_p(rho.data_ptr()),
                                               ctypes.c_void_p(y.data_ptr()), B, _stream(rho)),
              "tsp_segments_forward")
        return y if rho.dim() == 4 else y[0]

    def adjoint(self, y: torch.Tensor, out: torch.Tensor | None = None, accumulate: bool = False) -> torch.Tensor:
        _require_cuda(y, "y")
        nd = len(self.geom.det_shape)
        if tuple(y.shape[-nd:]) != self.geom.det_shape or y.dim() not in (nd, nd + 1):
            raise ValueError(f"y shape {tuple(y.shape)} does not match geometry {self.geom.det_shape}")
        y = y.contiguous()
        B = y.shape[0] if y.dim() == nd + 1 else 1
        if out is None:
            out = torch.empty((B,) + self.grid.shape, device=y.device, dtype=torch.float32)
            accumulate = False
        else:
            _require_cuda(out, "out")
            if out.numel() != B * self.grid.voxels or not out.is_contiguous():
                raise ValueError("out has the wrong size or is not contiguous")
        check(_lib.load().tsp_segments_adjoint(self.handle, ctypes.c_void_p(y.data_ptr()),
                                               ctypes.c_void_p(out.data_ptr()), B, int(accumulate), _stream(y)),
              "tsp_segments_adjoint")
        return out.view((B,) + self.grid.shape) if y.dim() == nd + 1 else out.view(self.grid.shape)

    def sirt_workspace(self) -> torch.Tensor:
        n = ctypes.c_size_t()
        check(_lib.load().tsp_segments_sirt_workspace_bytes(self.handle, ctypes.byref(n)),
              "tsp_segments_sirt_workspace_bytes")
        return torch.empty(n.value, dtype=torch.uint8, device=torch.device("cuda", self.geom.device))

    def sirt_weights(self):
        """(R [n_rays], C [grid shape]): the SIRT weights as tsp_segments_sirt forms them."""
        dev = torch.device("cuda", self.geom.device)
        R = torch.empty(self.geom.n_rays, device=dev)
        C = torch.empty(self.grid.shape, device=dev)
        st = torch.cuda.current_stream(dev).cuda_stream
        check(_lib.load().tsp_segments_sirt_weights(self.handle, ctypes.c_void_p(R.data_ptr()),
                                                    ctypes.c_void_p(C.data_ptr()), ctypes.c_void_p(st)),
              "tsp_segments_sirt_weights")
        return R, C

    def sirt(self, y: torch.Tensor, x: torch.Tensor, n_iter: int, nonneg: bool = False,
             workspace: torch.Tensor | None = None, reuse_weights: bool = False) -> torch.Tensor:
        """n_iter SIRT updates of x in place (as tsp_sirt), projections from the lists."""
        _require_cuda(y, "y")
        _require_cuda(x, "x")
        if x.numel() != self.grid.voxels or y.numel() != self.geom.n_rays:
            raise ValueError("x must match the grid and y the geometry")
        if reuse_weights and workspace is None:
            raise ValueError("reuse_weights needs the workspace of an earlier call")
        ws = self.sirt_workspace() if workspace is None else workspace
        flags = (_lib.TSP_SIRT_NONNEG if nonneg else 0) | (_lib.TSP_SIRT_REUSE_WEIGHTS if reuse_weights else 0)
        check(_lib.load().tsp_segments_sirt(self.handle, ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                            int(n_iter), flags, ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                            _stream(x)), "tsp_segments_sirt")
        return x

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            try:
                _lib.load(build_if_missing=False).tsp_segments_destroy(h)
            except Exception:
                pass
            self.handle = None


def sirt_chunked(items, n_iter: int, nonneg: bool = False, budget_bytes: int = 0):
    """SIRT over independent (grid, geom, y, x) items from stored segment
    lists built one memory-bounded chunk at a time (tsp_sirt_chunked); x is
    updated in place. Returns (chunks, peak list bytes)."""
    L = _lib.load()
    items = list(items)
    arr = (_lib.tsp_batch_item * len(items))()
    for i, (grid, geom, y, x) in enumerate(items):
        _require_cuda(y, "y")
        _require_cuda(x, "x")
        if y.numel() != geom.n_rays or x.numel() != grid.voxels:
            raise ValueError(f"item {i}: y or x has the wrong size")
        arr[i] = _lib.tsp_batch_item(grid.handle.value, geom.handle.value, y.data_ptr(), x.data_ptr())
    nc = ctypes.c_int()
    peak = ctypes.c_size_t()
    check(L.tsp_sirt_chunked(arr, len(items), n_iter, 1 if nonneg else 0, int(budget_bytes), ctypes.byref(nc),
                             ctypes.byref(peak), _stream(items[0][2])), "tsp_sirt_chunked")
    return nc.value, peak.value


def tsp_device_status(device_tensor: torch.Tensor | None = None) -> int:
    L = _lib.load()
    code = ctypes.c_int(0)
    st = torch.cuda.current_stream().cuda_stream
    L.tsp_device_status(ctypes.c_void_p(st), ctypes.byref(code))
    return code.value


class ProjectorFn(torch.autograd.Function):
    """Autograd function: forward = tsp_forward, backward = tsp_adjoint (the
    hand-written F^T), so parametric models (Eq. 7, Listing 8) differentiate
    through the projector."""

    @staticmethod
    def forward(ctx, rho, grid, geom, launch=None):
        ctx.grid, ctx.geom, ctx.launch = grid, geom, launch
        return tsp_forward(grid, geom, rho.contiguous(), launch)

    @staticmethod
    def backward(ctx, gy):
        g = tsp_adjoint(ctx.grid, ctx.geom, gy.contiguous(), launch=ctx.launch)
        return g, None, None, None


def _views(geom: Geometry) -> int:
    return geom.det_shape[0] if len(geom.det_shape) == 3 else 1


def tsp_forward_dynamic(grid: Grid, geom: Geometry, rho: torch.Tensor) -> torch.Tensor:
    """Dynamic object (Sec. 4.4): y[k] = F_k rho[k], view k of the collection
    seeing volume k. rho: (n_views, N_r, N_e, N_a); y shaped like the detector."""
    _require_cuda(rho, "rho")
    nv = _views(geom)
    if tuple(rho.shape) != (nv,) + grid.shape:
        raise ValueError(f"rho shape {tuple(rho.shape)} must be (views={nv},) + {grid.shape}")
    y = torch.empty(geom.det_shape, device=rho.device, dtype=torch.float32)
    check(_lib.load().tsp_forward_dynamic(grid.handle, geom.handle, ctypes.c_void_p(rho.data_ptr()),
                                          ctypes.c_void_p(y.data_ptr()), _stream(rho)), "tsp_forward_dynamic")
    return y


def tsp_adjoint_dynamic(grid: Grid, geom: Geometry, y: torch.Tensor, out: torch.Tensor | None = None,
                        accumulate: bool = False) -> torch.Tensor:
    """rho[k] (+)= F_k^T y[k]; returns (n_views, N_r, N_e, N_a)."""
    _require_cuda(y, "y")
    if tuple(y.shape) != geom.det_shape:
        raise ValueError(f"y shape {tuple(y.shape)} does not match geometry {geom.det_shape}")
    shape = (_views(geom),) + grid.shape
    if out is None:
        out = torch.empty(shape, device=y.device, dtype=torch.float32)
        accumulate = False
    else:
        _require_cuda(out, "out")
        if tuple(out.shape) != shape:
            raise ValueError("out has the wrong shape")
    check(_lib.load().tsp_adjoint_dynamic(grid.handle, geom.handle, ctypes.c_void_p(y.data_ptr()),
                                          ctypes.c_void_p(out.data_ptr()), int(accumulate), _stream(y)),
          "tsp_adjoint_dynamic")
    return out


class DynamicProjectorFn(torch.autograd.Function):
    """Autograd function of the dynamic projection: backward = tsp_adjoint_dynamic."""

    @staticmethod
    def forward(ctx, rho, grid, geom):
        ctx.grid, ctx.geom = grid, geom
        return tsp_forward_dynamic(grid, geom, rho.contiguous())

    @staticmethod
    def backward(ctx, gy):
        return tsp_adjoint_dynamic(ctx.grid, ctx.geom, gy.contiguous()), None, None


class ListProjectorFn(torch.autograd.Function):
    """Autograd function over stored segment lists: forward = the lists' F,
    backward = their F^T (the voxel-major gather when the lists were
    transposed), for repeated projections through one geometry."""

    @staticmethod
    def forward(ctx, rho, segments):
        ctx.segments = segments
        return segments.forward(rho)

    @staticmethod
    def backward(ctx, gy):
        return ctx.segments.adjoint(gy.contiguous()), None


class Operator:
    """Operator(grid, geom): callable F with autograd (Sec. 4.4, Listing 6).
    Called with a 3D object it projects it through every view; a 4D object
    is a batch of independent objects, or, with dynamic=True, a dynamic
    object whose k-th volume is seen by the k-th view (Sec. 4.4). With
    segments (a Segments of the same grid and geometry) F and F^T run from
    the stored lists instead of re-tracing every ray."""

    def __init__(self, grid: Grid, geom: Geometry, launch=None, dynamic: bool = False, segments=None):
        if segments is not None and (dynamic or segments.grid is not grid or segments.geom is not geom):
            raise ValueError("segments must belong to this grid and geometry (and the operator be static)")
        self.grid, self.geom, self.launch, self.dynamic = grid, geom, launch, dynamic
        self.segments = segments

    def __call__(self, rho: torch.Tensor) -> torch.Tensor:
        if self.dynamic and rho.dim() == 4:
            return DynamicProjectorFn.apply(rho, self.grid, self.geom)
        if self.segments is not None:
            return ListProjectorFn.apply(rho, self.segments)
        return ProjectorFn.apply(rho, self.grid, self.geom, self.launch)

    def T(self, y: torch.Tensor) -> torch.Tensor:
        if self.dynamic:
            return tsp_adjoint_dynamic(self.grid, self.geom, y)
        if self.segments is not None:
            return self.segments.adjoint(y)
        return tsp_adjoint(self.grid, self.geom, y, launch=self.launch)


class Batch:
    """Batched SIRT over independent (grid, geometry, y, x) items of uneven
    sizes: persistent per-stage launches, optionally one captured CUDA graph."""

    def __init__(self, items):
        L = _lib.load()
        self._items = list(items)  # keep handles and tensors alive
        arr = (_lib.tsp_batch_item * len(self._items))()
        for i, (grid, geom, y, x) in enumerate(self._items):
            _require_cuda(y, "y")
            _require_cuda(x, "x")
            if y.numel() != geom.n_rays or x.numel() != grid.voxels:
                raise ValueError(f"item {i}: y or x has the wrong size")
            arr[i] = _lib.tsp_batch_item(grid.handle.value, geom.handle.value, y.data_ptr(), x.data_ptr())
        h = ctypes.c_void_p()
        check(L.tsp_batch_create(arr, len(self._items), ctypes.byref(h)), "tsp_batch_create")
        self.handle = h
        self.device = torch.cuda.current_device()
        self._ws = None

    def info(self):
        L = _lib.load()
        r, v, b = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int()
        check(L.tsp_batch_info(self.handle, ctypes.byref(r), ctypes.byref(v), ctypes.byref(b)), "tsp_batch_info")
        return r.value, v.value, b.value

    def workspace(self, n_iter):
        L = _lib.load()
        n = ctypes.c_size_t()
        check(L.tsp_batch_workspace_bytes(self.handle, n_iter, ctypes.byref(n)), "tsp_batch_workspace_bytes")
        if self._ws is None or self._ws.numel() < n.value:
            self._ws = torch.empty(n.value, dtype=torch.uint8, device=torch.device("cuda", self.device))
        return self._ws

    def sirt(self, n_iter, nonneg=False):
        ws = self.workspace(n_iter)
        check(_lib.load().tsp_batch_sirt(self.handle, n_iter, _lib.TSP_SIRT_NONNEG if nonneg else 0,
                                         ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)), "tsp_batch_sirt")

    def capture(self, n_iter, nonneg=False):
        ws = self.workspace(n_iter)
        check(_lib.load().tsp_batch_sirt_capture(self.handle, n_iter, _lib.TSP_SIRT_NONNEG if nonneg else 0,
                                                 ctypes.c_void_p(ws.data_ptr()), ws.numel()), "tsp_batch_sirt_capture")

    def launch(self):
        check(_lib.load().tsp_batch_sirt_launch(self.handle, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)),
              "tsp_batch_sirt_launch")

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            try:
                _lib.load(build_if_missing=False).tsp_batch_destroy(h)
            except Exception:
                pass
            self.handle = None


# ---------------------------------------------------------------------------
# Attenuated projection (Sec. 9.3, Eq. 14-18)
# ---------------------------------------------------------------------------

def _vol_batch(grid: Grid, t: torch.Tensor, name: str) -> int:
    _require_cuda(t, name)
    if tuple(t.shape[-3:]) != grid.shape or t.dim() not in (3, 4):
        raise ValueError(f"{name} shape {tuple(t.shape)} does not match grid {grid.shape}")
    return t.shape[0] if t.dim() == 4 else 1


def sunward_rays(grid: Grid, sun, device=None):
    """F_1's rays (Fig. 16b): for every voxel (flat order) its centroid and the
    unit sun direction, as CUDA float32 (3, V) tensors (starts, dirs)."""
    L = _lib.load()
    dev = torch.device("cuda") if device is None else torch.device(device)
    s = np.ascontiguousarray(np.asarray(sun, dtype=np.float64).reshape(3))
    starts = torch.empty((3, grid.voxels), device=dev, dtype=torch.float32)
    dirs = torch.empty((3, grid.voxels), device=dev, dtype=torch.float32)
    check(L.tsp_sunward_rays(grid.handle, _dptr(s), ctypes.c_void_p(starts.data_ptr()),
                             ctypes.c_void_p(dirs.data_ptr()), _stream(starts)), "tsp_sunward_rays")
    return starts, dirs


def sunward_geometry(grid: Grid, sun, device=None) -> Geometry:
    """F_1's geometry: one ray per voxel from its centroid toward the sun
    (`sun`: 3 numbers pointing toward the sun)."""
    starts, dirs = sunward_rays(grid, sun, device)
    return Geometry.rays(starts, dirs, copy=True)


def optical_depth(grid: Grid, sun_geom: Geometry, rho: torch.Tensor, sigma: torch.Tensor) -> torch.Tensor:
    """tau_1 = F_1(sigma rho) (Eq. 14, 17), shaped like rho."""
    B = _vol_batch(grid, rho, "rho")
    if _vol_batch(grid, sigma, "sigma") != B or sigma.shape != rho.shape:
        raise ValueError("sigma must have the shape of rho")
    tau1 = torch.empty_like(rho)
    L = _lib.load()
    check(L.tsp_atten_optical_depth(grid.handle, sun_geom.handle, ctypes.c_void_p(rho.data_ptr()),
                                    ctypes.c_void_p(sigma.data_ptr()), ctypes.c_void_p(tau1.data_ptr()), B,
                                    _stream(rho)), "tsp_atten_optical_depth")
    return tau1


def optical_depth_adjoint(grid: Grid, sun_geom: Geometry, rho: torch.Tensor, sigma: torch.Tensor,
                          g_tau1: torch.Tensor, need_sigma: bool = True, out=None, accumulate: bool = False):
    """(sigma F_1^T g, rho F_1^T g): gradients of <g, F_1(sigma rho)>, written
    to (or, with accumulate, added to) out = (g_rho, g_sigma or None) if given."""
    B = _vol_batch(grid, rho, "rho")
    for t, nm in ((sigma, "sigma"), (g_tau1, "g_tau1")):
        _vol_batch(grid, t, nm)
        if t.shape != rho.shape:
            raise ValueError(f"{nm} must have the shape of rho")
    if out is not None:
        g_rho, g_sigma = out
    else:
        g_rho = torch.empty_like(rho)
        g_sigma = torch.empty_like(rho) if need_sigma else None
        accumulate = False
    L = _lib.load()
    check(L.tsp_atten_optical_depth_adjoint(
        grid.handle, sun_geom.handle, ctypes.c_void_p(rho.data_ptr()), ctypes.c_void_p(sigma.data_ptr()),
        ctypes.c_void_p(g_tau1.data_ptr()), ctypes.c_void_p(g_rho.data_ptr()),
        ctypes.c_void_p(g_sigma.data_ptr()) if g_sigma is not None else None, B, int(accumulate), _stream(rho)),
        "tsp_atten_optical_depth_adjoint")
    return g_rho, g_sigma


def atten_forward(grid: Grid, geom: Geometry, rho: torch.Tensor, sigma: torch.Tensor,
                  tau1: torch.Tensor) -> torch.Tensor:
    """Attenuated y (Eq. 16-18), shaped like tsp_forward's."""
    B = _vol_batch(grid, rho, "rho")
    for t, nm in ((sigma, "sigma"), (tau1, "tau1")):
        _vol_batch(grid, t, nm)
        if t.shape != rho.shape:
            raise ValueError(f"{nm} must have the shape of rho")
    y = torch.empty((B,) + geom.det_shape, device=rho.device, dtype=torch.float32)
    L = _lib.load()
    check(L.tsp_atten_forward(grid.handle, geom.handle, ctypes.c_void_p(rho.data_ptr()),
                              ctypes.c_void_p(sigma.data_ptr()), ctypes.c_void_p(tau1.data_ptr()),
                              ctypes.c_void_p(y.data_ptr()), B, _stream(rho)), "tsp_atten_forward")
    return y if rho.dim() == 4 else y[0]


def atten_backward(grid: Grid, geom: Geometry, rho, sigma, tau1, y, gy, need_sigma=True, need_tau1=True, out=None,
                   accumulate: bool = False):
    """Gradients of <gy, y> (y = atten_forward(rho, sigma, tau1)) with respect
    to rho, sigma and tau1 (None where not needed), written to (or, with
    accumulate, added to) out = (g_rho, g_sigma, g_tau1) if given (entries of
    out may be None)."""
    B = _vol_batch(grid, rho, "rho")
    for t, nm in ((y, "y"), (gy, "gy")):
        _require_cuda(t, nm)
        if t.numel() != B * geom.n_rays:
            raise ValueError(f"{nm} has the wrong size")
    if out is not None:
        g_rho, g_sigma, g_tau1 = out
    else:
        g_rho = torch.empty_like(rho)
        g_sigma = torch.empty_like(rho) if need_sigma else None
        g_tau1 = torch.empty_like(rho) if need_tau1 else None
        accumulate = False
    ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
    L = _lib.load()
    check(L.tsp_atten_backward(grid.handle, geom.handle, ptr(rho), ptr(sigma), ptr(tau1), ptr(y), ptr(gy),
                               ptr(g_rho), ptr(g_sigma), ptr(g_tau1), B, int(accumulate), _stream(rho)),
          "tsp_atten_backward")
    return g_rho, g_sigma, g_tau1


class OpticalDepthFn(torch.autograd.Function):
    """tau_1 = F_1(sigma rho) with its hand-written adjoint as backward."""

    @staticmethod
    def forward(ctx, rho, sigma, grid, sun_geom):
        rho, sigma = rho.contiguous(), sigma.contiguous()
        ctx.save_for_backward(rho, sigma)
        ctx.grid, ctx.sun = grid, sun_geom
        return optical_depth(grid, sun_geom, rho, sigma)

    @staticmethod
    def backward(ctx, g_tau1):
        rho, sigma = ctx.saved_tensors
        g_rho, g_sigma = optical_depth_adjoint(ctx.grid, ctx.sun, rho, sigma, g_tau1.contiguous(),
                                               need_sigma=ctx.needs_input_grad[1])
        return g_rho, g_sigma, None, None


class AttenuatedProjectionFn(torch.autograd.Function):
    """y = Eq. 17-18 given rho, sigma and tau_1, with the hand-written gradient."""

    @staticmethod
    def forward(ctx, rho, sigma, tau1, grid, geom):
        rho, sigma, tau1 = rho.contiguous(), sigma.contiguous(), tau1.contiguous()
        y = atten_forward(grid, geom, rho, sigma, tau1)
        ctx.save_for_backward(rho, sigma, tau1, y)
        ctx.grid, ctx.geom = grid, geom
        return y

    @staticmethod
    def backward(ctx, gy):
        rho, sigma, tau1, y = ctx.saved_tensors
        g = atten_backward(ctx.grid, ctx.geom, rho, sigma, tau1, y, gy.contiguous(),
                           need_sigma=ctx.needs_input_grad[1], need_tau1=ctx.needs_input_grad[2])
        return g[0], g[1], g[2], None, None


class AttenuatedOperator:
    """rho -> y of Eq. 16-17 with tau_1 = F_1(sigma rho) computed from the same
    rho (Eq. 17), differentiable in rho and sigma."""

    def __init__(self, grid: Grid, geom: Geometry, sun, device=None):
        self.grid, self.geom = grid, geom
        self.sun = sunward_geometry(grid, sun, device)

    def optical_depth(self, rho: torch.Tensor, sigma: torch.Tensor) -> torch.Tensor:
        return OpticalDepthFn.apply(rho, sigma, self.grid, self.sun)

    def __call__(self, rho: torch.Tensor, sigma: torch.Tensor) -> torch.Tensor:
        tau1 = self.optical_depth(rho, sigma)
        return AttenuatedProjectionFn.apply(rho, sigma, tau1, self.grid, self.geom)
