"""FP64 oracle of SIRT on the spherical-grid projector (test infrastructure only).

The paper lists SIRT among the iterative reconstructions its operator serves
(Sec. 1, ref. [10]) without spelling it out; this is the standard
simultaneous iterative reconstruction technique (Gilbert 1972; Kak and
Slaney, "Principles of Computerized Tomographic Imaging", ch. 7):

    R = 1 / (F 1)      (per ray; 0 where a ray misses the grid)
    C = 1 / (F^T 1)    (per voxel; 0 where no ray touches the voxel)
    x <- x + C * F^T( R * (y - F x) ),   optionally clamped at 0 after each step.

F and F^T are the oracle's own FP64 forward and adjoint.
"""
from __future__ import annotations

import numpy as np

from . import adjoint, forward


def weights(edges, starts, dirs):
    ones_v = np.ones(edges.shape)
    fl = forward(edges, starts, dirs, ones_v)
    R = np.where(fl > 0, 1.0 / np.where(fl > 0, fl, 1.0), 0.0)
    ct = adjoint(edges, starts, dirs, np.ones(len(fl)))
    C = np.where(ct > 0, 1.0 / np.where(ct > 0, ct, 1.0), 0.0)
    return R, C


def sirt(edges, starts, dirs, y, x0, n_iter: int, nonneg: bool = False, weights_rc=None):
    """n_iter SIRT steps from x0; y is (n_rays,), x0 is (N_r, N_e, N_a). Returns x."""
    R, C = weights(edges, starts, dirs) if weights_rc is None else weights_rc
    x = np.array(x0, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64).reshape(-1)
    for _ in range(n_iter):
        r = R * (y - forward(edges, starts, dirs, x))
        x = x + C * adjoint(edges, starts, dirs, r)
        if nonneg:
            x = np.maximum(x, 0.0)
    return x
