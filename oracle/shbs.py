"""FP64 oracle of the parametric density model and of Adam (test infrastructure only).

Model (Sec. 4.5 Eq. 7; Sec. 6 Eq. 10 uses spherical harmonics per shell):
    rho[ir, ie, ia] = sum_j sum_q B[ir, j] c[j, q] Y[q](theta_ie, phi_ia)
with B the clamped cubic B-splines on uniform interior knots over [r_min, r_max]
(scipy.interpolate.BSpline.design_matrix) and Y the real orthonormal spherical
harmonics built from scipy.special.sph_harm_y (the routine the paper names as
its analogue, Sec. 6 footnote 2):
    Y_l0 = Re Y_l^0,  Y_lm = sqrt(2) (-1)^m Re Y_l^m,  Y_l,-m = sqrt(2) (-1)^m Im Y_l^m  (m > 0),
index q = l^2 + l + m.

Adam: Kingma and Ba, "Adam: A method for stochastic optimization", ICLR 2015,
Algorithm 1, with L2 weight decay added to the gradient.
"""
from __future__ import annotations

import numpy as np
from scipy.interpolate import BSpline
from scipy.special import sph_harm_y


def bspline_matrix(r, r_min, r_max, n_basis, k=3):
    n_int = n_basis - k - 1
    inner = r_min + (r_max - r_min) * np.arange(1, n_int + 1) / (n_int + 1)
    t = np.concatenate([[r_min] * (k + 1), inner, [r_max] * (k + 1)])
    return BSpline.design_matrix(np.clip(np.asarray(r, float), r_min, r_max), t, k).toarray()


def real_sh(L, theta, phi):
    """(len(theta), (L+1)^2) real orthonormal spherical harmonics."""
    theta = np.asarray(theta, float)
    phi = np.asarray(phi, float)
    out = np.zeros(theta.shape + ((L + 1) ** 2,))
    for l in range(L + 1):
        out[..., l * l + l] = sph_harm_y(l, 0, theta, phi).real
        for m in range(1, l + 1):
            y = sph_harm_y(l, m, theta, phi)
            out[..., l * l + l + m] = np.sqrt(2.0) * (-1) ** m * y.real
            out[..., l * l + l - m] = np.sqrt(2.0) * (-1) ** m * y.imag
    return out


def centres(edges):
    return (0.5 * (edges.r[:-1] + edges.r[1:]), 0.5 * (edges.theta[:-1] + edges.theta[1:]),
            0.5 * (edges.phi[:-1] + edges.phi[1:]))


def model_tables(edges, n_basis, L):
    rc, tc, pc = centres(edges)
    B = bspline_matrix(rc, edges.r[0], edges.r[-1], n_basis)
    T, P = np.meshgrid(tc, pc, indexing="ij")
    Y = real_sh(L, T.ravel(), P.ravel())  # (Ne*Na, nq)
    return B, Y


def render(edges, coeffs, n_basis, L, tables=None):
    B, Y = model_tables(edges, n_basis, L) if tables is None else tables
    nr, ne, na = edges.shape
    return (B @ np.asarray(coeffs, float) @ Y.T).reshape(nr, ne, na)


def render_adjoint(edges, grad_rho, n_basis, L, tables=None):
    B, Y = model_tables(edges, n_basis, L) if tables is None else tables
    nr = edges.shape[0]
    return B.T @ np.asarray(grad_rho, float).reshape(nr, -1) @ Y


def adam(p, grads, lr, betas=(0.9, 0.999), eps=1e-8, weight_decay=0.0):
    """Run len(grads) Adam steps from p with the given gradient sequence."""
    p = np.array(p, float)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    b1, b2 = betas
    for t, g in enumerate(grads, start=1):
        g = np.asarray(g, float) + weight_decay * p
        m = b1 * m + (1 - b1) * g
        v = b2 * v + (1 - b2) * g * g
        p = p - lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)
    return p
