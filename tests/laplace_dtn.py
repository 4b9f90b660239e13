"""Independent reference for the surface vertical velocity: a direct numerical
solution of the Laplace problem of Sec. 2.1 in a periodic 2-D (x, z) fluid layer.

Test infrastructure only.  It shares nothing with the oracle's recursion: the
fluid domain -h0 + delta(x) <= z <= eta(x) is mapped onto 0 <= sigma <= 1 with
sigma = (z + h)/(eta + h), h = h0 - delta, and the transformed Laplace equation

    Phi_xx + 2 s_x Phi_xs + (s_x^2 + s_z^2) Phi_ss + s_xx Phi_s = 0

is collocated with a Fourier basis in x and Chebyshev-Gauss-Lobatto points in
sigma (Trefethen, Spectral Methods in MATLAB, ch. 6), with Phi = phi~ on the
surface and the impermeable seabed condition phi_z - delta_x phi_x = 0
(Eq. bottomBC).  The dense system is solved directly.  The returned
V = phi_z (1 + eta_x^2) - eta_x phi~_x is the exact vertical velocity of the
surface (Sec. 2.2) up to the discretisation error, which is spectrally small
for smooth inputs.
"""
from __future__ import annotations

import numpy as np


def cheb(n: int):
    """Chebyshev-Gauss-Lobatto points x_j = cos(pi j / n) and the
    differentiation matrix (negative-sum diagonal)."""
    x = np.cos(np.pi * np.arange(n + 1) / n)
    c = np.ones(n + 1)
    c[0] = c[-1] = 2.0
    c *= (-1.0) ** np.arange(n + 1)
    X = np.tile(x, (n + 1, 1)).T
    dX = X - X.T
    D = np.outer(c, 1.0 / c) / (dX + np.eye(n + 1))
    D -= np.diag(D.sum(axis=1))
    return x, D


def fourier_diff(n: int, L: float):
    """First-derivative matrix of the periodic trigonometric interpolant
    (Nyquist mode dropped)."""
    k = 2.0 * np.pi * np.fft.fftfreq(n, d=L / n)
    k[n // 2] = 0.0
    eye = np.eye(n)
    return np.real(np.fft.ifft(1j * k[:, None] * np.fft.fft(eye, axis=0), axis=0))


def exact_vertical_velocity(eta, phi, delta, h0: float, L: float, n_sigma: int = 32,
                            return_phi_grad: bool = False):
    """Surface vertical velocity V of the 1-D problem (eta, phi~, delta)."""
    eta = np.asarray(eta, dtype=np.float64).ravel()
    phi = np.asarray(phi, dtype=np.float64).ravel()
    nx = eta.size
    delta = np.zeros(nx) if delta is None else np.asarray(delta, dtype=np.float64).ravel()
    Dx = fourier_diff(nx, L)
    xi, Dxi = cheb(n_sigma)
    sig = 0.5 * (xi + 1.0)                # xi = 1 -> sigma = 1 (surface)
    Ds = 2.0 * Dxi
    Dss = Ds @ Ds
    h = h0 - delta
    D = eta + h
    hx, Dxv = Dx @ h, Dx @ D
    hxx, Dxx = Dx @ hx, Dx @ Dxv
    S = sig[:, None]                       # (n_sigma+1, 1)
    sx = (hx[None, :] - S * Dxv[None, :]) / D[None, :]
    sxx = (hxx[None, :] - 2.0 * sx * Dxv[None, :] - S * Dxx[None, :]) / D[None, :]
    sz2 = (1.0 / D[None, :]) ** 2 * np.ones_like(S)
    Ix, Is = np.eye(nx), np.eye(n_sigma + 1)
    A = (np.kron(Is, Dx @ Dx)
         + np.diag((2.0 * sx).ravel()) @ np.kron(Ds, Dx)
         + np.diag((sx * sx + sz2).ravel()) @ np.kron(Dss, Ix)
         + np.diag(sxx.ravel()) @ np.kron(Ds, Ix))
    rhs = np.zeros((n_sigma + 1) * nx)
    # surface rows (sigma index 0): Dirichlet Phi = phi~
    A[:nx, :] = 0.0
    A[:nx, :nx] = Ix
    rhs[:nx] = phi
    # bottom rows (sigma index n_sigma): Phi_s / D - delta_x (Phi_x + h_x/D Phi_s) = 0
    dx_delta = Dx @ delta
    b0 = n_sigma * nx
    rowsel = slice(b0, b0 + nx)
    Phi_s_bottom = np.kron(Ds[n_sigma:n_sigma + 1, :], Ix)           # (nx, N)
    Phi_x_bottom = np.zeros((nx, (n_sigma + 1) * nx))
    Phi_x_bottom[:, b0:b0 + nx] = Dx
    coef_s = (1.0 - dx_delta * hx) / D
    A[rowsel, :] = coef_s[:, None] * Phi_s_bottom - dx_delta[:, None] * Phi_x_bottom
    rhs[rowsel] = 0.0
    Phi = np.linalg.solve(A, rhs).reshape(n_sigma + 1, nx)
    Phi_s_top = (Ds[0:1, :] @ Phi).ravel()
    phi_z = Phi_s_top / D
    eta_x = Dx @ eta
    phi_x_s = Dx @ phi
    V = phi_z * (1.0 + eta_x ** 2) - eta_x * phi_x_s
    if return_phi_grad:
        u = phi_x_s - eta_x * phi_z       # horizontal velocity at the surface
        return V, u, phi_z
    return V
