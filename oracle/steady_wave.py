"""Steady periodic gravity waves of permanent form (Stokes waves), FP64: the
fully nonlinear reference solution of the ESBI/HOS accuracy comparison.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: only the tests,
``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` may use it.  It
shares no code with the CUDA library, nor with the oracle's recursion.

The section of the paper that compares ESBI with HOS measures the error of the
surface vertical velocity V of both diagnostics against a numerically exact
steady Stokes wave (Fenton's Fourier-approximation solution), one wavelength
on 64 points, for steepness 0.1 ... 0.35 and orders 1 ... 7.  This module
computes such a wave by the Fourier-approximation (stream-function
collocation) method of Rienecker & Fenton (J. Fluid Mech. 104, 1981), written
here from its equations:

In the frame that moves with the wave (phase speed c, crest at x = 0, wave
number k, still-water depth d or deep water) the flow is steady and its
stream function is

    Psi(x, z) = -c (z + d) + sum_{j=1}^{N} B_j S_j(z) cos(j k x),

with S_j(z) = sinh(j k (z + d)) / cosh(j k d) (deep water: e^{j k z} and
-c z).  Psi is harmonic and Psi = 0 on the bed.  The wave-frame velocities are
U = Psi_z = -c + sum_j j k B_j C_j(z) cos(j k x) and
W = sum_j j k B_j S_j(z) sin(j k x), C_j(z) = cosh(j k (z + d)) / cosh(j k d)
(deep water e^{j k z}).  The unknowns are the surface elevations eta_m at the
N + 1 collocation points x_m = m pi / (k N) (crest to trough), the B_j, c, the
volume flux Q and the Bernoulli constant R; the equations are

    Psi(x_m, eta_m) = -Q                          (the surface is a streamline)
    (U^2 + W^2) / 2 + g eta_m = R                  (Bernoulli on the surface)
    mean of eta over a wavelength = 0               (z = 0 is the mean level)
    eta_0 - eta_N = H                               (the wave height),

2N + 4 equations for 2N + 4 unknowns, solved by Newton's method (central
difference Jacobian) with continuation in H from a linear wave.  There is no
uniform current in the potential below, so the mean horizontal velocity
under the waves vanishes in the fixed frame (Stokes' first definition of the
wave speed): the fixed-frame potential

    phi(x, z, t) = sum_j B_j C_j(z) sin(j k (x - c t))

is periodic, and its surface value phi~(x) = phi(x, eta(x), 0) together with
eta(x) is an input of the diagnostics.  Because the wave translates without
change of form, eta_t = -c eta_x, so the kinematic condition gives the exact
surface vertical velocity V = phi_z - eta_x phi_x = -c eta_x.

Reading R14: the steepness of the comparison is eps = k H / 2 (the height
measured crest to trough), and its error measure is the largest pointwise
error of V divided by the largest |V|.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class SteadyWave:
    """A converged steady wave.  Lengths in metres, g in m/s^2; ``depth`` is
    math.inf for deep water."""
    k: float
    H: float
    depth: float
    g: float
    c: float                 # phase speed (fixed frame, no mean current)
    Q: float                 # volume flux per unit width (wave frame)
    R: float                 # Bernoulli constant (wave frame)
    E: np.ndarray            # eta(x) = sum_{j=0}^{N} E_j cos(j k x)
    B: np.ndarray            # B[j - 1] = B_j, j = 1..N
    eta_nodes: np.ndarray    # eta at x_m = m pi / (k N), m = 0..N
    residual: float          # max |F| at the Newton solution

    @property
    def N(self) -> int:
        return len(self.B)

    def eta(self, x):
        x = np.asarray(x, dtype=np.float64)
        j = np.arange(self.N + 1)
        return np.cos(np.multiply.outer(x, j * self.k)) @ self.E

    def eta_x(self, x):
        x = np.asarray(x, dtype=np.float64)
        j = np.arange(self.N + 1)
        return -np.sin(np.multiply.outer(x, j * self.k)) @ (j * self.k * self.E)

    def surface_potential(self, x):
        """phi~(x) = phi(x, eta(x), t = 0) in the fixed frame."""
        x = np.asarray(x, dtype=np.float64)
        z = self.eta(x)
        j = np.arange(1, self.N + 1)
        Cz = _vertical(j, self.k, self.depth, z, cosh_part=True)
        return np.sum(self.B * Cz * np.sin(np.multiply.outer(x, j * self.k)), axis=-1)

    def vertical_velocity(self, x):
        """The exact V = -c eta_x of a wave of permanent form."""
        return -self.c * self.eta_x(x)

    def surface_conditions(self, x):
        """(Psi + Q, Bernoulli - R) on the surface at arbitrary x: both vanish
        for an exact solution, not only at the collocation points."""
        x = np.asarray(x, dtype=np.float64)
        z = self.eta(x)
        return _surface_residuals(x, z, self.B, self.c, self.Q, self.R, self.k, self.depth, self.g)


def _vertical(j, k, depth, z, cosh_part: bool):
    """C_j(z) (cosh_part) or S_j(z) for every j (last axis), evaluated without
    overflow: cosh(a (z + d)) / cosh(a d) = e^{a z} (1 + e^{-2 a (z + d)}) / (1 + e^{-2 a d})."""
    a = np.asarray(j, dtype=np.float64) * k
    z = np.asarray(z, dtype=np.float64)[..., None]
    ez = np.exp(a * z)
    if math.isinf(depth):
        return ez
    sgn = 1.0 if cosh_part else -1.0
    return ez * (1.0 + sgn * np.exp(-2.0 * a * (z + depth))) / (1.0 + np.exp(-2.0 * a * depth))


def _surface_residuals(x, z, B, c, Q, R, k, depth, g):
    j = np.arange(1, len(B) + 1)
    jk = j * k
    cx = np.cos(np.multiply.outer(x, jk))
    sx = np.sin(np.multiply.outer(x, jk))
    S = _vertical(j, k, depth, z, cosh_part=False)
    C = _vertical(j, k, depth, z, cosh_part=True)
    zb = z if math.isinf(depth) else z + depth
    psi = -c * zb + np.sum(B * S * cx, axis=-1)
    U = -c + np.sum(jk * B * C * cx, axis=-1)
    W = np.sum(jk * B * S * sx, axis=-1)
    return psi + Q, 0.5 * (U * U + W * W) + g * z - R


def _residual(u, N, k, depth, g, H):
    eta = u[:N + 1]
    B = u[N + 1:2 * N + 1]
    c, Q, R = u[2 * N + 1:]
    x = np.arange(N + 1) * math.pi / (k * N)
    f1, f2 = _surface_residuals(x, eta, B, c, Q, R, k, depth, g)
    w = np.ones(N + 1)
    w[0] = w[-1] = 0.5
    mean = np.dot(w, eta) / N             # trapezoid over half a period of an even function
    return np.concatenate([f1, f2, [mean, eta[0] - eta[-1] - H]])


def _newton(u, N, k, depth, g, H, tol=1e-13, maxit=40):
    for _ in range(maxit):
        F = _residual(u, N, k, depth, g, H)
        if np.max(np.abs(F)) < tol:
            return u, float(np.max(np.abs(F)))
        J = np.empty((len(F), len(u)))
        for i in range(len(u)):
            h = 1e-7 * max(1.0, abs(u[i]))
            up, um = u.copy(), u.copy()
            up[i] += h
            um[i] -= h
            J[:, i] = (_residual(up, N, k, depth, g, H) - _residual(um, N, k, depth, g, H)) / (2 * h)
        u = u - np.linalg.solve(J, F)
    F = _residual(u, N, k, depth, g, H)
    return u, float(np.max(np.abs(F)))


def solve(k: float, H: float, depth: float = math.inf, g: float = 9.81, N: int = 28,
          steps: int | None = None) -> SteadyWave:
    """The steady wave of wave number k and height H over depth ``depth``
    (math.inf: deep water) with N Fourier modes.  Solved in units where
    k = g = 1 and scaled back."""
    if not (k > 0 and H > 0 and g > 0 and N >= 2):
        raise ValueError("k, H, g must be positive and N >= 2")
    d = depth * k if not math.isinf(depth) else math.inf
    Hn = H * k
    if steps is None:
        steps = max(1, math.ceil(Hn / 2 / 0.05))
    # linear start: eta = a cos x; B_1 = a c (deep) or a / c (depth d)
    x = np.arange(N + 1) * math.pi / N
    sols = []
    res = math.inf
    for s in range(1, steps + 1):
        Hs = Hn * s / steps
        if not sols:
            a = Hs / 2
            c0 = 1.0 if math.isinf(d) else math.sqrt(math.tanh(d))
            guess = np.zeros(2 * N + 4)
            guess[:N + 1] = a * np.cos(x)
            guess[N + 1] = a * c0 if math.isinf(d) else a / c0
            guess[2 * N + 1] = c0
            guess[2 * N + 2] = 0.0 if math.isinf(d) else c0 * d
            guess[2 * N + 3] = 0.5 * c0 * c0
        elif len(sols) == 1:
            guess = sols[-1]
        else:
            guess = 2.0 * sols[-1] - sols[-2]     # linear extrapolation in H
        sol, res = _newton(guess, N, 1.0, d, 1.0, Hs)
        sols.append(sol)
    u = sols[-1]
    if res > 1e-10:
        raise RuntimeError(f"steady wave did not converge (residual {res:.3e})")
    eta_n = u[:N + 1]
    # cosine coefficients of the interpolant through the nodes (DCT-I)
    j = np.arange(N + 1)
    w = np.ones(N + 1)
    w[0] = w[-1] = 0.5
    E = (2.0 / N) * (np.cos(np.outer(j, j) * math.pi / N) @ (w * eta_n))
    E[0] *= 0.5
    E[-1] *= 0.5
    sv = math.sqrt(g / k)                 # velocity scale
    return SteadyWave(k=k, H=H, depth=depth, g=g,
                      c=float(u[2 * N + 1]) * sv,
                      Q=float(u[2 * N + 2]) * sv / k,
                      R=float(u[2 * N + 3]) * g / k,
                      E=E / k, B=u[N + 1:2 * N + 1] * sv / k,
                      eta_nodes=eta_n / k, residual=res)
