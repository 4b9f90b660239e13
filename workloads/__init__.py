"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds the input generators that both the oracle-side tests and the
CUDA-side tests and benchmark use.  It contains none of the method's arithmetic
(no vertical-velocity recursion, no time stepping): only initial conditions,
bathymetries, sponge weights and random phases.

Every random number comes from PCG32 (O'Neill 2014: 64-bit LCG state,
multiplier 6364136223846793005, output = rotr32(((s >> 18) ^ s) >> 27, s >> 59)),
so the inputs are bit-identical on every machine.

The five workloads (sizes as used throughout the tests and the benchmark):

1. ``solitary_1d``  1-D flat bottom h=1 m, L=100 m, N=256, g=9.81; a Rayleigh
   solitary wave a/h=0.3 centred at x=25 m; dt=0.01 s.
2. ``bar_1d``       1-D submerged trapezoidal bar (the Beji-Battjes
   geometry of the paper's submerged-bar test): N=4096, L=80 m, still depth 0.4 m, toe at 30 m, 1:20 up to a
   0.1 m deep 2 m crest, 1:10 down; Gaussian-modulated train T=2.02 s,
   a=0.01 m; sponge layers over 10 m at each end; dt=0.005 s.
3. ``stokes_2d``    2-D 512x512 periodic box, flat kh=1, third-order Stokes wave
   ka=0.25 on the grid direction (17, 10) (30.47 deg); dt=T/64.
4. ``crossing_batch`` 96 deep-water (kp h = 5) crossing seas: 64 on 256x256
   (10x10 peak wavelengths) and 32 on 512x512 (20x20); two JONSWAP systems
   (gamma=3.3, cos^2 spreading) at +-20 deg, Hs=0.05 m each with
   kp=0.28/(0.05 sqrt 2); random phases from PCG32 seeded 1000+member;
   low-pass filter on; dt=Tp/32.
5. ``large_variable`` 4096x2048 on 64x32 peak wavelengths, mean kp h=1.5, ten
   sinusoidal bars of amplitude 0.3h and wavelength lambda_p/2 across x,
   raised-cosine ends; the crossing sea above with seed 7; filter on; dt=Tp/32.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

G = 9.81
_MASK64 = (1 << 64) - 1


# --------------------------------------------------------------------------
# PCG32 (vectorised over independent streams is not needed: one stream)
# --------------------------------------------------------------------------

class PCG32:
    """PCG-XSH-RR 64/32 generator (O'Neill 2014), standard seeding."""

    MULT = 6364136223846793005

    def __init__(self, seed: int, stream: int = 54):
        self.inc = ((stream << 1) | 1) & _MASK64
        self.state = 0
        self._next()
        self.state = (self.state + (seed & _MASK64)) & _MASK64
        self._next()

    def _next(self) -> int:
        old = self.state
        self.state = (old * self.MULT + self.inc) & _MASK64
        xorshifted = (((old >> 18) ^ old) >> 27) & 0xFFFFFFFF
        rot = old >> 59
        return ((xorshifted >> rot) | (xorshifted << ((-rot) & 31))) & 0xFFFFFFFF

    def uniform(self, n: int) -> np.ndarray:
        """n doubles in [0, 1) built from one 32-bit output each."""
        out = np.empty(n, dtype=np.float64)
        for i in range(n):
            out[i] = self._next() * (1.0 / 4294967296.0)
        return out


def _uniform_fast(seed: int, n: int) -> np.ndarray:
    """Same sequence as PCG32(seed).uniform(n), vectorised in blocks.

    The LCG is advanced with the closed-form jump a^j, c (a^j - 1)/(a - 1) so a
    block of states is produced with numpy uint64 arithmetic (which wraps mod 2^64).
    """
    g = PCG32(seed)
    a = PCG32.MULT
    c = g.inc
    block = 4096
    # multipliers and increments for jumps of 0..block-1 steps
    mul = np.empty(block, dtype=np.uint64)
    add = np.empty(block, dtype=np.uint64)
    m, ad = 1, 0
    for j in range(block):
        mul[j] = m
        add[j] = ad
        m = (m * a) & _MASK64
        ad = (ad * a + c) & _MASK64
    jump_mul, jump_add = m, ad
    out = np.empty(n, dtype=np.float64)
    state = g.state
    pos = 0
    with np.errstate(over="ignore"):
        while pos < n:
            cnt = min(block, n - pos)
            s = np.uint64(state) * mul[:cnt] + add[:cnt]
            xs = (((s >> np.uint64(18)) ^ s) >> np.uint64(27)) & np.uint64(0xFFFFFFFF)
            rot = s >> np.uint64(59)
            left = (np.uint64(32) - rot) & np.uint64(31)
            r = ((xs >> rot) | (xs << left)) & np.uint64(0xFFFFFFFF)
            out[pos:pos + cnt] = r.astype(np.float64) * (1.0 / 4294967296.0)
            state = (state * jump_mul + jump_add) & _MASK64
            pos += cnt
    return out


# --------------------------------------------------------------------------
# Workload description
# --------------------------------------------------------------------------

@dataclass
class Member:
    nx: int
    ny: int
    Lx: float
    Ly: float
    h0: float
    eta: np.ndarray
    phi: np.ndarray
    delta: np.ndarray | None = None


@dataclass
class Workload:
    name: str
    gravity: float
    dt: float
    steps: int
    members: list = field(default_factory=list)
    alpha: float = 0.5
    order: int = 7
    filt_beta1: float = 0.0
    filt_beta2: float = 0.0
    k_ref: float = 1.0
    sponge_w: np.ndarray | None = None      # same grid as every member
    sponge_nu: float = 0.0
    # pneumatic wavemaker: {"amp": [...], "omega": [...], "phase": [...], "x0": float}
    wavemaker: dict | None = None
    notes: dict = field(default_factory=dict)

    @property
    def points(self) -> int:
        return sum(m.nx * m.ny for m in self.members)


def dispersion_k(omega: float, h: float, g: float = G) -> float:
    """Solve omega^2 = g k tanh(k h) for k (Newton)."""
    k = omega * omega / g
    for _ in range(100):
        f = g * k * math.tanh(k * h) - omega * omega
        df = g * math.tanh(k * h) + g * k * h / math.cosh(k * h) ** 2
        dk = f / df
        k -= dk
        if abs(dk) < 1e-15 * k:
            break
    return k


def _spectral_integrate_1d(u: np.ndarray, L: float) -> np.ndarray:
    """Zero-mean periodic antiderivative of (u - mean u)."""
    n = u.size
    k = 2.0 * np.pi * np.fft.fftfreq(n, d=L / n)
    U = np.fft.fft(u)
    P = np.zeros_like(U)
    nz = k != 0
    P[nz] = U[nz] / (1j * k[nz])
    P[n // 2] = 0.0
    return np.real(np.fft.ifft(P))


# --------------------------------------------------------------------------
# 1. Rayleigh solitary wave
# --------------------------------------------------------------------------

def solitary_1d(n: int = 256, L: float = 100.0, h: float = 1.0, a: float = 0.3,
                x0: float = 25.0, g: float = G) -> Workload:
    x = np.arange(n) * (L / n)
    kappa = math.sqrt(3.0 * a / (4.0 * h * h * (h + a)))
    c = math.sqrt(g * (h + a))
    eta = a / np.cosh(kappa * (x - x0)) ** 2
    u = c * eta / (h + eta)
    phi = _spectral_integrate_1d(u, L)
    m = Member(n, 1, L, 1.0, h, eta.reshape(1, n), phi.reshape(1, n))
    return Workload("solitary_1d", g, 0.01, 1000, [m],
                    notes={"c": c, "a": a, "x0": x0, "kappa": kappa})


# --------------------------------------------------------------------------
# 2. Submerged trapezoidal bar
# --------------------------------------------------------------------------

def bar_depth(x: np.ndarray, h0: float = 0.4, toe: float = 30.0) -> np.ndarray:
    """Still-water depth h(x) of the trapezoidal bar: 1:20 up from the toe to a
    0.1 m deep, 2 m long crest, then 1:10 down."""
    h = np.full_like(x, h0)
    up = (x >= toe) & (x < toe + 6.0)
    h[up] = h0 - (x[up] - toe) / 20.0
    top = (x >= toe + 6.0) & (x < toe + 8.0)
    h[top] = 0.1
    down = (x >= toe + 8.0) & (x < toe + 11.0)
    h[down] = 0.1 + (x[down] - (toe + 8.0)) / 10.0
    return h


def gaussian_damping(x: np.ndarray, x0: float, k: float, L: float) -> np.ndarray:
    """Weight of the damping pressure in the submerged-bar section: a Gaussian
    exp(-(k (x - x0) / (4 pi))^2) centred at x0 (periodic distance), the
    printed form being in units of 1/k_p."""
    d = np.mod(x - x0 + 0.5 * L, L) - 0.5 * L
    return np.exp(-(k * d / (4.0 * np.pi)) ** 2)


def bar_1d(n: int = 4096, L: float = 80.0, h0: float = 0.4, a: float = 0.01,
           T: float = 2.02, g: float = G) -> Workload:
    x = np.arange(n) * (L / n)
    delta = h0 - bar_depth(x, h0)
    omega = 2.0 * np.pi / T
    k0 = dispersion_k(omega, h0, g)
    env = np.exp(-((x - 20.0) ** 2) / (2.0 * 4.0 ** 2))
    eta = a * env * np.cos(k0 * x)
    phi = (g * a / omega) * env * np.sin(k0 * x)
    w = np.zeros(n)
    left = x < 10.0
    w[left] = np.sin(0.5 * np.pi * (10.0 - x[left]) / 10.0) ** 2
    right = x > 70.0
    w[right] = np.sin(0.5 * np.pi * (x[right] - 70.0) / 10.0) ** 2
    m = Member(n, 1, L, 1.0, h0, eta.reshape(1, n), phi.reshape(1, n),
               delta.reshape(1, n))
    return Workload("bar_1d", g, 0.005, 8000, [m], sponge_w=w.reshape(1, n),
                    sponge_nu=omega, notes={"k0": k0, "omega": omega})


def bar_wavemaker_1d(n: int = 1024, L: float = 64.0, h0: float = 0.4, a: float = 0.01,
                     T: float = 2.02, toe: float = 10.0, g: float = G) -> Workload:
    """Numerical flume of the submerged-bar section: 64 m on 1024 points, still
    depth 0.4 m, the bar with its toe at 10 m, waves of period T and amplitude
    a from the pneumatic wavemaker split at both ends of the box (x0 = 0), the
    Gaussian damping pressure centred at 7/8 L with strength omega.  Starts
    from rest; dt = T/40."""
    x = np.arange(n) * (L / n)
    delta = h0 - bar_depth(x, h0, toe)
    omega = 2.0 * np.pi / T
    k0 = dispersion_k(omega, h0, g)
    w = gaussian_damping(x, 7.0 / 8.0 * L, k0, L)
    m = Member(n, 1, L, 1.0, h0, np.zeros((1, n)), np.zeros((1, n)), delta.reshape(1, n))
    return Workload("bar_wavemaker_1d", g, T / 40.0, 4000, [m], sponge_w=w.reshape(1, n),
                    sponge_nu=omega,
                    wavemaker={"amp": [a], "omega": [omega], "phase": [0.0], "x0": 0.0},
                    notes={"k0": k0, "omega": omega})


# --------------------------------------------------------------------------
# 3. Third-order Stokes wave (Fenton 1985 coefficients, finite depth)
# --------------------------------------------------------------------------

def stokes3(theta: np.ndarray, k: float, d: float, eps: float, g: float = G):
    """Third-order Stokes wave: surface eta(theta) and the potential
    phi(theta, z) as a callable, and the phase speed.  eps = k H / 2."""
    S = 1.0 / math.cosh(2.0 * k * d)
    sh = math.sinh(k * d)
    B22 = (1.0 / math.tanh(k * d)) * (1.0 + 2.0 * S) / (2.0 * (1.0 - S))
    B31 = -3.0 * (1.0 + 3.0 * S + 3.0 * S * S + 2.0 * S ** 3) / (8.0 * (1.0 - S) ** 3)
    A11 = 1.0 / sh
    A22 = 3.0 * S * S / (2.0 * (1.0 - S) ** 2)
    A31 = (-4.0 - 20.0 * S + 10.0 * S * S - 13.0 * S ** 3) / (8.0 * sh * (1.0 - S) ** 3)
    A33 = (-2.0 * S * S + 11.0 * S ** 3) / (8.0 * sh * (1.0 - S) ** 3)
    C0 = math.sqrt(math.tanh(k * d))
    C2 = C0 * (2.0 + 7.0 * S * S) / (4.0 * (1.0 - S) ** 2)
    eta = (eps * np.cos(theta) + eps ** 2 * B22 * np.cos(2 * theta)
           + eps ** 3 * B31 * (np.cos(theta) - np.cos(3 * theta))) / k
    scale = C0 * math.sqrt(g / k ** 3)

    def phi(th, z):
        zb = d + z
        return scale * ((eps * A11 + eps ** 3 * A31) * np.cosh(k * zb) * np.sin(th)
                        + eps ** 2 * A22 * np.cosh(2 * k * zb) * np.sin(2 * th)
                        + eps ** 3 * A33 * np.cosh(3 * k * zb) * np.sin(3 * th))

    c = C0 * math.sqrt(g / k) * (1.0 + eps * eps * C2 / C0)
    return eta, phi, c


def stokes_2d(n: int = 512, mode=(17, 10), kh: float = 1.0, ka: float = 0.25,
              k: float = 1.0, g: float = G) -> Workload:
    mx, my = mode
    L = 2.0 * np.pi * math.hypot(mx, my) / k
    d = kh / k
    x = np.arange(n) * (L / n)
    X, Y = np.meshgrid(x, x)
    kx, ky = 2.0 * np.pi * mx / L, 2.0 * np.pi * my / L
    theta = kx * X + ky * Y
    eps = ka  # first-harmonic steepness to leading order
    eta, phi_fn, c = stokes3(theta, k, d, eps, g)
    phi = phi_fn(theta, eta)
    omega = c * k
    T = 2.0 * np.pi / omega
    m = Member(n, n, L, L, d, eta, phi)
    return Workload("stokes_2d", g, T / 64.0, 2000, [m],
                    notes={"c": c, "kx": kx, "ky": ky, "T": T})


def stokes_1d(n: int, L: float, m: int, d: float, eps: float, g: float = G):
    """One-dimensional Stokes wave with wavenumber 2 pi m / L (test helper)."""
    k = 2.0 * np.pi * m / L
    x = np.arange(n) * (L / n)
    theta = k * x
    eta, phi_fn, c = stokes3(theta, k, d, eps, g)
    return eta, phi_fn(theta, eta), c, k


# --------------------------------------------------------------------------
# 4./5. Crossing JONSWAP seas
# --------------------------------------------------------------------------

KP_CROSSING = 0.28 / (0.05 * math.sqrt(2.0))


def crossing_sea(nx: int, ny: int, Lx: float, Ly: float, h: float, seed: int,
                 kp: float = KP_CROSSING, hs: float = 0.05, gamma: float = 3.3,
                 angle_deg: float = 20.0, g: float = G):
    """Linear superposition of two JONSWAP systems at +-angle with cos^2 spreading.

    Returns (eta, phi) with phi the linear surface potential of each travelling
    mode (phi^ = -i g/omega eta^).
    """
    kx = 2.0 * np.pi * np.fft.fftfreq(nx, d=Lx / nx)
    ky = 2.0 * np.pi * np.fft.fftfreq(ny, d=Ly / ny)
    KX, KY = np.meshgrid(kx, ky)
    K = np.hypot(KX, KY)
    dkx, dky = 2.0 * np.pi / Lx, 2.0 * np.pi / Ly
    with np.errstate(divide="ignore", invalid="ignore"):
        omega = np.sqrt(g * K * np.tanh(K * h))
        omega_p = math.sqrt(g * kp * math.tanh(kp * h))
        sig = np.where(omega <= omega_p, 0.07, 0.09)
        r = np.exp(-((omega - omega_p) ** 2) / (2.0 * sig ** 2 * omega_p ** 2))
        S = np.where(K > 0, omega ** -5.0 * np.exp(-1.25 * (omega_p / omega) ** 4)
                     * gamma ** r, 0.0)
        cg = np.where(K > 0, 0.5 * omega / K * (1.0 + 2.0 * K * h / np.sinh(2.0 * K * h)), 0.0)
        Fk = np.where(K > 0, S * cg / np.where(K > 0, K, 1.0), 0.0)  # S(w) dw/dk / k
    Fk = np.nan_to_num(Fk)
    theta = np.arctan2(KY, KX)
    # keep modes resolved well inside the dealiased band
    band = (np.abs(np.fft.fftfreq(nx, d=1.0 / nx))[None, :] < nx / 4) & \
           (np.abs(np.fft.fftfreq(ny, d=1.0 / ny))[:, None] < ny / 4)
    phases = _uniform_fast(seed, 2 * nx * ny).reshape(2, ny, nx) * 2.0 * np.pi
    C = np.zeros((ny, nx), dtype=np.complex128)
    for i, th0 in enumerate((math.radians(angle_deg), -math.radians(angle_deg))):
        dth = np.angle(np.exp(1j * (theta - th0)))
        D = np.where(np.abs(dth) < np.pi / 2, (2.0 / np.pi) * np.cos(dth) ** 2, 0.0)
        amp2 = 2.0 * Fk * D * dkx * dky * band
        m0 = 0.5 * np.sum(amp2)
        if m0 > 0:
            amp2 *= (hs / 4.0) ** 2 / m0
        C += np.sqrt(amp2) * np.exp(1j * phases[i])
    eta = np.real(np.fft.ifft2(C) * (nx * ny))
    with np.errstate(divide="ignore", invalid="ignore"):
        P = np.where(K > 0, -1j * g / np.where(omega > 0, omega, 1.0) * C, 0.0)
    phi = np.real(np.fft.ifft2(P) * (nx * ny))
    return eta, phi


def crossing_batch(n_small: int = 64, n_large: int = 32, kp: float = KP_CROSSING,
                   g: float = G, seed0: int = 1000) -> Workload:
    lam = 2.0 * np.pi / kp
    h = 5.0 / kp
    members = []
    idx = 0
    for n, nl, cnt in ((256, 10, n_small), (512, 20, n_large)):
        for _ in range(cnt):
            L = nl * lam
            eta, phi = crossing_sea(n, n, L, L, h, seed0 + idx, kp=kp, g=g)
            members.append(Member(n, n, L, L, h, eta, phi))
            idx += 1
    omega_p = math.sqrt(g * kp * math.tanh(kp * h))
    Tp = 2.0 * np.pi / omega_p
    return Workload("crossing_batch", g, Tp / 32.0, 1000, members,
                    filt_beta1=8.0, filt_beta2=30.0, k_ref=kp,
                    notes={"kp": kp, "Tp": Tp, "h": h})


def bars_delta(x: np.ndarray, Lx: float, lam_p: float, amp: float) -> np.ndarray:
    """Ten sinusoidal bars of wavelength lam_p/2 centred at Lx/2, each end
    tapered by a half-bar raised cosine."""
    lb = 0.5 * lam_p
    xs = 0.5 * Lx - 5.0 * lb
    xe = xs + 10.0 * lb
    d = np.zeros_like(x)
    inside = (x >= xs) & (x <= xe)
    d[inside] = amp * np.sin(2.0 * np.pi * (x[inside] - xs) / lb)
    ramp = 0.5 * lb
    w = np.ones_like(x)
    a = inside & (x < xs + ramp)
    w[a] = 0.5 * (1.0 - np.cos(np.pi * (x[a] - xs) / ramp))
    b = inside & (x > xe - ramp)
    w[b] = 0.5 * (1.0 - np.cos(np.pi * (xe - x[b]) / ramp))
    return d * w


def large_variable(nx: int = 4096, ny: int = 2048, nlx: int = 64, nly: int = 32,
                   kp: float = KP_CROSSING, seed: int = 7, g: float = G) -> Workload:
    lam = 2.0 * np.pi / kp
    h = 1.5 / kp
    Lx, Ly = nlx * lam, nly * lam
    eta, phi = crossing_sea(nx, ny, Lx, Ly, h, seed, kp=kp, g=g)
    x = np.arange(nx) * (Lx / nx)
    delta = np.broadcast_to(bars_delta(x, Lx, lam, 0.3 * h), (ny, nx)).copy()
    omega_p = math.sqrt(g * kp * math.tanh(kp * h))
    Tp = 2.0 * np.pi / omega_p
    m = Member(nx, ny, Lx, Ly, h, eta, phi, delta)
    return Workload("large_variable", g, Tp / 32.0, 5000, [m],
                    filt_beta1=8.0, filt_beta2=30.0, k_ref=kp,
                    notes={"kp": kp, "Tp": Tp, "h": h})


# --------------------------------------------------------------------------
# Generic band-limited random fields for parity tests
# --------------------------------------------------------------------------

def random_field(nx: int, ny: int, seed: int, amplitude: float = 1.0,
                 band: float = 0.5, slope: float = 2.0) -> np.ndarray:
    """Zero-mean real field whose Fourier modes satisfy |m| < band nx/2 and
    |n| < band ny/2, with amplitudes falling as (1+|index|)^-slope."""
    u = _uniform_fast(seed, 2 * nx * ny).reshape(2, ny, nx)
    m = np.fft.fftfreq(nx, d=1.0 / nx)
    n = np.fft.fftfreq(ny, d=1.0 / ny) if ny > 1 else np.zeros(1)
    M, N = np.meshgrid(m, n)
    keep = (np.abs(M) < band * nx / 2) & ((np.abs(N) < band * ny / 2) | (ny == 1))
    keep &= (M != 0) | (N != 0)
    amp = keep / (1.0 + np.hypot(M, N)) ** slope
    C = amp * np.exp(2j * np.pi * u[0]) * (0.5 + u[1])
    f = np.real(np.fft.ifft2(C))
    s = np.max(np.abs(f))
    return f * (amplitude / s) if s > 0 else f
