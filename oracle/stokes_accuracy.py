"""Accuracy of the oracle's ESBI and HOS diagnostics against steady Stokes
waves: the comparison of the section on ESBI and HOS (deep water, one
wavelength on 64 points, 16 alias-free modes).  Prints, for each steepness
kH/2 and order M = 1..7, the largest error of V divided by the largest |V|
(deep water, then finite depth kd = 1, 2 at orders 3, 5, 7),
the exact V being -c eta_x of the Fourier-approximation solution
(oracle/steady_wave.py); then, for the implicit form of Appendix A (reading
R15), how its iterations behave against the steepness and how accurate its
solution is beside the successive scheme's.

TEST INFRASTRUCTURE: a documentation script that calls only ``oracle/``.
Usage: python -m oracle.stokes_accuracy
"""
from __future__ import annotations

import math

import numpy as np

from . import sbi_oracle as O
from . import steady_wave as sw


def errors(eps: float, n: int = 64, g: float = 9.81, depth: float = math.inf):
    L = 2 * math.pi
    w = sw.solve(k=1.0, H=2 * eps, depth=depth, g=g)
    grid = O.Grid(n, 1, L)
    x = np.arange(n) * L / n
    eta, phi, Vx = w.eta(x), w.surface_potential(x), w.vertical_velocity(x)
    scale = np.max(np.abs(Vx))
    esbi, hos = [], []
    for M in range(1, O.MAX_ORDER + 1):
        V = O.vertical_velocity(eta, phi, None, depth, grid, order=M).ravel()
        Vh, _ = O.hos_surface_velocity(eta, phi, depth, grid, order=M)
        esbi.append(float(np.max(np.abs(V - Vx)) / scale))
        hos.append(float(np.max(np.abs(Vh.ravel() - Vx)) / scale))
    return esbi, hos


def implicit(eps: float, n: int = 64, g: float = 9.81):
    L = 2 * math.pi
    w = sw.solve(k=1.0, H=2 * eps, g=g)
    grid = O.Grid(n, 1, L)
    x = np.arange(n) * L / n
    eta, phi, Vx = w.eta(x), w.surface_potential(x), w.vertical_velocity(x)
    scale = np.max(np.abs(Vx))
    _, _, inc = O.implicit_vertical_velocity(eta, phi, math.inf, grid, tol=1e-6, maxit=12)
    fixed = next((i + 1 for i, v in enumerate(inc) if v <= 1e-6), None)
    _, a3, _ = O.implicit_vertical_velocity(eta, phi, math.inf, grid, tol=1e-3, solver="gmres")
    V, a6, _ = O.implicit_vertical_velocity(eta, phi, math.inf, grid, tol=1e-6, solver="gmres")
    Vs = O.vertical_velocity(eta, phi, None, math.inf, grid)
    return (fixed, a3, a6, float(np.max(np.abs(V.ravel() - Vx)) / scale),
            float(np.max(np.abs(Vs.ravel() - Vx)) / scale))


def main():
    print("| kH/2 | diagnostic | " + " | ".join(f"M={m}" for m in range(1, 8)) + " |")
    print("|---|---|" + "---:|" * 7)
    for eps in (0.1, 0.2, 0.3, 0.35):
        e, h = errors(eps)
        print(f"| {eps} | ESBI | " + " | ".join(f"{v:.2e}" for v in e) + " |")
        print(f"| {eps} | HOS | " + " | ".join(f"{v:.2e}" for v in h) + " |")
    print()
    print("| kd | kH/2 | ESBI M=3 | M=5 | M=7 | HOS M=3 | M=5 | M=7 |")
    print("|---|---|" + "---:|" * 6)
    for kd in (1.0, 2.0):
        for eps in (0.1, 0.2):
            e, h = errors(eps, depth=kd)
            print(f"| {kd} | {eps} | " + " | ".join(f"{v:.1e}" for v in (e[2], e[4], e[6], h[2], h[4], h[6])) + " |")
    print()
    print("| kH/2 | fixed-point iterations to 1e-6 | GMRES applications to 1e-3 | to 1e-6 "
          "| error of the implicit solution | error of the successive scheme (M = 7) |")
    print("|---|---:|---:|---:|---:|---:|")
    for eps in (0.1, 0.2, 0.3, 0.35):
        f, a3, a6, ei, es = implicit(eps)
        print(f"| {eps} | {f if f is not None else 'diverges'} | {a3} | {a6} | {ei:.2e} | {es:.2e} |")


if __name__ == "__main__":
    main()
