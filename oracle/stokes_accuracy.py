"""Accuracy of the oracle's ESBI and HOS diagnostics against steady Stokes
waves: the comparison of the section on ESBI and HOS (deep water, one
wavelength on 64 points, 16 alias-free modes).  Prints, for each steepness
kH/2 and order M = 1..7, the largest error of V divided by the largest |V|,
the exact V being -c eta_x of the Fourier-approximation solution
(oracle/steady_wave.py).

TEST INFRASTRUCTURE: a documentation script that calls only ``oracle/``.
Usage: python -m oracle.stokes_accuracy
"""
from __future__ import annotations

import math

import numpy as np

from . import sbi_oracle as O
from . import steady_wave as sw


def errors(eps: float, n: int = 64, g: float = 9.81):
    L = 2 * math.pi
    w = sw.solve(k=1.0, H=2 * eps, g=g)
    grid = O.Grid(n, 1, L)
    x = np.arange(n) * L / n
    eta, phi, Vx = w.eta(x), w.surface_potential(x), w.vertical_velocity(x)
    scale = np.max(np.abs(Vx))
    esbi, hos = [], []
    for M in range(1, O.MAX_ORDER + 1):
        V = O.vertical_velocity(eta, phi, None, math.inf, grid, order=M).ravel()
        Vh, _ = O.hos_surface_velocity(eta, phi, math.inf, grid, order=M)
        esbi.append(float(np.max(np.abs(V - Vx)) / scale))
        hos.append(float(np.max(np.abs(Vh.ravel() - Vx)) / scale))
    return esbi, hos


def main():
    print("| kH/2 | diagnostic | " + " | ".join(f"M={m}" for m in range(1, 8)) + " |")
    print("|---|---|" + "---:|" * 7)
    for eps in (0.1, 0.2, 0.3, 0.35):
        e, h = errors(eps)
        print(f"| {eps} | ESBI | " + " | ".join(f"{v:.2e}" for v in e) + " |")
        print(f"| {eps} | HOS | " + " | ".join(f"{v:.2e}" for v in h) + " |")


if __name__ == "__main__":
    main()
