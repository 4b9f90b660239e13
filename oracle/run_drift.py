"""Run the FP64 oracle over a workload's full run and record what it conserves.

TEST INFRASTRUCTURE ONLY (calls nothing but the oracle and the seeded input
generators).  It writes a small JSON file with the oracle's own mass and
energy drift over the run (Sec. 3.1 reports energy conserved to about 1e-5)
and the final state at a fixed set of sampled grid points, which the GPU tests
compare with the library after the same number of steps:

    python -m oracle.run_drift solitary_1d stokes_2d --out tests/golden

Both sides start from the projected (dealiased, filtered) initial state of the
workload.  Sample points: 64 flat indices drawn by PCG32 (seed 4242) from the
member's grid, sorted.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import sbi_oracle as O  # noqa: E402


def sample_indices(n_points: int, count: int = 64, seed: int = 4242):
    u = W.PCG32(seed).uniform(count)
    return sorted(set(int(v * n_points) for v in u))


def problem_of(wl, m):
    grid = O.Grid(m.nx, m.ny, m.Lx, m.Ly if m.ny > 1 else 1.0)
    return O.Problem(grid, wl.gravity, m.h0, delta=m.delta, order=wl.order, alpha=wl.alpha,
                     sponge_w=wl.sponge_w, sponge_nu=wl.sponge_nu, filt_beta1=wl.filt_beta1,
                     filt_beta2=wl.filt_beta2, k_ref=wl.k_ref)


def run(name: str, steps: int | None = None, every: int = 100):
    wl = getattr(W, name)()
    m = wl.members[0]
    pb = problem_of(wl, m)
    steps = wl.steps if steps is None else steps
    eta, phi = O.project(pb, m.eta), O.project(pb, m.phi)
    m0, e0 = O.invariants(pb, eta, phi)
    series = [(0, m0, e0)]
    t0 = time.perf_counter()
    done = 0
    while done < steps:
        k = min(every, steps - done)
        eta, phi = O.step(pb, eta, phi, wl.dt, k)
        done += k
        mk, ek = O.invariants(pb, eta, phi)
        series.append((done, mk, ek))
        print(f"{name}: step {done}/{steps}  energy drift {(ek - e0) / e0:+.3e}", flush=True)
    wall = time.perf_counter() - t0
    idx = sample_indices(m.nx * m.ny)
    return {
        "workload": name, "steps": steps, "dt": wl.dt, "grid": [m.nx, m.ny],
        "source": "oracle/run_drift.py (FP64 oracle, classical RK4, projected initial state)",
        "mass0": m0, "energy0": e0,
        "mass_drift": (series[-1][1] - m0), "energy_drift_rel": (series[-1][2] - e0) / e0,
        "series": [{"step": s, "mass": a, "energy": b} for s, a, b in series],
        "sample_index": idx,
        "eta_samples": [float(v) for v in eta.ravel()[idx]],
        "phi_samples": [float(v) for v in phi.ravel()[idx]],
        "oracle_seconds": wall,
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("workloads", nargs="+")
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--out", default=None, help="folder for oracle_run_<workload>.json")
    a = ap.parse_args()
    for name in a.workloads:
        res = run(name, a.steps)
        text = json.dumps(res, indent=1)
        if a.out:
            with open(os.path.join(a.out, f"oracle_run_{name}.json"), "w") as f:
                f.write(text + "\n")
        else:
            print(text)


if __name__ == "__main__":
    main()
