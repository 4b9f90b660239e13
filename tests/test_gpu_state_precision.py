"""The RK4 state of the FP32 path: double-single float pairs (the default)
against FP64 (``state_fp64 = 1``), both fed with the same FP32 stage values.

The FP32 path evaluates every right-hand side in FP32 but keeps eta, phi~ and
the RK sums k1 + 2 k2 + 2 k3 + k4 in a wider format, either as double-single
pairs (about 48 significant bits, updated by error-free float
transformations) or in FP64.  These tests bound what the format itself adds,
separately from the FP32 error of the right-hand sides.

* Exact stage values: on a 256 x 256 member with constant eta = a and
  phi~ = b every stage of the dynamic condition is the single float
  s = fl(-g a) (V and every gradient vanish, and the transforms of a constant
  row or column are exact), so after n RK4 steps phi~ = b + n dt s and eta = a
  exactly.  The runs must reach that value to about 48 bits (double-single)
  and 53 bits (FP64), i.e. far below the FP32 rounding of one stage value,
  and eta must not move.
* A crossing-sea member (filter on), step by step over 1000 steps: both
  formats start every step from the same state (the FP64 run's, handed to the
  double-single context).  Their FP32 working copies are then the same
  floats, hence so are all stage values, and the states after the step differ
  by the format alone (about 1.5e-15 relative: the 48-bit representation plus
  the double-single update).  In a few steps one working copy lies so close
  to a float rounding boundary that the two formats round it apart; that one
  ulp then spreads through the FP32 transforms of the step, and the states
  differ at the FP32 right-hand side's own rounding level (about 1e-7).
  The test bounds the typical step at the format's level, the share of such
  steps, and every step at the right-hand side's level.
"""
from fractions import Fraction

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sbi():
    import __graft_entry__ as g
    g.build()
    from paper_2310_19840_gb300 import sbi as s
    return s


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.mark.parametrize("state_fp64,bar", [(0, 2e-11), (1, 5e-13)])
def test_constant_state_accumulates_exact_stage_values(sbi, state_fp64, bar):
    n, L, g, dt, steps = 256, 10.0, 9.81, 0.01, 1000
    a, b = 0.03, 0.4
    ctx = sbi.Context([(n, n, L, L)], g, None, h0=1.0, precision=sbi.SBI_FP32,
                      state_fp64=state_fp64, set_state_dealias=0)
    ctx.set_state(0, np.full((n, n), a), np.full((n, n), b))
    ctx.step(dt, steps)
    eta, phi = ctx.get_state(0)
    ctx.close()
    s = np.float32(-np.float32(g) * np.float32(a))          # the FP32 stage value
    exact = Fraction(b) + steps * Fraction(dt) * Fraction(float(s))
    err = np.max(np.abs(phi - float(exact))) / abs(float(exact - Fraction(b)))
    print(f"state_fp64={state_fp64}: phi~ error relative to the total increment {err:.2e}")
    assert err < bar
    # a float dt (the old update) would be off by |fl(dt) - dt| / dt
    assert err < 1e-3 * abs(float(np.float32(dt)) - dt) / dt
    # eta: its stage values are exact zeros, so it stays a (stored to 48 or 53 bits)
    assert np.max(np.abs(eta - a)) <= (2.0 ** -46 if state_fp64 == 0 else 0.0) * a


def test_double_single_state_tracks_fp64_state_step_by_step(sbi):
    wl = W.crossing_batch(n_small=1, n_large=0)
    m = wl.members[0]
    spec = [(m.nx, m.ny, m.Lx, m.Ly)]
    kw = dict(h0=m.h0, order=wl.order, alias_frac=wl.alpha, precision=sbi.SBI_FP32,
              filt_beta1=wl.filt_beta1, filt_beta2=wl.filt_beta2, k_ref=wl.k_ref,
              set_state_dealias=0)
    ds = sbi.Context(spec, wl.gravity, None, state_fp64=0, **kw)
    f64 = sbi.Context(spec, wl.gravity, None, state_fp64=1, **kw)
    f64.set_state(0, m.eta, m.phi)
    d = []
    for _ in range(1000):
        e0, p0 = f64.get_state(0)
        ds.set_state(0, e0, p0)
        f64.step(wl.dt, 1)
        ds.step(wl.dt, 1)
        e64, p64 = f64.get_state(0)
        eds, pds = ds.get_state(0)
        d.append(max(rel(eds, e64), rel(pds, p64)))
    ds.close()
    f64.close()
    d = np.array(d)
    same = d[d < 1e-12]
    print(f"double-single vs FP64 state per step: median {np.median(d):.2e}, same stage values in "
          f"{same.size} of 1000 steps (max {same.max():.2e}), worst step {d.max():.2e}")
    assert np.median(d) < 5e-15
    assert same.size >= 900 and same.max() < 1e-14
    assert d.max() < 5e-7
