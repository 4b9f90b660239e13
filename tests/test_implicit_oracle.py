"""Pins of the oracle's implicit form of Appendix A (flat bottom), reading R15:
its fixed point against the successive scheme of Sec. 2.4 and Appendix C, and
the behaviour of its iterations against steady Stokes waves."""
import math

import numpy as np
import pytest

from oracle import sbi_oracle as O
from oracle import steady_wave as sw

G = 9.81


def _band_limited(n, L, seed, modes=5):
    r = np.random.default_rng(seed)
    x = np.arange(n) * L / n
    f = np.zeros(n)
    for m in range(1, modes + 1):
        f += r.normal() * np.cos(2 * math.pi * m * x / L + r.uniform(0, 2 * math.pi)) / m
    return f / np.max(np.abs(f))


@pytest.mark.parametrize("h0", [math.inf, 1.0, 3.0])
def test_fixed_point_agrees_with_successive_scheme_to_eighth_order(h0):
    # Appendix A and Appendix C describe the same operator up to the order
    # kept: with no dealiasing (alpha = 1) and inputs band-limited so that no
    # product aliases, the fixed point and sum_{l<=7} V_l differ by O(eps^8)
    n, L = 128, 8 * math.pi
    grid = O.Grid(n, 1, L)
    kmax = 2 * math.pi * 5 / L
    e0, p0 = _band_limited(n, L, 1) / kmax, _band_limited(n, L, 2)
    d = {}
    for s in (0.2, 0.1):
        eta, phi = 0.5 * s * e0, s * p0
        Vi, _, _ = O.implicit_vertical_velocity(eta, phi, h0, grid, alpha=1.0, tol=1e-14,
                                                solver="gmres")
        Vs = O.vertical_velocity(eta, phi, None, h0, grid, alpha=1.0)
        d[s] = np.max(np.abs(Vi - Vs))
        assert d[s] < 1e-8 * np.max(np.abs(Vs))
    assert 180.0 < d[0.2] / d[0.1] < 330.0


def test_still_surface_is_linear_and_one_step():
    n, L = 64, 6.0
    grid = O.Grid(n, 1, L)
    phi = O.project(O.Problem(grid, G, 0.8), _band_limited(n, L, 3))
    V, it, inc = O.implicit_vertical_velocity(np.zeros(n), phi, 0.8, grid, tol=1e-15)
    Vl = O.vertical_velocity(np.zeros(n), phi, None, 0.8, grid, order=1)
    assert it == 1 and inc[0] == 0.0
    assert np.max(np.abs(V - Vl)) < 1e-14 * np.max(np.abs(Vl))


def _stokes(eps, depth=math.inf, n=64):
    L = 2 * math.pi
    w = sw.solve(k=1.0, H=2 * eps, depth=depth, g=G)
    x = np.arange(n) * L / n
    return O.Grid(n, 1, L), w.eta(x), w.surface_potential(x), w.vertical_velocity(x)


def test_iterations_against_steepness():
    # kH/2 = 0.1: both iterations converge and reach the successive scheme's
    # accuracy; the fixed-point map stops contracting above that, GMRES needs
    # more applications as the wave steepens (more than three at 0.35)
    grid, eta, phi, Vx = _stokes(0.1)
    sc = np.max(np.abs(Vx))
    Vf, nf, incf = O.implicit_vertical_velocity(eta, phi, math.inf, grid, tol=1e-9, maxit=20)
    Vg, ng, _ = O.implicit_vertical_velocity(eta, phi, math.inf, grid, tol=1e-9, solver="gmres")
    Vs = O.vertical_velocity(eta, phi, None, math.inf, grid)
    assert incf[-1] <= 1e-9 and nf <= 6
    assert np.max(np.abs(Vf - Vg)) < 1e-8 * sc
    assert np.max(np.abs(Vf - Vx)) < 2 * np.max(np.abs(Vs - Vx))
    apps = []
    for eps in (0.1, 0.2, 0.3, 0.35):
        grid, eta, phi, Vx = _stokes(eps)
        _, n_apps, hist = O.implicit_vertical_velocity(eta, phi, math.inf, grid, tol=1e-6,
                                                       solver="gmres")
        assert hist[-1] <= 1e-6
        apps.append(n_apps)
        if eps >= 0.2:
            _, _, inc = O.implicit_vertical_velocity(eta, phi, math.inf, grid, tol=0.0, maxit=8)
            assert inc[-1] > 1e-2           # the fixed-point iteration diverges
    assert apps == sorted(apps) and apps[-1] > 3


def test_steep_fixed_point_is_less_accurate_than_successive_scheme():
    grid, eta, phi, Vx = _stokes(0.35)
    sc = np.max(np.abs(Vx))
    Vg, _, _ = O.implicit_vertical_velocity(eta, phi, math.inf, grid, tol=1e-10, solver="gmres")
    Vs = O.vertical_velocity(eta, phi, None, math.inf, grid)
    assert np.max(np.abs(Vs - Vx)) / sc < 5e-3 < np.max(np.abs(Vg - Vx)) / sc


@pytest.mark.parametrize("h0", [1.0, 2.0])
def test_variable_bottom_fixed_point_agrees_with_successive_scheme(h0):
    # Appendices A and B together (R17): with no dealiasing and inputs whose
    # products do not alias, the fixed point and the successive scheme of
    # Appendix C differ by O(eps^8) when eta, phi~ and delta are scaled together
    n, L = 128, 8 * math.pi
    grid = O.Grid(n, 1, L)
    kmax = 2 * math.pi * 5 / L
    e0, p0, d0 = _band_limited(n, L, 1) / kmax, _band_limited(n, L, 2), 0.5 * h0 * _band_limited(n, L, 3)
    d = {}
    for s in (0.2, 0.1):
        eta, phi, delta = 0.5 * s * e0, s * p0, s * d0
        Vi, _, _ = O.implicit_vertical_velocity(eta, phi, h0, grid, alpha=1.0, tol=1e-14,
                                                solver="gmres", delta=delta)
        Vs = O.vertical_velocity(eta, phi, delta, h0, grid, alpha=1.0)
        d[s] = np.max(np.abs(Vi - Vs))
        assert d[s] < 1e-6 * np.max(np.abs(Vs))
    assert 180.0 < d[0.2] / d[0.1] < 330.0


def test_printed_varphi5_equals_the_pattern_form():
    # R17: the printed varphi~^(5) terms and the pattern of the other orders
    # are the same operator (their difference is a vanishing nested commutator)
    n, L, h0 = 128, 8 * math.pi, 1.0
    grid = O.Grid(n, 1, L)
    kmax = 2 * math.pi * 5 / L
    eta, phi = 0.1 * _band_limited(n, L, 4) / kmax, 0.2 * _band_limited(n, L, 5)
    delta = 0.1 * h0 * _band_limited(n, L, 6)
    Va, _, _ = O.implicit_vertical_velocity(eta, phi, h0, grid, alpha=1.0, tol=1e-14, solver="gmres",
                                            delta=delta, b5="printed")
    Vb, _, _ = O.implicit_vertical_velocity(eta, phi, h0, grid, alpha=1.0, tol=1e-14, solver="gmres",
                                            delta=delta, b5="pattern")
    assert np.max(np.abs(Va - Vb)) < 1e-13 * np.max(np.abs(Va))
    # and a zero bottom variation is the flat form
    Vf, _, _ = O.implicit_vertical_velocity(eta, phi, h0, grid, alpha=1.0, tol=1e-14, solver="gmres")
    V0, _, _ = O.implicit_vertical_velocity(eta, phi, h0, grid, alpha=1.0, tol=1e-14, solver="gmres",
                                            delta=np.zeros(n))
    assert np.array_equal(Vf, V0)


def test_variable_bottom_iterations_and_accuracy():
    # A wave over a bump (delta up to 0.3 h0, k h0 = 1): GMRES solves the
    # implicit form of Appendices A and B in a few applications; against the
    # independent Laplace solution the successive scheme is the more accurate
    from laplace_dtn import exact_vertical_velocity
    n, L, h0, g = 64, 4 * math.pi, 1.0, 9.81
    grid = O.Grid(n, 1, L)
    x = np.arange(n) * L / n
    delta = 0.3 * h0 * np.exp(-((x - L / 2) / 1.5) ** 2)
    pb = O.Problem(grid, g, h0, delta=delta)
    k = 4 * math.pi / L
    om = math.sqrt(g * k * math.tanh(k * h0))
    for eps in (0.05, 0.1, 0.2):
        a = eps / k
        eta = O.project(pb, a * np.cos(k * x))
        phi = O.project(pb, a * g / om * np.sin(k * x))
        Vx = exact_vertical_velocity(eta, phi, delta, h0, L, n_sigma=32)
        sc = np.max(np.abs(Vx))
        Vs = np.ravel(O.vertical_velocity(eta, phi, delta, h0, grid))
        Vg, apps, hist = O.implicit_vertical_velocity(eta, phi, h0, grid, tol=1e-6, solver="gmres",
                                                      delta=delta)
        ei, es = np.max(np.abs(np.ravel(Vg) - Vx)) / sc, np.max(np.abs(Vs - Vx)) / sc
        print(f"kH/2 = {eps}: GMRES {apps} applications, implicit {ei:.2e}, successive {es:.2e}")
        assert hist[-1] <= 1e-6 and 3 < apps <= 12
        assert es < ei < 1e-4
