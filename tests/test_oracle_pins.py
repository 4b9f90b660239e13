"""Pins of the FP64 oracle against results fixed by the paper and by mathematics
(no GPU).  Each test names the property and the passage it comes from.

Plausible mistakes and the pin that catches them:
* a wrong coefficient, sign, power of k, tanh/sech factor or (-1)^j in any
  order of V_l or varphi_l  -> constant-(eta, delta) Taylor pin (per order).
* a misplaced product (F{eta^j} F{V} instead of F{eta^j V}), a gradient on the
  wrong factor, a transposed kx/ky  -> Laplace-solver convergence pin (1-D) and
  the oblique 2-D embedding pin.
* a wrong term in the dynamic condition  -> Bernoulli pin.
* a wrong RK4 weight  -> linear amplification-factor pin.
"""
import math

import numpy as np
import pytest

from oracle import sbi_oracle as O
from laplace_dtn import exact_vertical_velocity
import workloads as W


def _dft2(f):
    ny, nx = f.shape
    m = np.arange(nx)
    n = np.arange(ny)
    Ex = np.exp(-2j * np.pi * np.outer(m, m) / nx)
    Ey = np.exp(-2j * np.pi * np.outer(n, n) / ny)
    return Ey @ f @ Ex.T


def test_fft_matches_brute_force_dft():
    rng = np.random.default_rng(1)
    for shape in ((8, 16), (1, 32), (4, 8)):
        f = rng.standard_normal(shape)
        F = O.fft(f)
        D = _dft2(f)
        assert np.max(np.abs(F - D)) <= 1e-13 * np.max(np.abs(D)) * shape[0] * shape[1]
        assert np.max(np.abs(O.ifft(F) - f)) < 1e-14


def test_dealias_mask_reading():
    # Reading R5: strict |m| < alpha n/2.  64 points keep m = 0..15 (16 modes on
    # each side), as in the paper's "first 16 Fourier modes" of 64 points.
    g = O.Grid(64, 1, 1.0)
    mk = O.dealias_mask(g, 0.5)[0]
    kept = np.nonzero(mk)[0]
    m = np.fft.fftfreq(64, d=1.0 / 64)[kept]
    assert set(np.abs(m).astype(int)) == set(range(16))
    # alpha = 1 removes only the Nyquist mode
    assert O.dealias_mask(g, 1.0).sum() == 63
    g2 = O.Grid(16, 8, 1.0, 1.0)
    assert O.dealias_mask(g2, 0.5).sum() == 7 * 3


@pytest.mark.parametrize("dim", [1, 2])
@pytest.mark.parametrize("h0", [0.3, 1.0, np.inf])
def test_linear_operator_closed_form(dim, h0):
    # eta = 0, delta = 0: V = F^{-1}{k tanh(kh) F{phi~}} (Sec. 2.4, order 1).
    nx, ny = 32, (1 if dim == 1 else 16)
    g = O.Grid(nx, ny, 5.0, 3.0 if dim == 2 else 1.0)
    phi = W.random_field(nx, ny, seed=3, band=0.5)
    V = O.vertical_velocity(np.zeros((ny, nx)), phi, None, h0, g)
    KX, KY, K = O.wavenumbers(g)
    mult = K * (np.tanh(K * h0) if np.isfinite(h0) else 1.0)
    ref = np.real(np.fft.ifft2(mult * np.fft.fft2(phi)))
    assert np.max(np.abs(V - ref)) < 1e-13 * np.max(np.abs(ref))


def _taylor_tables(max_deg=6):
    """Homogeneous parts (degree d in (a, b)) of k tanh(k(h+a-b)) and
    sech(k(h+a-b)), as sympy lambdas of (a, b, k, h)."""
    sp = pytest.importorskip("sympy")
    a, b, k, h, s = sp.symbols("a b k h s")
    V = sp.series(k * sp.tanh(k * (h + s * (a - b))), s, 0, max_deg + 1).removeO()
    B = sp.series(sp.sech(k * (h + s * (a - b))), s, 0, max_deg + 1).removeO()
    vfun = [sp.lambdify((a, b, k, h), sp.simplify(V.coeff(s, d))) for d in range(max_deg + 1)]
    bfun = [sp.lambdify((a, b, k, h), sp.simplify(B.coeff(s, d))) for d in range(max_deg + 1)]
    return vfun, bfun


@pytest.mark.parametrize("dim", [1, 2])
def test_constant_elevation_and_depth_match_taylor_per_order(dim):
    # With constant eta = a and delta = b a single Fourier mode of phi~ has the
    # exact V = k tanh(k(h0+a-b)) phi^ and bottom potential sech(k(h0+a-b)) phi^
    # (the constant-delta idea of the applicability section).  V_l of the
    # successive scheme is O(eps^m zeta^{l-m}), so it must equal the Taylor part of
    # total degree l-1 in (a, b); varphi_l likewise for sech.
    vfun, bfun = _taylor_tables()
    if dim == 1:
        g = O.Grid(32, 1, 2 * np.pi)
        modes = [(1, 0), (3, 0), (6, 0)]
    else:
        g = O.Grid(32, 16, 2 * np.pi, 2 * np.pi)
        modes = [(1, 1), (3, 2), (2, 5)]
    x = np.arange(g.nx) * g.Lx / g.nx
    y = np.arange(g.ny) * g.Ly / g.ny
    X, Y = np.meshgrid(x, y)
    for (a, b, h0) in [(0.05, 0.0, 1.0), (0.03, 0.04, 0.7), (-0.02, 0.05, 1.3), (0.04, -0.03, 0.5)]:
        for (mx, my) in modes:
            kx, ky = 2 * np.pi * mx / g.Lx, 2 * np.pi * my / g.Ly
            kk = math.hypot(kx, ky)
            carrier = np.cos(kx * X + ky * Y)
            eta = np.full((g.ny, g.nx), a)
            delta = np.full((g.ny, g.nx), b) if b != 0 else None
            _, terms = O.vertical_velocity(eta, carrier, delta, h0, g, alpha=1.0,
                                           return_terms=True)
            for l, Vl in enumerate(terms["V"], start=1):
                amp = np.sum(Vl * carrier) / np.sum(carrier * carrier)
                ref = vfun[l - 1](a, b, kk, h0)
                assert abs(amp - ref) < 1e-12 * max(1.0, kk), (l, a, b, mx, my)
                assert np.max(np.abs(Vl - amp * carrier)) < 1e-12 * max(1.0, kk)
            if delta is not None:
                for l, Bl in enumerate(terms["varphi"], start=1):
                    amp = np.sum(Bl * carrier) / np.sum(carrier * carrier)
                    ref = bfun[l - 1](a, b, kk, h0)
                    assert abs(amp - ref) < 1e-12, (l, a, b, mx, my)


@pytest.mark.parametrize("order,ratio", [(3, 8.0), (5, 32.0), (7, 128.0)])
@pytest.mark.parametrize("variable", [False, True])
def test_truncation_error_scaling_vs_laplace_solver(order, ratio, variable):
    # Sec. 2.4: the omitted terms are O(eps^m zeta^{M+1-m}).  Scaling eta and delta
    # by s at fixed phi~, the error of the order-M sum against the exact
    # Dirichlet-Neumann operator (independent Laplace solve) falls as s^M.
    L, nx, h0 = 2 * np.pi, 64, 1.0
    x = np.arange(nx) * L / nx
    eta0 = 0.3 * np.cos(x) + 0.2 * np.sin(2 * x + 0.4)
    del0 = 0.25 * np.cos(x + 0.5) + 0.15 * np.sin(3 * x)
    phi = np.cos(x) + 0.5 * np.sin(2 * x + 0.3)
    g = O.Grid(nx, 1, L)
    errs = []
    for s in (0.4, 0.2, 0.1):
        d = s * del0 if variable else None
        Ve = exact_vertical_velocity(s * eta0, phi, d, h0, L, n_sigma=32)
        Vo = O.vertical_velocity(s * eta0, phi, d, h0, g, order=order, alpha=1.0)
        errs.append(np.linalg.norm(Vo - Ve) / np.linalg.norm(Ve))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 0.7 * ratio < r2 < 1.4 * ratio, errs
    assert 0.6 * ratio < r1 < 1.5 * ratio, errs
    if order == 7:
        assert errs[0] < 1e-5


def test_oblique_2d_matches_1d():
    # A 2-D field varying only along the grid direction (2, 1) must give the 1-D
    # result with the same wavenumbers (checks ik. on both components).
    n, L, h0 = 32, 2 * np.pi, 0.8
    # x carries harmonic p at index 2p: 64 points keep degree-7 products unaliased
    g2 = O.Grid(2 * n, n, L, L)
    L1 = L / math.sqrt(5.0)
    g1 = O.Grid(n, 1, L1)
    s1 = np.arange(n) * L1 / n

    def f1(c):  # 1-D functions of the coordinate along the direction
        return c[0] * np.cos(2 * np.pi * s1 / L1) + c[1] * np.sin(4 * np.pi * s1 / L1 + 0.3)

    x = np.arange(2 * n) * L / (2 * n)
    y = np.arange(n) * L / n
    X, Y = np.meshgrid(x, y)
    arg = 2 * np.pi * (2 * X + Y) / L      # phase of mode (2,1)

    def f2(c):
        return c[0] * np.cos(arg) + c[1] * np.sin(2 * arg + 0.3)

    ce, cd, cp = (0.12, 0.05), (0.1, -0.06), (1.0, 0.4)
    V1 = O.vertical_velocity(f1(ce)[None, :], f1(cp)[None, :], f1(cd)[None, :], h0, g1, alpha=1.0)
    V2 = O.vertical_velocity(f2(ce), f2(cp), f2(cd), h0, g2, alpha=1.0)
    # compare Fourier coefficients of harmonics p = 1..6 along the direction
    F1 = np.fft.fft(V1[0]) / n
    F2 = np.fft.fft2(V2) / (2 * n * n)
    for p in range(1, 7):
        assert abs(F1[p] - F2[p % n, (2 * p) % (2 * n)]) < 1e-12 * np.max(np.abs(F1)), p


def test_dynamic_condition_matches_bernoulli():
    # phi~_t of Eq. (prognostic) equals -g eta - |u|^2/2 - w^2/2 + w V (Bernoulli at
    # the surface plus the chain rule), with u, w taken from the Laplace solution.
    L, nx, h0, grav = 2 * np.pi, 64, 1.0, 9.81
    x = np.arange(nx) * L / nx
    eta = 0.06 * np.cos(x) + 0.03 * np.sin(2 * x + 0.4)
    phi = np.cos(x) + 0.5 * np.sin(2 * x + 0.3)
    delta = 0.1 * np.cos(x + 0.5)
    Ve, u, w = exact_vertical_velocity(eta, phi, delta, h0, L, return_phi_grad=True)
    g = O.Grid(nx, 1, L)
    got = O.dynamic_rhs(eta[None, :], phi[None, :], Ve[None, :], grav, g, alpha=1.0)[0]
    ref = -grav * eta - 0.5 * (u * u + w * w) + w * Ve
    assert np.max(np.abs(got - ref)) < 1e-9 * np.max(np.abs(ref))


def test_rk4_linear_amplification_factor():
    # For an infinitesimal single mode the system is linear,
    # d/dt (eta^, phi^) = A (eta^, phi^), A = [[0, k t], [-g, 0]], and one classical
    # RK4 step multiplies by I + Ad + (Ad)^2/2 + (Ad)^3/6 + (Ad)^4/24 exactly.
    nx, L, h0, grav, dt = 32, 10.0, 0.7, 9.81, 0.05
    g = O.Grid(nx, 1, L)
    pb = O.Problem(g, grav, h0)
    x = np.arange(nx) * L / nx
    m = 3
    k = 2 * np.pi * m / L
    a = 1e-9
    eta = a * np.cos(k * x)
    phi = 0.3 * a * np.sin(k * x)
    e1, p1 = O.step(pb, eta, phi, dt, 1)
    A = np.array([[0.0, k * math.tanh(k * h0)], [-grav, 0.0]]) * dt
    R = np.eye(2) + A + A @ A / 2 + A @ A @ A / 6 + A @ A @ A @ A / 24
    ce, se = 1.0, 0.0     # eta = ce cos + se sin (in units of a)
    cp, sp_ = 0.0, 0.3
    new_c = R @ np.array([ce, cp])
    new_s = R @ np.array([se, sp_])
    ref_eta = a * (new_c[0] * np.cos(k * x) + new_s[0] * np.sin(k * x))
    ref_phi = a * (new_c[1] * np.cos(k * x) + new_s[1] * np.sin(k * x))
    assert np.max(np.abs(e1[0] - ref_eta)) < 1e-6 * a
    assert np.max(np.abs(p1[0] - ref_phi)) < 1e-6 * a


def test_linear_dispersion_relation():
    # omega^2 = g k tanh(k h) at small amplitude: a standing-free progressive mode
    # returns to its phase after one period up to O((omega dt)^4).
    nx, L, h0, grav = 32, 8.0, 0.5, 9.81
    g = O.Grid(nx, 1, L)
    pb = O.Problem(g, grav, h0)
    m = 2
    k = 2 * np.pi * m / L
    om = math.sqrt(grav * k * math.tanh(k * h0))
    T = 2 * np.pi / om
    nsteps = 200
    dt = T / nsteps
    x = np.arange(nx) * L / nx
    a = 1e-6
    eta = a * np.cos(k * x)
    phi = (grav * a / om) * np.sin(k * x)
    e, p = O.step(pb, eta, phi, dt, nsteps)
    assert np.max(np.abs(e[0] - eta)) < 1e-6 * a * 10


def test_mass_conserved_exactly():
    # R4: F{V_l}(0) = 0, so int eta dA is constant to round-off.
    g = O.Grid(16, 8, 3.0, 2.0)
    pb = O.Problem(g, 9.81, 0.5, delta=W.random_field(16, 8, 11, amplitude=0.05))
    eta = W.random_field(16, 8, 12, amplitude=0.03) + 0.01
    phi = W.random_field(16, 8, 13, amplitude=0.1)
    m0, _ = O.invariants(pb, eta, phi)
    e, p = O.step(pb, eta, phi, 0.01, 5)
    m1, _ = O.invariants(pb, e, p)
    assert abs(m1 - m0) < 1e-14 * np.sum(np.abs(eta)) * g.dA * 10


def test_sponge_constant_weight_closed_form():
    # R7: with a constant weight w the damping pressure reduces to nu w phi~.
    g = O.Grid(32, 1, 4.0)
    phi = W.random_field(32, 1, 5)
    pd = O.damping_pressure(phi, np.full((1, 32), 0.7), 2.0, g)
    assert np.max(np.abs(pd - 1.4 * phi)) < 1e-13


@pytest.mark.slow
def test_solitary_wave_energy_and_speed():
    # Sec. 3.1: the total energy of a solitary wave stays constant (the paper
    # reports |E-E0|/E0 ~ 1e-5); the crest moves at about sqrt(g (h + a)).
    wl = W.solitary_1d()
    m = wl.members[0]
    g = O.Grid(m.nx, 1, m.Lx)
    pb = O.Problem(g, wl.gravity, m.h0)
    eta = O.project(pb, m.eta)
    phi = O.project(pb, m.phi)
    _, E0 = O.invariants(pb, eta, phi)
    nsteps = 400
    e, p = O.step(pb, eta, phi, wl.dt, nsteps)
    _, E1 = O.invariants(pb, e, p)
    assert abs(E1 - E0) / E0 < 1e-4
    # crest position by a parabolic fit around the maximum
    def crest(f):
        f = f[0]
        i = int(np.argmax(f))
        fm, f0, fp = f[i - 1], f[i], f[(i + 1) % f.size]
        off = 0.5 * (fm - fp) / (fm - 2 * f0 + fp)
        return (i + off) * m.Lx / m.nx
    speed = (crest(e) - crest(eta)) / (nsteps * wl.dt)
    c = wl.notes["c"]
    assert abs(speed - c) / c < 0.03


def test_translating_stokes_wave():
    # A wave of permanent form eta(x - c t) has V = eta_t = -c eta_x exactly.  The
    # third-order Stokes initial condition leaves an absolute residual O(eps^4)
    # (relative O(eps^3)); by the parity of the Stokes expansion the first and
    # third harmonics of the residual are O(eps^5).
    res, h1, h3 = [], [], []
    for eps in (0.1, 0.05):
        eta, phi, c, k = W.stokes_1d(64, 2 * np.pi, 1, 1.0, eps)
        g = O.Grid(64, 1, 2 * np.pi)
        V = O.vertical_velocity(eta[None, :], phi[None, :], None, 1.0, g, alpha=1.0)[0]
        kx = 2 * np.pi * np.fft.fftfreq(64, d=2 * np.pi / 64)
        eta_x = np.real(np.fft.ifft(1j * kx * np.fft.fft(eta)))
        r = V + c * eta_x
        res.append(np.linalg.norm(r) / np.linalg.norm(V))
        F = np.abs(np.fft.fft(r))
        h1.append(F[1])
        h3.append(F[3])
    assert res[0] / res[1] > 6.5, res
    assert h1[0] / h1[1] > 20.0 and h3[0] / h3[1] > 20.0, (h1, h3)


def test_adaptive_order_stops_at_first_small_taylor_increment():
    # R9 (Sec. 2.4: the series is truncated once further orders stop changing
    # V).  With constant eta = a over a flat bottom, a single mode of phi~ has
    # order-l increments equal to the degree-(l-1) Taylor coefficients of
    # k tanh(k(h+a)) (sympy), so the order at which the test first holds and
    # the truncated sum are known independently of the oracle's recursion.
    vfun, _ = _taylor_tables()
    g = O.Grid(32, 1, 2 * np.pi)
    a, h0, mode = 0.06, 0.8, 3
    kk = 2 * np.pi * mode / g.Lx
    c = [vfun[d](a, 0.0, kk, h0) for d in range(7)]          # increments V_1..V_7
    part = np.cumsum(c)
    ratio = [abs(c[l]) / abs(part[l]) for l in range(7)]
    for L in (3, 4, 5):
        tol = math.sqrt(ratio[L - 1] * ratio[L - 2])          # between orders L-1 and L
        assert all(ratio[l] > tol for l in range(1, L - 1)) and ratio[L - 1] <= tol
        x = np.arange(g.nx) * g.Lx / g.nx
        carrier = np.cos(kk * x)[None, :]
        V, terms = O.vertical_velocity(np.full((1, g.nx), a), carrier, None, h0, g, alpha=1.0,
                                       tol=tol, return_terms=True)
        assert terms["used"] == L
        amp = np.sum(V * carrier) / np.sum(carrier * carrier)
        assert abs(amp - part[L - 1]) < 1e-12 * kk
    # tol = 0 keeps every order
    _, terms = O.vertical_velocity(np.full((1, g.nx), a), np.cos(kk * np.arange(g.nx) * g.Lx / g.nx)[None, :],
                                   None, h0, g, alpha=1.0, return_terms=True)
    assert terms["used"] == 7


def test_low_pass_filter_special_values():
    # R8 (Eq. filter): Lambda = exp(-|k/(beta1 k_ref)|^beta2) is 1/e at the
    # cut-off k = beta1 k_ref for every beta2, about 1 well below it and about 0
    # well above it for a steep beta2 (the paper's 30).
    g = O.Grid(128, 1, 2 * np.pi)
    x = np.arange(g.nx) * g.Lx / g.nx
    k_ref, b1, b2 = 2.0, 8.0, 30.0                  # cut-off at wavenumber 16
    pb = O.Problem(g, 9.81, 1.0, alpha=1.0, filt_beta1=b1, filt_beta2=b2, k_ref=k_ref)
    modes = {4: 1.0, 8: 1.0, 16: math.exp(-1.0), 24: 0.0, 40: 0.0}
    f = sum(np.cos(m * x) for m in modes)[None, :]
    out = O.project(pb, f)
    for m, lam in modes.items():
        amp = 2.0 * np.mean(out[0] * np.cos(m * x))
        assert abs(amp - lam) < 1e-8, (m, amp, lam)
    pb2 = O.Problem(g, 9.81, 1.0, alpha=1.0, filt_beta1=b1, filt_beta2=4.0, k_ref=k_ref)
    out2 = O.project(pb2, np.cos(16 * x)[None, :])
    assert abs(2.0 * np.mean(out2[0] * np.cos(16 * x)) - math.exp(-1.0)) < 1e-12


@pytest.mark.parametrize("h0,T,L,xs", [(0.5, 1.2, 60.0, (10.0, 50.0)), (0.5, 3.0, 120.0, (20.0, 100.0))])
def test_wavemaker_radiates_waves_of_amplitude_a(h0, T, L, xs):
    # R10: with the pressure of the submerged-bar section (scaled by g), linear
    # theory gives a radiated wave of amplitude a_j on each side: the Fourier
    # transform of the bell at k_j cancels sqrt(e/2pi) and the shoaling factor
    # [1 + 2kh/sinh 2kh] cancels the group velocity.  A small-amplitude run
    # (order 1) with the paper's Gaussian damping zone (centred at L/2, width
    # 4 pi / k) is fitted at two gauges after the front has passed.  Cases
    # kh = 1.53 (factor 1.29) and kh = 0.5 (factor 1.85).
    g, nx, a = 9.81, 512, 1e-4
    w = 2 * math.pi / T
    k = O.dispersion_wavenumber(w, h0, g)
    grid = O.Grid(nx, 1, L)
    x = np.arange(nx) * L / nx
    damp = np.exp(-(k * (x - L / 2) / (4 * math.pi)) ** 2)[None, :]
    wm = O.Wavemaker(np.array([a]), np.array([w]), np.array([0.0]), 0.0)
    pb = O.Problem(grid, g, h0, order=1, sponge_w=damp, sponge_nu=w, wavemaker=wm)
    dt = T / 40
    idx = [int(round(xi / (L / nx))) for xi in xs]
    eta, phi = np.zeros((1, nx)), np.zeros((1, nx))
    t_end = 10.0 * T if T > 2 else 20.0 * T
    n = int(round(t_end / dt))
    rec = []
    for i in range(n):
        eta, phi = O.step(pb, eta, phi, dt, 1, t0=i * dt)
        rec.append(eta[0, idx])
    rec = np.array(rec)
    t = (np.arange(n) + 1) * dt
    sel = t >= t_end - 4 * T
    basis = np.stack([np.cos(w * t[sel]), np.sin(w * t[sel]), np.ones(sel.sum())], 1)
    for c in range(len(idx)):
        coef, *_ = np.linalg.lstsq(basis, rec[sel, c], rcond=None)
        amp = math.hypot(coef[0], coef[1])
        assert abs(amp / a - 1.0) < 0.02, (h0, T, xs[c], amp / a)


def test_wavemaker_pressure_shape():
    # R10: the bell is centred at x0 on the periodic box, symmetric, of
    # e-folding half-width sqrt(2)/k, and proportional to sin(omega t + theta).
    g, h0 = 9.81, 0.4
    grid = O.Grid(256, 1, 20.0)
    wm = O.Wavemaker(np.array([0.01]), np.array([4.0]), np.array([0.3]), 5.0)
    k = O.dispersion_wavenumber(4.0, h0, g)
    t = 0.7
    p = O.wavemaker_pressure(wm, grid, h0, g, t)[0]
    x = np.arange(256) * 20.0 / 256
    i0 = int(round(5.0 / (20.0 / 256)))
    peak = g * 0.01 * math.sqrt(math.e / (2 * math.pi)) * (1 + 2 * k * h0 / math.sinh(2 * k * h0)) * math.sin(4.0 * t + 0.3)
    assert abs(p[i0] - peak) < 1e-12 * abs(peak)
    for m in (1, 5, 17):
        assert abs(p[i0 + m] - p[i0 - m]) < 1e-14
        d = m * 20.0 / 256
        assert abs(p[i0 + m] - peak * math.exp(-0.5 * (k * d) ** 2)) < 1e-12
    # periodic: the bell wraps around the ends
    wm2 = O.Wavemaker(np.array([0.01]), np.array([4.0]), np.array([0.3]), 0.0)
    p2 = O.wavemaker_pressure(wm2, grid, h0, g, t)[0]
    assert abs(p2[1] - p2[-1]) < 1e-14
    # deep water: the shoaling factor is 1
    p3 = O.wavemaker_pressure(wm, grid, math.inf, g, t)[0]
    k3 = 16.0 / g
    assert abs(p3[i0] - g * 0.01 * math.sqrt(math.e / (2 * math.pi)) * math.sin(4.0 * t + 0.3)) < 1e-12
    assert abs(p3[i0 + 3] / p3[i0] - math.exp(-0.5 * (k3 * 3 * 20.0 / 256) ** 2)) < 1e-12


@pytest.mark.parametrize("h0", [0.4, math.inf])
def test_lawson_step_is_exact_for_linear_waves(h0):
    # R11: the integrating factor carries the linear part exactly, so for an
    # infinitesimal travelling wave one step of any length gives
    # eta = a cos(kx - w dt), phi~ = (g a / w) sin(kx - w dt) with
    # w^2 = g k tanh(k h0), here at w dt = 2.5 where classical RK4 is unstable.
    g, a, nx, L, m = 9.81, 1e-8, 64, 4.0, 3
    grid = O.Grid(nx, 1, L)
    k = 2 * math.pi * m / L
    w = math.sqrt(g * k * (math.tanh(k * h0) if math.isfinite(h0) else 1.0))
    x = np.arange(nx) * L / nx
    eta = a * np.cos(k * x)[None, :]
    phi = (g * a / w) * np.sin(k * x)[None, :]
    dt = 2.5 / w
    pb = O.Problem(grid, g, h0, order=1, integrator="lawson")
    e, p = O.step(pb, eta, phi, dt, 1)
    assert np.max(np.abs(e[0] - a * np.cos(k * x - w * dt))) < 1e-6 * a
    assert np.max(np.abs(p[0] - (g * a / w) * np.sin(k * x - w * dt))) < 1e-6 * g * a / w
    pb_rk = O.Problem(grid, g, h0, order=1)
    e_rk, _ = O.step(pb_rk, eta, phi, dt, 1)
    assert np.max(np.abs(e_rk[0] - a * np.cos(k * x - w * dt))) > 0.1 * a


def test_lawson_is_fourth_order_and_agrees_with_rk4():
    # R11: on a nonlinear variable-depth problem the Lawson scheme converges
    # at fourth order (a wrong stage weight or propagator would lower it) to
    # the solution of classical RK4 at a tiny step.
    nx, ny, Lx, Ly, h0 = 32, 16, 6.0, 3.0, 0.7
    grid = O.Grid(nx, ny, Lx, Ly)
    delta = W.random_field(nx, ny, 111, amplitude=0.05, band=0.3)
    pb = O.Problem(grid, 9.81, h0, delta=delta, order=4, integrator="lawson")
    eta = O.project(pb, W.random_field(nx, ny, 112, amplitude=0.04, band=0.3))
    phi = O.project(pb, W.random_field(nx, ny, 113, amplitude=0.1, band=0.3))
    T_end = 0.4
    ref_pb = O.Problem(grid, 9.81, h0, delta=delta, order=4)
    e_ref, p_ref = O.step(ref_pb, eta, phi, T_end / 128, 128)
    errs = []
    for n in (4, 8, 16):
        e, p = O.step(pb, eta, phi, T_end / n, n)
        errs.append(np.linalg.norm(e - e_ref) + np.linalg.norm(p - p_ref))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 12.0 < r1 < 20.0 and 12.0 < r2 < 20.0, (errs, r1, r2)


@pytest.mark.parametrize("order", [1, 3, 5, 7])
def test_hos_constant_elevation_matches_taylor(order):
    # R12: with a constant elevation a over a flat bottom the HOS sum of order
    # M keeps exactly the terms of degree <= M-1 in a of the exact
    # W = V = k tanh(k(h + a)) (sympy), mode by mode.
    vfun, _ = _taylor_tables()
    g = O.Grid(32, 16, 2 * np.pi, 2 * np.pi)
    x = np.arange(g.nx) * g.Lx / g.nx
    y = np.arange(g.ny) * g.Ly / g.ny
    X, Y = np.meshgrid(x, y)
    for (a, h0) in [(0.05, 1.0), (-0.03, 0.6)]:
        for (mx, my) in [(1, 1), (3, 2)]:
            kk = math.hypot(mx, my)
            carrier = np.cos(mx * X + my * Y)
            V, Wz = O.hos_surface_velocity(np.full((g.ny, g.nx), a), carrier, h0, g, order=order,
                                           alpha=1.0)
            ref = sum(vfun[d](a, 0.0, kk, h0) for d in range(order))
            for f in (V, Wz):
                amp = np.sum(f * carrier) / np.sum(carrier * carrier)
                assert abs(amp - ref) < 1e-12 * kk, (order, a, mx, my, amp, ref)
                assert np.max(np.abs(f - amp * carrier)) < 1e-12 * kk


@pytest.mark.parametrize("order,ratio", [(3, 8.0), (5, 32.0), (7, 128.0)])
def test_hos_truncation_error_scaling_vs_laplace_solver(order, ratio):
    # R12: scaling eta by s at fixed phi~, the HOS error against the exact
    # Dirichlet-Neumann operator (independent Laplace solve) falls as s^M;
    # both V and the Eulerian W = (V + eta_x phi_x) / (1 + eta_x^2).
    L, nx, h0 = 2 * np.pi, 64, 1.0
    x = np.arange(nx) * L / nx
    eta0 = 0.3 * np.cos(x) + 0.2 * np.sin(2 * x + 0.4)
    phi = np.cos(x) + 0.5 * np.sin(2 * x + 0.3)
    phi_x = -np.sin(x) + np.cos(2 * x + 0.3)
    g = O.Grid(nx, 1, L)
    errs, errw = [], []
    for s in (0.4, 0.2, 0.1):
        eta = s * eta0
        eta_x = s * (-0.3 * np.sin(x) + 0.4 * np.cos(2 * x + 0.4))
        Ve = exact_vertical_velocity(eta, phi, None, h0, L, n_sigma=32)
        We = (Ve + eta_x * phi_x) / (1 + eta_x ** 2)
        Vh, Wh = O.hos_surface_velocity(eta, phi, h0, g, order=order, alpha=1.0)
        errs.append(np.linalg.norm(Vh[0] - Ve) / np.linalg.norm(Ve))
        errw.append(np.linalg.norm(Wh[0] - We) / np.linalg.norm(We))
    for e in (errs, errw):
        r1, r2 = e[0] / e[1], e[1] / e[2]
        assert 0.6 * ratio < r1 < 1.5 * ratio and 0.7 * ratio < r2 < 1.4 * ratio, e


def test_rk45_tableau_conditions():
    # R13: Cash-Karp 5(4) pair, the consistency conditions of an explicit RK
    # pair: rows of A sum to the nodes, both weight vectors sum to 1, and the
    # order conditions sum b c = 1/2, sum b c^2 = 1/3, sum b c^3 = 1/4 hold for
    # both (order 4 and 5), sum b c^4 = 1/5 for the order-5 weights only.
    c, A, b5, b4 = O.CK_C, O.CK_A, O.CK_B5, O.CK_B4
    for i in range(6):
        assert abs(sum(A[i]) - c[i]) < 1e-15
    for b in (b5, b4):
        assert abs(sum(b) - 1.0) < 1e-15
        for q, val in ((1, 0.5), (2, 1 / 3), (3, 0.25)):
            assert abs(sum(bi * ci ** q for bi, ci in zip(b, c)) - val) < 1e-14
    assert abs(sum(bi * ci ** 4 for bi, ci in zip(b5, c)) - 0.2) < 1e-14
    assert abs(sum(bi * ci ** 4 for bi, ci in zip(b4, c)) - 0.2) > 1e-4


@pytest.mark.parametrize("h0", [0.4, math.inf])
def test_rk45_exact_for_linear_waves(h0):
    # R13: the integrating factor carries an infinitesimal travelling wave
    # exactly for any step, and both solutions of the pair agree.
    g, a, nx, L, m = 9.81, 1e-8, 64, 4.0, 3
    grid = O.Grid(nx, 1, L)
    k = 2 * math.pi * m / L
    w = math.sqrt(g * k * (math.tanh(k * h0) if math.isfinite(h0) else 1.0))
    x = np.arange(nx) * L / nx
    pb = O.Problem(grid, g, h0, order=1, integrator="rk45")
    y5, y4 = O.if_rk45_step(pb, a * np.cos(k * x)[None, :], (g * a / w) * np.sin(k * x)[None, :], 3.0 / w)
    assert np.max(np.abs(y5[0][0] - a * np.cos(k * x - 3.0))) < 1e-6 * a
    assert np.max(np.abs(y4[0][0] - y5[0][0])) < 1e-6 * a


def _rk45_case():
    nx, ny, Lx, Ly, h0 = 32, 16, 6.0, 3.0, 0.7
    grid = O.Grid(nx, ny, Lx, Ly)
    delta = W.random_field(nx, ny, 111, amplitude=0.05, band=0.3)
    pb = O.Problem(grid, 9.81, h0, delta=delta, order=4, integrator="rk45")
    eta = O.project(pb, W.random_field(nx, ny, 112, amplitude=0.04, band=0.3))
    phi = O.project(pb, W.random_field(nx, ny, 113, amplitude=0.1, band=0.3))
    return grid, delta, pb, eta, phi


def test_rk45_fifth_order_and_embedded_estimate():
    # R13: the order-5 solution converges at fifth order to the classical RK4
    # solution at a tiny step (error ratio ~32 per halving); the embedded
    # estimate |u5 - u4| of one step shrinks like h^5 too.
    grid, delta, pb, eta, phi = _rk45_case()
    T_end = 0.4
    ref = O.step(O.Problem(grid, 9.81, 0.7, delta=delta, order=4), eta, phi, T_end / 1024, 1024)
    errs = []
    for n in (4, 8, 16):
        e, p = O.step(pb, eta, phi, T_end / n, n)
        errs.append(np.linalg.norm(e - ref[0]) + np.linalg.norm(p - ref[1]))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 22.0 < r1 < 45.0 and 22.0 < r2 < 45.0, (errs, r1, r2)
    est = []
    for h in (0.2, 0.1, 0.05):
        y5, y4 = O.if_rk45_step(pb, eta, phi, h)
        est.append(O.step_error(eta, phi, y5, y4))
    q1, q2 = est[0] / est[1], est[1] / est[2]
    assert 20.0 < q1 < 48.0 and 20.0 < q2 < 48.0, (est, q1, q2)


def test_rk45_adaptive_run():
    # R13: the adaptive run lands on t_end, its error against the reference is
    # of the order of the tolerance, and a looser tolerance takes fewer steps.
    grid, delta, pb, eta, phi = _rk45_case()
    T_end = 0.6
    ref = O.step(O.Problem(grid, 9.81, 0.7, delta=delta, order=4), eta, phi, T_end / 512, 512)
    steps = {}
    for tol in (1e-6, 1e-8):
        e, p, h, acc, rej = O.step_adaptive(pb, eta, phi, 0.0, T_end, tol, 0.05)
        err = max(np.linalg.norm(e - ref[0]) / np.linalg.norm(ref[0]),
                  np.linalg.norm(p - ref[1]) / np.linalg.norm(ref[1]))
        assert err < 50 * tol, (tol, err)
        steps[tol] = acc
    assert steps[1e-6] < steps[1e-8]


def test_crest_position():
    # R16: the parabola through the largest sample and its neighbours places a
    # smooth peak within a small fraction of a cell; the height is the sample
    n, L = 64, 10.0
    dx = L / n
    grid = O.Grid(n, 1, L)
    x = np.arange(n) * dx
    for x0 in (3.0, 3.0 + 0.37 * dx, 9.9):
        f = np.cos(2 * np.pi * (x - x0) / L)
        cx, cy, h = O.crest(grid, f)
        d = (cx - x0 + L / 2) % L - L / 2
        assert abs(d) < 0.01 * dx and cy == 0.0 and h == f.max()
        g = 0.3 / np.cosh(1.2 * ((x - x0 + L / 2) % L - L / 2)) ** 2
        cx, _, h = O.crest(grid, g)
        assert abs((cx - x0 + L / 2) % L - L / 2) < 0.05 * dx and h == g.max()
    # 2-D: a Gaussian bump; the first of equal samples wins
    grid2 = O.Grid(32, 16, 4.0, 2.0)
    X, Y = np.meshgrid(np.arange(32) * 4.0 / 32, np.arange(16) * 2.0 / 16)
    b = np.exp(-((X - 1.3) ** 2 + (Y - 0.7) ** 2) / 0.5)
    cx, cy, h = O.crest(grid2, b)
    assert abs(cx - 1.3) < 0.05 * 4.0 / 32 and abs(cy - 0.7) < 0.05 * 2.0 / 16 and h == b.max()
    flat = np.zeros((16, 32))
    flat[3, 5] = flat[7, 2] = 1.0
    assert O.crest(grid2, flat)[:2] == (5 * 4.0 / 32, 3 * 2.0 / 16)
