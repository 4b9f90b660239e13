"""Plain FP64 CPU oracle of the enhanced spectral boundary integral (ESBI) hot path.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import this module:
only the tests, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference
legs of ``bench.py`` use it.  It shares no code with the CUDA library.

What it computes (Wang, "An enhanced spectral boundary integral method for
modeling highly nonlinear water waves in variable depth", arXiv 2310.19840):

* ``vertical_velocity``: the surface vertical velocity V = sqrt(1+|grad eta|^2)
  dphi/dn (definition under Eq. (prognostic), Sec. 2.2) from the surface
  elevation eta, the surface potential phi~ and the bottom variation delta, by the
  successive approximation of Sec. 2.4: V = sum_{l=1..M} V_l (Eq. app-V) with
  the bottom potential varphi~ = sum_{l=1..M-1} varphi_l (Eq. app-phi).  The
  order-l terms are taken from the explicit forms of Appendix C (Eqs. v2..v7),
  written with the index pattern of the general recursion (Eqs. app-V-scs,
  app-phi-scs) where the two agree; where they disagree the appendix is followed
  (readings R1-R3 below).
* ``surface_rhs``: the kinematic and dynamic free-surface conditions in the
  Zakharov form of Eq. (prognostic): eta_t = V and
  phi~_t = -g eta + 1/2 [(V + grad eta . grad phi~)^2 / (1+|grad eta|^2) - |grad phi~|^2] - p_d,
  with the optional damping pressure p_d of Eq. (pd).
* ``rk4_step``: classical fourth-order Runge-Kutta with a fixed step on the
  physical-space pair (eta, phi~) (the paper's Sec. 2.2 uses an integrating-factor
  RK5(4); this oracle follows the fixed-step RK4 workload definition).
* ``invariants``: mass int eta dA and total energy E = 1/2 int (V phi~ + g eta^2) dA
  (Eq. energy, written dimensionally).

Readings of passages where the paper is silent, ambiguous or inconsistent:

R1  F{V_l}: the general recursion puts tanh(kh) on the grad-phi~ term for every
    l, Appendix C has it only for odd l (V2 and V4 carry none).  Appendix C is
    followed: the factor is T_l = tanh(kh) for odd l, 1 for even l.
R2  F{varphi_l}: the general recursion omits the eta^{l-1} grad phi~ term and
    gives every delta^j term a minus sign; Appendix C has -sech(kh) k^{l-3}/(l-1)!
    ik.F{eta^{l-1} grad phi~} for odd l and a sign (-1)^j on the delta^j terms.
    Appendix C is followed.
R3  <j/2> is the remainder of j divided by 2, so tanh^{<j/2>} is tanh for odd j
    and 1 for even j, and <j/2> sech is sech for odd j and 0 for even j.
R4  k = 0: every multiplier that carries ik or a positive power of k vanishes
    there; k^{-1} tanh(kh) ik also vanishes (its limit is h ik -> 0).  Hence
    F{V_l}(0) = 0 and the mean of eta is conserved exactly.
R5  Dealiasing ("2/(l+1)-rule", Sec. 2.4): a rectangular mask that keeps the
    Fourier modes with |m| < alpha nx/2 and |n| < alpha ny/2 (strict, after the
    submerged-bar section's "waves longer than 4 grid cells are alias free"),
    alpha = 0.5 by default.  The mask is applied to F{phi~}, to every order
    F{V_l}, F{varphi_l}, to the dynamic-condition right-hand side and to the
    state after each full step.  The Nyquist modes are always removed.
R6  Reference depth h0 is an explicit input, delta = h0 - h(x, y).  sech(kh0) is
    evaluated as 2 e^{-kh0} / (1 + e^{-2kh0}); h0 = inf gives deep water.
R7  Damping pressure (Eq. pd): p_d = nu F^{-1}{ ik/(-k^2) . F{w grad phi~} },
    zero at k = 0, with a user weight w(x, y) and strength nu [1/s].  It enters
    the dynamic condition with a minus sign (a surface pressure).
R8  Low-pass filter (Eq. filter): Lambda = exp(-|k/(beta1 k_ref)|^beta2), applied
    to the spectra of eta and phi~ after each full step when beta1 > 0.
R9  Order truncation: the scheme is explicit with a fixed maximum order M <= 7.
    An optional tolerance stops at the first l whose increment satisfies
    ||F{V_l}||_2 <= tol ||sum_{m<=l} F{V_m}||_2.
R10 Pneumatic wavemaker (Eq. for p_g, submerged-bar section): the printed
    pressure is nondimensional (g = 1); dimensionally
    p_g / rho = g sum_j a_j sqrt(e/2pi) [1 + 2 k_j h0 / sinh(2 k_j h0)]
                  exp(-(k_j d)^2 / 2) sin(omega_j t + theta_j),
    with omega_j^2 = g k_j tanh(k_j h0), d the periodic distance in x from the
    centre x0 (the bell "split in halves at both ends" is the bell centred at
    x0 = 0 of the periodic box) and, in 2-D, no dependence on y (a line
    source).  It enters the dynamic condition like p_d: phi~_t gets -p_g/rho,
    inside the dealiasing of that right-hand side.  With this scaling linear
    theory gives radiated waves of amplitude a_j on each side.
R11 Integrating factor (Sec. 2.2, the reformulation of Eq. (prognostic) with
    e^{-A(t-t0)}): A is the linearisation of the system about rest in
    spectral space, d/dt (eta^, phi^) = [[0, k tanh(k h0)], [-g, 0]] (eta^, phi^)
    on the dealiased modes (the first order of Sec. 2.4 and the -g eta of the
    dynamic condition); everything else is the nonlinear part N: eta_t - V_1
    and phi~_t + g eta.  e^{A tau} = [[cos w tau, (k t / w) sin w tau],
    [-(g / w) sin w tau, cos w tau]] with w^2 = g k t (t = tanh k h0), and at
    k = 0 [[1, 0], [-g tau, 1]].  The paper integrates the transformed system
    with an adaptive embedded RK5(4); this oracle provides the integrating
    factor with classical RK4 stages and a fixed step (the Lawson scheme).
R13 Adaptive integrating factor (Sec. 2.2: six-stage fifth-order RK with an
    embedded fourth-order solution, step size from their difference): the
    tableau is Cash and Karp's 5(4) pair; in the integrating-factor form
    stage i is E(c_i h) u_n + h sum_j a_ij E((c_i - c_j) h) k_j and the
    solutions E(h) u_n + h sum_j b_j E((1 - c_j) h) k_j (b of order 5 and 4).
    The error of a step is max over eta and phi~ of ||u5 - u4|| / ||u_n||
    (L2 over the member, fields whose norm is 0 skipped); a step is accepted
    when the error is at most tol, and the next step is
    h min(5, max(0.2, 0.9 (tol / err)^(1/5))) (5 h when err = 0), cut to end
    at t_end.  The order-5 solution is kept.
R12 HOS diagnostic (the section comparing ESBI and HOS, Eqs. HOS-HOSZ), flat
    bottom at the reference depth h0: the eigenfunctions are
    cosh(k(z + h0)) / cosh(k h0) (deep water e^{kz}), so d^n/dz^n at z = 0
    multiplies mode k by k^n T_n (T_n = tanh(k h0) for odd n, 1 for even n).
    phi^(1) = phi~, phi^(m) = -sum_{n=1}^{m-1} eta^n/n! d^n_z phi^(m-n),
    W = sum_m sum_{n=0}^{M-m} eta^n/n! d^{n+1}_z phi^(m); every phi^(m) and W
    are dealiased with the mask of R5 after their forward transform, and the
    ESBI quantity is V = W (1 + |grad eta|^2) - grad eta . grad phi~ (the
    kinematic condition), dealiased as well.
R15 Implicit form (Appendix A, the "iterative approach" that the successive
    scheme of Sec. 2.4 replaces), flat bottom only (delta = 0, so the bottom
    potential of Appendix B drops out) and without the remaining integral
    I^(S).  Every printed flat-bottom term of V^(2)..V^(7) has the form
    C_h k c F{eta^a F^{-1}{ mult F{eta^b X} }} with m = j - 1 = a + b and
    X = V or the vector grad phi~ under ik. (an a = 0 term has no inner
    transform): for a term of grad phi~ when m is odd, or of V when m is even,
    c = (-1)^{a+1}/(a! b!) and mult = C_h^{-1} (a even) or D_h^{-1} (a odd)
    times k^{m-2} (grad phi~) or k^{m-1} (V); for a term of grad phi~ when m
    is even, or of V when m is odd, c = 1/(a! b!) and mult = e_h k^{m-2}
    (grad phi~) or e_h k^{m-1} (V); e_h = e^{-2kh}, C_h = 1/(1 + e_h),
    D_h = 1/(1 - e_h); V^(1) = k tanh(kh) F{phi~}.  (Each printed term was
    checked against this pattern.)  k^{-1} multiplies only ik.F{...} terms
    and is 0 at k = 0 (R4).  Every forward transform is dealiased (R5).  The
    equation F{V} = G + L(V) (G: V^(1) and the grad phi~ terms; L: the V
    terms) is solved either by the fixed-point iteration
    V_{n+1} = F^{-1}{G + L(V_n)} from V_0 = F^{-1}{V^(1)}, stopped when the
    relative L2 change ||V_{n+1} - V_n|| / ||V_{n+1}|| is at most tol, or by
    GMRES on (I - F^{-1} L) V = F^{-1} G from the same start (relative
    residual tol, no restart), counting applications of L.  The paper does
    not say which iteration its "iterative approach" uses.
R17 Implicit form over a variable bottom (Appendices A and B together,
    without I^(S) and I^(B)): the unknowns are V and the bottom potential
    varphi~.  Besides the terms of R15, V^(j) (j = 2..M) carries
    C_h k 2 (-1)^a/(a! b!) F{eta^a F^{-1}{sqrt(e_h) k^{j-3} ik.F{delta^b grad varphi~}}}
    for odd b, a + b = j - 1; varphi~^(j) (j = 1..M-1) is D_h times
      2/(a! c!) F{delta^c F^{-1}{sqrt(e_h) k^{j-2} F{eta^a V}}}          (even a),
      2/(a! c!) F{delta^c F^{-1}{sqrt(e_h) k^{j-3} ik.F{eta^a grad phi~}}} (odd a),
    c + a = j - 1, and for j >= 2
      s/(c! b!) F{delta^c F^{-1}{X k^{j-3} ik.F{delta^b grad varphi~}}},
    c + b = j - 1, with s X = -C_h^{-1} for odd b and +D_h^{-1} for even b.
    (Each printed term was checked against these patterns.)  The printed
    varphi~^(5) has -e_h on every varphi~ term instead; the two differ by
    sum_{c+b=4} (-1)^b/(c! b!) delta^c K delta^b, K = k^2 ik., the fourth
    nested commutator of a multiplication with a third-order differential
    operator, which vanishes: both forms are the same operator (the printed
    one is the default).  D_h = 1/(1 - e_h) is taken as 0 at k = 0 (R4).
R16 Crest (the crest position and speed of the solitary-wave runs, Sec. 3.1):
    the largest sample of eta (the first in row-major order among equal
    samples), its position refined along each axis by the parabola through
    it and its two periodic neighbours, x = (i + (f_- - f_+) / (2 (f_- - 2 f_0
    + f_+))) dx (no shift where the denominator vanishes); the reported
    height is the sample itself.  The crest speed is the change of position
    over time.

Grid convention: fields are arrays of shape (ny, nx), x fastest; a 1-D problem
has ny = 1 (Ly is then the unit width).  Horizontal vectors are lists of
components [x] (1-D) or [x, y] (2-D).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

MAX_ORDER = 7


@dataclass(frozen=True)
class Grid:
    nx: int
    ny: int
    Lx: float
    Ly: float = 1.0

    @property
    def dim(self) -> int:
        return 1 if self.ny == 1 else 2

    @property
    def dA(self) -> float:
        return (self.Lx / self.nx) * (self.Ly / self.ny)


# --------------------------------------------------------------------------
# Spectral primitives (Sec. 2.2: F{.} is evaluated by the FFT)
# --------------------------------------------------------------------------

def fft(f):
    return np.fft.fft2(f)


def ifft(F):
    return np.real(np.fft.ifft2(F))


def wavenumbers(grid: Grid):
    """Angular wavenumbers (kx, ky) on the full FFT grid and |k|."""
    kx = 2.0 * np.pi * np.fft.fftfreq(grid.nx, d=grid.Lx / grid.nx)
    if grid.ny == 1:
        ky = np.zeros(1)
    else:
        ky = 2.0 * np.pi * np.fft.fftfreq(grid.ny, d=grid.Ly / grid.ny)
    KX, KY = np.meshgrid(kx, ky)
    return KX, KY, np.sqrt(KX * KX + KY * KY)


def dealias_mask(grid: Grid, alpha: float = 0.5):
    """Reading R5: keep |m| < alpha nx/2 and |n| < alpha ny/2 (Nyquist always off)."""
    m = np.abs(np.fft.fftfreq(grid.nx, d=1.0 / grid.nx))
    keep_x = (m < alpha * grid.nx / 2) & (m < grid.nx / 2)
    if grid.ny == 1:
        keep_y = np.ones(1, dtype=bool)
    else:
        n = np.abs(np.fft.fftfreq(grid.ny, d=1.0 / grid.ny))
        keep_y = (n < alpha * grid.ny / 2) & (n < grid.ny / 2)
    return (keep_y[:, None] & keep_x[None, :]).astype(np.float64)


def depth_multipliers(K, h0: float):
    """tanh(k h0) and sech(k h0) (reading R6; h0 = inf -> deep water)."""
    with np.errstate(invalid="ignore", over="ignore"):
        kh = np.where(K > 0, K * h0, 0.0)
    e = np.exp(-kh)
    t = np.tanh(kh)
    s = 2.0 * e / (1.0 + e * e)
    return t, s


def gradient(f_hat, KX, KY, dim):
    """grad f = F^{-1}{ik f^} (component list)."""
    comps = [ifft(1j * KX * f_hat)]
    if dim == 2:
        comps.append(ifft(1j * KY * f_hat))
    return comps


def ik_dot(vec, KX, KY):
    """ik . F{vec} = i kx F{vec_x} + i ky F{vec_y}."""
    out = 1j * KX * fft(vec[0])
    if len(vec) == 2:
        out = out + 1j * KY * fft(vec[1])
    return out


# --------------------------------------------------------------------------
# Diagnostic: successive approximation of V (Sec. 2.4, Appendix C)
# --------------------------------------------------------------------------

def vertical_velocity(eta, phi, delta, h0, grid: Grid, order: int = MAX_ORDER,
                      alpha: float = 0.5, tol: float = 0.0, return_terms: bool = False):
    """V from (eta, phi~, delta) by the successive approximation of Sec. 2.4.

    delta may be None (flat bottom: every delta term drops out).  With
    ``return_terms`` the per-order lists [V_1..V_M] and [varphi_1..varphi_{M-1}]
    (physical space) and the number of orders used are returned as well.
    """
    if not 1 <= order <= MAX_ORDER:
        raise ValueError("order must be in 1..7")
    eta = np.asarray(eta, dtype=np.float64).reshape(grid.ny, grid.nx)
    phi = np.asarray(phi, dtype=np.float64).reshape(grid.ny, grid.nx)
    flat = delta is None or not np.any(delta)
    if not flat:
        delta = np.asarray(delta, dtype=np.float64).reshape(grid.ny, grid.nx)
    KX, KY, K = wavenumbers(grid)
    mask = dealias_mask(grid, alpha)
    t, s = depth_multipliers(K, h0)
    with np.errstate(divide="ignore", invalid="ignore"):
        k_inv_t = np.where(K > 0, t / np.where(K > 0, K, 1.0), 0.0)   # R4
    dim = grid.dim

    def T(j):  # R3
        return t if j % 2 == 1 else 1.0

    def S(j):  # R3
        return s if j % 2 == 1 else 0.0

    def kpow(p):  # k^p for p >= 0
        return K ** p if p > 0 else np.ones_like(K)

    phi_hat = mask * fft(phi)
    grad_phi_s = gradient(phi_hat, KX, KY, dim)            # grad phi~

    # Order 1 (Sec. 2.4): F{V_1} = k tanh(kh) F{phi~}, F{varphi_1} = sech(kh) F{phi~}
    V_hat = [None, K * t * phi_hat]
    V = [None, ifft(V_hat[1])]
    grad_b = [None]
    if not flat:
        b_hat1 = s * phi_hat
        grad_b.append(gradient(b_hat1, KX, KY, dim))
        b_phys = [None, ifft(b_hat1)]
    total_hat = V_hat[1].copy()
    used = 1
    for l in range(2, order + 1):
        # F{V_l}: Eq. app-V-scs with Appendix C's T_l on the grad phi~ term (R1)
        acc = np.zeros_like(phi_hat)
        for j in range(1, l):
            acc -= kpow(j) / math.factorial(j) * T(j) * fft(eta ** j * V[l - j])
        prod = [eta ** (l - 1) * g for g in grad_phi_s]
        acc -= T(l) * kpow(l - 2) / math.factorial(l - 1) * ik_dot(prod, KX, KY)
        if not flat:
            for j in range(1, l, 2):   # S_j = 0 for even j
                prod = [delta ** j * g for g in grad_b[l - j]]
                acc += kpow(j - 1) / math.factorial(j) * s * ik_dot(prod, KX, KY)
        V_hat.append(mask * acc)
        V.append(ifft(V_hat[l]))
        # F{varphi_l}: Appendix C (R2); needed for l <= order-1 only
        if not flat and l <= order - 1:
            bcc = np.zeros_like(phi_hat)
            for j in range(1, l, 2):
                bcc -= kpow(j - 1) / math.factorial(j) * s * fft(eta ** j * V[l - j])
            if l % 2 == 1:
                prod = [eta ** (l - 1) * g for g in grad_phi_s]
                bcc -= s * kpow(l - 3) / math.factorial(l - 1) * ik_dot(prod, KX, KY)
            for j in range(1, l):
                prod = [delta ** j * g for g in grad_b[l - j]]
                if j == 1:
                    coef = -k_inv_t                     # (-1)^1 k^{-1} tanh / 1!
                elif j % 2 == 1:
                    coef = -kpow(j - 2) / math.factorial(j) * t
                else:
                    coef = kpow(j - 2) / math.factorial(j)
                bcc += coef * ik_dot(prod, KX, KY)
            b_hat = mask * bcc
            grad_b.append(gradient(b_hat, KX, KY, dim))
            b_phys.append(ifft(b_hat))
        total_hat = total_hat + V_hat[l]
        used = l
        if tol > 0.0:
            inc = np.sqrt(np.sum(np.abs(V_hat[l]) ** 2))
            tot = np.sqrt(np.sum(np.abs(total_hat) ** 2))
            if inc <= tol * tot:
                break
    Vsum = ifft(total_hat)
    if return_terms:
        terms = {"V": V[1:used + 1], "used": used}
        if not flat:
            terms["varphi"] = b_phys[1:]
        return Vsum, terms
    return Vsum


def hos_surface_velocity(eta, phi, h0, grid: Grid, order: int = MAX_ORDER, alpha: float = 0.5):
    """(V, W) by the HOS perturbation expansion (R12): W = dphi/dz at the
    surface, V = sqrt(1+|grad eta|^2) dphi/dn as in Eq. (prognostic)."""
    if not 1 <= order <= MAX_ORDER:
        raise ValueError("order must be in 1..7")
    eta = np.asarray(eta, dtype=np.float64).reshape(grid.ny, grid.nx)
    phi = np.asarray(phi, dtype=np.float64).reshape(grid.ny, grid.nx)
    KX, KY, K = wavenumbers(grid)
    mask = dealias_mask(grid, alpha)
    t, _ = depth_multipliers(K, h0)

    def dz(f_hat, n):          # d^n/dz^n at z = 0 (R12)
        return ifft(K ** n * (t if n % 2 == 1 else 1.0) * f_hat)

    phis = [None, mask * fft(phi)]                      # Eq. HOSM, phi^(1) = phi~
    for m in range(2, order + 1):
        acc = np.zeros_like(eta)
        for n in range(1, m):
            acc -= eta ** n / math.factorial(n) * dz(phis[m - n], n)
        phis.append(mask * fft(acc))
    W = np.zeros_like(eta)                              # Eq. HOSZ
    for m in range(1, order + 1):
        for n in range(0, order - m + 1):
            W += eta ** n / math.factorial(n) * dz(phis[m], n + 1)
    W = ifft(mask * fft(W))
    ge = gradient(mask * fft(eta), KX, KY, grid.dim)
    gp = gradient(phis[1], KX, KY, grid.dim)
    V = W * (1.0 + sum(a * a for a in ge)) - sum(a * b for a, b in zip(ge, gp))
    return ifft(mask * fft(V)), W


# --------------------------------------------------------------------------
# Implicit convolution form (Appendix A, flat bottom) by iteration (R15)
# --------------------------------------------------------------------------

def implicit_system(eta, phi, h0, grid: Grid, order: int = MAX_ORDER, alpha: float = 0.5):
    """The implicit equations of Appendix A on a flat bottom of depth h0
    (math.inf: deep water), reading R15, as F{V} = G + L(V): returns the
    spectrum G driven by phi~ (V^(1) and the grad phi~ terms of V^(2..M)) and
    the linear map L from a physical V to the spectrum of the V terms."""
    if not 1 <= order <= MAX_ORDER:
        raise ValueError("order must be in 1..7")
    eta = np.asarray(eta, dtype=np.float64).reshape(grid.ny, grid.nx)
    phi = np.asarray(phi, dtype=np.float64).reshape(grid.ny, grid.nx)
    KX, KY, K = wavenumbers(grid)
    mask = dealias_mask(grid, alpha)
    t, _ = depth_multipliers(K, h0)
    if math.isinf(h0):
        e_h = np.zeros_like(K)
    else:
        e_h = np.exp(-2.0 * K * h0)
    C = 1.0 / (1.0 + e_h)                   # C_h
    X = (1.0 + e_h, 1.0 - e_h)              # C_h^{-1} (a even), D_h^{-1} (a odd)
    image = bool(np.any(e_h > 0.0))

    def kpow(p):
        if p >= 0:
            return K ** p if p > 0 else np.ones_like(K)
        with np.errstate(divide="ignore"):
            return np.where(K > 0, 1.0 / np.where(K > 0, K, 1.0) ** (-p), 0.0)

    def outer(a, spec):                     # F{eta^a F^{-1}{spec}}, dealiased
        return mask * spec if a == 0 else mask * fft(eta ** a * ifft(spec))

    M1 = order - 1
    phi_hat = mask * fft(phi)
    grad_phi = gradient(phi_hat, KX, KY, grid.dim)
    P = [mask * ik_dot([eta ** b * g for g in grad_phi], KX, KY) for b in range(M1 + 1)]
    # the part driven by phi~: V^(1) and the grad phi~ terms of V^(2..M)
    G = K * t * phi_hat
    for m in range(1, M1 + 1):
        for a in range(m + 1):
            b = m - a
            f = math.factorial(a) * math.factorial(b)
            if m % 2 == 1:
                mult = (-1.0) ** (a + 1) / f * X[a % 2] * kpow(m - 2)
            elif image:
                mult = e_h / f * kpow(m - 2)
            else:
                continue
            G = G + C * K * outer(a, mult * P[b])

    def implicit_part(Vp):                  # the V terms of V^(2..M)
        Q = [mask * fft(eta ** b * Vp) for b in range(M1 + 1)]
        out = np.zeros_like(G)
        for m in range(1, M1 + 1):
            for a in range(m + 1):
                b = m - a
                f = math.factorial(a) * math.factorial(b)
                if m % 2 == 0:
                    mult = (-1.0) ** (a + 1) / f * X[a % 2] * kpow(m - 1)
                elif image:
                    mult = e_h / f * kpow(m - 1)
                else:
                    continue
                out = out + C * K * outer(a, mult * Q[b])
        return out

    return mask * G, lambda Vp: mask * implicit_part(np.asarray(Vp, dtype=np.float64).reshape(grid.ny, grid.nx))


def implicit_system_variable(eta, phi, delta, h0, grid: Grid, order: int = MAX_ORDER,
                             alpha: float = 0.5, b5: str = "pattern"):
    """The implicit equations of Appendices A and B over a variable bottom
    (reading R17) for the unknowns u = (V, varphi~) in physical space:
    F{u} = G + L(u).  Returns (G, L) with G = (G_V, G_B) spectra and L(u)
    the pair of spectra of the terms in V and varphi~.  ``b5`` selects the
    reading of the varphi~ terms of varphi~^(5): "pattern" (the signs and
    depth factors of the other orders) or "printed" (-e_h on every term)."""
    if not 1 <= order <= MAX_ORDER:
        raise ValueError("order must be in 1..7")
    if math.isinf(h0):
        raise ValueError("a variable bottom needs a finite reference depth")
    shape = (grid.ny, grid.nx)
    eta = np.asarray(eta, dtype=np.float64).reshape(shape)
    phi = np.asarray(phi, dtype=np.float64).reshape(shape)
    delta = np.asarray(delta, dtype=np.float64).reshape(shape)
    KX, KY, K = wavenumbers(grid)
    mask = dealias_mask(grid, alpha)
    t, _ = depth_multipliers(K, h0)
    e_h = np.exp(-2.0 * K * h0)
    C = 1.0 / (1.0 + e_h)
    X = (1.0 + e_h, 1.0 - e_h)               # C_h^{-1} (even), D_h^{-1} (odd)
    with np.errstate(divide="ignore"):
        D = np.where(K > 0, 1.0 / np.where(K > 0, 1.0 - e_h, 1.0), 0.0)   # D_h, 0 at k = 0 (R4)
    se = np.sqrt(e_h)
    M1 = order - 1
    fa = math.factorial

    def kpow(p):
        if p >= 0:
            return K ** p if p > 0 else np.ones_like(K)
        with np.errstate(divide="ignore"):
            return np.where(K > 0, 1.0 / np.where(K > 0, K, 1.0) ** (-p), 0.0)

    def outer(f, a, spec):                   # F{f^a F^{-1}{spec}}, dealiased
        return mask * spec if a == 0 else mask * fft(f ** a * ifft(spec))

    def ikdot(f, b, vec):                    # ik . F{f^b vec}, dealiased
        return mask * ik_dot([f ** b * v for v in vec], KX, KY)

    phi_hat = mask * fft(phi)
    gphi = gradient(phi_hat, KX, KY, grid.dim)
    # G_V: V^(1) and the grad phi~ terms of V^(2..M) (Appendix A, flat part)
    GV = K * t * phi_hat
    GB = np.zeros_like(GV)
    for m in range(1, M1 + 1):
        for a in range(m + 1):
            b = m - a
            if m % 2 == 1:
                mult = (-1.0) ** (a + 1) / (fa(a) * fa(b)) * X[a % 2] * kpow(m - 2)
            else:
                mult = e_h / (fa(a) * fa(b)) * kpow(m - 2)
            GV = GV + C * K * outer(eta, a, mult * ikdot(eta, b, gphi))
    # G_B: the grad phi~ terms of varphi~^(j), j = 2..M-1 (Appendix B)
    for j in range(2, M1 + 1):
        for a in range(1, j, 2):
            c = j - 1 - a
            GB = GB + D * outer(delta, c, 2.0 / (fa(a) * fa(c)) * se * kpow(j - 3) * ikdot(eta, a, gphi))

    def L(u):
        Vp, Bp = (np.asarray(w, dtype=np.float64).reshape(shape) for w in u)
        gB = gradient(mask * fft(Bp), KX, KY, grid.dim)
        LV = np.zeros_like(GV)
        # V terms of Appendix A (as on a flat bottom)
        for m in range(1, M1 + 1):
            for a in range(m + 1):
                b = m - a
                if m % 2 == 0:
                    mult = (-1.0) ** (a + 1) / (fa(a) * fa(b)) * X[a % 2] * kpow(m - 1)
                else:
                    mult = e_h / (fa(a) * fa(b)) * kpow(m - 1)
                LV = LV + C * K * outer(eta, a, mult * mask * fft(eta ** b * Vp))
        # delta grad varphi~ terms of V^(j), j = 2..M
        for j in range(2, order + 1):
            for b in range(1, j, 2):
                a = j - 1 - b
                LV = LV + C * K * outer(eta, a, 2.0 * (-1.0) ** a / (fa(a) * fa(b)) * se * kpow(j - 3)
                                        * ikdot(delta, b, gB))
        LB = np.zeros_like(GV)
        for j in range(1, M1 + 1):
            # V terms of varphi~^(j)
            for a in range(0, j, 2):
                c = j - 1 - a
                LB = LB + D * outer(delta, c, 2.0 / (fa(a) * fa(c)) * se * kpow(j - 2) * mask * fft(eta ** a * Vp))
            # varphi~ terms of varphi~^(j), j >= 2
            if j >= 2:
                for b in range(j):
                    c = j - 1 - b
                    if j == 5 and b5 == "printed":
                        mult = -e_h / (fa(c) * fa(b))
                    elif b % 2 == 1:
                        mult = -X[0] / (fa(c) * fa(b))
                    else:
                        mult = X[1] / (fa(c) * fa(b))
                    LB = LB + D * outer(delta, c, mult * kpow(j - 3) * ikdot(delta, b, gB))
        return LV, LB

    return (mask * GV, mask * GB), L


def implicit_vertical_velocity(eta, phi, h0, grid: Grid, order: int = MAX_ORDER,
                               alpha: float = 0.5, tol: float = 1e-12, maxit: int = 200,
                               solver: str = "fixed_point", delta=None, b5: str = "printed"):
    """V from the implicit equations of Appendix A (flat bottom, reading R15)
    or of Appendices A and B together (variable bottom ``delta``, reading
    R17; unknowns V and varphi~), by the fixed-point iteration
    (``solver="fixed_point"``) or by GMRES (``solver="gmres"``), both from
    the first orders V^(1) (and varphi~_1 = sech(k h0) F{phi~}).

    Returns (V, applications, history): the number of applications of L and,
    per application, the relative L2 change of the iterate (fixed point) or
    the relative residual (GMRES)."""
    shape = (grid.ny, grid.nx)
    npts = grid.nx * grid.ny
    KX, KY, K = wavenumbers(grid)
    t, s = depth_multipliers(K, h0)
    mask = dealias_mask(grid, alpha)
    phi_hat = mask * fft(np.asarray(phi, dtype=np.float64).reshape(shape))
    variable = delta is not None and bool(np.any(delta))
    if variable:
        G, Lv = implicit_system_variable(eta, phi, delta, h0, grid, order, alpha, b5)
        u0 = [ifft(K * t * phi_hat), ifft(s * phi_hat)]
        L = lambda u: list(Lv(u))
    else:
        G1, L1 = implicit_system(eta, phi, h0, grid, order, alpha)
        G, u0 = [G1], [ifft(K * t * phi_hat)]
        L = lambda u: [L1(u[0])]
    nf = len(u0)

    def pack(fields):
        return np.concatenate([np.asarray(f, dtype=np.float64).ravel() for f in fields])

    def unpack(v):
        return [v[q * npts:(q + 1) * npts].reshape(shape) for q in range(nf)]

    def step(u):                            # F^{-1}{G + L(u)}, per unknown
        return [ifft(g + l) for g, l in zip(G, L(u))]

    if solver == "gmres":
        import scipy.sparse.linalg as spla
        count = [0]
        Gp = pack([ifft(g) for g in G])

        def apply(v):
            count[0] += 1
            return v - (pack(step(unpack(v))) - Gp)

        history = []
        A = spla.LinearOperator((nf * npts, nf * npts), matvec=apply, dtype=np.float64)
        sol, info = spla.gmres(A, Gp, x0=pack(u0), rtol=tol, atol=0.0,
                               restart=min(nf * npts, maxit), maxiter=1,
                               callback=history.append, callback_type="pr_norm")
        if info < 0:
            raise RuntimeError("gmres failed")
        return unpack(sol)[0], count[0], history
    if solver != "fixed_point":
        raise ValueError("solver must be 'fixed_point' or 'gmres'")
    u = u0
    increments = []
    n = 0
    for n in range(1, maxit + 1):
        with np.errstate(over="ignore", invalid="ignore"):
            un = step(u)
            inc = float(np.linalg.norm(un[0] - u[0]) / max(np.linalg.norm(un[0]), 1e-300))
        u = un
        increments.append(inc)
        if inc <= tol or not math.isfinite(inc):   # converged, or diverged
            break
    return u[0], n, increments


# --------------------------------------------------------------------------
# Prognostic right-hand side (Sec. 2.2) and damping pressure (Eq. pd)
# --------------------------------------------------------------------------

def damping_pressure(phi, weight, nu, grid: Grid, alpha: float = 0.5):
    """R7: p_d = nu F^{-1}{ mask ik/(-k^2) . F{w grad phi~} }."""
    KX, KY, K = wavenumbers(grid)
    mask = dealias_mask(grid, alpha)
    phi_hat = mask * fft(np.asarray(phi, dtype=np.float64).reshape(grid.ny, grid.nx))
    w = np.asarray(weight, dtype=np.float64).reshape(grid.ny, grid.nx)
    prod = [w * g for g in gradient(phi_hat, KX, KY, grid.dim)]
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = np.where(K > 0, -1.0 / np.where(K > 0, K * K, 1.0), 0.0)
    return nu * ifft(mask * inv * ik_dot(prod, KX, KY))


def dynamic_rhs(eta, phi, V, gravity, grid: Grid, alpha: float = 0.5, pressure=None):
    """phi~_t without the damping pressure: the second line of Eq. (prognostic)
    written in physical space, -g eta + 1/2[(V + grad eta.grad phi~)^2/(1+|grad eta|^2)
    - |grad phi~|^2] (minus a surface pressure / rho when given), dealiased (R5)."""
    KX, KY, K = wavenumbers(grid)
    mask = dealias_mask(grid, alpha)
    eta = np.asarray(eta, dtype=np.float64).reshape(grid.ny, grid.nx)
    phi = np.asarray(phi, dtype=np.float64).reshape(grid.ny, grid.nx)
    ge = gradient(mask * fft(eta), KX, KY, grid.dim)
    gp = gradient(mask * fft(phi), KX, KY, grid.dim)
    dot = sum(a * b for a, b in zip(ge, gp))
    ge2 = sum(a * a for a in ge)
    gp2 = sum(a * a for a in gp)
    n2 = -gravity * eta + 0.5 * ((V + dot) ** 2 / (1.0 + ge2) - gp2)
    if pressure is not None:
        n2 = n2 - pressure
    return ifft(mask * fft(n2))


@dataclass
class Wavemaker:
    """Components of the pneumatic wavemaker (R10): amplitudes a_j [m], angular
    frequencies omega_j [rad/s], phases theta_j, and the centre x0 [m]."""
    amp: np.ndarray
    omega: np.ndarray
    phase: np.ndarray
    x0: float = 0.0


def dispersion_wavenumber(omega: float, h0: float, gravity: float) -> float:
    """k with omega^2 = g k tanh(k h0) (Newton from the deep-water value)."""
    k = omega * omega / gravity
    if math.isinf(h0):
        return k
    for _ in range(100):
        t = math.tanh(k * h0)
        f = gravity * k * t - omega * omega
        df = gravity * (t + k * h0 * (1.0 - t * t))
        dk = f / df
        k -= dk
        if abs(dk) <= 1e-15 * k:
            break
    return k


def wavemaker_pressure(wm: Wavemaker, grid: Grid, h0: float, gravity: float, t: float):
    """p_g / rho of R10 at time t on the grid, shape (ny, nx)."""
    x = np.arange(grid.nx) * (grid.Lx / grid.nx)
    d = np.mod(x - wm.x0 + 0.5 * grid.Lx, grid.Lx) - 0.5 * grid.Lx
    p = np.zeros(grid.nx)
    for a, w, th in zip(np.atleast_1d(wm.amp), np.atleast_1d(wm.omega), np.atleast_1d(wm.phase)):
        k = dispersion_wavenumber(float(w), h0, gravity)
        shoal = 1.0 if math.isinf(h0) else 1.0 + 2.0 * k * h0 / math.sinh(2.0 * k * h0)
        p += (gravity * a * math.sqrt(math.e / (2.0 * math.pi)) * shoal
              * np.exp(-0.5 * (k * d) ** 2) * math.sin(w * t + th))
    return np.broadcast_to(p, (grid.ny, grid.nx)).copy()


@dataclass
class Problem:
    grid: Grid
    gravity: float
    h0: float
    delta: np.ndarray | None = None
    order: int = MAX_ORDER
    alpha: float = 0.5
    sponge_w: np.ndarray | None = None
    sponge_nu: float = 0.0
    filt_beta1: float = 0.0
    filt_beta2: float = 0.0
    k_ref: float = 1.0
    adapt_tol: float = 0.0      # R9: 0 = fixed order
    wavemaker: "Wavemaker | None" = None   # R10
    integrator: str = "rk4"                 # "rk4" (classical), "lawson" (R11) or "rk45" (R13)
    diagnostic: str = "esbi"                # "esbi" (Sec. 2.4) or "hos" (R12, flat bottom)


def diagnose(pb: "Problem", eta, phi):
    """V of the problem's diagnostic: ESBI (Sec. 2.4) or HOS (R12)."""
    if pb.diagnostic == "hos":
        return hos_surface_velocity(eta, phi, pb.h0, pb.grid, pb.order, pb.alpha)[0]
    return vertical_velocity(eta, phi, pb.delta, pb.h0, pb.grid, pb.order, pb.alpha, tol=pb.adapt_tol)


def surface_rhs(pb: Problem, eta, phi, t: float = 0.0):
    """(eta_t, phi~_t) of Eq. (prognostic) in physical space at time t."""
    V = diagnose(pb, eta, phi)
    pg = None
    if pb.wavemaker is not None:
        pg = wavemaker_pressure(pb.wavemaker, pb.grid, pb.h0, pb.gravity, t)
    phi_t = dynamic_rhs(eta, phi, V, pb.gravity, pb.grid, pb.alpha, pressure=pg)
    if pb.sponge_w is not None and pb.sponge_nu != 0.0:
        phi_t = phi_t - damping_pressure(phi, pb.sponge_w, pb.sponge_nu, pb.grid, pb.alpha)
    return V, phi_t


def project(pb: Problem, f):
    """Dealias (R5) and, when enabled, low-pass filter (R8) a state field."""
    KX, KY, K = wavenumbers(pb.grid)
    m = dealias_mask(pb.grid, pb.alpha)
    if pb.filt_beta1 > 0.0:
        m = m * np.exp(-np.abs(K / (pb.filt_beta1 * pb.k_ref)) ** pb.filt_beta2)
    return ifft(m * fft(np.asarray(f, dtype=np.float64).reshape(pb.grid.ny, pb.grid.nx)))


def linear_propagator(pb: "Problem", tau: float):
    """R11: entries (cos w tau, (k t / w) sin w tau, (g / w) sin w tau) of
    e^{A tau} on the full FFT grid."""
    KX, KY, K = wavenumbers(pb.grid)
    t, _ = depth_multipliers(K, pb.h0)
    w = np.sqrt(pb.gravity * K * t)
    C = np.cos(w * tau)
    with np.errstate(divide="ignore", invalid="ignore"):
        Sk = np.where(K > 0, K * t * np.sin(w * tau) / np.where(w > 0, w, 1.0), 0.0)
        Sg = np.where(K > 0, pb.gravity * np.sin(w * tau) / np.where(w > 0, w, 1.0), pb.gravity * tau)
    return C, Sk, Sg


def nonlinear_part(pb: "Problem", eta, phi, t: float):
    """R11: N = (eta_t - V_1, phi~_t + g eta) in physical space, with V_1 the
    first order of Sec. 2.4 and eta dealiased as in the dynamic condition."""
    KX, KY, K = wavenumbers(pb.grid)
    mask = dealias_mask(pb.grid, pb.alpha)
    tk, _ = depth_multipliers(K, pb.h0)
    V, phi_t = surface_rhs(pb, eta, phi, t)
    V1 = ifft(mask * K * tk * fft(phi))
    return V - V1, phi_t + pb.gravity * ifft(mask * fft(eta))


def lawson_rk4_step(pb: "Problem", eta, phi, dt: float, t: float = 0.0):
    """One step of the integrating-factor scheme (R11) with classical RK4
    stages (Lawson): with E(tau) = e^{A tau} and h = dt,
      k1 = N(u_n),  u2 = E(h/2)(u_n + h/2 k1),  k2 = N(u2),
      u3 = E(h/2) u_n + h/2 k2,  k3 = N(u3),  u4 = E(h) u_n + h E(h/2) k3,
      k4 = N(u4),  u_{n+1} = E(h) u_n + h/6 (E(h) k1 + 2 E(h/2)(k2 + k3) + k4),
    the stages evaluated at t, t + h/2, t + h/2, t + h."""
    half, full = linear_propagator(pb, 0.5 * dt), linear_propagator(pb, dt)

    def E(P, a, b):
        C, Sk, Sg = P
        return C * a + Sk * b, -Sg * a + C * b

    def N(a, b, tt):
        ne, nph = nonlinear_part(pb, ifft(a), ifft(b), tt)
        return fft(ne), fft(nph)

    u = (fft(np.asarray(eta, dtype=np.float64).reshape(pb.grid.ny, pb.grid.nx)),
         fft(np.asarray(phi, dtype=np.float64).reshape(pb.grid.ny, pb.grid.nx)))
    k1 = N(*u, t)
    u2 = E(half, u[0] + 0.5 * dt * k1[0], u[1] + 0.5 * dt * k1[1])
    k2 = N(*u2, t + 0.5 * dt)
    Eu_half = E(half, *u)
    u3 = (Eu_half[0] + 0.5 * dt * k2[0], Eu_half[1] + 0.5 * dt * k2[1])
    k3 = N(*u3, t + 0.5 * dt)
    Eu_full = E(full, *u)
    Ek3 = E(half, *k3)
    u4 = (Eu_full[0] + dt * Ek3[0], Eu_full[1] + dt * Ek3[1])
    k4 = N(*u4, t + dt)
    Ek1 = E(full, *k1)
    Ek23 = E(half, k2[0] + k3[0], k2[1] + k3[1])
    new = tuple(Eu_full[i] + dt / 6.0 * (Ek1[i] + 2.0 * Ek23[i] + k4[i]) for i in range(2))
    return ifft(new[0]), ifft(new[1])


# Cash-Karp 5(4) tableau (R13): nodes, stage weights, order-5 and order-4 weights
CK_C = (0.0, 1.0 / 5.0, 3.0 / 10.0, 3.0 / 5.0, 1.0, 7.0 / 8.0)
CK_A = ((),
        (1.0 / 5.0,),
        (3.0 / 40.0, 9.0 / 40.0),
        (3.0 / 10.0, -9.0 / 10.0, 6.0 / 5.0),
        (-11.0 / 54.0, 5.0 / 2.0, -70.0 / 27.0, 35.0 / 27.0),
        (1631.0 / 55296.0, 175.0 / 512.0, 575.0 / 13824.0, 44275.0 / 110592.0, 253.0 / 4096.0))
CK_B5 = (37.0 / 378.0, 0.0, 250.0 / 621.0, 125.0 / 594.0, 0.0, 512.0 / 1771.0)
CK_B4 = (2825.0 / 27648.0, 0.0, 18575.0 / 48384.0, 13525.0 / 55296.0, 277.0 / 14336.0, 1.0 / 4.0)


def if_rk45_step(pb: "Problem", eta, phi, dt: float, t: float = 0.0):
    """One integrating-factor step with the 5(4) pair of R13: returns the
    order-5 pair (eta, phi~) and the order-4 pair."""
    def E(tau, a, b):
        C, Sk, Sg = linear_propagator(pb, tau)
        return C * a + Sk * b, -Sg * a + C * b

    def N(a, b, tt):
        ne, nph = nonlinear_part(pb, ifft(a), ifft(b), tt)
        return fft(ne), fft(nph)

    u = (fft(np.asarray(eta, dtype=np.float64).reshape(pb.grid.ny, pb.grid.nx)),
         fft(np.asarray(phi, dtype=np.float64).reshape(pb.grid.ny, pb.grid.nx)))
    ks = []
    for i in range(6):
        st = list(E(CK_C[i] * dt, *u))
        for j in range(i):
            if CK_A[i][j] != 0.0:
                ek = E((CK_C[i] - CK_C[j]) * dt, *ks[j])
                st[0] = st[0] + dt * CK_A[i][j] * ek[0]
                st[1] = st[1] + dt * CK_A[i][j] * ek[1]
        ks.append(N(st[0], st[1], t + CK_C[i] * dt))
    out = []
    for b in (CK_B5, CK_B4):
        acc = list(E(dt, *u))
        for j in range(6):
            if b[j] != 0.0:
                ek = E((1.0 - CK_C[j]) * dt, *ks[j])
                acc[0] = acc[0] + dt * b[j] * ek[0]
                acc[1] = acc[1] + dt * b[j] * ek[1]
        out.append((ifft(acc[0]), ifft(acc[1])))
    return out[0], out[1]


def step_error(eta0, phi0, y5, y4):
    """R13: max over the fields of ||u5 - u4|| / ||u_n|| (fields of norm 0 skipped)."""
    err = 0.0
    for f0, a, b in ((eta0, y5[0], y4[0]), (phi0, y5[1], y4[1])):
        n0 = float(np.linalg.norm(f0))
        if n0 > 0.0:
            err = max(err, float(np.linalg.norm(a - b)) / n0)
    return err


def next_step(h: float, err: float, tol: float) -> float:
    """R13: the step after an error err at step h."""
    if err == 0.0:
        return 5.0 * h
    return h * min(5.0, max(0.2, 0.9 * (tol / err) ** 0.2))


def step_adaptive(pb: "Problem", eta, phi, t0: float, t_end: float, tol: float, h: float,
                  max_steps: int = 100000):
    """Integrate from t0 to t_end with the adaptive integrating factor of R13;
    each accepted step is followed by the projection of R5/R8.  Returns
    (eta, phi~, h_next, accepted, rejected)."""
    y = (np.asarray(eta, dtype=np.float64).reshape(pb.grid.ny, pb.grid.nx),
         np.asarray(phi, dtype=np.float64).reshape(pb.grid.ny, pb.grid.nx))
    t, acc, rej = t0, 0, 0
    while t < t_end and acc + rej < max_steps:
        last = t + h >= t_end
        hh = t_end - t if last else h
        y5, y4 = if_rk45_step(pb, y[0], y[1], hh, t)
        err = step_error(y[0], y[1], y5, y4)
        if err <= tol:
            y = (project(pb, y5[0]), project(pb, y5[1]))
            t = t_end if last else t + hh
            acc += 1
            h = next_step(hh, err, tol) if not last else max(h, next_step(hh, err, tol))
        else:
            rej += 1
            h = next_step(hh, err, tol)
    return y[0], y[1], h, acc, rej


def rk4_step(f, y, dt, t=0.0):
    """Classical RK4 for y' = f(t, y) from time t; y is a tuple of arrays."""
    def axpy(a, x, b):
        return tuple(xi + a * bi for xi, bi in zip(x, b))
    k1 = f(t, y)
    k2 = f(t + 0.5 * dt, axpy(0.5 * dt, y, k1))
    k3 = f(t + 0.5 * dt, axpy(0.5 * dt, y, k2))
    k4 = f(t + dt, axpy(dt, y, k3))
    return tuple(yi + dt / 6.0 * (a + 2.0 * b + 2.0 * c + d)
                 for yi, a, b, c, d in zip(y, k1, k2, k3, k4))


def step(pb: Problem, eta, phi, dt: float, n: int = 1, t0: float = 0.0):
    """n RK4 steps of (eta, phi~) from time t0, each followed by the
    projection of R5/R8."""
    y = (np.asarray(eta, dtype=np.float64).reshape(pb.grid.ny, pb.grid.nx),
         np.asarray(phi, dtype=np.float64).reshape(pb.grid.ny, pb.grid.nx))
    for i in range(n):
        if pb.integrator == "lawson":
            y = lawson_rk4_step(pb, y[0], y[1], dt, t0 + i * dt)
        elif pb.integrator == "rk45":
            y = if_rk45_step(pb, y[0], y[1], dt, t0 + i * dt)[0]
        else:
            y = rk4_step(lambda t, s: surface_rhs(pb, s[0], s[1], t), y, dt, t0 + i * dt)
        y = (project(pb, y[0]), project(pb, y[1]))
    return y


def crest(grid: Grid, eta):
    """(x, y, height) of the crest, reading R16 (y = 0 in 1-D)."""
    f = np.asarray(eta, dtype=np.float64).reshape(grid.ny, grid.nx)
    j, i = divmod(int(np.argmax(f)), grid.nx)

    def shift(fm, f0, fp):
        den = fm - 2.0 * f0 + fp
        return 0.5 * (fm - fp) / den if den != 0.0 else 0.0

    x = (i + shift(f[j, (i - 1) % grid.nx], f[j, i], f[j, (i + 1) % grid.nx])) * (grid.Lx / grid.nx)
    y = 0.0
    if grid.ny > 1:
        y = (j + shift(f[(j - 1) % grid.ny, i], f[j, i], f[(j + 1) % grid.ny, i])) * (grid.Ly / grid.ny)
    return x, y, float(f[j, i])


def invariants(pb: Problem, eta, phi):
    """Mass int eta dA and energy 1/2 int (V phi~ + g eta^2) dA (Eq. energy)."""
    eta = np.asarray(eta, dtype=np.float64).reshape(pb.grid.ny, pb.grid.nx)
    phi = np.asarray(phi, dtype=np.float64).reshape(pb.grid.ny, pb.grid.nx)
    V = diagnose(pb, eta, phi)
    mass = float(np.sum(eta) * pb.grid.dA)
    energy = float(0.5 * np.sum(V * phi + pb.gravity * eta * eta) * pb.grid.dA)
    return mass, energy
