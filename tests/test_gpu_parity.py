"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: the FP32 path must reach 1e-5 relative L2 on V after one
evaluation; the FP64 path 1e-12 (FFT round-off grows like eps log N and the
order-7 terms multiply it by at most a few hundred at these amplitudes; every
case here stays below 1e-12).
Inputs are seeded band-limited fields shaped like the workloads (red spectra,
amplitudes k|eta| up to ~0.3), projected by the oracle so both sides start
from the same band-limited state.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import sbi_oracle as O

pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 1: 1e-12}   # SBI_FP32, SBI_FP64


@pytest.fixture(scope="module")
def sbi():
    import __graft_entry__ as g
    g.build()
    from paper_2310_19840_gb300 import sbi as s
    return s


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def maxrel(a, b):
    """Largest pointwise error relative to the largest |b|."""
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


# largest pointwise error of V relative to max|V| after one evaluation
TOL_MAX = {0: 1e-5, 1: 1e-11}


def _case(nx, ny, Lx, Ly, h0, variable, seed, amp_eta=0.04, amp_phi=0.3, amp_delta=0.1):
    grid = O.Grid(nx, ny, Lx, Ly if ny > 1 else 1.0)
    delta = W.random_field(nx, ny, seed, amplitude=amp_delta * h0) if variable else None
    pb = O.Problem(grid, 9.81, h0, delta=delta)
    eta = O.project(pb, W.random_field(nx, ny, seed + 1, amplitude=amp_eta))
    phi = O.project(pb, W.random_field(nx, ny, seed + 2, amplitude=amp_phi))
    return grid, pb, eta, phi


CASES = [
    # nx, ny, Lx, Ly, h0, variable
    (64, 1, 6.0, 1.0, 0.7, False),
    (256, 1, 12.0, 1.0, 0.5, True),
    (32, 16, 4.0, 3.0, 0.6, False),
    (64, 32, 6.0, 4.0, 0.8, True),
    (128, 8, 8.0, 1.5, 1.0, True),
    (16, 64, 2.0, 5.0, 0.9, False),
]


@pytest.mark.parametrize("prec", [1, 0])
@pytest.mark.parametrize("case", CASES)
def test_vertical_velocity_matches_oracle(sbi, prec, case):
    nx, ny, Lx, Ly, h0, variable = case
    grid, pb, eta, phi = _case(nx, ny, Lx, Ly, h0, variable, seed=100 + nx + ny)
    depth = (h0 - pb.delta) if variable else None
    ctx = sbi.Context([(nx, ny, Lx, Ly)], 9.81, [depth], h0=h0, precision=prec)
    ctx.set_state(0, eta, phi)
    V = ctx.vertical_velocity(0)
    Vo = O.vertical_velocity(eta, phi, pb.delta, h0, grid)
    assert rel(V, Vo) < TOL[prec]


@pytest.mark.parametrize("order", [1, 2, 3, 4, 5, 6])
def test_every_order(sbi, order):
    nx, ny, Lx, Ly, h0 = 64, 16, 5.0, 3.0, 0.6
    grid, pb, eta, phi = _case(nx, ny, Lx, Ly, h0, True, seed=7)
    ctx = sbi.Context([(nx, ny, Lx, Ly)], 9.81, [h0 - pb.delta], h0=h0, precision=1, order=order)
    ctx.set_state(0, eta, phi)
    V = ctx.vertical_velocity(0)
    Vo = O.vertical_velocity(eta, phi, pb.delta, h0, grid, order=order)
    assert rel(V, Vo) < TOL[1]


def test_deep_water(sbi):
    nx, ny, L = 64, 64, 10.0
    grid = O.Grid(nx, ny, L, L)
    pb = O.Problem(grid, 9.81, np.inf)
    eta = O.project(pb, W.random_field(nx, ny, 5, amplitude=0.1))
    phi = O.project(pb, W.random_field(nx, ny, 6, amplitude=0.5))
    for prec in (1, 0):
        ctx = sbi.Context([(nx, ny, L, L)], 9.81, None, h0=np.inf, precision=prec)
        ctx.set_state(0, eta, phi)
        assert rel(ctx.vertical_velocity(0), O.vertical_velocity(eta, phi, None, np.inf, grid)) < TOL[prec]


@pytest.mark.parametrize("prec", [1, 0])
def test_rk4_steps_match_oracle(sbi, prec):
    nx, ny, Lx, Ly, h0 = 64, 32, 6.0, 4.0, 0.8
    grid, pb, eta, phi = _case(nx, ny, Lx, Ly, h0, True, seed=40)
    ctx = sbi.Context([(nx, ny, Lx, Ly)], 9.81, [h0 - pb.delta], h0=h0, precision=prec)
    ctx.set_state(0, eta, phi)
    ctx.step(0.02, 3)
    e, p = ctx.get_state(0)
    eo, po = O.step(pb, eta, phi, 0.02, 3)
    assert rel(e, eo) < TOL[prec] and rel(p, po) < TOL[prec]


def test_sponge_matches_oracle(sbi):
    wl = W.bar_1d(n=512, L=40.0)
    m = wl.members[0]
    grid = O.Grid(m.nx, 1, m.Lx)
    x = np.arange(m.nx) * m.Lx / m.nx
    w = (np.sin(np.pi * x / m.Lx) ** 8).reshape(1, -1)
    pb = O.Problem(grid, wl.gravity, m.h0, delta=m.delta, sponge_w=w, sponge_nu=wl.sponge_nu)
    eta, phi = O.project(pb, m.eta), O.project(pb, m.phi)
    for prec in (1, 0):
        ctx = sbi.Context([(m.nx, 1, m.Lx, 1.0)], wl.gravity, [m.h0 - m.delta], h0=m.h0,
                          precision=prec, sponge_w=w, sponge_nu=wl.sponge_nu)
        ctx.set_state(0, eta, phi)
        ctx.step(wl.dt, 4)
        e, p = ctx.get_state(0)
        eo, po = O.step(pb, eta, phi, wl.dt, 4)
        assert rel(e, eo) < TOL[prec] and rel(p, po) < TOL[prec]


def test_filter_matches_oracle(sbi):
    nx, ny, L = 64, 64, 8.0
    grid = O.Grid(nx, ny, L, L)
    kref = 2 * np.pi / L * 3
    pb = O.Problem(grid, 9.81, 1.0, filt_beta1=2.0, filt_beta2=8.0, k_ref=kref)
    eta = O.project(pb, W.random_field(nx, ny, 50, amplitude=0.05))
    phi = O.project(pb, W.random_field(nx, ny, 51, amplitude=0.3))
    for prec in (1, 0):
        ctx = sbi.Context([(nx, ny, L, L)], 9.81, None, h0=1.0, precision=prec,
                          filt_beta1=2.0, filt_beta2=8.0, k_ref=kref)
        ctx.set_state(0, eta, phi)
        ctx.step(0.02, 2)
        e, p = ctx.get_state(0)
        eo, po = O.step(pb, eta, phi, 0.02, 2)
        assert rel(e, eo) < TOL[prec] and rel(p, po) < TOL[prec]


@pytest.mark.parametrize("prec", [0, 1])
def test_autotuned_block_shapes_give_identical_results(sbi, prec):
    # The autotuner only changes rows / columns per block: a context with it
    # and one without produce the same bits after diagnostics and steps, and
    # it reports one choice per distinct pass shape.
    specs = [(256, 128, 12.0, 8.0), (512, 64, 20.0, 4.0)]
    depth = [0.6 - W.random_field(256, 128, 71, amplitude=0.05), None]
    out = {}
    for tune in (0, 1):
        ctx = sbi.Context(specs, 9.81, depth, h0=0.6, precision=prec, autotune=tune,
                          filt_beta1=8.0, filt_beta2=30.0, k_ref=1.0)
        for i, (nx, ny, Lx, Ly) in enumerate(specs):
            ctx.set_state(i, W.random_field(nx, ny, 72 + i, amplitude=0.03),
                          W.random_field(nx, ny, 74 + i, amplitude=0.2))
        V = ctx.vertical_velocity(0)
        ctx.step(0.01, 3)
        out[tune] = (V, ctx.get_state(0), ctx.get_state(1))
        if tune:
            rep = ctx.autotune_report().strip().splitlines()
            assert any(": rpc " in ln for ln in rep) and any(": cpb " in ln for ln in rep)
            assert len(set(ln.split(":")[0] for ln in rep)) == len(rep)
        else:
            assert ctx.autotune_report() == ""
    assert np.array_equal(out[0][0], out[1][0])
    for m in (1, 2):
        for f in (0, 1):
            assert np.array_equal(out[0][m][f], out[1][m][f])


@pytest.mark.parametrize("buf", ["numpy", "pinned", "device"])
@pytest.mark.parametrize("dealias", [0, 1])
def test_batch_state_calls_equal_per_member_calls(sbi, dealias, buf):
    # sbi_set_state_all / sbi_get_state_all on members of interleaved sizes
    # give the same bits as one sbi_set_state / sbi_get_state per member, from
    # pageable host buffers (copied through staging), pinned host buffers and
    # device buffers (read and written by the conversion kernels directly).
    import torch
    specs = [(64, 32, 6.0, 4.0), (32, 16, 3.0, 2.0), (64, 32, 6.0, 4.0), (128, 1, 9.0, 1.0)]
    eta = [W.random_field(nx, ny, 80 + i, amplitude=0.03).ravel() for i, (nx, ny, _, _) in enumerate(specs)]
    phi = [W.random_field(nx, ny, 90 + i, amplitude=0.2).ravel() for i, (nx, ny, _, _) in enumerate(specs)]
    a = sbi.Context(specs, 9.81, None, h0=0.7, precision=0, set_state_dealias=dealias)
    b = sbi.Context(specs, 9.81, None, h0=0.7, precision=0, set_state_dealias=dealias)
    for i in range(len(specs)):
        a.set_state(i, eta[i], phi[i])

    def wrap(x):
        if buf == "numpy":
            return x
        t = torch.from_numpy(np.ascontiguousarray(x))
        return t.pin_memory() if buf == "pinned" else t.cuda()

    b.set_state_all(wrap(np.concatenate(eta)), wrap(np.concatenate(phi)))
    for ctx in (a, b):
        ctx.step(0.01, 2)
    ea, pa = a.get_state_all()
    if buf != "numpy":
        eb, pb_ = wrap(np.zeros_like(ea)), wrap(np.zeros_like(pa))
        b.get_state_all(eb, pb_)
        torch.cuda.synchronize()
        assert np.array_equal(eb.cpu().numpy(), ea) and np.array_equal(pb_.cpu().numpy(), pa)
    for i in range(len(specs)):
        e1, p1 = a.get_state(i)
        e2, p2 = b.get_state(i)
        assert np.array_equal(e1, e2) and np.array_equal(p1, p2)
        assert np.array_equal(a.split(ea)[i], e1) and np.array_equal(a.split(pa)[i], p1)


def test_batch_of_uneven_grids_equals_single(sbi):
    specs = [(64, 32, 6.0, 4.0), (32, 16, 3.0, 2.0), (64, 32, 6.0, 4.0), (128, 1, 9.0, 1.0)]
    states = []
    for i, (nx, ny, Lx, Ly) in enumerate(specs):
        grid, pb, eta, phi = _case(nx, ny, Lx, Ly, 0.7, False, seed=60 + 3 * i)
        states.append((eta, phi))
    batch = sbi.Context(specs, 9.81, None, h0=0.7, precision=0)
    for i, (e, p) in enumerate(states):
        batch.set_state(i, e, p)
    batch.step(0.01, 2)
    for i, spec in enumerate(specs):
        single = sbi.Context([spec], 9.81, None, h0=0.7, precision=0)
        single.set_state(0, *states[i])
        single.step(0.01, 2)
        eb, pb_ = batch.get_state(i)
        es, ps = single.get_state(0)
        assert np.array_equal(eb, es) and np.array_equal(pb_, ps)


@pytest.mark.parametrize("prec", [1, 0])
def test_invariants_match_oracle(sbi, prec):
    nx, ny, Lx, Ly, h0 = 64, 32, 6.0, 4.0, 0.8
    grid, pb, eta, phi = _case(nx, ny, Lx, Ly, h0, True, seed=70)
    eta = eta + 0.01
    ctx = sbi.Context([(nx, ny, Lx, Ly)], 9.81, [h0 - pb.delta], h0=h0, precision=prec)
    ctx.set_state(0, eta, phi)
    m, e = ctx.invariants(0)
    mo, eo = O.invariants(pb, eta, phi)
    assert abs(m - mo) <= 1e-12 * abs(mo)
    assert abs(e - eo) <= TOL[prec] * abs(eo)


@pytest.mark.parametrize("nx,ny", [(4096, 1), (16, 2048), (4096, 8), (1024, 1024), (512, 512),
                                   (256, 256), (2048, 16), (4096, 2048)])
def test_every_kernel_size_matches_oracle(sbi, nx, ny):
    # Largest and extreme grids (variable depth): each size instantiation of
    # the row and column kernels launches in both precisions and matches the
    # FP64 oracle, in relative L2 and pointwise.  At 4096 x 2048 the FP32 path
    # is compared with the FP64 path instead: the same instantiations meet the
    # oracle on the 4096 x 2048 variable-depth sea (test_gpu_workloads.py).
    # The grid spacing is fixed (0.05 m) so k|delta| stays below ~1 at every
    # size: FP32 round-off is amplified by (k delta)^j / j! in the delta terms.
    # The spectra are spread over the band (as in the wave workloads): with all
    # the energy in the box-scale mode V would be ~k_max/k_1 times smaller
    # than the FP32 round-off of the short modes.
    Lx, Ly, h0 = 0.05 * nx, (0.05 * ny if ny > 1 else 1.0), 0.6
    delta = W.random_field(nx, ny, 3, amplitude=0.06, band=0.2, slope=0.5)
    eta = W.random_field(nx, ny, 4, amplitude=0.03, band=0.2, slope=0.5)
    phi = W.random_field(nx, ny, 5, amplitude=0.2, band=0.2, slope=0.5)
    out = {}
    for prec in (1, 0):
        ctx = sbi.Context([(nx, ny, Lx, Ly)], 9.81, [h0 - delta], h0=h0, precision=prec,
                          set_state_dealias=0)
        ctx.set_state(0, eta, phi)
        out[prec] = ctx.vertical_velocity(0)
        ctx.close()
    assert np.all(np.isfinite(out[1]))
    if nx * ny > 2 ** 22:
        assert rel(out[0], out[1]) < TOL[0] and maxrel(out[0], out[1]) < TOL_MAX[0]
        return
    grid = O.Grid(nx, ny, Lx, Ly)
    Vo = O.vertical_velocity(eta, phi, delta, h0, grid)
    for prec in (1, 0):
        print(f"{nx}x{ny} prec {prec}: rel {rel(out[prec], Vo):.2e} max {maxrel(out[prec], Vo):.2e}")
        assert rel(out[prec], Vo) < TOL[prec] and maxrel(out[prec], Vo) < TOL_MAX[prec], prec


@pytest.mark.parametrize("prec", [1, 0])
@pytest.mark.parametrize("case", [(256, 1, 12.0, 1.0, 0.5, True), (64, 32, 6.0, 4.0, 0.8, True),
                                  (128, 64, 8.0, 4.0, math.inf, False)])
def test_eulerian_w_matches_oracle(sbi, prec, case):
    # sbi_vertical_velocity(..., eulerian_w = 1): the Eulerian vertical
    # velocity at the surface w = (V + grad eta . grad phi~) / (1 + |grad eta|^2)
    # (Sec. 2.2, the definition of V through the normal derivative), built
    # here from the oracle's V and the spectral gradients of the dealiased
    # state.
    nx, ny, Lx, Ly, h0, variable = case
    grid, pb, eta, phi = _case(nx, ny, Lx, Ly, h0, variable, seed=300 + nx)
    depth = (h0 - pb.delta) if variable else None
    ctx = sbi.Context([(nx, ny, Lx, Ly)], 9.81, [depth], h0=h0, precision=prec)
    ctx.set_state(0, eta, phi)
    w = ctx.vertical_velocity(0, eulerian_w=True)
    V = ctx.vertical_velocity(0)
    Vo = O.vertical_velocity(eta, phi, pb.delta, h0, grid)
    KX, KY, _ = O.wavenumbers(grid)
    mask = O.dealias_mask(grid)
    ge = O.gradient(mask * O.fft(eta), KX, KY, grid.dim)
    gp = O.gradient(mask * O.fft(phi), KX, KY, grid.dim)
    dot = sum(a * b for a, b in zip(ge, gp))
    ge2 = sum(a * a for a in ge)
    wo = (Vo + dot) / (1.0 + ge2)
    assert not np.allclose(wo, Vo)          # the slope terms matter for this state
    assert rel(w, wo) < TOL[prec] and maxrel(w, wo) < TOL_MAX[prec]
    assert rel(V, Vo) < TOL[prec]             # the V output is unchanged by the w call


def _ratios(eta, phi, delta, h0, grid):
    """||F{V_l}|| / ||F{V_1 + .. + V_l}|| per order l >= 2 (oracle)."""
    _, terms = O.vertical_velocity(eta, phi, delta, h0, grid, return_terms=True)
    out, tot = [], np.zeros_like(np.fft.fft2(terms["V"][0]))
    for l, Vl in enumerate(terms["V"], start=1):
        Vh = np.fft.fft2(Vl)
        tot = tot + Vh
        if l >= 2:
            out.append(np.sqrt(np.sum(np.abs(Vh) ** 2) / np.sum(np.abs(tot) ** 2)))
    return out


@pytest.mark.parametrize("prec", [1, 0])
def test_adaptive_order_matches_oracle(sbi, prec):
    # Reading R9: stop at the first l with ||F{V_l}|| <= tol ||sum F{V_m}||.  The
    # tolerance sits midway (geometrically) between two consecutive ratios so
    # that round-off cannot flip the decision.
    nx, ny, Lx, Ly, h0 = 64, 32, 6.0, 4.0, 0.8
    grid, pb, eta, phi = _case(nx, ny, Lx, Ly, h0, True, seed=90, amp_eta=0.06)
    r = _ratios(eta, phi, pb.delta, h0, grid)
    L = 4                                   # stop at order 4
    tol = math.sqrt(r[L - 2] * r[L - 3])    # r[i] belongs to order i + 2
    assert r[L - 2] < tol < r[L - 3]
    ctx = sbi.Context([(nx, ny, Lx, Ly)], 9.81, [h0 - pb.delta], h0=h0, precision=prec,
                      adapt_tol=tol)
    ctx.set_state(0, eta, phi)
    V = ctx.vertical_velocity(0)
    assert ctx.orders_used(0) == L
    Vo = O.vertical_velocity(eta, phi, pb.delta, h0, grid, tol=tol)
    assert rel(V, Vo) < TOL[prec]
    # the RK4 step uses the adaptive order in every stage
    pb.adapt_tol = tol
    ctx.step(0.02, 1)
    e, p = ctx.get_state(0)
    eo, po = O.step(pb, eta, phi, 0.02, 1)
    assert rel(e, eo) < TOL[prec] and rel(p, po) < TOL[prec]


def test_adaptive_order_not_met_is_reported(sbi):
    nx, ny, Lx, Ly, h0 = 32, 16, 4.0, 3.0, 0.6
    grid, pb, eta, phi = _case(nx, ny, Lx, Ly, h0, False, seed=95, amp_eta=0.08)
    ctx = sbi.Context([(nx, ny, Lx, Ly)], 9.81, None, h0=h0, precision=1, adapt_tol=1e-30)
    ctx.set_state(0, eta, phi)
    with pytest.raises(sbi.SbiError) as ei:
        ctx.vertical_velocity(0)
    assert ei.value.code == sbi.SBI_ENOTCONVERGED
    assert ctx.orders_used(0) == 7


LAWSON_CASES = {
    # name: (nx, ny, Lx, Ly, h0, variable, filter, sponge)
    "flat2d": (64, 32, 6.0, 4.0, 0.8, False, False, False),
    "var1d": (256, 1, 12.0, 1.0, 0.5, True, False, False),
    "var2d_filter_sponge": (64, 32, 6.0, 4.0, 0.7, True, True, True),
}


@pytest.mark.parametrize("prec,tol", [(1, 1e-10), (0, 1e-5)])
@pytest.mark.parametrize("name", list(LAWSON_CASES))
def test_lawson_steps_match_oracle(sbi, prec, tol, name):
    # Integrating-factor (Lawson) RK4 steps on the GPU path against the oracle.
    nx, ny, Lx, Ly, h0, variable, filt, sponge = LAWSON_CASES[name]
    grid, pb, eta, phi = _case(nx, ny, Lx, Ly, h0, variable, seed=120)
    kw = {}
    if filt:
        pb.filt_beta1, pb.filt_beta2, pb.k_ref = 8.0, 30.0, 1.0
        kw.update(filt_beta1=8.0, filt_beta2=30.0, k_ref=1.0)
    if sponge:
        x = np.arange(nx) * Lx / nx
        w = np.broadcast_to(np.exp(-((x - 0.75 * Lx) / (0.1 * Lx)) ** 2), (ny, nx)).copy()
        pb.sponge_w, pb.sponge_nu = w, 2.0
        kw.update(sponge_w=w, sponge_nu=2.0)
    pb.integrator = "lawson"
    eta, phi = O.project(pb, eta), O.project(pb, phi)
    depth = [h0 - pb.delta] if variable else None
    ctx = sbi.Context([(nx, ny, Lx, Ly)], 9.81, depth, h0=h0, precision=prec,
                      integrator=sbi.SBI_LAWSON_RK4, **kw)
    ctx.set_state(0, eta, phi)
    ctx.step(0.03, 3)
    e, p = ctx.get_state(0)
    eo, po = O.step(pb, eta, phi, 0.03, 3)
    assert rel(e, eo) < tol and rel(p, po) < tol


@pytest.mark.parametrize("prec,tol", [(1, 1e-6), (0, 2e-5)])
def test_lawson_exact_linear_propagation(sbi, prec, tol):
    # One integrating-factor step of w dt = 2.5 carries an infinitesimal
    # travelling wave exactly (order 1), where classical RK4 cannot: the
    # closed form holds to the size of the nonlinear terms, k a ~ 5e-8, and
    # the FP64 path equals the oracle to round-off.
    g, a, nx, L, m, h0 = 9.81, 1e-8, 64, 4.0, 3, 0.4
    k = 2 * math.pi * m / L
    w = math.sqrt(g * k * math.tanh(k * h0))
    x = np.arange(nx) * L / nx
    ctx = sbi.Context([(nx, 1, L, 1.0)], g, None, h0=h0, order=1, precision=prec,
                      integrator=sbi.SBI_LAWSON_RK4)
    ctx.set_state(0, a * np.cos(k * x), (g * a / w) * np.sin(k * x))
    ctx.step(2.5 / w, 1)
    e, p = ctx.get_state(0)
    assert rel(e, a * np.cos(k * x - 2.5)) < tol
    assert rel(p, (g * a / w) * np.sin(k * x - 2.5)) < tol
    if prec == 1:
        pb = O.Problem(O.Grid(nx, 1, L), g, h0, order=1, integrator="lawson")
        eo, po = O.step(pb, a * np.cos(k * x), (g * a / w) * np.sin(k * x), 2.5 / w, 1)
        assert rel(e, eo) < 1e-10 and rel(p, po) < 1e-10


@pytest.mark.parametrize("prec,tol", [(1, 1e-10), (0, 1e-5)])
def test_lawson_with_wavemaker_stage_times(sbi, prec, tol):
    nx, Lx, h0 = 256, 16.0, 0.5
    grid = O.Grid(nx, 1, Lx)
    amp, omega, phase = [0.005], [4.0], [0.4]
    wm = O.Wavemaker(np.array(amp), np.array(omega), np.array(phase), 0.0)
    pb = O.Problem(grid, 9.81, h0, wavemaker=wm, integrator="lawson")
    eta = O.project(pb, W.random_field(nx, 1, 130, amplitude=0.01))
    phi = O.project(pb, W.random_field(nx, 1, 131, amplitude=0.05))
    ctx = sbi.Context([(nx, 1, Lx, 1.0)], 9.81, None, h0=h0, precision=prec,
                      integrator=sbi.SBI_LAWSON_RK4)
    ctx.set_wavemaker(amp, omega, phase)
    ctx.set_time(1.1)
    ctx.set_state(0, eta, phi)
    ctx.step(0.04, 5)
    e, p = ctx.get_state(0)
    eo, po = O.step(pb, eta, phi, 0.04, 5, t0=1.1)
    assert rel(e, eo) < tol and rel(p, po) < tol


def test_lawson_option_validation(sbi):
    with pytest.raises(sbi.SbiError) as ei:
        sbi.Context([(32, 1, 3.0, 1.0)], 9.81, None, h0=1.0, integrator=7)
    assert ei.value.code == sbi.SBI_EINVAL
    with pytest.raises(sbi.SbiError) as ei:
        sbi.Context([(32, 1, 3.0, 1.0)], 9.81, None, h0=1.0, integrator=sbi.SBI_LAWSON_RK4,
                    adapt_tol=1e-3)
    assert ei.value.code == sbi.SBI_EINVAL


HOS_CASES = [
    # nx, ny, Lx, Ly, h0, order
    (64, 32, 6.0, 4.0, 0.8, 7),
    (64, 32, 6.0, 4.0, 0.8, 3),
    (128, 1, 9.0, 1.0, 0.5, 7),
    (64, 32, 6.0, 4.0, math.inf, 5),
    (32, 16, 3.0, 2.0, 0.6, 1),
]


@pytest.mark.parametrize("prec", [1, 0])
@pytest.mark.parametrize("case", HOS_CASES)
def test_hos_diagnostic_matches_oracle(sbi, prec, case):
    # The HOS perturbation expansion (flat bottom) on the GPU path against the
    # oracle's, V after one evaluation.
    nx, ny, Lx, Ly, h0, order = case
    grid, pb, eta, phi = _case(nx, ny, Lx, Ly, h0 if math.isfinite(h0) else 1.0, False, seed=140)
    ctx = sbi.Context([(nx, ny, Lx, Ly)], 9.81, None, h0=h0, order=order, precision=prec,
                      diagnostic=sbi.SBI_DIAG_HOS)
    ctx.set_state(0, eta, phi)
    V = ctx.vertical_velocity(0)
    Vo, _ = O.hos_surface_velocity(eta, phi, h0, grid, order=order)
    assert rel(V, Vo) < TOL[prec]


@pytest.mark.parametrize("prec,tol", [(1, 1e-10), (0, 1e-5)])
@pytest.mark.parametrize("integrator", ["rk4", "lawson"])
def test_hos_steps_match_oracle(sbi, prec, tol, integrator):
    nx, ny, Lx, Ly, h0 = 64, 32, 6.0, 4.0, 0.8
    grid, pb, eta, phi = _case(nx, ny, Lx, Ly, h0, False, seed=150)
    pb.diagnostic, pb.integrator = "hos", integrator
    ctx = sbi.Context([(nx, ny, Lx, Ly)], 9.81, None, h0=h0, precision=prec,
                      diagnostic=sbi.SBI_DIAG_HOS,
                      integrator=sbi.SBI_LAWSON_RK4 if integrator == "lawson" else sbi.SBI_RK4)
    ctx.set_state(0, eta, phi)
    ctx.step(0.03, 3)
    e, p = ctx.get_state(0)
    eo, po = O.step(pb, eta, phi, 0.03, 3)
    assert rel(e, eo) < tol and rel(p, po) < tol


@pytest.mark.parametrize("prec", [1, 0])
@pytest.mark.parametrize("diag", ["esbi", "hos"])
@pytest.mark.parametrize("order", [4, 7])
def test_steep_stokes_wave(sbi, prec, diag, order):
    # A steep steady Stokes wave (kH/2 = 0.35, deep water, one wavelength on
    # 64 points, 16 alias-free modes), the comparison of the section on ESBI
    # and HOS: the GPU V against the oracle's, and against the exact V = -c eta_x
    # of a wave of permanent form (Fourier-approximation solution).
    from oracle import steady_wave as SW
    n, L = 64, 2 * math.pi
    w = SW.solve(k=1.0, H=0.7, g=9.81)
    grid = O.Grid(n, 1, L)
    pb = O.Problem(grid, 9.81, math.inf)
    x = np.arange(n) * L / n
    eta, phi = O.project(pb, w.eta(x)), O.project(pb, w.surface_potential(x))
    ctx = sbi.Context([(n, 1, L, 1.0)], 9.81, None, h0=math.inf, order=order, precision=prec,
                      diagnostic=sbi.SBI_DIAG_HOS if diag == "hos" else sbi.SBI_DIAG_ESBI)
    ctx.set_state(0, eta, phi)
    V = np.asarray(ctx.vertical_velocity(0)).ravel()
    if diag == "hos":
        Vo = O.hos_surface_velocity(eta, phi, math.inf, grid, order=order)[0].ravel()
    else:
        Vo = O.vertical_velocity(eta, phi, None, math.inf, grid, order=order).ravel()
    assert rel(V, Vo) < TOL[prec]
    Vx = w.vertical_velocity(x)
    err = np.max(np.abs(V - Vx)) / np.max(np.abs(Vx))
    err_o = np.max(np.abs(Vo - Vx)) / np.max(np.abs(Vx))
    assert abs(err - err_o) < 1e-4 * (1.0 if prec == 0 else 1e-4)
    if order == 7 or diag == "esbi":
        assert err < 5e-3       # within 0.5 %
    else:
        assert err > 5e-3       # HOS at order 4 is not


@pytest.mark.parametrize("prec,tol", [(1, 1e-10), (0, 1e-5)])
@pytest.mark.parametrize("depth,eps", [(math.inf, 0.3), (2.0, 0.2)])
def test_steady_stokes_wave_translates(sbi, prec, tol, depth, eps):
    # A steady Stokes wave stepped a quarter period on the GPU: the state
    # matches the oracle's and the exactly translated wave (phi~ up to its
    # uniform Bernoulli drift).
    from oracle import steady_wave as SW
    n, L, g = 64, 2 * math.pi, 9.81
    w = SW.solve(k=1.0, H=2 * eps, depth=depth, g=g)
    grid = O.Grid(n, 1, L)
    pb = O.Problem(grid, g, depth)
    x = np.arange(n) * L / n
    eta0, phi0 = O.project(pb, w.eta(x)), O.project(pb, w.surface_potential(x))
    dt = L / w.c / 64
    ctx = sbi.Context([(n, 1, L, 1.0)], g, None, h0=depth, precision=prec)
    ctx.set_state(0, eta0, phi0)
    ctx.step(dt, 16)
    e, p = (np.ravel(a) for a in ctx.get_state(0))
    eo, po = (np.ravel(a) for a in O.step(pb, eta0, phi0, dt, 16))
    assert rel(e, eo) < tol and rel(p, po) < tol
    t = 16 * dt
    ex = np.ravel(O.project(pb, w.eta(x - w.c * t)))
    px = np.ravel(O.project(pb, w.surface_potential(x - w.c * t)))
    assert np.max(np.abs(e - ex)) < 2e-4 * np.max(np.abs(ex))
    d = (p - p.mean()) - (px - px.mean())
    assert np.max(np.abs(d)) < 2e-4 * np.max(np.abs(px - px.mean()))


def _implicit_case(depth, eps, n=64):
    from oracle import steady_wave as SW
    L = 2 * math.pi
    w = SW.solve(k=1.0, H=2 * eps, depth=depth, g=9.81)
    grid = O.Grid(n, 1, L)
    pb = O.Problem(grid, 9.81, depth)
    x = np.arange(n) * L / n
    return grid, O.project(pb, w.eta(x)), O.project(pb, w.surface_potential(x))


@pytest.mark.parametrize("prec,tol", [(1, 1e-10), (0, 1e-5)])
@pytest.mark.parametrize("depth,eps,order", [(math.inf, 0.1, 7), (2.0, 0.1, 7), (1.0, 0.05, 4)])
def test_implicit_iteration_matches_oracle(sbi, prec, tol, depth, eps, order):
    # The implicit form of Appendix A (flat bottom) by fixed-point iteration on
    # a steady wave: V and the increment of every iteration against the oracle.
    grid, eta, phi = _implicit_case(depth, eps)
    its = 4
    ctx = sbi.Context([(grid.nx, 1, grid.Lx, 1.0)], 9.81, None, h0=depth, order=order, precision=prec)
    ctx.set_state(0, eta, phi)
    V, inc = ctx.vertical_velocity_implicit(0, its)
    Vo, _, inco = O.implicit_vertical_velocity(eta, phi, depth, grid, order=order, tol=0.0, maxit=its)
    assert rel(V, Vo) < tol
    assert np.all(np.abs(inc - np.array(inco)) < 1e3 * tol * np.array(inco) + tol)
    assert inc[-1] < 1e-3 * inc[0]      # converging


@pytest.mark.parametrize("prec,tol", [(1, 1e-10), (0, 1e-5)])
def test_implicit_iteration_2d_matches_oracle(sbi, prec, tol):
    nx, ny, Lx, Ly, h0 = 64, 32, 6.0, 4.0, 0.8
    grid, pb, eta, phi = _case(nx, ny, Lx, Ly, h0, False, seed=170)
    ctx = sbi.Context([(nx, ny, Lx, Ly)], 9.81, None, h0=h0, precision=prec)
    ctx.set_state(0, eta, phi)
    V, inc = ctx.vertical_velocity_implicit(0, 3)
    Vo, _, inco = O.implicit_vertical_velocity(eta, phi, h0, grid, tol=0.0, maxit=3)
    assert rel(V, Vo) < tol
    assert abs(inc[0] - inco[0]) < 1e3 * tol * inco[0]


def test_implicit_iteration_diverges_like_the_oracle(sbi):
    # kH/2 = 0.3: the fixed-point map is expansive; the GPU iterates follow
    # the oracle's (FP64) while the increments grow
    grid, eta, phi = _implicit_case(math.inf, 0.3)
    ctx = sbi.Context([(grid.nx, 1, grid.Lx, 1.0)], 9.81, None, h0=math.inf, precision=1)
    ctx.set_state(0, eta, phi)
    V, inc = ctx.vertical_velocity_implicit(0, 4)
    Vo, _, inco = O.implicit_vertical_velocity(eta, phi, math.inf, grid, tol=0.0, maxit=4)
    assert rel(V, Vo) < 1e-8
    assert np.all(np.abs(inc - np.array(inco)) < 1e-6 * np.array(inco))
    assert inc[-1] > 0.1 and inc[-1] > inc[0]


@pytest.mark.parametrize("prec,tol", [(1, 1e-10), (0, 1e-5)])
def test_implicit_iteration_variable_bottom_1d(sbi, prec, tol):
    # Appendices A and B together over a bump (delta up to 0.3 h0): V and the
    # increment of every fixed-point iteration against the oracle's
    n, L, h0, g = 64, 4 * math.pi, 1.0, 9.81
    grid = O.Grid(n, 1, L)
    x = np.arange(n) * L / n
    delta = 0.3 * h0 * np.exp(-((x - L / 2) / 1.5) ** 2)
    pb = O.Problem(grid, g, h0, delta=delta)
    k = 4 * math.pi / L
    a = 0.1 / k
    om = math.sqrt(g * k * math.tanh(k * h0))
    eta = O.project(pb, a * np.cos(k * x))
    phi = O.project(pb, a * g / om * np.sin(k * x))
    ctx = sbi.Context([(n, 1, L, 1.0)], g, [h0 - delta], h0=h0, precision=prec)
    ctx.set_state(0, eta, phi)
    V, inc = ctx.vertical_velocity_implicit(0, 5)
    Vo, _, inco = O.implicit_vertical_velocity(eta, phi, h0, grid, tol=0.0, maxit=5, delta=delta)
    assert rel(V, Vo) < tol
    assert np.all(np.abs(inc - np.array(inco)) < 1e3 * tol * np.array(inco) + tol)


@pytest.mark.parametrize("prec,tol", [(1, 1e-10), (0, 1e-5)])
def test_implicit_iteration_variable_bottom_2d(sbi, prec, tol):
    nx, ny, Lx, Ly, h0 = 64, 32, 6.0, 4.0, 0.8
    grid, pb, eta, phi = _case(nx, ny, Lx, Ly, h0, True, seed=190)
    ctx = sbi.Context([(nx, ny, Lx, Ly)], 9.81, [h0 - pb.delta], h0=h0, precision=prec)
    ctx.set_state(0, eta, phi)
    V, inc = ctx.vertical_velocity_implicit(0, 3)
    Vo, _, inco = O.implicit_vertical_velocity(eta, phi, h0, grid, tol=0.0, maxit=3, delta=pb.delta)
    assert rel(V, Vo) < tol
    assert abs(inc[0] - inco[0]) < 1e3 * tol * inco[0]


def test_implicit_iteration_validation(sbi):
    flat = sbi.Context([(32, 1, 3.0, 1.0)], 9.81, None, h0=0.7, precision=1)
    for bad in (0, 65):
        with pytest.raises(sbi.SbiError):
            flat.vertical_velocity_implicit(0, bad)


@pytest.mark.parametrize("prec", [1, 0])
@pytest.mark.parametrize("case", [(256, 1, 12.0, 1.0), (64, 32, 6.0, 4.0)])
def test_crest_matches_oracle(sbi, prec, case):
    # sbi_crest against the oracle's crest of the same state (read back)
    nx, ny, Lx, Ly = case
    grid, pb, eta, phi = _case(nx, ny, Lx, Ly, 0.7, False, seed=180)
    ctx = sbi.Context([(nx, ny, Lx, Ly)], 9.81, None, h0=0.7, precision=prec)
    ctx.set_state(0, eta, phi)
    ctx.step(0.01, 2)
    e, _ = ctx.get_state(0)
    x, y, h = ctx.crest(0)
    xo, yo, ho = O.crest(grid, e)
    assert h == ho
    assert abs(x - xo) <= 1e-12 * Lx and abs(y - yo) <= 1e-12 * Ly


@pytest.mark.parametrize("prec", [1, 0])
@pytest.mark.parametrize("spec", [(16, 1, 2.0, 1.0), (16, 8, 2.0, 1.5), (32, 16, 3.0, 2.0)])
def test_degenerate_states(sbi, prec, spec):
    # the smallest grids with degenerate states: rest stays rest exactly; a
    # uniform potential carries no flow (k = 0 has no multiplier, R4); a
    # uniformly raised surface under one potential mode gives the oracle's V
    nx, ny, Lx, Ly = spec
    grid = O.Grid(nx, ny, Lx, Ly)
    h0 = 0.6
    ctx = sbi.Context([spec], 9.81, None, h0=h0, precision=prec)
    z = np.zeros((ny, nx))
    ctx.set_state(0, z, z)
    assert np.all(ctx.vertical_velocity(0) == 0.0)
    ctx.step(0.01, 3)
    e, p = ctx.get_state(0)
    assert np.all(e == 0.0) and np.all(p == 0.0)
    ctx.set_state(0, z, z + 0.7)
    assert np.max(np.abs(ctx.vertical_velocity(0))) < (1e-12 if prec == 1 else 1e-5)
    X, Y = np.meshgrid(np.arange(nx) * Lx / nx, np.arange(ny) * Ly / ny)
    phi = 0.1 * np.cos(2 * np.pi * X / Lx) + (0.05 * np.sin(2 * np.pi * Y / Ly) if ny > 1 else 0.0)
    eta = z + 0.05
    ctx.set_state(0, eta, phi)
    V = ctx.vertical_velocity(0)
    assert rel(V, O.vertical_velocity(eta, phi, None, h0, grid)) < TOL[prec]
    m0, _ = ctx.invariants(0)
    ctx.step(0.01, 3)
    m1, _ = ctx.invariants(0)
    assert abs(m1 - m0) <= 1e-12 * abs(m0) if prec == 1 else abs(m1 - m0) <= 1e-6 * abs(m0)


# Fixed upper limits of the bar of the wide-mask cases.  The oracle's change
# of V under input perturbations of one rounding of the path's precision is
# 2e-6 at alpha = 1/2, 1.5e-5 at 0.75 and 1.6e-3 at 1 for FP32; the GPU path
# rounds at every transform stage, not only at its input, and its FP32 error
# on the steep wave was measured at up to 1.3e-4 (alpha = 0.75) and 2.0e-3
# (alpha = 1), pointwise.  The caps sit about 2.5 times above those.
MASK_BAR_CAP = {0: {1.0 / 3.0: 1e-5, 0.75: 3e-4, 1.0: 5e-3}, 1: {1.0 / 3.0: 1e-12, 0.75: 1e-12, 1.0: 1e-10}}


@pytest.mark.parametrize("prec", [1, 0])
@pytest.mark.parametrize("alpha", [1.0 / 3.0, 0.75, 1.0])
def test_other_mask_widths_match_oracle(sbi, prec, alpha):
    # The dealiasing fraction alias_frac (R5) away from 1/2: the steep wave
    # (ESBI and HOS) and a 2-D variable bottom (ESBI) against the oracle.  A
    # wide mask keeps modes whose order-7 terms amplify round-off.  The bar is
    # the usual one or 50 times the oracle's own change of V under input
    # perturbations at the path's rounding level (the median over five
    # perturbations; the GPU path rounds each value about 50 times in
    # sequence, each rounding amplified like the input's), whichever is
    # larger, but never above a fixed cap per width; the largest pointwise
    # error is held to the same bar, so a single wrong mode cannot hide in the
    # L2 norm.
    grid, eta, phi = _implicit_case(math.inf, 0.3)
    unit = 2.0 ** -24 if prec == 0 else 2.0 ** -53
    for diag in (sbi.SBI_DIAG_ESBI, sbi.SBI_DIAG_HOS):
        ctx = sbi.Context([(grid.nx, 1, grid.Lx, 1.0)], 9.81, None, h0=math.inf, precision=prec,
                          alias_frac=alpha, diagnostic=diag, set_state_dealias=0)
        ctx.set_state(0, eta, phi)
        V = ctx.vertical_velocity(0)
        if diag == sbi.SBI_DIAG_HOS:
            f = lambda e, p: O.hos_surface_velocity(e, p, math.inf, grid, alpha=alpha)[0]
        else:
            f = lambda e, p: O.vertical_velocity(e, p, None, math.inf, grid, alpha=alpha)
        Vo = f(eta, phi)
        conds = []
        for seed in range(210, 215):
            r = np.random.default_rng(seed)
            de = eta * (1 + unit * r.standard_normal(eta.shape))
            dp = phi * (1 + unit * r.standard_normal(phi.shape))
            conds.append(rel(f(de, dp), Vo))
        bar = min(max(TOL[prec], 50.0 * float(np.median(conds))), MASK_BAR_CAP[prec][alpha])
        print(f"alpha {alpha:.3f} diag {diag} prec {prec}: rel {rel(V, Vo):.2e} "
              f"max {maxrel(V, Vo):.2e} bar {bar:.2e}")
        assert rel(V, Vo) < bar and maxrel(V, Vo) < bar
    nx, ny, Lx, Ly, h0 = 64, 32, 6.0, 4.0, 0.8
    g2, pb, e2, p2 = _case(nx, ny, Lx, Ly, h0, True, seed=200)
    ctx = sbi.Context([(nx, ny, Lx, Ly)], 9.81, [h0 - pb.delta], h0=h0, precision=prec, alias_frac=alpha,
                      set_state_dealias=0)
    ctx.set_state(0, e2, p2)
    V2 = ctx.vertical_velocity(0)
    Vo2 = O.vertical_velocity(e2, p2, pb.delta, h0, g2, alpha=alpha)
    assert rel(V2, Vo2) < TOL[prec] and maxrel(V2, Vo2) < TOL_MAX[prec]


def test_hos_option_validation(sbi):
    depth = 0.7 - W.random_field(32, 1, 160, amplitude=0.05)
    with pytest.raises(sbi.SbiError) as ei:
        sbi.Context([(32, 1, 3.0, 1.0)], 9.81, [depth], h0=0.7, diagnostic=sbi.SBI_DIAG_HOS)
    assert ei.value.code == sbi.SBI_EINVAL
    with pytest.raises(sbi.SbiError) as ei:
        sbi.Context([(32, 1, 3.0, 1.0)], 9.81, None, h0=1.0, diagnostic=sbi.SBI_DIAG_HOS, adapt_tol=1e-3)
    assert ei.value.code == sbi.SBI_EINVAL
    with pytest.raises(sbi.SbiError) as ei:
        sbi.Context([(32, 1, 3.0, 1.0)], 9.81, None, h0=1.0, diagnostic=5)
    assert ei.value.code == sbi.SBI_EINVAL


RK45_CASES = {
    "flat2d_filter": (64, 32, 6.0, 4.0, 0.8, False, True),
    "var1d": (256, 1, 12.0, 1.0, 0.5, True, False),
}


@pytest.mark.parametrize("prec,tol", [(1, 1e-10), (0, 1e-5)])
@pytest.mark.parametrize("name", list(RK45_CASES))
def test_rk45_fixed_steps_match_oracle(sbi, prec, tol, name):
    # Fixed steps of the integrating factor with the 5(4) pair (order-5
    # solution) against the oracle.
    nx, ny, Lx, Ly, h0, variable, filt = RK45_CASES[name]
    grid, pb, eta, phi = _case(nx, ny, Lx, Ly, h0, variable, seed=170)
    kw = {}
    if filt:
        pb.filt_beta1, pb.filt_beta2, pb.k_ref = 8.0, 30.0, 1.0
        kw.update(filt_beta1=8.0, filt_beta2=30.0, k_ref=1.0)
    pb.integrator = "rk45"
    eta, phi = O.project(pb, eta), O.project(pb, phi)
    depth = [h0 - pb.delta] if variable else None
    ctx = sbi.Context([(nx, ny, Lx, Ly)], 9.81, depth, h0=h0, precision=prec,
                      integrator=sbi.SBI_IF_RK45, **kw)
    ctx.set_state(0, eta, phi)
    ctx.step(0.04, 3)
    e, p = ctx.get_state(0)
    eo, po = O.step(pb, eta, phi, 0.04, 3)
    assert rel(e, eo) < tol and rel(p, po) < tol


def _rk45_adaptive_case():
    nx, ny, Lx, Ly, h0 = 64, 32, 6.0, 4.0, 0.7
    grid, pb, eta, phi = _case(nx, ny, Lx, Ly, h0, True, seed=180, amp_eta=0.05)
    pb.integrator = "rk45"
    return (nx, ny, Lx, Ly, h0), grid, pb, eta, phi


def test_rk45_adaptive_fp64_follows_the_oracle(sbi):
    # The FP64 path takes the same accepted and rejected steps as the
    # oracle's controller, proposes the same next step and ends in the same
    # state at t_end.
    (nx, ny, Lx, Ly, h0), grid, pb, eta, phi = _rk45_adaptive_case()
    t_end, tol, h = 0.5, 1e-6, 0.2
    eo, po, ho, acc_o, rej_o = O.step_adaptive(pb, eta, phi, 0.0, t_end, tol, h)
    assert rej_o >= 1
    ctx = sbi.Context([(nx, ny, Lx, Ly)], 9.81, [h0 - pb.delta], h0=h0, precision=1,
                      integrator=sbi.SBI_IF_RK45)
    ctx.set_state(0, eta, phi)
    hg, acc, rej = ctx.step_adaptive(t_end, tol, h)
    assert (acc, rej) == (acc_o, rej_o)
    assert abs(hg - ho) < 1e-6 * ho
    assert abs(ctx.get_time() - t_end) < 1e-15
    e, p = ctx.get_state(0)
    assert rel(e, eo) < 1e-9 and rel(p, po) < 1e-9


def test_rk45_adaptive_fp32_reaches_t_end(sbi):
    (nx, ny, Lx, Ly, h0), grid, pb, eta, phi = _rk45_adaptive_case()
    out = {}
    for prec in (1, 0):
        ctx = sbi.Context([(nx, ny, Lx, Ly)], 9.81, [h0 - pb.delta], h0=h0, precision=prec,
                          integrator=sbi.SBI_IF_RK45)
        ctx.set_state(0, eta, phi)
        ctx.step_adaptive(0.5, 1e-6, 0.2)
        assert abs(ctx.get_time() - 0.5) < 1e-15
        out[prec] = ctx.get_state(0)
    assert rel(out[0][0], out[1][0]) < 1e-5 and rel(out[0][1], out[1][1]) < 1e-5


def test_rk45_option_validation(sbi):
    ctx = sbi.Context([(32, 1, 3.0, 1.0)], 9.81, None, h0=1.0, integrator=sbi.SBI_IF_RK45)
    with pytest.raises(sbi.SbiError) as ei:
        ctx.set_wavemaker([0.01], [3.0], [0.0])
    assert ei.value.code == sbi.SBI_EINVAL
    with pytest.raises(sbi.SbiError) as ei:
        ctx.step_adaptive(1.0, -1.0, 0.1)
    assert ei.value.code == sbi.SBI_EINVAL
    plain = sbi.Context([(32, 1, 3.0, 1.0)], 9.81, None, h0=1.0)
    with pytest.raises(sbi.SbiError) as ei:
        plain.step_adaptive(1.0, 1e-6, 0.1)
    assert ei.value.code == sbi.SBI_EINVAL
