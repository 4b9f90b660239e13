"""GPU checks on the workloads at their full sizes, in the launch configuration
the benchmark uses, plus failure detection and checkpoint/restart.

Full-size outputs are compared with the oracle element by element: the 1-D
grids, the 512^2 Stokes wave, the edge members of every graph branch of the
96-member batch, and V of the 4096 x 2048 variable-depth sea (one oracle
evaluation, about a minute of CPU time).  Each comparison bounds the relative
L2 error and the largest pointwise error relative to max|V| (``maxrel``), so
that one wrong row or block tail cannot hide in the L2 norm of a large field.
For the 4096 x 2048 grid a few properties that hold at any size are checked as
well: equivariance under a shift by one grid cell, linearity of V in phi~ and
exact mass conservation.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import sbi_oracle as O

pytestmark = pytest.mark.gpu


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


# V after one evaluation: relative L2 (the stated tolerance) and the largest
# pointwise error relative to max|V|, per precision (SBI_FP32 = 0, SBI_FP64 = 1)
TOL_L2 = {0: 1e-5, 1: 1e-12}
TOL_MAX = {0: 1e-5, 1: 1e-11}


def problem_of(wl, m):
    g = O.Grid(m.nx, m.ny, m.Lx, m.Ly if m.ny > 1 else 1.0)
    wm = None
    if wl.wavemaker:
        wm = O.Wavemaker(np.array(wl.wavemaker["amp"]), np.array(wl.wavemaker["omega"]),
                         np.array(wl.wavemaker["phase"]), wl.wavemaker["x0"])
    return O.Problem(g, wl.gravity, m.h0, delta=m.delta, order=wl.order, alpha=wl.alpha,
                     sponge_w=wl.sponge_w, sponge_nu=wl.sponge_nu, filt_beta1=wl.filt_beta1,
                     filt_beta2=wl.filt_beta2, k_ref=wl.k_ref, wavemaker=wm)


def context_of(sbi, wl, members, prec, **kw):
    ms = [wl.members[i] for i in members]
    grids = [(m.nx, m.ny, m.Lx, m.Ly) for m in ms]
    depths = [(m.h0 - m.delta) if m.delta is not None else None for m in ms]
    ctx = sbi.Context(grids, wl.gravity, depths, h0=ms[0].h0, order=wl.order,
                      alias_frac=wl.alpha, precision=prec, filt_beta1=wl.filt_beta1,
                      filt_beta2=wl.filt_beta2, k_ref=wl.k_ref, sponge_w=wl.sponge_w,
                      sponge_nu=wl.sponge_nu, **kw)
    if wl.wavemaker:
        ctx.set_wavemaker(wl.wavemaker["amp"], wl.wavemaker["omega"], wl.wavemaker["phase"],
                          wl.wavemaker["x0"])
    return ctx


def test_solitary_wave_run_energy_and_speed(sbi):
    # The 1-D solitary wave (N=256, h=1, a/h=0.3), FP64 GPU path over 400 steps:
    # energy conserved to 1e-4 (Sec. 3.1 reports ~1e-5), crest speed within 3% of
    # sqrt(g(h+a)), and the state equal to the oracle's to 1e-9.
    wl = W.solitary_1d()
    m = wl.members[0]
    pb = problem_of(wl, m)
    eta, phi = O.project(pb, m.eta), O.project(pb, m.phi)
    ctx = context_of(sbi, wl, [0], 1)
    ctx.set_state(0, eta, phi)
    _, E0 = ctx.invariants(0)
    x0, _, _ = ctx.crest(0)
    ctx.step(wl.dt, 400)
    e, p = ctx.get_state(0)
    _, E1 = ctx.invariants(0)
    assert abs(E1 - E0) / E0 < 1e-4
    eo, po = O.step(pb, eta, phi, wl.dt, 400)
    assert rel(e, eo) < 1e-9 and rel(p, po) < 1e-9
    # crest speed from the library's crest (sbi_crest), against sqrt(g (h + a))
    x1, _, _ = ctx.crest(0)
    assert abs(x1 - O.crest(pb.grid, e)[0]) < 1e-12 * m.Lx
    speed = (x1 - x0) / (400 * wl.dt)
    assert abs(speed - wl.notes["c"]) / wl.notes["c"] < 0.03


@pytest.mark.parametrize("name,steps", [("stokes_2d", 200), ("solitary_1d", 400)])
def test_fp32_run_tracks_fp64_run(sbi, name, steps):
    # Over a run the FP32 path stays with the FP64 path: eta within 1e-4
    # relative L2, and the relative energy drifts within 1e-4 of each other.
    wl = getattr(W, name)()
    m = wl.members[0]
    pb = problem_of(wl, m)
    eta, phi = O.project(pb, m.eta), O.project(pb, m.phi)
    res = {}
    for prec in (1, 0):
        ctx = context_of(sbi, wl, [0], prec)
        ctx.set_state(0, eta, phi)
        _, E0 = ctx.invariants(0)
        ctx.step(wl.dt, steps)
        e, _ = ctx.get_state(0)
        _, E1 = ctx.invariants(0)
        res[prec] = (e, (E1 - E0) / E0)
        ctx.close()
    print(f"{name}: FP32 vs FP64 eta {rel(res[0][0], res[1][0]):.2e}, drifts {res[0][1]:.2e} {res[1][1]:.2e}")
    assert rel(res[0][0], res[1][0]) < 1e-4
    assert abs(res[0][1] - res[1][1]) < 1e-4


@pytest.mark.parametrize("prec,tol", [(1, 1e-10), (0, 1e-5)])
def test_submerged_bar_full_size_steps(sbi, prec, tol):
    # N=4096 bar with sponge layers: a few RK4 steps against the oracle.
    wl = W.bar_1d()
    m = wl.members[0]
    pb = problem_of(wl, m)
    eta, phi = O.project(pb, m.eta), O.project(pb, m.phi)
    ctx = context_of(sbi, wl, [0], prec)
    ctx.set_state(0, eta, phi)
    V = ctx.vertical_velocity(0)
    assert rel(V, O.vertical_velocity(eta, phi, m.delta, m.h0, pb.grid)) < tol
    ctx.step(wl.dt, 3)
    e, p = ctx.get_state(0)
    eo, po = O.step(pb, eta, phi, wl.dt, 3)
    assert rel(e, eo) < tol and rel(p, po) < tol


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name", ["solitary_1d", "bar_1d", "stokes_2d"])
def test_v_after_one_evaluation_per_workload(sbi, name, prec):
    # V of the workload's (projected) initial state against the oracle, in
    # the workload's own configuration: relative L2 and pointwise.
    wl = getattr(W, name)()
    m = wl.members[0]
    pb = problem_of(wl, m)
    eta, phi = O.project(pb, m.eta), O.project(pb, m.phi)
    ctx = context_of(sbi, wl, [0], prec)
    ctx.set_state(0, eta, phi)
    V = ctx.vertical_velocity(0)
    ctx.close()
    Vo = O.vertical_velocity(eta, phi, m.delta, m.h0, pb.grid, order=wl.order, alpha=wl.alpha)
    print(f"{name} prec {prec}: V rel {rel(V, Vo):.2e} max {maxrel(V, Vo):.2e}")
    assert rel(V, Vo) < TOL_L2[prec] and maxrel(V, Vo) < TOL_MAX[prec]


@pytest.mark.parametrize("prec,tol", [(1, 1e-11), (0, 1e-5)])
def test_stokes_full_size_diagnostic(sbi, prec, tol):
    wl = W.stokes_2d()
    m = wl.members[0]
    pb = problem_of(wl, m)
    eta, phi = O.project(pb, m.eta), O.project(pb, m.phi)
    ctx = context_of(sbi, wl, [0], prec)
    ctx.set_state(0, eta, phi)
    assert rel(ctx.vertical_velocity(0), O.vertical_velocity(eta, phi, None, m.h0, pb.grid)) < tol


# The first and last member of every graph branch of the benchmark batch: the
# 256^2 group (members 0..63) runs as one branch, the 512^2 group as two
# (64..79 and 80..95).
BATCH_EDGE_MEMBERS = (0, 63, 64, 79, 80, 95)


def test_crossing_members_in_the_bench_batch(sbi):
    # The benchmark's 96-member batch (FP32) after one RK4 step: the edge
    # members of every graph branch against the oracle, state and V.
    wl = W.crossing_batch()
    ctx = context_of(sbi, wl, list(range(len(wl.members))), 0, check_finite=1)
    start = {}
    for i, m in enumerate(wl.members):
        if i in BATCH_EDGE_MEMBERS:
            # both sides start from the same projected (dealiased, filtered) state
            pb = problem_of(wl, m)
            start[i] = (pb, O.project(pb, m.eta), O.project(pb, m.phi))
            ctx.set_state(i, start[i][1], start[i][2])
        else:
            ctx.set_state(i, m.eta, m.phi)
    for i in BATCH_EDGE_MEMBERS:
        pb, e0, p0 = start[i]
        Vo = O.vertical_velocity(e0, p0, None, pb.h0, pb.grid, order=wl.order, alpha=wl.alpha)
        V = ctx.vertical_velocity(i)
        print(f"member {i}: V rel {rel(V, Vo):.2e} max {maxrel(V, Vo):.2e}")
        assert rel(V, Vo) < TOL_L2[0] and maxrel(V, Vo) < TOL_MAX[0], i
    ctx.step(wl.dt, 1)
    for i in BATCH_EDGE_MEMBERS:
        pb, e0, p0 = start[i]
        eo, po = O.step(pb, e0, p0, wl.dt, 1)
        e, p = ctx.get_state(i)
        print(f"member {i}: eta rel {rel(e, eo):.2e} max {maxrel(e, eo):.2e}, "
              f"phi rel {rel(p, po):.2e} max {maxrel(p, po):.2e}")
        assert rel(e, eo) < 1e-5 and rel(p, po) < 1e-5, i
        assert maxrel(e, eo) < 1e-5 and maxrel(p, po) < 1e-5, i


@pytest.fixture(scope="module")
def large_variable_oracle():
    """The 4096 x 2048 variable-depth sea, its projected state and the
    oracle's V of that state (evaluated once for the module)."""
    wl = W.large_variable()
    m = wl.members[0]
    pb = problem_of(wl, m)
    eta, phi = O.project(pb, m.eta), O.project(pb, m.phi)
    Vo = O.vertical_velocity(eta, phi, m.delta, m.h0, pb.grid, order=wl.order, alpha=wl.alpha)
    return wl, m, eta, phi, Vo


@pytest.mark.parametrize("prec", [0, 1])
def test_large_variable_matches_oracle(sbi, large_variable_oracle, prec):
    # Config 5 at full size (k_row<4096>, k_col<2048>, variable depth with
    # delta up to 0.3 h): V after one evaluation against the FP64 oracle.
    wl, m, eta, phi, Vo = large_variable_oracle
    ctx = context_of(sbi, wl, [0], prec)
    ctx.set_state(0, eta, phi)
    V = ctx.vertical_velocity(0)
    ctx.close()
    print(f"large_variable prec {prec}: V rel {rel(V, Vo):.2e} max {maxrel(V, Vo):.2e}")
    assert rel(V, Vo) < TOL_L2[prec]
    assert maxrel(V, Vo) < TOL_MAX[prec]


def test_large_variable_depth_properties(sbi):
    # 4096 x 2048 variable-depth crossing sea: FP32 vs FP64 paths, shift
    # equivariance, linearity in phi~ and exact mass conservation.
    wl = W.large_variable()
    m = wl.members[0]
    grid = (m.nx, m.ny, m.Lx, m.Ly)
    out = {}
    dA = (m.Lx / m.nx) * (m.Ly / m.ny)
    for prec in (1, 0):
        ctx = context_of(sbi, wl, [0], prec)
        ctx.set_state(0, m.eta, m.phi)
        out[prec] = ctx.vertical_velocity(0)
        # mass: F{V}(0) = 0, so the change over a step is the round-off of the
        # increment dt sum(V) in the path's precision
        mass0, _ = ctx.invariants(0)
        ctx.step(wl.dt, 1)
        mass1, _ = ctx.invariants(0)
        eps = 2.0 ** -52 if prec == 1 else 2.0 ** -23
        bound = 20.0 * eps * wl.dt * np.sum(np.abs(out[prec])) * dA
        assert abs(mass1 - mass0) <= bound, (prec, mass1 - mass0, bound)
        ctx.close()
    err = rel(out[0], out[1])
    print(f"large_variable FP32 vs FP64 V rel L2 = {err:.3e}")
    assert err < 1e-5
    # shift by one cell in x (delta, eta and phi~ together): V shifts with them
    ctx = sbi.Context([grid], wl.gravity, [np.roll(m.h0 - m.delta, 1, axis=1)], h0=m.h0,
                      precision=1, filt_beta1=wl.filt_beta1, filt_beta2=wl.filt_beta2, k_ref=wl.k_ref)
    ctx.set_state(0, np.roll(m.eta, 1, axis=1), np.roll(m.phi, 1, axis=1))
    Vs = ctx.vertical_velocity(0)
    assert rel(Vs, np.roll(out[1], 1, axis=1)) < 1e-11
    # linearity in phi~ at fixed eta, delta (same shifted configuration)
    ctx.set_state(0, np.roll(m.eta, 1, axis=1), 2.5 * np.roll(m.phi, 1, axis=1))
    assert rel(ctx.vertical_velocity(0), 2.5 * Vs) < 1e-11
    ctx.close()


@pytest.mark.parametrize("prec", [1, 0])
def test_checkpoint_restart_is_bit_exact(sbi, prec):
    # step(n) equals step(k) + get_state / set_state + step(n - k) bit for bit.
    nx, ny, Lx, Ly, h0 = 64, 32, 6.0, 4.0, 0.8
    grid = O.Grid(nx, ny, Lx, Ly)
    delta = W.random_field(nx, ny, 41, amplitude=0.05)
    pb = O.Problem(grid, 9.81, h0, delta=delta)
    eta = O.project(pb, W.random_field(nx, ny, 42, amplitude=0.03))
    phi = O.project(pb, W.random_field(nx, ny, 43, amplitude=0.2))
    a = sbi.Context([(nx, ny, Lx, Ly)], 9.81, [h0 - delta], h0=h0, precision=prec,
                    set_state_dealias=0)
    a.set_state(0, eta, phi)
    a.step(0.02, 5)
    ea, pa = a.get_state(0)
    b = sbi.Context([(nx, ny, Lx, Ly)], 9.81, [h0 - delta], h0=h0, precision=prec,
                    set_state_dealias=0)
    b.set_state(0, eta, phi)
    b.step(0.02, 2)
    e2, p2 = b.get_state(0)
    c = sbi.Context([(nx, ny, Lx, Ly)], 9.81, [h0 - delta], h0=h0, precision=prec,
                    set_state_dealias=0)
    c.set_state(0, e2, p2)
    c.step(0.02, 3)
    ec, pc = c.get_state(0)
    assert np.array_equal(ea, ec) and np.array_equal(pa, pc)


def test_nonfinite_state_is_reported(sbi):
    # A NaN in the state is detected on the device after the step and reported
    # as SBI_ENONFINITE (a flag the kernel sets; nothing traps).
    nx, ny = 32, 16
    eta = W.random_field(nx, ny, 51, amplitude=0.02)
    phi = W.random_field(nx, ny, 52, amplitude=0.1)
    eta[3, 5] = np.nan
    ctx = sbi.Context([(nx, ny, 3.0, 2.0)], 9.81, None, h0=1.0, precision=0, set_state_dealias=0)
    ctx.set_state(0, eta, phi)
    with pytest.raises(sbi.SbiError) as ei:
        ctx.step(0.01, 1)
    assert ei.value.code == sbi.SBI_ENONFINITE
    # the context stays usable
    ctx.set_state(0, np.zeros((ny, nx)), np.zeros((ny, nx)))


def test_bad_calls_fail_cleanly(sbi):
    ctx = sbi.Context([(32, 1, 3.0, 1.0)], 9.81, None, h0=1.0)
    with pytest.raises(sbi.SbiError) as ei:
        ctx.set_state(3, np.zeros(32), np.zeros(32))
    assert ei.value.code == sbi.SBI_EINVAL
    with pytest.raises(sbi.SbiError) as ei:
        ctx.step(-1.0, 1)
    assert ei.value.code == sbi.SBI_EINVAL
    with pytest.raises(sbi.SbiError) as ei:
        ctx.step(math.nan, 1)
    assert ei.value.code == sbi.SBI_EINVAL


@pytest.mark.parametrize("prec,tol", [(1, 1e-10), (0, 1e-5)])
def test_wavemaker_flume_matches_oracle(sbi, prec, tol):
    # The flume of the submerged-bar section driven by the pneumatic wavemaker
    # from rest, started at t0 != 0: the state after 60 steps and after 20 more
    # (the device time carried across calls) equals the oracle's.
    wl = W.bar_wavemaker_1d()
    m = wl.members[0]
    pb = problem_of(wl, m)
    ctx = context_of(sbi, wl, [0], prec)
    t0 = 0.37
    ctx.set_time(t0)
    ctx.set_state(0, m.eta, m.phi)
    ctx.step(wl.dt, 60)
    assert abs(ctx.get_time() - (t0 + 60 * wl.dt)) < 1e-12
    e, p = ctx.get_state(0)
    eo, po = O.step(pb, m.eta, m.phi, wl.dt, 60, t0=t0)
    assert np.max(np.abs(eo)) > 1e-3          # waves have been generated
    assert rel(e, eo) < tol and rel(p, po) < tol
    ctx.step(wl.dt, 20)
    e, p = ctx.get_state(0)
    eo, po = O.step(pb, eo, po, wl.dt, 20, t0=t0 + 60 * wl.dt)
    assert rel(e, eo) < tol and rel(p, po) < tol


@pytest.mark.parametrize("prec,tol", [(1, 1e-10), (0, 1e-5)])
def test_wavemaker_line_source_2d(sbi, prec, tol):
    # Two components, off-centre bell, a 2-D variable-depth member in motion.
    nx, ny, Lx, Ly, h0 = 64, 32, 8.0, 4.0, 0.6
    grid = O.Grid(nx, ny, Lx, Ly)
    delta = W.random_field(nx, ny, 101, amplitude=0.04)
    amp, omega, phase, x0 = [0.004, 0.002], [3.0, 5.5], [0.2, 1.1], 1.3
    wm = O.Wavemaker(np.array(amp), np.array(omega), np.array(phase), x0)
    pb = O.Problem(grid, 9.81, h0, delta=delta, wavemaker=wm)
    eta = O.project(pb, W.random_field(nx, ny, 102, amplitude=0.02))
    phi = O.project(pb, W.random_field(nx, ny, 103, amplitude=0.1))
    ctx = sbi.Context([(nx, ny, Lx, Ly)], 9.81, [h0 - delta], h0=h0, precision=prec)
    ctx.set_wavemaker(amp, omega, phase, x0)
    ctx.set_state(0, eta, phi)
    ctx.step(0.02, 6)
    e, p = ctx.get_state(0)
    eo, po = O.step(pb, eta, phi, 0.02, 6)
    assert rel(e, eo) < tol and rel(p, po) < tol
    # removing the wavemaker restores the free evolution
    ctx.set_wavemaker([], [], [])
    ctx.set_state(0, eta, phi)
    ctx.step(0.02, 2)
    pb0 = O.Problem(grid, 9.81, h0, delta=delta)
    e, p = ctx.get_state(0)
    eo, po = O.step(pb0, eta, phi, 0.02, 2)
    assert rel(e, eo) < tol and rel(p, po) < tol


def test_wavemaker_bad_calls(sbi):
    ctx = sbi.Context([(32, 1, 3.0, 1.0)], 9.81, None, h0=1.0)
    for args in (([0.01], [-1.0], [0.0]), ([math.nan], [2.0], [0.0]), ([0.01], [2.0], [math.inf])):
        with pytest.raises(sbi.SbiError) as ei:
            ctx.set_wavemaker(*args)
        assert ei.value.code == sbi.SBI_EINVAL
    with pytest.raises(sbi.SbiError) as ei:
        ctx.set_time(math.nan)
    assert ei.value.code == sbi.SBI_EINVAL
