"""Step schedules: how the members of a batch are split into graph branches.

A step's passes may run over any partition of the batch into units (member
ranges of one group), as concurrent branches or one after another.  Each
member's arithmetic is the same under every split, so every schedule must give
the same bits: through sbi_step and through the streamed step, with the
autotuner's timed choice (whose timing runs advance the state and put it back)
as well.  The batch interleaves two grid sizes in the caller's member order
(so member ranges are not runs of the caller's buffer), one group has a
variable bottom, and the low-pass filter makes the step non-idempotent.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

A = (64, 32, 6.0, 4.0)
B = (128, 16, 9.0, 2.0)
SPECS = [A, A, B, A, B, A, A, B, A]
H0 = 0.6


@pytest.fixture(scope="module")
def sbi():
    import __graft_entry__ as g
    g.build()
    from paper_2310_19840_gb300 import sbi as s
    return s


def depths():
    return [None if s is A else H0 - W.random_field(s[0], s[1], 40 + i, amplitude=0.04)
            for i, s in enumerate(SPECS)]


def initial():
    eta = [W.random_field(nx, ny, 60 + i, amplitude=0.03).ravel() for i, (nx, ny, _, _) in enumerate(SPECS)]
    phi = [W.random_field(nx, ny, 70 + i, amplitude=0.2).ravel() for i, (nx, ny, _, _) in enumerate(SPECS)]
    return np.concatenate(eta), np.concatenate(phi)


def make(sbi, prec, schedule, autotune):
    return sbi.Context(SPECS, 9.81, depths(), h0=H0, precision=prec, autotune=autotune,
                       schedule=schedule, filt_beta1=6.0, filt_beta2=20.0, k_ref=1.0)


def run(sbi, prec, schedule, autotune, streamed):
    eta, phi = initial()
    ctx = make(sbi, prec, schedule, autotune)
    if streamed:
        eo, po = np.empty_like(eta), np.empty_like(phi)
        ctx.step_streamed(eta, phi, 0.01, 3, eo, po)
        out = (eo, po)
    else:
        ctx.set_state_all(eta, phi)
        ctx.step(0.01, 3)
        out = ctx.get_state_all()
    rep = ctx.schedule_report()
    launches = ctx.step_launches()
    ctx.close()
    return out, rep, launches


@pytest.mark.parametrize("prec", [0, 1])
def test_every_schedule_gives_the_same_bits(sbi, prec):
    (e0, p0), rep0, l0 = run(sbi, prec, 1, 0, False)
    assert rep0.startswith("forced one") or rep0.startswith("forced split total/1"), rep0
    seen = {}
    for schedule in (-1, 2, 3, 4, 6):
        for streamed in (False, True):
            (e, p), rep, nl = run(sbi, prec, schedule, 1, streamed)
            assert rep.startswith("forced"), rep
            assert np.array_equal(e, e0) and np.array_equal(p, p0), (schedule, streamed)
            seen[schedule] = (rep, nl)
    # more units, more (smaller) launches: every unit runs its group's passes
    units = {b: int(r.split(" units:")[0].split()[-1]) for b, (r, _) in seen.items()}
    assert units[-1] == 2 and units[2] == 3 and units[4] == 5 and units[6] == 6, units
    assert seen[-1][1] == l0 and seen[2][1] > l0 and seen[6][1] > seen[4][1] > seen[2][1]


@pytest.mark.parametrize("streamed", [False, True])
def test_timed_choice_gives_the_same_bits(sbi, streamed):
    (e0, p0), _, _ = run(sbi, 0, 1, 0, False)
    (e, p), rep, _ = run(sbi, 0, 0, 1, streamed)
    lines = rep.strip().splitlines()
    # every candidate timed, one chosen; the state after the timing runs was
    # put back exactly, so the three steps give the same bits
    assert sum(ln.startswith("chosen ") for ln in lines) == 1, rep
    assert sum(" ms per step: " in ln for ln in lines) >= 3, rep
    assert all(float(ln.split()[1]) > 0 for ln in lines if " ms per step: " in ln), rep
    assert np.array_equal(e, e0) and np.array_equal(p, p0)


def test_untimed_default_and_bad_schedule(sbi):
    (_, _), rep, _ = run(sbi, 0, 0, 0, False)
    assert rep.startswith("default split total/3"), rep
    with pytest.raises(sbi.SbiError):
        make(sbi, 0, -2, 0)


def test_streamed_split_is_timed_and_gives_the_same_bits(sbi):
    # The streamed step cuts each schedule unit into k member ranges (k = 1, 2,
    # 3, 4, 6 timed on the first call when the outputs overlap no input); every k
    # gives the bits of the three calls.  An in-place call is not timed.
    (e0, p0), _, _ = run(sbi, 0, 3, 0, False)
    eta, phi = initial()
    ctx = make(sbi, 0, 3, 1)
    eo, po = np.empty_like(eta), np.empty_like(phi)
    ctx.step_streamed(eta, phi, 0.01, 3, eo, po)
    rep = ctx.schedule_report()
    ks = [ln for ln in rep.splitlines() if ln.startswith("streamed-")]
    assert sum(ln.startswith("streamed-chosen ") for ln in ks) == 1 and len(ks) >= 2, rep
    assert np.array_equal(eo, e0) and np.array_equal(po, p0)
    # later calls reuse the choice (no new report lines) and give the same bits
    ctx.step_streamed(eta, phi, 0.01, 3, eo, po)
    assert ctx.schedule_report() == rep
    assert np.array_equal(eo, e0) and np.array_equal(po, p0)
    ctx.close()
    ctx = make(sbi, 0, 3, 1)
    e, p = eta.copy(), phi.copy()
    ctx.step_streamed(e, p, 0.01, 3, e, p)
    assert not any(ln.startswith("streamed-") for ln in ctx.schedule_report().splitlines())
    assert np.array_equal(e, e0) and np.array_equal(p, p0)
    ctx.close()
