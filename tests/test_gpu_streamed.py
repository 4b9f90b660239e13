"""sbi_step_streamed against the three calls it stands for.

The streamed call copies every member's state in, runs n steps and copies the
state out, with each member group on its own stream.  Its launches and their
arguments are those of sbi_set_state_all + sbi_step + sbi_get_state_all, so
the two must agree bit for bit: on an uneven batch whose first group's members
are not consecutive in the caller's buffer (two copies per field), in both
precisions, with and without the dealiasing entry pass, with pageable numpy
buffers, pinned host tensors, device tensors and in place.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

GRIDS = [(64, 64, 6.0, 6.0), (128, 128, 12.0, 12.0), (64, 64, 6.0, 6.0)]


@pytest.fixture(scope="module")
def sbi():
    import __graft_entry__ as g
    g.build()
    from paper_2310_19840_gb300 import sbi as s
    return s


def smooth_fields(seed):
    """Every member's eta and phi~, concatenated: a few random low modes each."""
    rng = np.random.default_rng(seed)
    etas, phis = [], []
    for nx, ny, Lx, Ly in GRIDS:
        x = np.arange(nx) * Lx / nx
        y = np.arange(ny) * Ly / ny
        X, Y = np.meshgrid(x, y)
        e = np.zeros((ny, nx))
        p = np.zeros((ny, nx))
        for _ in range(4):
            kx, ky = rng.integers(1, 5, size=2)
            a, b, ph = rng.normal(size=3)
            arg = 2 * math.pi * (kx * X / Lx + ky * Y / Ly) + ph
            e += 0.01 * a * np.cos(arg)
            p += 0.01 * b * np.sin(arg)
        etas.append(e.ravel())
        phis.append(p.ravel())
    return np.concatenate(etas), np.concatenate(phis)


def make(sbi, prec, dealias):
    return sbi.Context(GRIDS, 9.81, None, h0=1.0, order=7, alias_frac=0.5, precision=prec,
                       set_state_dealias=dealias)


def three_calls(sbi, prec, dealias, eta, phi, dt, n):
    ctx = make(sbi, prec, dealias)
    ctx.set_state_all(eta, phi)
    ctx.step(dt, n)
    out = ctx.get_state_all()
    ctx.close()
    return out


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("dealias", [1, 0])
def test_streamed_equals_three_calls(sbi, prec, dealias):
    eta, phi = smooth_fields(7 + prec)
    dt, n = 0.02, 3
    (e_ref, p_ref) = three_calls(sbi, prec, dealias, eta, phi, dt, n)
    ctx = make(sbi, prec, dealias)
    e, p = ctx.step_streamed(eta, phi, dt, n)
    # a second call continues from the caller's buffers, not from the device state
    e2, p2 = ctx.step_streamed(eta, phi, dt, n)
    ctx.close()
    assert np.array_equal(e, e_ref) and np.array_equal(p, p_ref)
    assert np.array_equal(e2, e_ref) and np.array_equal(p2, p_ref)
    assert not np.array_equal(e, eta)          # the steps did move the state


def test_streamed_buffers_in_place_pinned_and_device(sbi):
    import torch
    eta, phi = smooth_fields(11)
    dt, n = 0.02, 2
    (e_ref, p_ref) = three_calls(sbi, 0, 1, eta, phi, dt, n)
    ctx = make(sbi, 0, 1)
    # pinned host tensors, outputs written over the inputs
    te = torch.from_numpy(eta.copy()).pin_memory()
    tp = torch.from_numpy(phi.copy()).pin_memory()
    ctx.step_streamed(te, tp, dt, n, te, tp)
    assert np.array_equal(te.numpy(), e_ref) and np.array_equal(tp.numpy(), p_ref)
    # device tensors
    de = torch.from_numpy(eta).cuda()
    dp = torch.from_numpy(phi).cuda()
    oe, op = torch.empty_like(de), torch.empty_like(dp)
    ctx.step_streamed(de, dp, dt, n, oe, op)
    assert np.array_equal(oe.cpu().numpy(), e_ref) and np.array_equal(op.cpu().numpy(), p_ref)
    # n = 0: the entry state (dealiased) comes back
    z_e, z_p = ctx.step_streamed(eta, phi, dt, 0)
    ctx.close()
    c2 = make(sbi, 0, 1)
    c2.set_state_all(eta, phi)
    g_e, g_p = c2.get_state_all()
    c2.close()
    assert np.array_equal(z_e, g_e) and np.array_equal(z_p, g_p)


def test_streamed_advances_time_and_rejects_bad_arguments(sbi):
    eta, phi = smooth_fields(3)
    ctx = make(sbi, 0, 1)
    ctx.step_streamed(eta, phi, 0.02, 5)
    t_expect = 0.0
    for _ in range(5):
        t_expect += 0.02        # the same sum as five sbi_step steps
    assert ctx.get_time() == t_expect
    with pytest.raises(Exception):
        ctx.step_streamed(eta, phi, -1.0, 1)
    with pytest.raises(Exception):
        ctx.step_streamed(eta, phi, 0.02, -1)
    with pytest.raises(ValueError):
        ctx.step_streamed(eta[:-1], phi, 0.02, 1)
    with pytest.raises(ValueError):
        ctx.step_streamed(eta, phi, 0.02, 1, np.empty(eta.size, dtype=np.float32), np.empty(eta.size))
    ctx.close()


def test_streamed_one_group_runs_the_three_calls(sbi):
    eta, phi = smooth_fields(5)
    n0 = GRIDS[0][0] * GRIDS[0][1]
    ctx = sbi.Context(GRIDS[:1], 9.81, None, h0=1.0, order=7, alias_frac=0.5, precision=0)
    e, p = ctx.step_streamed(eta[:n0], phi[:n0], 0.02, 2)
    ctx.set_state_all(eta[:n0], phi[:n0])
    ctx.step(0.02, 2)
    e_ref, p_ref = ctx.get_state_all()
    ctx.close()
    assert np.array_equal(e, e_ref) and np.array_equal(p, p_ref)
