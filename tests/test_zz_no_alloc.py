"""The allocation-free reduction entry point (sbi_invariants_noalloc) against
the context's sbi_invariants.

It serves callers that may not allocate device memory (memory-pool or arena
hosts, plugins handed device buffers only); it keeps its partial sums in a
fixed device array, so it is checked on two calls in a row (the second call
reuses the array the first one left behind).  This file is collected last.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [0, 1])
def test_invariants_noalloc_matches_context(prec):
    torch = pytest.importorskip("torch")
    import __graft_entry__ as g
    g.build()
    from paper_2310_19840_gb300 import sbi

    nx, ny, Lx, Ly, h0, grav = 256, 128, 12.0, 6.0, 0.7, 9.81
    delta = W.random_field(nx, ny, 81, amplitude=0.05, band=0.25)
    ctx = sbi.Context([(nx, ny, Lx, Ly)], grav, [h0 - delta], h0=h0, precision=prec)
    dev = torch.device("cuda")
    for call, seed in enumerate((82, 90)):
        eta = W.random_field(nx, ny, seed, amplitude=0.03, band=0.25) + 0.002 * (call + 1)
        phi = W.random_field(nx, ny, seed + 1, amplitude=0.2, band=0.25)
        ctx.set_state(0, eta, phi)
        m_ref, e_ref = ctx.invariants(0)
        e_d = torch.empty((ny, nx), dtype=torch.float64, device=dev)
        p_d = torch.empty((ny, nx), dtype=torch.float64, device=dev)
        v_d = torch.empty((ny, nx), dtype=torch.float64, device=dev)
        ctx.get_state(0, e_d, p_d)
        ctx.vertical_velocity(0, v_d)
        torch.cuda.synchronize()
        m, e = sbi.invariants_noalloc((nx, ny, Lx, Ly), grav, e_d, p_d, v_d)
        assert abs(m - m_ref) <= 1e-12 * abs(m_ref), (call, m, m_ref)
        assert abs(e - e_ref) <= 1e-12 * abs(e_ref), (call, e, e_ref)
    ctx.close()


def test_invariants_noalloc_rejects_bad_calls_before_any_launch():
    # Every rejection happens on the host, before a kernel is launched: the
    # C entry point's NULL, grid, gravity and size checks (called directly),
    # and the binding's check that each field holds nx*ny values.
    import ctypes as C
    torch = pytest.importorskip("torch")
    import __graft_entry__ as g
    g.build()
    from paper_2310_19840_gb300 import sbi

    lib = sbi.load()
    x = torch.zeros(64, dtype=torch.float64, device="cuda")
    p = x.data_ptr()
    m, e = C.c_double(), C.c_double()

    def call(grid, gravity, eta=p, phi=p, V=p):
        gr = sbi.sbi_grid(*grid)
        rc = lib.sbi_invariants_noalloc(C.byref(gr), gravity, eta, phi, V, None,
                                        C.byref(m), C.byref(e))
        return rc, lib.sbi_noalloc_last_error().decode()

    rc, msg = call((8, 8, 1.0, 1.0), 9.81, eta=None)
    assert rc == sbi.SBI_EINVAL and "NULL" in msg
    rc, msg = call((0, 8, 1.0, 1.0), 9.81)
    assert rc == sbi.SBI_EINVAL and "bad grid" in msg
    rc, msg = call((8, 8, 1.0, 1.0), 0.0)
    assert rc == sbi.SBI_EINVAL and "gravity" in msg
    rc, msg = call((8192, 8192, 1.0, 1.0), 9.81)
    assert rc == sbi.SBI_EINVAL and "limit" in msg
    # a valid call still works after the rejected ones
    rc, msg = call((8, 8, 1.0, 1.0), 9.81)
    assert rc == sbi.SBI_OK and m.value == 0.0 and e.value == 0.0
    # the binding refuses fields shorter than the grid (the kernel would read
    # past them) and host arrays
    with pytest.raises(ValueError):
        sbi.invariants_noalloc((16, 8, 1.0, 1.0), 9.81, x, x, x)
    with pytest.raises(ValueError):
        sbi.invariants_noalloc((8, 8, 1.0, 1.0), 9.81, x.cpu(), x, x)
