"""Python binding of the C ABI in include/sbi.h (ctypes; argument marshalling only).

Every computation runs in the CUDA library ``_build/libsbi.so``; importing this
module fails loudly when the library has not been built.  The functions carry
the C names (sbi_create, sbi_set_state, sbi_vertical_velocity, sbi_step,
sbi_invariants, ...); ``Context`` wraps them for numpy arrays and torch tensors.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

from . import build as _build

SBI_OK, SBI_EINVAL, SBI_ENOMEM, SBI_ECUDA, SBI_ENONFINITE, SBI_ENOTCONVERGED, SBI_ETIMEOUT = range(7)
SBI_FP32, SBI_FP64 = 0, 1
SBI_RK4, SBI_LAWSON_RK4, SBI_IF_RK45 = 0, 1, 2
SBI_DIAG_ESBI, SBI_DIAG_HOS = 0, 1


class SbiError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"sbi error {code}: {msg}")
        self.code = code


class sbi_grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("Lx", C.c_double), ("Ly", C.c_double)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class sbi_options(C.Structure):
    _fields_ = [("order", C.c_int), ("alias_frac", C.c_double), ("h0", C.c_double),
                ("precision", C.c_int), ("adapt_tol", C.c_double),
                ("filt_beta1", C.c_double), ("filt_beta2", C.c_double), ("k_ref", C.c_double),
                ("sponge_w", C.POINTER(C.c_double)), ("sponge_nu", C.c_double),
                ("cuda_stream", C.c_void_p), ("check_finite", C.c_int),
                ("set_state_dealias", C.c_int),
                ("dev_alloc", ALLOC_FN), ("dev_free", FREE_FN), ("alloc_user", C.c_void_p),
                ("autotune", C.c_int), ("integrator", C.c_int), ("diagnostic", C.c_int),
                ("state_fp64", C.c_int), ("schedule", C.c_int),
                ("col_staging", C.c_int)]


EXPORTS = {
    "sbi_default_options": (None, [C.POINTER(sbi_options)]),
    "sbi_create": (C.c_int, [C.POINTER(sbi_grid), C.c_double, C.POINTER(C.c_double),
                             C.POINTER(sbi_options), C.POINTER(C.c_void_p)]),
    "sbi_create_batch": (C.c_int, [C.c_int, C.POINTER(sbi_grid), C.c_double,
                                   C.POINTER(C.POINTER(C.c_double)), C.POINTER(sbi_options),
                                   C.POINTER(C.c_void_p)]),
    "sbi_num_members": (C.c_int, [C.c_void_p]),
    "sbi_set_state": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int]),
    "sbi_get_state": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int]),
    "sbi_set_state_all": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "sbi_get_state_all": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "sbi_vertical_velocity": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_int]),
    "sbi_vertical_velocity_implicit": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int,
                                                 C.POINTER(C.c_double)]),
    "sbi_crest": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double),
                            C.POINTER(C.c_double)]),
    "sbi_step": (C.c_int, [C.c_void_p, C.c_double, C.c_int]),
    "sbi_step_streamed": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_int,
                                    C.c_void_p, C.c_void_p]),
    "sbi_invariants": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "sbi_set_time": (C.c_int, [C.c_void_p, C.c_double]),
    "sbi_get_time": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "sbi_set_wavemaker": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                    C.POINTER(C.c_double), C.c_double]),
    "sbi_orders_used": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int)]),
    "sbi_profile_enable": (C.c_int, [C.c_void_p, C.c_int]),
    "sbi_profile_read": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_char_p),
                                   C.POINTER(C.c_longlong), C.POINTER(C.c_double),
                                   C.POINTER(C.c_int)]),
    "sbi_step_bytes": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double)]),
    "sbi_step_transforms": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double)]),
    "sbi_step_launches": (C.c_int, [C.c_void_p, C.POINTER(C.c_int)]),
    "sbi_step_adaptive": (C.c_int, [C.c_void_p, C.c_double, C.c_double, C.POINTER(C.c_double),
                                    C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "sbi_autotune_report": (C.c_int, [C.c_void_p, C.c_char_p, C.c_size_t, C.POINTER(C.c_size_t)]),
    "sbi_schedule_report": (C.c_int, [C.c_void_p, C.c_char_p, C.c_size_t, C.POINTER(C.c_size_t)]),
    "sbi_test_stall_staged_copies": (C.c_int, [C.c_void_p, C.c_int]),
    "sbi_invariants_noalloc": (C.c_int, [C.POINTER(sbi_grid), C.c_double, C.c_void_p, C.c_void_p,
                                         C.c_void_p, C.c_void_p, C.POINTER(C.c_double),
                                         C.POINTER(C.c_double)]),
    "sbi_noalloc_last_error": (C.c_char_p, []),
    "sbi_last_error": (C.c_char_p, [C.c_void_p]),
    "sbi_destroy": (None, [C.c_void_p]),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load() -> C.CDLL:
    """Load libsbi.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(path)
    for name, (res, args) in EXPORTS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def default_options(**kw) -> sbi_options:
    o = sbi_options()
    load().sbi_default_options(C.byref(o))
    for k, v in kw.items():
        if k == "sponge_w":
            continue
        setattr(o, k, v)
    return o


def _ptr(a, dtype=np.float64):
    """(address, on_device, keepalive) of a numpy array or torch tensor of float64."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.dtype != torch.float64 or not a.is_contiguous():
                raise ValueError("torch tensors must be contiguous float64")
            return a.data_ptr(), 1 if a.is_cuda else 0, a
    except ImportError:
        pass
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr.ctypes.data, 0, arr


def invariants_noalloc(grid, gravity, eta, phi, V, stream=None):
    """Mass and energy from device arrays without any device allocation
    (sbi_invariants_noalloc); eta, phi, V are contiguous float64 CUDA tensors."""
    import torch
    lib = load()
    g = sbi_grid(grid[0], grid[1], grid[2], grid[3] if len(grid) > 3 else 1.0)
    npts = int(grid[0]) * int(grid[1])
    ptrs = []
    for a in (eta, phi, V):
        # the kernel reads nx*ny doubles from each pointer on the current
        # device: anything shorter, or elsewhere, is refused before the call
        if not isinstance(a, torch.Tensor) or not a.is_cuda:
            raise ValueError("sbi_invariants_noalloc takes CUDA tensors")
        if a.numel() != npts:
            raise ValueError(f"sbi_invariants_noalloc: a field holds {a.numel()} values, "
                             f"the grid {npts}")
        if a.device.index != torch.cuda.current_device():
            raise ValueError("sbi_invariants_noalloc: the fields must be on the current device")
        p, dev, keep = _ptr(a)
        ptrs.append(p)
    m, e = C.c_double(), C.c_double()
    st = C.c_void_p(int(stream)) if stream is not None else None
    rc = lib.sbi_invariants_noalloc(C.byref(g), float(gravity), ptrs[0], ptrs[1], ptrs[2], st,
                                    C.byref(m), C.byref(e))
    if rc != SBI_OK:
        raise SbiError(rc, lib.sbi_noalloc_last_error().decode())
    return m.value, e.value


class Context:
    """Owner of one sbi_ctx (one member or a batch of members)."""

    def __init__(self, grids, gravity, depths=None, *, h0=math.nan, order=7, alias_frac=0.5,
                 precision=SBI_FP32, adapt_tol=0.0, filt_beta1=0.0, filt_beta2=0.0, k_ref=1.0,
                 sponge_w=None, sponge_nu=0.0, stream=None, check_finite=1, set_state_dealias=1,
                 autotune=1, integrator=SBI_RK4, diagnostic=SBI_DIAG_ESBI, state_fp64=0,
                 schedule=0, col_staging=0):
        self.lib = load()
        if isinstance(grids, tuple):
            grids = [grids]
        self.grids = [tuple(g) for g in grids]
        n = len(self.grids)
        opt = default_options(order=order, alias_frac=alias_frac, h0=h0, precision=precision,
                              adapt_tol=adapt_tol, filt_beta1=filt_beta1, filt_beta2=filt_beta2,
                              k_ref=k_ref, sponge_nu=sponge_nu, check_finite=check_finite,
                              set_state_dealias=set_state_dealias, autotune=autotune,
                              integrator=integrator, diagnostic=diagnostic,
                              state_fp64=state_fp64, schedule=schedule,
                              col_staging=col_staging)
        keep = []
        if sponge_w is not None:
            w = np.ascontiguousarray(sponge_w, dtype=np.float64).ravel()
            keep.append(w)
            opt.sponge_w = w.ctypes.data_as(C.POINTER(C.c_double))
        if stream is not None:
            opt.cuda_stream = C.c_void_p(int(stream))
        garr = (sbi_grid * n)(*[sbi_grid(g[0], g[1], g[2], g[3] if len(g) > 3 else 1.0)
                                for g in self.grids])
        harr = (C.POINTER(C.c_double) * n)()
        if depths is not None:
            if not isinstance(depths, (list, tuple)):
                depths = [depths]
            for i, d in enumerate(depths):
                if d is None:
                    continue
                a = np.ascontiguousarray(d, dtype=np.float64).ravel()
                keep.append(a)
                harr[i] = a.ctypes.data_as(C.POINTER(C.c_double))
        out = C.c_void_p()
        rc = self.lib.sbi_create_batch(n, garr, gravity, harr, C.byref(opt), C.byref(out))
        if rc != SBI_OK:
            raise SbiError(rc, self.lib.sbi_last_error(None).decode())
        self.ctx = out
        self.precision = precision

    # -- helpers --------------------------------------------------------------
    def _check(self, rc):
        if rc != SBI_OK:
            raise SbiError(rc, self.lib.sbi_last_error(self.ctx).decode())

    def shape(self, member=0):
        g = self.grids[member]
        return (g[1], g[0])

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.sbi_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- C ABI ------------------------------------------------------------------
    def set_state(self, member, eta, phi):
        pe, de, ke = _ptr(eta)
        pp, dp, kp = _ptr(phi)
        if de != dp:
            raise ValueError("eta and phi must both be host or both be device buffers")
        self._check(self.lib.sbi_set_state(self.ctx, member, pe, pp, de))

    def get_state(self, member, eta=None, phi=None):
        if eta is None:
            eta = np.empty(self.shape(member))
            phi = np.empty(self.shape(member))
        pe, de, _ = _ptr(eta)
        pp, dp, _ = _ptr(phi)
        self._check(self.lib.sbi_get_state(self.ctx, member, pe, pp, de))
        return eta, phi

    def total_points(self):
        return sum(g[0] * g[1] for g in self.grids)

    def split(self, flat):
        """Per-member (ny, nx) views of a concatenated field (member order)."""
        out, o = [], 0
        for g in self.grids:
            n = g[0] * g[1]
            out.append(flat[o:o + n].reshape(g[1], g[0]))
            o += n
        return out

    def set_state_all(self, eta, phi):
        """sbi_set_state_all: eta, phi hold every member's field concatenated
        in member order (numpy arrays or contiguous float64 torch tensors)."""
        pe, de, ke = _ptr(eta)
        pp, dp, kp = _ptr(phi)
        if de != dp:
            raise ValueError("eta and phi must both be host or both be device buffers")
        for a in (ke, kp):
            if int(np.prod(a.shape)) != self.total_points():
                raise ValueError("eta and phi must hold every member's points")
        self._check(self.lib.sbi_set_state_all(self.ctx, pe, pp, de))

    def get_state_all(self, eta=None, phi=None):
        if eta is None:
            eta = np.empty(self.total_points())
            phi = np.empty(self.total_points())
        pe, de, ke = _ptr(eta)
        pp, dp, kp = _ptr(phi)
        if de != dp:
            raise ValueError("eta and phi must both be host or both be device buffers")
        for a in (ke, kp):
            if int(np.prod(a.shape)) != self.total_points():
                raise ValueError("eta and phi must hold every member's points")
        self._check(self.lib.sbi_get_state_all(self.ctx, pe, pp, de))
        return eta, phi

    def vertical_velocity(self, member=0, out=None, eulerian_w=False):
        if out is None:
            out = np.empty(self.shape(member))
        po, do, _ = _ptr(out)
        self._check(self.lib.sbi_vertical_velocity(self.ctx, member, po, do, int(eulerian_w)))
        return out

    def crest(self, member=0):
        """sbi_crest: (x, y, height) of the crest of the current surface."""
        x, y, h = C.c_double(), C.c_double(), C.c_double()
        self._check(self.lib.sbi_crest(self.ctx, member, C.byref(x), C.byref(y), C.byref(h)))
        return x.value, y.value, h.value

    def vertical_velocity_implicit(self, member=0, iterations=1, out=None):
        """sbi_vertical_velocity_implicit: V after `iterations` fixed-point
        iterations of the implicit form (flat bottom) and the relative L2
        change of each iteration."""
        if out is None:
            out = np.empty(self.shape(member))
        po, do, _ = _ptr(out)
        inc = (C.c_double * int(iterations))()
        self._check(self.lib.sbi_vertical_velocity_implicit(self.ctx, member, int(iterations), po, do, inc))
        return out, np.array(inc[:])

    def step(self, dt, n=1):
        self._check(self.lib.sbi_step(self.ctx, float(dt), int(n)))

    def step_streamed(self, eta_in, phi_in, dt, n=1, eta_out=None, phi_out=None):
        """sbi_step_streamed: every member's state in (concatenated in member
        order), n steps, the state out.  The outputs are new numpy arrays unless
        given (contiguous float64 numpy arrays or torch tensors, host or
        device; they may be the inputs)."""
        if eta_out is None:
            eta_out = np.empty(self.total_points())
        if phi_out is None:
            phi_out = np.empty(self.total_points())
        ptrs, keeps = [], []   # keeps: converted inputs stay alive over the call
        for a, is_out in ((eta_in, False), (phi_in, False), (eta_out, True), (phi_out, True)):
            p, _, keep = _ptr(a)
            if is_out and keep is not a:
                raise ValueError("eta_out and phi_out must be contiguous float64 arrays or tensors")
            if int(np.prod(keep.shape)) != self.total_points():
                raise ValueError("every buffer must hold every member's points")
            ptrs.append(p)
            keeps.append(keep)
        self._check(self.lib.sbi_step_streamed(self.ctx, ptrs[0], ptrs[1], float(dt), int(n),
                                               ptrs[2], ptrs[3]))
        return eta_out, phi_out

    def step_adaptive(self, t_end, tol, h):
        """sbi_step_adaptive: returns (proposed next step, accepted, rejected)."""
        hh, acc, rej = C.c_double(float(h)), C.c_int(), C.c_int()
        self._check(self.lib.sbi_step_adaptive(self.ctx, float(t_end), float(tol), C.byref(hh),
                                               C.byref(acc), C.byref(rej)))
        return hh.value, acc.value, rej.value

    def invariants(self, member=0):
        m, e = C.c_double(), C.c_double()
        self._check(self.lib.sbi_invariants(self.ctx, member, C.byref(m), C.byref(e)))
        return m.value, e.value

    def set_time(self, t):
        self._check(self.lib.sbi_set_time(self.ctx, float(t)))

    def get_time(self):
        t = C.c_double()
        self._check(self.lib.sbi_get_time(self.ctx, C.byref(t)))
        return t.value

    def set_wavemaker(self, amp, omega, phase, x0=0.0):
        """sbi_set_wavemaker; empty sequences remove the wavemaker."""
        arrs = [np.ascontiguousarray(np.atleast_1d(a), dtype=np.float64) for a in (amp, omega, phase)]
        n = arrs[0].size
        if any(a.size != n for a in arrs):
            raise ValueError("amp, omega and phase must have the same length")
        ptrs = [a.ctypes.data_as(C.POINTER(C.c_double)) for a in arrs]
        self._check(self.lib.sbi_set_wavemaker(self.ctx, n, *ptrs, float(x0)))

    def orders_used(self, member=0):
        o = C.c_int()
        self._check(self.lib.sbi_orders_used(self.ctx, member, C.byref(o)))
        return o.value

    def profile_enable(self, on=True):
        self._check(self.lib.sbi_profile_enable(self.ctx, int(on)))

    def profile_read(self):
        cap = 8
        names = (C.c_char_p * cap)()
        launches = (C.c_longlong * cap)()
        ms = (C.c_double * cap)()
        cnt = C.c_int()
        self._check(self.lib.sbi_profile_read(self.ctx, cap, names, launches, ms, C.byref(cnt)))
        return [(names[i].decode(), launches[i], ms[i]) for i in range(cnt.value)]

    def step_bytes(self, family=-1):
        b = C.c_double()
        self._check(self.lib.sbi_step_bytes(self.ctx, family, C.byref(b)))
        return b.value

    def autotune_report(self):
        need = C.c_size_t()
        self._check(self.lib.sbi_autotune_report(self.ctx, None, 0, C.byref(need)))
        buf = C.create_string_buffer(need.value + 1)
        self._check(self.lib.sbi_autotune_report(self.ctx, buf, len(buf), C.byref(need)))
        return buf.value.decode()

    def test_stall_staged_copies(self, on=True):
        """Test hook (sbi_test_stall_staged_copies): make the staged column
        pass's bounded waits run out, or restore normal operation."""
        self._check(self.lib.sbi_test_stall_staged_copies(self.ctx, int(on)))

    def schedule_report(self):
        """Lines of sbi_schedule_report: the step schedules tried, their times
        and the one chosen (empty before the first step)."""
        need = C.c_size_t()
        self._check(self.lib.sbi_schedule_report(self.ctx, None, 0, C.byref(need)))
        buf = C.create_string_buffer(need.value + 1)
        self._check(self.lib.sbi_schedule_report(self.ctx, buf, len(buf), C.byref(need)))
        return buf.value.decode()

    def step_transforms(self, family=-1):
        x = C.c_double()
        self._check(self.lib.sbi_step_transforms(self.ctx, family, C.byref(x)))
        return x.value

    def step_launches(self):
        n = C.c_int()
        self._check(self.lib.sbi_step_launches(self.ctx, C.byref(n)))
        return n.value
