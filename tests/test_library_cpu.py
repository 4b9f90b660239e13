"""Host-side checks of the C-ABI library (no GPU compute): it builds, loads,
exports every function include/sbi.h declares, and rejects bad arguments with
SBI_EINVAL before touching the device."""
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "sbi.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(sbi_[a-z_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2310_19840_gb300 import sbi
    return sbi.load()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("sbi_create", "sbi_set_state", "sbi_vertical_velocity", "sbi_step",
                     "sbi_invariants", "sbi_destroy", "sbi_last_error", "sbi_create_batch",
                     "sbi_get_state"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_2310_19840_gb300 import sbi
    assert set(_declared_functions()) <= set(sbi.EXPORTS)


def test_default_options(lib):
    from paper_2310_19840_gb300 import sbi
    o = sbi.default_options()
    assert o.order == 7 and o.alias_frac == 0.5 and math.isnan(o.h0)
    assert o.precision == sbi.SBI_FP32 and o.check_finite == 1 and o.set_state_dealias == 1
    assert o.autotune == 1


def test_binding_structs_match_the_header(tmp_path):
    # The ctypes mirrors of sbi_grid and sbi_options must have the C layout:
    # a C program compiled against include/sbi.h prints sizeof and offsetof.
    import ctypes
    import shutil
    import subprocess
    from paper_2310_19840_gb300 import sbi
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"sbi_grid": sbi.sbi_grid, "sbi_options": sbi.sbi_options}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "sbi.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name}.{field} %zu\\n", offsetof({name}, {field}));')
    lines.append("  return 0;\n}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(ln.split() for ln in subprocess.run([str(exe)], capture_output=True, text=True,
                                                    check=True).stdout.splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert int(got[f"{name}.{field}"]) == getattr(cls, field).offset, (name, field)


@pytest.mark.parametrize("grid,kw,msg", [
    ((100, 1, 1.0, 1.0), {}, "nx"),
    ((8, 1, 1.0, 1.0), {}, "nx"),
    ((64, 4, 1.0, 1.0), {}, "ny"),
    ((64, 1, -1.0, 1.0), {}, "box"),
    ((64, 1, 1.0, 1.0), {"order": 8}, "order"),
    ((64, 1, 1.0, 1.0), {"order": 0}, "order"),
    ((64, 1, 1.0, 1.0), {"alias_frac": 0.0}, "alias"),
    ((64, 1, 1.0, 1.0), {"h0": math.nan}, "h0"),
    ((64, 1, 1.0, 1.0), {"h0": 1.0, "filt_beta1": 8.0, "k_ref": 0.0}, "filter"),
])
def test_create_rejects_bad_arguments(lib, grid, kw, msg):
    from paper_2310_19840_gb300 import sbi
    with pytest.raises(sbi.SbiError) as ei:
        sbi.Context([grid], 9.81, None, **kw)
    assert ei.value.code == sbi.SBI_EINVAL
    assert msg in str(ei.value)


def test_create_rejects_nonpositive_depth(lib):
    from paper_2310_19840_gb300 import sbi
    h = np.ones(64)
    h[3] = 0.0
    with pytest.raises(sbi.SbiError) as ei:
        sbi.Context([(64, 1, 1.0, 1.0)], 9.81, [h])
    assert ei.value.code == sbi.SBI_EINVAL


def test_create_without_device_fails_cleanly(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    from paper_2310_19840_gb300 import sbi
    with pytest.raises(sbi.SbiError) as ei:
        sbi.Context([(64, 1, 1.0, 1.0)], 9.81, None, h0=1.0)
    assert ei.value.code == sbi.SBI_ECUDA
