"""The C-ABI library loads and exports every entry point its header declares;
host-side argument checks answer without touching a GPU."""
import ctypes
import os
import re

import pytest

import __graft_entry__ as entry

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    entry.build()
    from paper_2003_07720_gb300 import rpm
    return rpm.lib()


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(rpm_\w+)\s*\(", txt))
    return names


def test_every_declared_symbol_is_exported(L):
    names = _declared()
    assert "rpm_solve" in names and "rpm_apply_gamma" in names
    for n in sorted(names):
        assert hasattr(L, n), n


def test_binding_covers_header(L):
    from paper_2003_07720_gb300 import rpm
    assert set(rpm.EXPORTS) <= _declared()


def test_host_side_checks(L):
    from paper_2003_07720_gb300 import rpm
    o = rpm.rpm_default_options()
    assert (o.n_max, o.p_max, o.max_iters) == (10, 20, 5000) and o.tol == 1e-6
    assert rpm.rpm_grid_supported(128, 128, 128)
    assert rpm.rpm_grid_supported(64, 64, 1)
    assert rpm.rpm_grid_supported(96, 96, 96)
    assert not rpm.rpm_grid_supported(80, 80, 80)
    assert rpm.rpm_grid_supported(64, 32, 32)
    assert not rpm.rpm_grid_supported(512, 512, 8)
    h = ctypes.c_void_p()
    g = rpm.rpm_grid(40, 40, 40, 1.0, 1.0, 1.0)
    iso = (rpm.rpm_iso * 1)(rpm.rpm_iso(1.0, 1.0))
    ph = (ctypes.c_uint8 * (48 ** 3))()
    st = L.rpm_create(ctypes.byref(g), ctypes.cast(ph, ctypes.c_void_p), 0, 1, iso,
                      rpm.rpm_iso(1.0, 1.0), None, None, ctypes.byref(h))
    assert st == rpm.RPM_ERR_UNSUPPORTED_GRID and not h.value
    st = L.rpm_create(None, None, 0, 1, iso, rpm.rpm_iso(1.0, 1.0), None, None, ctypes.byref(h))
    assert st == rpm.RPM_ERR_INVALID_ARG
    g = rpm.rpm_grid(16, 16, 16, 1.0, 1.0, 1.0)
    st = L.rpm_create(ctypes.byref(g), ctypes.cast(ph, ctypes.c_void_p), 0, 1, iso,
                      rpm.rpm_iso(1.0, -1.0), None, None, ctypes.byref(h))
    assert st == rpm.RPM_ERR_INVALID_ARG
    bad = rpm.rpm_default_options(p_max=257)
    st = L.rpm_create(ctypes.byref(g), ctypes.cast(ph, ctypes.c_void_p), 0, 1, iso,
                      rpm.rpm_iso(1.0, 1.0), ctypes.byref(bad), None, ctypes.byref(h))
    assert st == rpm.RPM_ERR_INVALID_ARG
    assert L.rpm_status_string(5) == b"RPM_ERR_NOT_CONVERGED"
