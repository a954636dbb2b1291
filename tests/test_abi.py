"""The C-ABI library loads and exports every entry point its header declares;
host-side argument checks answer without touching a GPU."""
import ctypes
import os
import re

import numpy as np
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


def test_variant_profile_and_basis_options_are_checked_on_the_host(L):
    """Defaults of the kernel-variant, profiling and shared-basis options,
    and their range checks before any device work; the queries and the
    bounded-wait self-check refuse null arguments."""
    from paper_2003_07720_gb300 import rpm
    o = rpm.rpm_default_options()
    assert (o.autotune, o.plane_variant, o.pencil_variant, o.share_basis, o.profile) == \
        (0, 0, 0, 0, 0)
    h = ctypes.c_void_p()
    g = rpm.rpm_grid(16, 16, 16, 1.0, 1.0, 1.0)
    iso = (rpm.rpm_iso * 1)(rpm.rpm_iso(1.0, 1.0))
    ph = (ctypes.c_uint8 * (16 ** 3))()
    for field, value in (("plane_variant", 3), ("pencil_variant", 4), ("share_basis", 2),
                         ("profile", -1), ("autotune", 2)):
        bad = rpm.rpm_default_options(**{field: value})
        st = L.rpm_create(ctypes.byref(g), ctypes.cast(ph, ctypes.c_void_p), 0, 1, iso,
                          rpm.rpm_iso(1.0, 1.0), ctypes.byref(bad), None, ctypes.byref(h))
        assert st == rpm.RPM_ERR_INVALID_ARG and not h.value, field
    assert L.rpm_plane_variant(None) == -1
    assert L.rpm_pencil_tile(None) == 0
    assert L.rpm_bounded_wait_check(None, None, None) == rpm.RPM_ERR_INVALID_ARG


def test_fno_host_side_checks(L):
    import ctypes as ct
    from paper_2003_07720_gb300 import fno
    F = fno.lib()
    assert set(fno.EXPORTS) <= _declared()
    m, layers = 12, 4
    assert fno.param_count(m, layers) == 768 + layers * (272 + 2 * (2 * m * m) * (2 * m) * 256)
    assert fno.param_count(0, 1) == 0 and fno.param_count(13, 1) == 0
    assert fno.param_count(4, 0) == 0 and fno.param_count(4, 9) == 0
    h = ct.c_void_p()
    for cfg in [(20, 4, 1, 1), (32, 17, 1, 1), (36, 4, 1, 1), (32, 4, 0, 1), (32, 4, 1, 0),
                (136, 4, 1, 1), (24, 13, 1, 1), (32, 4, 1, 65)]:
        st = F.rpm_fno_create(ct.byref(fno.rpm_fno_config(*cfg)), None, ct.byref(h))
        assert st == 1 and not h.value, cfg
    assert F.rpm_fno_create(None, None, ct.byref(h)) == 1
    # layout round trip of the dictionary form
    import microstructure as ms
    p = ms.fno_params(3, 2, seed=1)
    back = fno.unpack_params(fno.pack_params(p, 3, 2), 3, 2)
    for k in p:
        assert np.allclose(back[k], p[k], atol=1e-6), k
