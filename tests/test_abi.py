"""The C-ABI library builds, loads and exports every symbol include/mdsip.h
declares (no compute calls: this runs without a GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "mdsip.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = set(re.findall(r"\b(mdsip_[a-z_0-9]+)\s*\(", txt))
    return sorted(n for n in names if not n.endswith("_t"))


@pytest.fixture(scope="module")
def lib():
    import paper_2605_13736_gb300 as m
    m.build()
    return m.lib()


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("mdsip_ctx_create", "mdsip_problem_create_synthetic", "mdsip_solve",
                 "mdsip_get_iterate", "mdsip_get_stats", "mdsip_debug_direction",
                 "mdsip_syrk_scaled", "mdsip_ldlt_factor", "mdsip_ldlt_solve"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    import paper_2605_13736_gb300 as m
    assert set(_declared()) == set(m.exported_symbols())


def test_status_strings(lib):
    import paper_2605_13736_gb300 as m
    assert m.mdsip_status_str(0) == "OK"
    assert m.mdsip_status_str(6) == "INERTIA"
    assert m.mdsip_status_str(11) == "DEVICE"
