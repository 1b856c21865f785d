"""The C-ABI library builds for sm_103a, loads, and exports every entry
point that include/qaoa.h declares (no device call is made)."""
import ctypes
import os
import re

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "qaoa.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qaoa_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("qaoa_plan_graph", "qaoa_plan_graphs", "qaoa_energy", "qaoa_energy_grad", "qaoa_plan_free",
                 "qaoa_last_error", "qaoa_cut_table", "qaoa_plan_info"):
        assert must in names


def test_library_exports_every_declared_symbol(qlib):
    h = ctypes.CDLL(qlib.LIB_PATH)
    missing = [n for n in _declared() if not hasattr(h, n)]
    assert not missing, missing
    assert qlib.lib().qaoa_version().decode().startswith("qaoa-gb300")


def test_binding_covers_every_declared_symbol(qlib):
    assert set(_declared()) <= set(qlib._SIGS)
