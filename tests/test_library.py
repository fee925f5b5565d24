"""CPU-only checks of the C ABI library: it builds for sm_103a, loads, and
exports every entry point that include/btmg.h declares.  No compute calls."""
import ctypes
import os
import re

from paper_2301_09991_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(btmg_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("btmg_create_problem", "btmg_apply_operator", "btmg_smooth", "btmg_mg_cycle",
                     "btmg_solve", "btmg_destroy_problem", "btmg_scalar_flux"):
        assert required in names


def test_library_builds_and_exports_every_declared_symbol():
    path = B.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_export():
    from paper_2301_09991_gb300 import btmg
    assert sorted(btmg.EXPORTS) == declared_symbols()


def test_error_strings_without_gpu():
    from paper_2301_09991_gb300 import btmg
    assert btmg.error_string(0) == "ok"
    assert "invalid" in btmg.error_string(-1)
