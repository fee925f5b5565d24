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


def test_library_stencils_match_the_pinned_oracle():
    """The library derives its ConvFEM stencils itself (exact polynomial
    integration, host code, no device needed); they must equal the oracle's,
    which the pins tie to the paper's printed tables (Appendix A.1-A.3), and
    the quadratic ones the closed forms."""
    import numpy as np
    import oracle as O
    from paper_2301_09991_gb300 import btmg
    for p in (1, 2, 3):
        m1, d1, s1 = btmg.convfem_stencils(p)
        om1, od1, os1, _ = O.convfem_1d(p)
        pad = 3 - p
        for got, ref in ((m1, om1), (d1, od1), (s1, os1)):
            np.testing.assert_allclose(got[pad:7 - pad], ref, rtol=0, atol=1e-13)
            assert np.all(got[:pad] == 0) and np.all(got[7 - pad:] == 0)
    m1, d1, s1 = btmg.convfem_stencils(2)
    np.testing.assert_allclose(m1[1:6], np.array([-1, 4, 24, 4, -1]) / 30, atol=1e-15)
    np.testing.assert_allclose(d1[1:6], np.array([1, -8, 0, 8, -1]) / 12, atol=1e-15)
    np.testing.assert_allclose(s1[1:6], np.array([1, -16, 30, -16, 1]) / 12, atol=1e-15)
