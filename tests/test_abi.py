"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/swnmg.h declares (no compute calls: this runs without a GPU)."""
import ctypes as C
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"SWNMG_API\s+[\w\s\*]+?\b(swnmg_\w+)\s*\(", txt)
    return names


def test_header_declares_entry_points():
    names = declared_symbols()
    for must in ("swnmg_create", "swnmg_residual", "swnmg_jacobian", "swnmg_vcycle", "swnmg_solve"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_1608_06721_gb300 import swnmg
    lib = swnmg.lib()
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_default_params_are_the_papers():
    from paper_1608_06721_gb300 import swnmg
    p1, p2 = swnmg.default_params(1), swnmg.default_params(2)
    assert p1["alpha"] == 3.0 and p1["fd_eps"] == 1e-8 and p1["tau"] == 1.0 and p1["h_eps"] == 1e-6
    assert p1["n_mg"] == 2 and p2["n_mg"] == 3 and p1["n_levels"] == 3 and p1["eps_p"] == 0.2
    assert p2["eps_r"] == 0.03 and p2["flux"] == 1 and p1["flux"] == 0
    assert p1["eps_f"] == 0.4 and p2["eps_f"] == 0.4


def test_struct_layouts_match_header():
    """ctypes mirrors of the ABI structs have the C sizes (natural alignment)."""
    from paper_1608_06721_gb300 import swnmg
    assert C.sizeof(swnmg._BC) == 32
    assert C.sizeof(swnmg.Problem) == 3 * 4 + 4 + 5 * 8 + 4 * 32
    assert C.sizeof(swnmg.Params) == 2 * 4 + 7 * 8 + 10 * 4 + 8 + 8   # smoother + padding
    assert C.sizeof(swnmg.Stats) == 3 * 4 + 16 * 4 + 4 + 2 * 8 + 512 * 8 + 2 * 8
