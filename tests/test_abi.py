"""The C-ABI library builds for sm_103a, loads, and exports every function that
include/jfnk.h declares (no GPU needed: nothing is called that touches a device)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "jfnk.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w \*]*?\b(\w+)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "defined")))


@pytest.fixture(scope="module")
def libpath():
    from paper_2505_24504_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("jfnk_create", "jfnk_destroy", "dg_residual", "jv_product", "mg_precondition", "implicit_step"):
        assert n in names


def test_library_exports_every_declared_function(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_calls(libpath):
    import paper_2505_24504_gb300 as P
    o = P.Opts.defaults()
    assert o.newton_tol == 1e-8 and o.mg_key == b"mg111111V" and o.gmres_restart == 30
    assert P.lib().jfnk_strerror(-4).decode().startswith("Newton")
    g = P.Grid(20, 10, 0.0, 20000.0, 0.0, 10000.0, 0)
    b20 = P.Context.workspace_bytes(g, 2, o)
    g2 = P.Grid(40, 20, 0.0, 20000.0, 0.0, 10000.0, 0)
    assert P.Context.workspace_bytes(g2, 2, o) > 3.0 * b20   # 4x the unknowns, fixed scratch aside
    assert P.Context.workspace_bytes(P.Grid(0, 10, 0, 1, 0, 1, 0), 2, o) == 0
    assert P.Context.workspace_bytes(g, 5, o) == 0
