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
    # the options struct of the binding has the header's size and field order
    assert o.precond_fd_eps == 0.0 and o.time_budget_ms == 0.0
    assert ctypes.sizeof(P.Opts) == _c_sizeof_opts()


def _c_sizeof_opts():
    """sizeof(jfnk_opts) as the C compiler lays it out (gcc on the header)."""
    import subprocess
    import tempfile
    src = '#include <stdio.h>\n#include "jfnk.h"\nint main(void){printf("%zu", sizeof(jfnk_opts));return 0;}\n'
    with tempfile.TemporaryDirectory() as d:
        c, exe = os.path.join(d, "s.c"), os.path.join(d, "s")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        return int(subprocess.run([exe], capture_output=True, text=True, check=True).stdout)


def test_norm_wrappers_reject_bad_arguments_before_any_launch():
    # a float32 vector or an n beyond the tensor would make the reduction read
    # past the buffer: the binding refuses both before the library is called
    torch = pytest.importorskip("torch")
    from paper_2505_24504_gb300 import jfnk
    x32 = torch.zeros(8, dtype=torch.float32)
    x64 = torch.zeros(8, dtype=torch.float64)
    out = torch.zeros(1, dtype=torch.float64)
    with pytest.raises(ValueError):
        jfnk.norm2_noalloc(x32, out)
    with pytest.raises(ValueError):
        jfnk.norm2_noalloc(x64, out, n=9)
    with pytest.raises(ValueError):
        jfnk.norm2_noalloc(x64, out, n=-1)
    with pytest.raises(ValueError):
        jfnk.norm2_noalloc(x64, torch.zeros(1, dtype=torch.float32))
