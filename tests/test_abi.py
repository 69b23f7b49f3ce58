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


def test_create_rejects_invalid_arguments_before_any_device_call(libpath):
    # jfnk_create checks the order, the grid, the physical constants and the
    # options before its first CUDA call, so every case below returns
    # JFNK_EINVAL (-1) on a host without a GPU as on one with a GPU
    import paper_2505_24504_gb300 as P
    from paper_2505_24504_gb300.jfnk import JfnkError

    def grid(**kw):
        a = dict(nx=4, nz=2, x0=0.0, x1=4000.0, z0=0.0, z1=2000.0, periodic_x=0)
        a.update(kw)
        return P.Grid(a["nx"], a["nz"], a["x0"], a["x1"], a["z0"], a["z1"], a["periodic_x"])

    def phys(**kw):
        a = dict(cp=1005.0, cv=717.95, g=9.81, p0=1e5, theta0=300.0, mu=0.0, background=0, ubg=0.0, wbg=0.0,
                 N_bv=0.0)
        a.update(kw)
        return P.Physics(*a.values())

    cases = [
        (grid(), 0, phys(), {}), (grid(), 5, phys(), {}),
        (grid(nx=0), 2, phys(), {}), (grid(nz=0), 2, phys(), {}), (grid(nx=-3), 2, phys(), {}),
        (grid(x1=0.0), 2, phys(), {}), (grid(z1=-1.0), 2, phys(), {}),
        (grid(), 2, phys(cp=700.0), {}), (grid(), 2, phys(cv=0.0), {}), (grid(), 2, phys(p0=0.0), {}),
        (grid(), 2, phys(theta0=-1.0), {}), (grid(), 2, phys(mu=-1.0), {}),
        (grid(), 2, phys(background=3), {}), (grid(), 2, phys(background=2, N_bv=0.0), {}),
        (grid(), 2, phys(), dict(gmres_restart=0)), (grid(), 2, phys(), dict(gmres_restart=65)),
        (grid(), 2, phys(), dict(gmres_max=0)), (grid(), 2, phys(), dict(newton_max=0)),
        (grid(), 2, phys(), dict(precond_prec=48)), (grid(), 2, phys(), dict(precond_fd_eps=-1.0)),
        (grid(), 2, phys(), dict(time_budget_ms=-5.0)), (grid(), 2, phys(), dict(dg_fused=3)),
        (grid(), 2, phys(), dict(rk_stages=5)), (grid(), 2, phys(), dict(rk_stages=2, rk_alpha=(0.5, 0.0))),
        (grid(), 2, phys(), dict(tile_faces=96)), (grid(), 2, phys(), dict(tile_volume=3)),
        (grid(), 2, phys(), dict(tile_fv=512)),
    ]
    for g, k, ph, opt in cases:
        with pytest.raises(JfnkError) as ei:
            P.Context(g, k, ph, P.Opts.defaults(**opt))
        assert ei.value.code == -1, (g.nx, g.nz, k, opt)
    # the valid arguments themselves are not what fails: on a GPU they create a
    # context, without one the first CUDA call reports JFNK_ECUDA (-3)
    try:
        c = P.Context(grid(), 2, phys(), P.Opts.defaults())
        c.close()
    except JfnkError as e:
        assert e.code == -3, e.code


def test_context_wrappers_reject_wrong_dtype_or_length_before_any_launch():
    # every array the library receives is indexed by the context's sizes: the
    # binding refuses a float32 array, a short one and a wrong member count
    # before it calls the library (objects built without a library context, so
    # a call that got through would fail on the null handle instead)
    torch = pytest.importorskip("torch")
    from paper_2505_24504_gb300 import jfnk
    ctx = object.__new__(jfnk.Context)
    ctx.N, ctx.h = 64, None
    good = torch.zeros(64, dtype=torch.float64)
    short = torch.zeros(63, dtype=torch.float64)
    f32 = torch.zeros(64, dtype=torch.float32)
    calls = [
        lambda: ctx.dg_residual(short, good), lambda: ctx.dg_residual(good, f32),
        lambda: ctx.jv_product(good, None, short, 1.0, 0.0, good), lambda: ctx.jv_product(good, f32, good, 1.0, 0.0, good),
        lambda: ctx.mg_precondition(good, 1.0, good, f32), lambda: ctx.implicit_step(short, 1.0),
        lambda: ctx.implicit_step(f32, 1.0), lambda: ctx.tangent_product(good, good, 1.0, short),
        lambda: ctx.jfnk_init_state(good, good), lambda: ctx.eos_pressure(good, short),
        lambda: ctx.time_operator(1, good, f32, 1), lambda: ctx.jfnk_autotune(short, good),
    ]
    for call in calls:
        with pytest.raises(ValueError, match="float64|elements"):
            call()
    b = object.__new__(jfnk.Batch)
    b.contexts, b.h = [ctx, ctx], None
    with pytest.raises(ValueError, match="members"):
        b.jfnk_batch_step([good], [1.0], [1])
    with pytest.raises(ValueError, match="elements"):
        b.jfnk_batch_step([good, short], [1.0, 1.0], [1, 1])
    with pytest.raises(ValueError, match="float64"):
        b.jfnk_batch_dg_residual([good, good], [good, f32])
