"""Degenerate grids and invalid calls on a live context.

Grids of one element row (both slip walls of every element's z faces at once),
one element column (both x walls), one periodic column (an element is its own
x neighbour) and single elements, against the FP64 oracle element by element:
the residual at 1e-12, the FD product at the bound its cancellation implies,
whole implicit steps (FP64 and FP32 preconditioner forms) at the solver
tolerance (relative to the step's increment, see the test), and the FV
hierarchy's level sizes.  Then every documented
JFNK_EINVAL of the calls on a context (null pointers, aliased outputs, a bad
multigrid key, out-of-range modes and levels)."""
import ctypes

import numpy as np
import pytest

import synth
from tests._common import gpu_context, oracle_dg, perturbed_state, rel, to_cpu, to_gpu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

W1 = synth.BUBBLE_Q2_20x10
CASES = {
    "row-q2-6x1": synth.scaled(W1, 6, 1, k=2, fv_levels=2),
    "col-q3-1x4": synth.scaled(W1, 1, 4, k=3, fv_levels=3),
    "periodic-col-q1-1x3": synth.scaled(W1, 1, 3, k=1, periodic_x=True, fv_levels=2),
    "single-q4-1x1": synth.scaled(W1, 1, 1, k=4, fv_levels=1),
    "single-q1-1x1": synth.scaled(W1, 1, 1, k=1, fv_levels=2),
}


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    w = CASES[request.param]
    dg = oracle_dg(w)
    return w, dg, perturbed_state(w, dg, seed=61, scale=0.2)


def test_residual_on_degenerate_grids(case):
    w, dg, Up = case
    ctx = gpu_context(w)
    f = torch.empty(ctx.N, dtype=torch.float64, device="cuda")
    ctx.dg_residual(to_gpu(Up), f)
    got, ref = to_cpu(f, dg.shape), dg.rhs(Up)
    assert rel(got, ref) <= 1e-12
    for v in range(4):
        assert np.abs(got[v] - ref[v]).max() <= 1e-12 * np.abs(ref[v]).max()


def test_jv_product_on_degenerate_grids(case):
    w, dg, Up = case
    ctx = gpu_context(w)
    y = synth.random_perturbation(dg.shape[1:], 62)
    adt, eps = 0.7 * w.dt, 1e-3
    fU = dg.rhs(Up)
    ref = dg.jv(Up, fU, y, adt, eps=eps)
    Jy = torch.empty(ctx.N, dtype=torch.float64, device="cuda")
    ctx.jv_product(to_gpu(Up), None, to_gpu(y), adt, eps, Jy)
    f1 = dg.rhs(Up + eps * y)
    bound = adt * 1e-12 * (np.linalg.norm(f1) + np.linalg.norm(fU)) / eps + 1e-13 * np.linalg.norm(ref)
    assert np.linalg.norm(to_cpu(Jy, dg.shape) - ref) <= bound


def test_fv_hierarchy_matches_the_oracle(case):
    from oracle.fv import Multigrid
    w, dg, _ = case
    ctx = gpu_context(w, precond_prec=32)
    mg = Multigrid(dg, w.fv_levels, w.mg_key)
    assert ctx.fv_levels() == [(lv.NX, lv.NZ) for lv in mg.levels]


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("scheme", [0, 1])
def test_implicit_step_on_degenerate_grids(case, prec, scheme):
    from oracle.fv import Multigrid
    from oracle.solver import implicit_step
    w, dg, Up = case
    ref = implicit_step(dg, Up, w.dt, scheme=scheme, tol=w.newton_tol,
                        precond=Multigrid(dg, w.fv_levels, w.mg_key))
    ctx = gpu_context(w, precond_prec=prec)
    U = to_gpu(Up)
    st = ctx.implicit_step(U, w.dt, scheme=scheme)
    assert st.status == 0
    got = to_cpu(U, dg.shape)
    # These seeded states are far from any balance: the step changes the state by
    # more than its final size (e.g. |U^{n+1}| = 0.07 against |dU| = 0.48 on the
    # single Q1 element), so the bar is the one the solver controls.  Newton
    # stops at |G_k| < 1e-8 |G_0| with |G_0| = alpha dt |f(U^n)| ~ |dU| (Sec. 3.1),
    # so two converged solvers differ by at most 2e-8 |G'^-1| |dU|; 1e-6 |dU|
    # allows |G'^-1| up to 50 (the 1e-8 |U'| bar of the other parity tests holds
    # where |U'| >> |dU|, as for the paper's bubble states).
    assert np.linalg.norm(got - ref) <= 1e-6 * np.linalg.norm(ref - Up)


def test_invalid_calls_on_a_context_return_einval():
    import paper_2505_24504_gb300 as P
    from paper_2505_24504_gb300.jfnk import JfnkError
    w = CASES["row-q2-6x1"]
    with pytest.raises(JfnkError) as ei:
        gpu_context(w, mg_key="mg11111V")          # eight characters
    assert ei.value.code == -1
    with pytest.raises(JfnkError) as ei:
        gpu_context(w, mg_key="mg1x1111V")
    assert ei.value.code == -1
    ctx = gpu_context(w, precond_prec=64)
    lib, h = P.lib(), ctx.h
    a = torch.zeros(ctx.N, dtype=torch.float64, device="cuda")
    b = torch.zeros(ctx.N, dtype=torch.float64, device="cuda")
    c = torch.zeros(ctx.N, dtype=torch.float64, device="cuda")
    pa, pb, pc = (ctypes.c_void_p(t.data_ptr()) for t in (a, b, c))
    ms = (ctypes.c_double * 2)()
    X, Z = ctypes.c_int(), ctypes.c_int()
    calls = {
        "dg_residual null U": lib.dg_residual(h, None, pb, None),
        "dg_residual null f": lib.dg_residual(h, pa, None, None),
        "dg_residual f == U": lib.dg_residual(h, pa, pa, None),
        "jv_product Jy == y": lib.jv_product(h, pa, None, pb, 1.0, 0.0, pb, None),
        "jv_product Jy == U": lib.jv_product(h, pa, None, pb, 1.0, 0.0, pa, None),
        "jv_product null y": lib.jv_product(h, pa, None, None, 1.0, 0.0, pc, None),
        "mg_precondition z == r": lib.mg_precondition(h, pa, 1.0, pb, pb, None),
        "mg_precondition z == U": lib.mg_precondition(h, pa, 1.0, pb, pa, None),
        "implicit_step null U": lib.implicit_step(h, None, 1.0, 1, None, None),
        "implicit_step dt 0": lib.implicit_step(h, pa, 0.0, 1, None, None),
        "implicit_step scheme 2": lib.implicit_step(h, pa, 1.0, 2, None, None),
        "time_operator which 5": lib.jfnk_time_operator(h, 5, pa, pb, 1, ms, None),
        "time_operator reps 0": lib.jfnk_time_operator(h, 0, pa, pb, 0, ms, None),
        "time_operator FP32 mode on FP64": lib.jfnk_time_operator(h, 2, pa, pb, 1, ms, None),
        "tangent_product on FP64": lib.jfnk_tangent_product(h, pa, pb, 1.0, pc, None),
        "fv_level_size beyond": lib.jfnk_fv_level_size(h, lib.jfnk_fv_levels(h), ctypes.byref(X), ctypes.byref(Z)),
        "fv_level_size negative": lib.jfnk_fv_level_size(h, -1, ctypes.byref(X), ctypes.byref(Z)),
        "fv_residual level beyond": lib.jfnk_fv_residual(h, lib.jfnk_fv_levels(h), pa, pb, None),
        "transfer_to_fv null": lib.jfnk_transfer_to_fv(h, None, pb, None),
        "init_state null": lib.jfnk_init_state(h, None, pa, None),
    }
    torch.cuda.synchronize()
    bad = {k: v for k, v in calls.items() if v != -1}
    assert not bad, bad
    # nothing was written by the rejected calls
    assert not a.any() and not b.any() and not c.any()
