"""The benchmark's own configuration against the FP64 oracle, element by
element: warm bubble on DG Q3 160 x 80 (819,200 unknowns), 5 FV levels, the
schedule and launch shapes of the benchmark (presets.WARM_BUBBLE_Q3_160x80),
FP64 and FP32 preconditioner forms; and the operators at the largest size of
any workload (the ensemble's DG Q4 member on 320 x 160 quads).  The oracle's
SDIRK2 step takes a few minutes on one host core, so this module is marked
slow; it still runs with -m gpu."""
import numpy as np
import pytest

import synth
from paper_2505_24504_gb300 import presets
from tests._common import gpu_context, initial_state, oracle_dg, perturbed_state, rel, to_cpu, to_gpu

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

W = synth.BUBBLE_Q3_160x80
P = presets.WARM_BUBBLE_Q3_160x80
C_FD = 1e-2     # FD step numerator of the tight preconditioner comparison (see test_gpu_parity)


def _ctx(prec, **kw):
    opt = dict(P)
    opt.update(kw)
    return gpu_context(W, precond_prec=prec, **opt)


@pytest.fixture(scope="module")
def dg():
    return oracle_dg(W)


@pytest.fixture(scope="module")
def state(dg):
    return perturbed_state(W, dg, seed=41, scale=0.2)


def test_residual_at_bench_size(dg, state):
    ctx = _ctx(32)
    f = torch.empty(ctx.N, dtype=torch.float64, device="cuda")
    ctx.dg_residual(to_gpu(state), f)
    got, ref = to_cpu(f, dg.shape), dg.rhs(state)
    assert rel(got, ref) <= 1e-12
    for v in range(4):
        assert np.abs(got[v] - ref[v]).max() <= 1e-12 * np.abs(ref[v]).max()


def test_jv_product_at_bench_size(dg, state):
    ctx = _ctx(32)
    y = synth.random_perturbation(dg.shape[1:], 42)
    adt, eps = (1 - 2 ** -0.5) * W.dt, 1e-3
    fU = dg.rhs(state)
    ref = dg.jv(state, fU, y, adt, eps=eps)
    Jy = torch.empty(ctx.N, dtype=torch.float64, device="cuda")
    ctx.jv_product(to_gpu(state), None, to_gpu(y), adt, eps, Jy)
    f1 = dg.rhs(state + eps * y)
    bound = adt * 1e-12 * (np.linalg.norm(f1) + np.linalg.norm(fU)) / eps + 1e-13 * np.linalg.norm(ref)
    assert np.linalg.norm(to_cpu(Jy, dg.shape) - ref) <= bound


@pytest.fixture(scope="module")
def precond_ref(dg, state):
    from oracle.fv import Multigrid
    r = synth.random_perturbation(dg.shape[1:], 43)
    adt = (1 - 2 ** -0.5) * W.dt
    mg = Multigrid(dg, W.fv_levels, fd_eps=C_FD, **presets.schedule(P))
    mg.linearize(state, adt)
    z = mg.apply(r)
    return r, adt, z, mg.stats["dg_calls"] + sum(mg.stats["fv_calls"])


def test_fp64_preconditioner_at_bench_size(dg, state, precond_ref):
    r, adt, ref, products = precond_ref
    ctx = _ctx(64, precond_fd_eps=C_FD)
    z = torch.empty(ctx.N, dtype=torch.float64, device="cuda")
    ctx.mg_precondition(to_gpu(state), adt, to_gpu(r), z)
    err = rel(to_cpu(z, dg.shape), ref)
    bound = min(1e-6, products * 2.0 ** -44 * 400.0 * np.sqrt(dg.N) / C_FD + 1e-12)
    assert err <= bound, (err, bound)


@pytest.mark.parametrize("prec", [32, 16])
def test_fp32_preconditioner_at_bench_size(dg, state, precond_ref, prec):
    # the FP32 form (exact FP32 tangents) applies the same Q^-1 as the FP64 oracle
    # (whose FD step C_FD keeps its own round-off far below FP32's)
    r, adt, ref, _ = precond_ref
    ctx = _ctx(prec)
    z = torch.empty(ctx.N, dtype=torch.float64, device="cuda")
    ctx.mg_precondition(to_gpu(state), adt, to_gpu(r), z)
    err = rel(to_cpu(z, dg.shape), ref)
    assert err <= (2e-3 if prec == 32 else 2e-2), err


@pytest.fixture(scope="module")
def oracle_step(dg):
    from oracle.fv import Multigrid
    from oracle.solver import implicit_step
    U0 = initial_state(W, dg)
    ref = implicit_step(dg, U0, W.dt, scheme=1, tol=W.newton_tol,
                        precond=Multigrid(dg, W.fv_levels, **presets.schedule(P)))
    return U0, ref


@pytest.mark.timeout(1800)
@pytest.mark.parametrize("prec", [64, 32])
def test_sdirk2_step_at_bench_size(dg, oracle_step, prec):
    U0, ref = oracle_step
    ctx = _ctx(prec)
    U = to_gpu(U0)
    st = ctx.implicit_step(U, W.dt, scheme=1)
    assert st.status == 0 and st.stages == 2
    got = to_cpu(U, dg.shape)
    assert np.linalg.norm(got - ref) <= 1e-8 * np.linalg.norm(ref)
    assert np.linalg.norm(got - ref) <= 1e-6 * np.linalg.norm(ref - U0)


# The largest configuration of any workload: the ensemble's biggest member,
# DG Q4 on 320 x 160 quads (5,120,000 unknowns).
BIG = max(synth.ensemble(64), key=lambda m: m.n_unknowns)


@pytest.fixture(scope="module")
def big():
    dg = oracle_dg(BIG)
    return dg, perturbed_state(BIG, dg, seed=71, scale=0.2)


def test_operators_at_the_largest_size(big):
    dg, Up = big
    assert BIG.k == 4 and BIG.n_unknowns == 5_120_000
    ctx = gpu_context(BIG, precond_prec=32)
    U = to_gpu(Up)
    # FP64 residual, element by element
    f = torch.empty(ctx.N, dtype=torch.float64, device="cuda")
    ctx.dg_residual(U, f)
    got, ref = to_cpu(f, dg.shape), dg.rhs(Up)
    assert rel(got, ref) <= 1e-12
    for v in range(4):
        assert np.abs(got[v] - ref[v]).max() <= 1e-12 * np.abs(ref[v]).max()
    # FP64 FD product at a large step (bound of its cancellation, as at the bench size)
    y = synth.random_perturbation(dg.shape[1:], 72)
    adt, eps = (1 - 2 ** -0.5) * BIG.dt, 1e-3
    refj = dg.jv(Up, ref, y, adt, eps=eps)
    Jy = torch.empty(ctx.N, dtype=torch.float64, device="cuda")
    ctx.jv_product(U, None, to_gpu(y), adt, eps, Jy)
    f1 = dg.rhs(Up + eps * y)
    bound = adt * 1e-12 * (np.linalg.norm(f1) + np.linalg.norm(ref)) / eps + 1e-13 * np.linalg.norm(refj)
    assert np.linalg.norm(to_cpu(Jy, dg.shape) - refj) <= bound
    # FP32 DG product of the preconditioner against the complex-step product
    exact = dg.jv_exact(Up, y, adt)
    out = torch.empty(ctx.N, dtype=torch.float64, device="cuda")
    ctx.tangent_product(U, to_gpu(y), adt, out)
    assert np.linalg.norm(to_cpu(out, dg.shape) - exact) <= 2e-3 * np.linalg.norm(exact - y)
