"""CUDA path vs the FP64 oracle, element by element on the same seeded inputs,
through the C ABI.  Tolerances: 1e-12 relative for the residual and the pieces
that involve no finite difference; FD products and the preconditioner at the
bound the FD quotient's cancellation implies (see each test)."""
import numpy as np
import pytest

import synth
from tests._common import gpu_context, initial_state, oracle_dg, perturbed_state, rel, to_cpu, to_gpu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

W1 = synth.BUBBLE_Q2_20x10
W3S = synth.scaled(synth.DENSITY_CURRENT_Q2_256x32, 24, 6, x1=4800.0 * 4, z1=6400.0)


def _cases():
    return {
        "q2-20x10": W1,
        "q1-9x5": synth.scaled(W1, 9, 5, k=1),
        "q3-11x6": synth.scaled(W1, 11, 6, k=3, fv_levels=4),
        "q4-7x5": synth.scaled(W1, 7, 5, k=4),
        "q3-periodic": synth.scaled(W1, 12, 6, k=3, periodic_x=True, fv_levels=4),
        "visc-q2-24x6": W3S,
        "visc-q3-10x4": synth.scaled(synth.DENSITY_CURRENT_Q2_256x32, 10, 4, k=3, x1=8000.0, fv_levels=3),
        "igw-q3-20x3": synth.scaled(synth.INERTIA_GRAVITY_Q3_80x3, 20, 3),
    }


@pytest.fixture(scope="module", params=list(_cases().keys()))
def case(request):
    w = _cases()[request.param]
    return w, gpu_context(w), oracle_dg(w)


def test_eos_power_against_cuda_pow():
    w = W1
    ctx = gpu_context(w)
    E = torch.linspace(20.0, 400.0, 200001, dtype=torch.float64, device="cuda")
    p = torch.empty_like(E)
    ctx.eos_pressure(E, p)
    R, gam = w.cp - w.cv, w.cp / w.cv
    x = ((R / w.p0) * E)                                    # the same rounded argument
    ref = w.p0 * torch.pow(x, gam)                          # CUDA's pow
    ulp = torch.abs(p - ref) / torch.abs(torch.nextafter(ref, ref * 2) - ref)
    assert float(ulp.max()) <= 4.0
    ref_cpu = w.p0 * x.cpu().numpy() ** gam                 # the oracle's (libm) pow
    assert np.max(np.abs(p.cpu().numpy() - ref_cpu) / ref_cpu) <= 3 * 2.0 ** -52


def test_well_balanced_exact_zero(case):
    w, ctx, dg = case
    U = torch.zeros(ctx.N, dtype=torch.float64, device="cuda")
    f = torch.full_like(U, 1.0)
    ctx.dg_residual(U, f)
    torch.cuda.synchronize()
    if w.mu == 0.0:
        assert torch.count_nonzero(f).item() == 0
    else:
        assert float(torch.abs(f).max()) < 1e-14 * w.mu * 300 / min(dg.hx, dg.hz) ** 2 * 100


def test_init_state_matches_oracle(case):
    w, ctx, dg = case
    x, z = ctx.node_coords()
    np.testing.assert_allclose(x, dg.X.ravel(), rtol=1e-15, atol=1e-9)
    np.testing.assert_allclose(z, dg.Z.ravel(), rtol=1e-15, atol=1e-9)
    th = w.theta_pert(dg.X, dg.Z)
    U = torch.empty(ctx.N, dtype=torch.float64, device="cuda")
    ctx.jfnk_init_state(to_gpu(th), U)
    ref = dg.init_state(th)
    got = to_cpu(U, dg.shape)
    # U' = U - Ubar is a difference of background-sized numbers (rho ~ 1,
    # rho theta ~ 300): its rounding is relative to those, not to |U'|
    bg = [1.3, 1.0, 1.0, 400.0]
    for v in range(4):
        scale = max(np.abs(ref[v]).max(), bg[v])
        assert np.abs(got[v] - ref[v]).max() <= 1e-12 * scale


def test_dg_residual_parity(case):
    w, ctx, dg = case
    Up = perturbed_state(w, dg, seed=11)
    f = torch.empty(ctx.N, dtype=torch.float64, device="cuda")
    ctx.dg_residual(to_gpu(Up), f)
    got = to_cpu(f, dg.shape)
    ref = dg.rhs(Up)
    assert rel(got, ref) <= 1e-12
    for v in range(4):
        assert np.abs(got[v] - ref[v]).max() <= 1e-12 * np.abs(ref[v]).max()


def test_jv_product_parity_large_step(case):
    # eps large enough that the FD quotient is well conditioned: tight parity
    w, ctx, dg = case
    Up = perturbed_state(w, dg, seed=12)
    y = synth.random_perturbation(dg.shape[1:], 13)
    adt = w.dt
    fU = dg.rhs(Up)
    eps = 1e-3
    ref = dg.jv(Up, fU, y, adt, eps=eps)
    Jy = torch.empty(ctx.N, dtype=torch.float64, device="cuda")
    ctx.jv_product(to_gpu(Up), None, to_gpu(y), adt, eps, Jy)
    got = to_cpu(Jy, dg.shape)
    # bound: adt (|df(U+eps y)| + |df(U)|) / eps with |df| <= 1e-12 |f|
    f1 = dg.rhs(Up + eps * y)
    bound = adt * 1e-12 * (np.linalg.norm(f1) + np.linalg.norm(fU)) / eps + 1e-13 * np.linalg.norm(ref)
    assert np.linalg.norm(got - ref) <= bound


def test_jv_product_small_step_same_states(case):
    # eps = 2^-32 (the paper's sqrt(eps_mach)/|y| is ~1e-10 here) and y with 20
    # fractional bits: eps y is exact, so U' + eps y rounds once on both sides and
    # both evaluate f at bit-identical states.  What remains is the residual
    # mismatch amplified by the FD quotient: |dJv| <= adt (|df1| + |df0|) / eps.
    w, ctx, dg = case
    Up = perturbed_state(w, dg, seed=14)
    y = np.round(synth.random_perturbation(dg.shape[1:], 15) * 2.0 ** 20) / 2.0 ** 20
    adt, eps = w.dt, 2.0 ** -32
    U1 = Up + eps * y
    f0, f1 = dg.rhs(Up), dg.rhs(U1)
    ref = y - adt * (f1 - f0) / eps
    Jy = torch.empty(ctx.N, dtype=torch.float64, device="cuda")
    ctx.jv_product(to_gpu(Up), None, to_gpu(y), adt, eps, Jy)
    got = to_cpu(Jy, dg.shape)
    g0 = torch.empty_like(Jy)
    g1 = torch.empty_like(Jy)
    ctx.dg_residual(to_gpu(Up), g0)
    ctx.dg_residual(to_gpu(U1), g1)
    df = np.linalg.norm(to_cpu(g0, dg.shape) - f0) + np.linalg.norm(to_cpu(g1, dg.shape) - f1)
    assert np.linalg.norm(got - ref) <= 1.01 * adt * df / eps + 1e-14 * np.linalg.norm(ref)


def test_jv_product_paper_eps(case):
    # default eps = sqrt(2^-52)/|y|_2 with |y| reduced on the device.  The GPU forms
    # U' + eps y with one rounding (FMA), numpy with two; with eps |y_i| ~ 1e-10
    # against rho theta ~ 300 (ulp 6e-14) the effective directions differ by
    # ~1e-4 relative, which the FD quotient passes straight into the product.
    # The tight checks of the FD composition are the two tests above.
    w, ctx, dg = case
    Up = perturbed_state(w, dg, seed=14)
    y = synth.random_perturbation(dg.shape[1:], 15)
    adt = w.dt
    fU = dg.rhs(Up)
    ref = dg.jv(Up, fU, y, adt)
    Jy = torch.empty(ctx.N, dtype=torch.float64, device="cuda")
    ctx.jv_product(to_gpu(Up), to_gpu(fU), to_gpu(y), adt, -1.0, Jy)
    assert rel(to_cpu(Jy, dg.shape), ref) <= 2e-3


def test_transfers_parity(case):
    from oracle.fv import Transfer
    w, ctx, dg = case
    T = Transfer(dg)
    u = perturbed_state(w, dg, seed=16)
    v = torch.empty(ctx.N, dtype=torch.float64, device="cuda")
    ctx.transfer_to_fv(to_gpu(u), v)
    vref = T.to_fv(u)
    assert rel(to_cpu(v, vref.shape), vref) <= 1e-14
    back = torch.empty_like(v)
    ctx.transfer_to_dg(v, back)
    assert rel(to_cpu(back, dg.shape), T.to_dg(to_cpu(v, vref.shape))) <= 1e-14
    assert rel(to_cpu(back, dg.shape), u) <= 1e-13


def test_transfers_l2_parity(case):
    from oracle.fv import Transfer
    w, _, dg = case
    ctx = gpu_context(w, transfer_l2=1)
    T = Transfer(dg, l2=True)
    u = perturbed_state(w, dg, seed=21)
    v = torch.empty(ctx.N, dtype=torch.float64, device="cuda")
    ctx.transfer_to_fv(to_gpu(u), v)
    vref = T.to_fv(u)
    assert rel(to_cpu(v, vref.shape), vref) <= 1e-14
    back = torch.empty_like(v)
    ctx.transfer_to_dg(v, back)
    assert rel(to_cpu(back, dg.shape), T.to_dg(to_cpu(v, vref.shape))) <= 1e-14
    assert rel(to_cpu(back, dg.shape), u) <= 1e-13


@pytest.mark.parametrize("split", [1, 1 << 30])
def test_fv_residual_parity_every_level(case, split):
    # split 1: one thread per cell on every level; 1 << 30: four lanes per cell
    from oracle.fv import Multigrid
    w, _, dg = case
    ctx = gpu_context(w, fv_split_cells=split)
    mg = Multigrid(dg, w.fv_levels, w.mg_key)
    assert ctx.fv_levels() == [(lev.NX, lev.NZ) for lev in mg.levels]
    for l, lev in enumerate(mg.levels):
        u = synth.random_perturbation(lev.shape[1:], 30 + l)
        f = torch.empty(u.size, dtype=torch.float64, device="cuda")
        ctx.fv_residual(l, to_gpu(u), f)
        ref = lev.rhs(u)
        assert rel(to_cpu(f, u.shape), ref) <= 1e-12


def test_preconditioner_without_fd_products_is_tight(case):
    # one FV level and only the first (zero-guess) pseudo-time step on it: no FD
    # quotient anywhere, so T^-1 dtau T r must agree to rounding
    from oracle.fv import Multigrid
    w, _, dg = case
    ctx = gpu_context(w, fv_levels=1, mg_key="mg001000V")
    Up = perturbed_state(w, dg, seed=17)
    r = synth.random_perturbation(dg.shape[1:], 18)
    z = torch.empty(ctx.N, dtype=torch.float64, device="cuda")
    ctx.mg_precondition(to_gpu(Up), w.dt, to_gpu(r), z)
    mg = Multigrid(dg, 1, "mg001000V")
    mg.linearize(Up, w.dt)
    assert rel(to_cpu(z, dg.shape), mg.apply(r)) <= 1e-12


@pytest.mark.parametrize("split", [0, 1])
def test_preconditioner_parity_at_fd_noise(case, split):
    # every FD product g'x amplifies rounding of f_low by alpha dt / eps with
    # eps = sqrt(eps_mach)/|x|, so two correct implementations differ at that
    # noise level.  Measure the oracle's own noise (input perturbed at 1e-15) and
    # require the GPU within a small multiple of it.  split 1: one thread per FV
    # cell on every level (the default runs these small levels four lanes per cell).
    from oracle.fv import Multigrid
    w, ctx, dg = case
    if split:
        ctx = gpu_context(w, fv_split_cells=split)
    Up = perturbed_state(w, dg, seed=19)
    r = synth.random_perturbation(dg.shape[1:], 20)
    z = torch.empty(ctx.N, dtype=torch.float64, device="cuda")
    ctx.mg_precondition(to_gpu(Up), w.dt, to_gpu(r), z)
    mg = Multigrid(dg, w.fv_levels, w.mg_key)
    mg.linearize(Up, w.dt)
    ref = mg.apply(r)
    noise = []
    for s in range(3):
        jit = 1.0 + 1e-15 * np.random.default_rng(s).standard_normal(Up.shape)
        mg.linearize(Up * jit, w.dt)
        noise.append(rel(mg.apply(r), ref))
    err = rel(to_cpu(z, dg.shape), ref)
    assert err <= max(10.0 * max(noise), 1e-10), (err, noise)


# FD step numerator of the preconditioner's products in the tight parity tests:
# eps = C_FD / |x|, so every perturbation eps x_i sits ~C_FD / sqrt(n) above the
# state instead of ~1e-8 / sqrt(n).  The two sides round u + eps x differently
# (one FMA rounding against two) by at most one ulp of |u| <= 400, so a product's
# relative difference is about ulp(400) sqrt(n) / C_FD <= 6e-14 * 1e3 / 1e-2 =
# 6e-9 per FD product; the preconditioner chains a few tens of them.
C_FD = 1e-2
FD_PARITY = 1e-6    # the FP64 mg_precondition bar


def _fd_bound(n, products):
    return min(FD_PARITY, products * 2.0 ** -44 * 400.0 * np.sqrt(n) / C_FD + 1e-12)


@pytest.mark.parametrize("key", ["mg111111V", "mg132211V", "mg111111W"])
def test_preconditioner_parity_fixed_fd_step(case, key):
    # the whole Q^-1 (DG smoothing, transfers, every FV level, V and W cycles) in
    # FP64 with the same FD step on both sides: agreement to the FD round-off
    # bound above, at most 1e-6 relative
    from oracle.fv import Multigrid
    w, _, dg = case
    ctx = gpu_context(w, mg_key=key, precond_fd_eps=C_FD)
    Up = perturbed_state(w, dg, seed=19)
    r = synth.random_perturbation(dg.shape[1:], 20)
    z = torch.empty(ctx.N, dtype=torch.float64, device="cuda")
    ctx.mg_precondition(to_gpu(Up), w.dt, to_gpu(r), z)
    mg = Multigrid(dg, w.fv_levels, key, fd_eps=C_FD)
    mg.linearize(Up, w.dt)
    ref = mg.apply(r)
    products = mg.stats["dg_calls"] + sum(mg.stats["fv_calls"])
    err = rel(to_cpu(z, dg.shape), ref)
    assert err <= _fd_bound(dg.N, products), (err, products)


@pytest.mark.parametrize("prec", [32, 16])
def test_fp32_preconditioner_close_to_oracle(case, prec):
    # the FP32 form (exact tangents in FP32 instead of FP64 difference quotients)
    # applies the same Q^-1: agreement to FP32 rounding and the oracle's FD noise,
    # far below the O(1) error a wrong tangent term would give
    from oracle.fv import Multigrid
    w, _, dg = case
    ctx = gpu_context(w, precond_prec=prec)
    Up = perturbed_state(w, dg, seed=19)
    r = synth.random_perturbation(dg.shape[1:], 20)
    z = torch.empty(ctx.N, dtype=torch.float64, device="cuda")
    ctx.mg_precondition(to_gpu(Up), w.dt, to_gpu(r), z)
    mg = Multigrid(dg, w.fv_levels, w.mg_key)
    mg.linearize(Up, w.dt)
    err = rel(to_cpu(z, dg.shape), mg.apply(r))
    assert err <= (2e-3 if prec == 32 else 2e-2), err


def _oracle_step(w, dg, U0, scheme, key=None, levels=None):
    from oracle.fv import Multigrid
    from oracle.solver import implicit_step
    pre = Multigrid(dg, levels or w.fv_levels, key or w.mg_key) if (key or w.mg_key) else None
    return implicit_step(dg, U0, w.dt, scheme=scheme, tol=w.newton_tol, precond=pre)


@pytest.mark.parametrize("scheme", [0, 1])
def test_implicit_step_parity(case, scheme):
    w, ctx, dg = case
    U0 = initial_state(w, dg)
    U = to_gpu(U0)
    st = ctx.implicit_step(U, w.dt, scheme=scheme)
    assert st.status == 0 and st.stages == (1 if scheme == 0 else 2)
    got = to_cpu(U, dg.shape)
    ref = _oracle_step(w, dg, U0, scheme)
    assert np.linalg.norm(got - ref) <= 1e-8 * np.linalg.norm(ref)
    assert np.linalg.norm(got - ref) <= 1e-6 * np.linalg.norm(ref - U0)


@pytest.mark.parametrize("name", ["q3-11x6", "igw-q3-20x3"])
def test_implicit_step_l2_transfer_parity(name):
    from oracle.fv import Multigrid
    from oracle.solver import implicit_step
    w = _cases()[name]
    dg = oracle_dg(w)
    ctx = gpu_context(w, transfer_l2=1)
    U0 = initial_state(w, dg)
    U = to_gpu(U0)
    st = ctx.implicit_step(U, w.dt, scheme=1)
    assert st.status == 0
    ref = implicit_step(dg, U0, w.dt, scheme=1, tol=w.newton_tol,
                        precond=Multigrid(dg, w.fv_levels, w.mg_key, l2=True))
    got = to_cpu(U, dg.shape)
    assert np.linalg.norm(got - ref) <= 1e-8 * np.linalg.norm(ref)
    assert np.linalg.norm(got - ref) <= 1e-6 * np.linalg.norm(ref - U0)


@pytest.mark.parametrize("name", ["q2-20x10", "q3-11x6", "visc-q2-24x6"])
@pytest.mark.parametrize("prec", [64, 32])
def test_implicit_step_w_cycle_parity(name, prec):
    # W cycle (the coarse correction applied twice, Sec. 3.4) inside the
    # implicit step: same converged answer as the oracle's step with the W cycle
    w = _cases()[name]
    dg = oracle_dg(w)
    ctx = gpu_context(w, mg_key="mg111111W", precond_prec=prec)
    U0 = initial_state(w, dg)
    U = to_gpu(U0)
    st = ctx.implicit_step(U, w.dt, scheme=1)
    assert st.status == 0
    ref = _oracle_step(w, dg, U0, 1, key="mg111111W")
    got = to_cpu(U, dg.shape)
    assert np.linalg.norm(got - ref) <= 1e-8 * np.linalg.norm(ref)
    assert np.linalg.norm(got - ref) <= 1e-6 * np.linalg.norm(ref - U0)


def test_inertia_gravity_steady_with_wind_and_periodic():
    # zero perturbation: the implicit step of the stratified atmosphere with mean
    # flow leaves U' = 0 exactly (well balanced, periodic x)
    w = synth.scaled(synth.INERTIA_GRAVITY_Q3_80x3, 20, 3)
    ctx = gpu_context(w)
    U = torch.zeros(ctx.N, dtype=torch.float64, device="cuda")
    st = ctx.implicit_step(U, w.dt, scheme=1)
    assert st.status == 0
    assert torch.count_nonzero(U).item() == 0


@pytest.mark.parametrize("prec", [64, 32])
def test_implicit_step_unpreconditioned_parity(prec):
    # no preconditioner: FGMRES keeps z_j = v_j in FP64 whatever precond_prec says
    w = synth.scaled(W1, 10, 5)
    from tests._common import oracle_dg as od
    dg = od(w)
    ctx = gpu_context(w, mg_key="", precond_prec=prec)
    U0 = initial_state(w, dg)
    U = to_gpu(U0)
    st = ctx.implicit_step(U, w.dt, scheme=0)
    from oracle.solver import implicit_step
    ref = implicit_step(dg, U0, w.dt, scheme=0, tol=w.newton_tol)
    assert np.linalg.norm(to_cpu(U, dg.shape) - ref) <= 1e-6 * np.linalg.norm(ref - U0)
    assert st.gmres_its > 0


@pytest.mark.parametrize("prec", [32, 16])
def test_implicit_step_fp32_preconditioner_same_answer(case, prec):
    # the preconditioner changes the iteration, not the converged answer
    w, _, dg = case
    ctx = gpu_context(w, precond_prec=prec)
    U0 = initial_state(w, dg)
    U = to_gpu(U0)
    st = ctx.implicit_step(U, w.dt, scheme=1)
    assert st.status == 0
    ref = _oracle_step(w, dg, U0, 1)
    got = to_cpu(U, dg.shape)
    assert np.linalg.norm(got - ref) <= 1e-8 * np.linalg.norm(ref)


@pytest.mark.parametrize("prec", [64, 32])
def test_graph_replay_bitwise_equals_direct_launches(prec):
    # the captured preconditioner graph issues the same kernels on the same
    # buffers: implicit steps with and without graphs agree bit for bit
    w = synth.scaled(W1, 12, 6, k=3, fv_levels=4)
    from tests._common import oracle_dg as od
    dg = od(w)
    U0 = initial_state(w, dg)
    out = []
    for g in (0, 1):
        ctx = gpu_context(w, precond_prec=prec, use_graphs=g)
        U = to_gpu(U0)
        for _ in range(2):
            ctx.implicit_step(U, w.dt, scheme=1)
        out.append(to_cpu(U))
    assert np.array_equal(out[0], out[1])


def test_norm2_entry_point():
    w = synth.scaled(W1, 10, 5)
    ctx = gpu_context(w)
    for n, seed in ((0, 1), (1, 2), (777, 3), (ctx.N, 4), (3_000_001, 5)):
        x = torch.from_numpy(synth.random_vector(max(n, 1), seed)).cuda()
        out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        ctx.norm2(x, out, n=n)
        ref = float(np.linalg.norm(x.cpu().numpy()[:n])) if n else 0.0
        assert abs(out.item() - ref) <= 1e-14 * max(ref, 1.0)



def test_launch_tiles_do_not_change_results_and_autotune_picks_valid_shapes():
    w = synth.scaled(W1, 12, 6, k=3, fv_levels=4)
    from tests._common import oracle_dg as od
    dg = od(w)
    U0 = initial_state(w, dg)
    outs = []
    for tf, tv, tfv in ((128, 2, 128), (64, 1, 64), (256, 2, 256)):
        ctx = gpu_context(w, precond_prec=32, tile_faces=tf, tile_volume=tv, tile_fv=tfv)
        U = to_gpu(U0)
        ctx.implicit_step(U, w.dt, scheme=1)
        outs.append(to_cpu(U))
    assert all(np.array_equal(outs[0], o) for o in outs[1:])
    ctx = gpu_context(w, precond_prec=32)
    y = to_gpu(synth.random_perturbation(dg.shape[1:], 3))
    best = ctx.jfnk_autotune(to_gpu(U0), y, reps=2)
    assert best["tile_faces"] in (64, 128, 256) and best["tile_volume"] in (1, 2)
    assert best["tile_fv"] in (64, 128, 256) and best["dg_ms"] > 0 and best["precond_ms"] > 0
    assert best["fv_split_cells"] >= 1
    U = to_gpu(U0)
    ctx.implicit_step(U, w.dt, scheme=1)
    # the lane split changes the FV summation order: same answer to the Newton tolerance
    got = to_cpu(U)
    assert np.linalg.norm(got - outs[0]) <= 1e-6 * np.linalg.norm(outs[0] - U0)


@pytest.mark.parametrize("prec", [64, 32])
def test_fv_lane_split_same_answer(prec):
    # one thread per FV cell on every level vs four lanes per cell on every level
    w = synth.scaled(W1, 12, 6, k=3, fv_levels=4)
    dg = oracle_dg(w)
    U0 = initial_state(w, dg)
    outs = []
    for split in (1, 1 << 30):
        ctx = gpu_context(w, precond_prec=prec, fv_split_cells=split)
        U = to_gpu(U0)
        st = ctx.implicit_step(U, w.dt, scheme=1)
        assert st.status == 0
        outs.append(to_cpu(U))
    assert np.linalg.norm(outs[0] - outs[1]) <= 1e-6 * np.linalg.norm(outs[0] - U0)


@pytest.mark.parametrize("name", ["q3-11x6", "visc-q2-24x6", "q1-9x5", "q4-7x5", "q3-periodic"])
def test_fused_and_two_launch_tangent_products_same_answer(name):
    # the FP32 tangent DG product as one fused launch per element strip or as a
    # face launch plus a volume launch: the same preconditioner up to FP32
    # rounding, so the same converged step
    w = _cases()[name]
    dg = oracle_dg(w)
    U0 = initial_state(w, dg)
    outs = []
    for fused in (1, 2):
        ctx = gpu_context(w, precond_prec=32, dg_fused=fused)
        U = to_gpu(U0)
        st = ctx.implicit_step(U, w.dt, scheme=1)
        assert st.status == 0
        outs.append(to_cpu(U))
    for o in outs[1:]:
        assert np.linalg.norm(outs[0] - o) <= 1e-6 * np.linalg.norm(outs[0] - U0)
    # and one product against the other directly
    ctxs = [gpu_context(w, precond_prec=32, dg_fused=f) for f in (1, 2)]
    Up = to_gpu(perturbed_state(w, dg, seed=5))
    y = to_gpu(synth.random_perturbation(dg.shape[1:], 6))
    res = []
    for c in ctxs:
        ms = c.time_operator(2, Up, y, 1)     # one FP32 tangent product z - adt J z into the workspace
        res.append(ms)
    assert all(m[0] > 0 for m in res)


@pytest.mark.parametrize("name", ["q2-20x10", "q1-9x5", "q3-11x6", "q4-7x5", "q3-periodic", "igw-q3-20x3",
                                  "visc-q2-24x6"])
def test_fp32_dg_product_against_oracle(name):
    # y - adt J(U) y in FP32, the product of the preconditioner's DG smoothing
    # steps, in both launch forms (one fused launch, dg_fused 1; face + volume
    # launches, dg_fused 2), against the oracle's complex-step product, element
    # by element relative to the size of the J part (FP32 rounding: the same
    # 2e-3 bar as the FP32 preconditioner); the two forms differ only in
    # rounding order
    w = _cases()[name]
    dg = oracle_dg(w)
    Up = perturbed_state(w, dg, seed=31)
    y = synth.random_perturbation(dg.shape[1:], 32)
    adt = w.dt
    ref = dg.jv_exact(Up, y, adt)
    jpart = np.linalg.norm(ref - y)
    outs = []
    for f in (1, 2):
        ctx = gpu_context(w, precond_prec=32, dg_fused=f)
        out = torch.empty(ctx.N, dtype=torch.float64, device="cuda")
        ctx.tangent_product(to_gpu(Up), to_gpu(y), adt, out)
        got = to_cpu(out, dg.shape)
        assert np.linalg.norm(got - ref) <= 2e-3 * jpart, (f, np.linalg.norm(got - ref) / jpart)
        for v in range(4):
            assert np.abs(got[v] - ref[v]).max() <= 2e-3 * np.abs(ref[v] - y[v]).max()
        outs.append(got)
    assert np.linalg.norm(outs[0] - outs[1]) <= 1e-4 * jpart


JST4 = (0.25, 1.0 / 3.0, 0.5, 1.0)   # Jameson-Schmidt-Turkel four-stage coefficients


@pytest.mark.parametrize("key", ["mg111111V", "mg132211V"])
def test_preconditioner_parity_multistage_smoother(case, key):
    # Q^-1 with the four-stage low-storage pseudo-time smoother (Sec. 3.5) on the
    # FV levels and the DG level: FP64 at the fixed FD step against the oracle, and
    # the FP32 form against the same oracle at FP32 rounding
    from oracle.fv import Multigrid
    w, _, dg = case
    Up = perturbed_state(w, dg, seed=23)
    r = synth.random_perturbation(dg.shape[1:], 24)
    mg = Multigrid(dg, w.fv_levels, key, fd_eps=C_FD, rk_alpha=JST4)
    mg.linearize(Up, w.dt)
    ref = mg.apply(r)
    products = mg.stats["dg_calls"] + sum(mg.stats["fv_calls"])
    for prec, bound in ((64, _fd_bound(dg.N, products)), (32, 2e-3)):
        ctx = gpu_context(w, mg_key=key, precond_prec=prec, precond_fd_eps=C_FD, rk_stages=4, rk_alpha=JST4)
        z = torch.empty(ctx.N, dtype=torch.float64, device="cuda")
        ctx.mg_precondition(to_gpu(Up), w.dt, to_gpu(r), z)
        err = rel(to_cpu(z, dg.shape), ref)
        assert err <= bound, (prec, err, bound)


@pytest.mark.parametrize("name", ["q2-20x10", "q3-11x6", "visc-q2-24x6", "igw-q3-20x3"])
@pytest.mark.parametrize("prec", [64, 32])
def test_implicit_step_multistage_smoother_parity(name, prec):
    w = _cases()[name]
    dg = oracle_dg(w)
    from oracle.fv import Multigrid
    from oracle.solver import implicit_step
    ctx = gpu_context(w, precond_prec=prec, rk_stages=4, rk_alpha=JST4)
    U0 = initial_state(w, dg)
    U = to_gpu(U0)
    st = ctx.implicit_step(U, w.dt, scheme=1)
    assert st.status == 0
    ref = implicit_step(dg, U0, w.dt, scheme=1, tol=w.newton_tol,
                        precond=Multigrid(dg, w.fv_levels, w.mg_key, rk_alpha=JST4))
    got = to_cpu(U, dg.shape)
    assert np.linalg.norm(got - ref) <= 1e-8 * np.linalg.norm(ref)
    assert np.linalg.norm(got - ref) <= 1e-6 * np.linalg.norm(ref - U0)


@pytest.mark.timeout(600)
def test_density_current_runs_past_the_landing_of_the_cold_air():
    # the viscous density current on its full grid (Q2 256x32, dt = 1 s, FP32
    # preconditioner) through t = 150 s, past the landing of the cold air near
    # t = 110 s: every step converges and the state stays finite (the interior
    # penalty acts on the jumps of u, w, theta; on the conserved variables a theta
    # jump at constant rho theta grew there until the step failed)
    w = synth.DENSITY_CURRENT_Q2_256x32
    dg = oracle_dg(w)
    ctx = gpu_context(w, precond_prec=32)
    U = to_gpu(dg.init_state(w.theta_pert(dg.X, dg.Z)))
    for i in range(150):
        st = ctx.implicit_step(U, w.dt, scheme=w.scheme, raise_on_error=False)
        assert st.status == 0, (i, st.status)
    assert torch.isfinite(U).all()
    ctx.close()
