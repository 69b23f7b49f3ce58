"""Pins of the oracle preconditioner pieces (Sec. 3.2-3.5)."""
import numpy as np
import pytest

import synth
from oracle.dg import DG
from oracle.fv import FVLevel, Multigrid, Transfer, hierarchy, parse_mg_key, prolong, restrict
from oracle.physics import Physics, UNIFORM
from oracle.solver import fgmres, norm
from oracle.tables import midpoint_weights

ROBERT = Physics(cp=1005.0, cv=717.95, g=9.80665, p0=1e5, theta0=300.0)
VISC = Physics(cp=1004.0, cv=717.0, g=9.81, p0=1e5, theta0=300.0, mu=75.0)


def test_mg_key_parser():
    assert parse_mg_key("mg111111V") == dict(dg_pre=1, dg_post=1, fine_pre=1, fine_post=1,
                                             mid_pre=1, mid_post=1, cycles=1)
    assert parse_mg_key("mg001121W")["cycles"] == 2
    assert parse_mg_key("mg001121W")["mid_pre"] == 2
    with pytest.raises(ValueError):
        parse_mg_key("mg11111V")


def test_hierarchy_level_counts_of_the_workloads():
    # Q2 20x10 -> 3 levels; Q3 160x80 -> 5 levels; Q2 256x32 -> 4 levels
    assert hierarchy(20, 10, 2, 3)[0] == [(60, 30), (20, 10), (10, 5)]
    assert hierarchy(160, 80, 3, 5)[0] == [(640, 320), (320, 160), (160, 80), (80, 40), (40, 20)]
    assert hierarchy(256, 32, 2, 4)[0] == [(768, 96), (256, 32), (128, 16), (64, 8)]
    # the paper's k = 3 case: the subgrid adds two levels above the DG grid (Sec. 4)
    s, f = hierarchy(8, 8, 3, 10)
    assert s[2] == (8, 8) and f[:2] == [2, 2]


@pytest.mark.parametrize("ph", [ROBERT, VISC])
def test_fv_well_balanced(ph):
    lev = FVLevel(12, 8, 0, 6000, 0, 4000, ph)
    f = lev.rhs(np.zeros(lev.shape))
    if ph.mu == 0:
        assert np.all(f == 0.0)
    else:
        assert np.abs(f).max() < 1e-14 * 75 * 300 / 500.0 ** 2 * 10


def test_fv_free_stream_and_conservation():
    ph = Physics(cp=3.5, cv=2.5, g=0.0, p0=1.0, theta0=1.0, background=UNIFORM, ubg=0.2)
    lev = FVLevel(6, 5, 0, 1, 0, 1, ph, periodic_x=True)
    up = np.zeros(lev.shape)
    up[0] += 0.1
    up[1] += 0.02
    up[3] += 0.1
    assert np.abs(lev.rhs(up)).max() < 1e-14
    lev = FVLevel(7, 5, 0, 7000, 0, 5000, VISC)
    up = synth.random_perturbation(lev.shape[1:], 4, scales=(1e-2, 2, 2, 1))
    f = lev.rhs(up)
    for v in (0, 3):
        assert abs(f[v].sum()) <= 1e-12 * np.abs(f[v]).sum()


def test_restriction_and_injection():
    u = np.random.default_rng(0).standard_normal((4, 6, 9))
    for fac in (3,):
        r = restrict(u, fac)
        assert np.allclose(r.sum(axis=(1, 2)) * fac * fac, u.sum(axis=(1, 2)), rtol=1e-14)
        v = np.random.default_rng(1).standard_normal((4, 2, 3))
        # R P = I (exact in real arithmetic; the mean of fac^2 equal values rounds)
        np.testing.assert_allclose(restrict(prolong(v, fac), fac), v, rtol=4e-16, atol=0)
    assert np.allclose(restrict(u[:, :4, :8], 2)[0, 0, 0], u[0, :2, :2].mean())


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_transfer_mass_conservative_and_invertible(k):
    dg = DG(3, 2, 0, 3000, 0, 2000, k, ROBERT)
    T = Transfer(dg)
    u = synth.random_perturbation(dg.shape[1:], 9)
    v = T.to_fv(u)
    cell = dg.hx * dg.hz / (k + 1) ** 2
    for var in range(4):
        m_dg = np.sum(dg.mass_weights() * u[var])
        m_fv = cell * v[var].sum()
        assert abs(m_fv - m_dg) <= 1e-14 * np.sum(np.abs(dg.mass_weights() * u[var]))
    np.testing.assert_allclose(T.to_dg(v), u, atol=1e-12 * np.abs(u).max())
    # without the mass fix T interpolates: a Q_k polynomial is sampled at the centres
    p = lambda x, z: 1 + x / 3000 + (z / 2000) ** k
    up = np.stack([p(dg.X, dg.Z)] * 4)
    vp = T.to_fv(up, massfix=False)
    n1 = k + 1
    cx = (np.arange(3 * n1) + 0.5) * dg.hx / n1
    cz = (np.arange(2 * n1) + 0.5) * dg.hz / n1
    np.testing.assert_allclose(vp[0], p(cx[None, :], cz[:, None]), rtol=1e-13)


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_midpoint_mass_equals_polynomial_mass(k):
    # Sec. 3.3: the element mass from the FV-centre values with the modified
    # Newton-Cotes weights equals the GL mass of the DG polynomial
    dg = DG(2, 2, 0, 2000, 0, 2000, k, ROBERT)
    u = synth.random_perturbation(dg.shape[1:], 2)
    Tu = Transfer(dg).to_fv(u, massfix=False)
    _, om = midpoint_weights(k)
    n1 = k + 1
    blk = Tu.reshape(4, 2, n1, 2, n1).transpose(0, 1, 3, 2, 4)
    m_nc = dg.hx * dg.hz * np.einsum('j,i,vzxji->vzx', om, om, blk)
    m_gl = np.einsum('ba,vzxba->vzx', dg.mass_weights(), u)
    np.testing.assert_allclose(m_nc, m_gl, rtol=1e-12, atol=1e-12 * np.abs(m_gl).max())


def _mg_case():
    w = synth.BUBBLE_Q2_20x10
    dg = DG(w.nx, w.nz, w.x0, w.x1, w.z0, w.z1, w.k, ROBERT)
    Up = dg.init_state(w.theta_pert(dg.X, dg.Z))
    return w, dg, Up


def test_multigrid_converges_as_a_solver_on_the_finest_fv_level():
    w, dg, Up = _mg_case()
    # moderate pseudo-CFL: alpha dt = dt/10 (at the workload's alpha dt the explicit
    # Euler smoother is not a convergent stand-alone iteration; it is used only
    # inside GMRES there, see test_preconditioner_cuts_gmres_iterations)
    mg = Multigrid(dg, w.fv_levels, "mg001111V")
    mg.linearize(Up, 0.1 * w.dt)
    b = np.random.default_rng(0).standard_normal(mg.levels[0].shape)
    x = np.zeros_like(b)
    res = [norm(b)]
    for _ in range(6):
        x = x + mg.mg(0, np.zeros_like(b), b - mg.gprime(0, x), True)
        res.append(norm(b - mg.gprime(0, x)))
    assert all(r1 < r0 for r0, r1 in zip(res, res[1:]))
    assert res[-1] < 1e-2 * res[0]


def test_preconditioner_cuts_gmres_iterations():
    # the paper's qualitative claim (Sec. 4.1, 4.2): MG preconditioning strongly
    # reduces the GMRES iteration count versus no preconditioner
    w, dg, Up = _mg_case()
    adt = w.dt
    fU = dg.rhs(Up)
    G, _ = dg.G(Up, adt, Up - 0.01 * fU, fU)
    A = lambda y: dg.jv(Up, fU, y, adt)
    _, its_none, _ = fgmres(A, -G, None, tol_abs=1e-6 * norm(G), m=30, maxit=600)
    mg = Multigrid(dg, w.fv_levels, "mg111111V")
    mg.linearize(Up, adt, fU)
    _, its_mg, _ = fgmres(A, -G, mg.apply, tol_abs=1e-6 * norm(G), m=30, maxit=600)
    assert its_mg * 3 <= its_none


def test_fv_other_hydrostatic_state_converges_to_balance():
    # u' = ubar(theta0=305) - ubar(theta0=300) at the cell centres: hydrostatic, so
    # f_low -> 0 in the interior (second order in the momentum); a wrong gravity
    # sign leaves an O(1) residual.  The rows next to the slip walls keep an O(1)
    # residual rho' g / 2: a k = 0 cell with a mirrored ghost sees its centre
    # pressure at the wall, so they are excluded.
    from oracle.physics import background
    hot = Physics(cp=1005.0, cv=717.95, g=9.80665, p0=1e5, theta0=305.0)
    res = []
    for n in (8, 16, 32):
        lev = FVLevel(2, n, 0, 1000, 0, 4000, ROBERT)
        uh, _ = background(lev.zc, hot)
        f = lev.rhs(np.broadcast_to(uh[:, :, None], lev.shape) - np.broadcast_to(lev.ub, lev.shape))
        res.append(np.abs(f[2, 1:-1]).max())
    assert res[0] < 0.01 * ROBERT.g * 0.017
    assert np.log2(res[1] / res[2]) > 1.8


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_l2_transfer_gives_cell_averages_and_conserves_mass(k):
    # Sec. 3.2.1: the L2 projection onto piecewise constants = subcell averages
    dg = DG(2, 2, 0, 2000, 0, 2000, k, ROBERT)
    T = Transfer(dg, l2=True)
    n1 = k + 1
    p = lambda x, z: 1 + (x / 2000) ** k + 2 * (z / 2000) ** (k - 1) * (x / 2000)
    u = np.stack([p(dg.X, dg.Z)] * 4)
    v = T.to_fv(u)
    # exact averages of p over each subcell by Gauss-Legendre with k+2 points
    from oracle.tables import gauss_legendre
    g, wg = gauss_legendre(k + 2)
    H = 1000.0 / n1
    for J in range(2 * n1):
        for I in range(2 * n1):
            xs = (I + 0.5 * (1 + g)) * H
            zs = (J + 0.5 * (1 + g)) * H
            avg = 0.25 * np.sum(wg[:, None] * wg[None, :] * p(xs[None, :], zs[:, None]))
            assert abs(v[0, J, I] - avg) <= 1e-12 * abs(avg)
    ur = synth.random_perturbation(dg.shape[1:], 9)
    vr = T.to_fv(ur)
    cell = dg.hx * dg.hz / n1 ** 2
    for var in range(4):
        m_dg = np.sum(dg.mass_weights() * ur[var])
        assert abs(cell * vr[var].sum() - m_dg) <= 1e-13 * np.sum(np.abs(dg.mass_weights() * ur[var]))
    np.testing.assert_allclose(T.to_dg(vr), ur, atol=1e-11 * np.abs(ur).max())


# ---- pins of the two-point viscous flux of f_low (reading of Sec. 3.2 / 4.3) ----

def _visc_level(NX, NZ, periodic):
    ph = Physics(cp=1004.0, cv=717.0, g=0.0, p0=1e5, theta0=300.0, mu=75.0, background=UNIFORM)
    return FVLevel(NX, NZ, 0.0, 16000.0, 0.0, 6000.0, ph, periodic_x=periodic), ph


def test_fv_viscous_flux_is_the_periodic_five_point_laplacian_in_x():
    # rho constant, no motion, theta = theta0 + a cos(2 pi m x / L) at the cell
    # centres, periodic in x: mu {rho} (theta_R - theta_L)/H summed over the two x
    # faces is mu rho times the periodic 3-point second difference, whose
    # eigenvalue on this mode is -(4/H^2) sin^2(pi m H / L) (closed form).  A
    # flipped sign, a wrong 1/2 in the face average or a wrong spacing fails.
    lev, ph = _visc_level(16, 3, True)
    rho0, a, m = 1.17, 0.8, 3
    xc = (np.arange(lev.NX) + 0.5) * lev.Hx
    th = 300.0 + a * np.cos(2 * np.pi * m * xc / 16000.0)
    U = np.zeros(lev.shape)
    U[0] = rho0
    U[3] = rho0 * th[None, :]
    V = lev._viscous(U)
    lam = -(4.0 / lev.Hx ** 2) * np.sin(np.pi * m * lev.Hx / 16000.0) ** 2
    ref = ph.mu * rho0 * lam * a * np.cos(2 * np.pi * m * xc / 16000.0)
    np.testing.assert_allclose(V[3], np.broadcast_to(ref, V[3].shape), rtol=1e-12, atol=1e-15)
    assert np.all(V[0] == 0.0) and np.abs(V[1:3]).max() < 1e-18


def test_fv_viscous_flux_has_no_wall_flux_in_z():
    # u = a cos(pi m (z - z0)/Lz) at the centres with slip walls at z0 and z1:
    # zero viscous flux through the walls makes this the cell-centred Neumann
    # second difference, eigenvalue -(4/H^2) sin^2(pi m H / (2 Lz)) on every row,
    # boundary rows included (a wall flux would change exactly those rows).
    lev, ph = _visc_level(4, 12, False)
    rho0, a, m = 0.93, 2.5, 2
    zc = (np.arange(lev.NZ) + 0.5) * lev.Hz
    u = a * np.cos(np.pi * m * zc / 6000.0)
    U = np.zeros(lev.shape)
    U[0] = rho0
    U[1] = rho0 * u[:, None]
    U[3] = rho0 * 300.0
    V = lev._viscous(U)
    lam = -(4.0 / lev.Hz ** 2) * np.sin(np.pi * m * lev.Hz / (2 * 6000.0)) ** 2
    ref = ph.mu * rho0 * lam * u
    np.testing.assert_allclose(V[1], np.broadcast_to(ref[:, None], V[1].shape), rtol=1e-12, atol=1e-15)
    assert np.abs(V[2]).max() < 1e-18 and np.abs(V[3]).max() < 1e-12


def test_fv_viscous_flux_of_a_linear_shear_with_variable_density():
    # u = s z with rho varying by row: the two-point flux mu {rho} (u_R - u_L)/H is
    # exact for a linear u, mu s (rho_j + rho_{j+1})/2 through face j+1/2, so the
    # interior divergence is mu s (rho_{j+1} - rho_{j-1}) / (2 H).  Differencing
    # the momentum instead of the velocity, or dropping the density average, fails.
    lev, ph = _visc_level(5, 9, True)
    s = 3.0e-3
    rho = 1.0 + 0.2 * np.random.default_rng(3).random(lev.NZ)
    zc = (np.arange(lev.NZ) + 0.5) * lev.Hz
    U = np.zeros(lev.shape)
    U[0] = rho[:, None]
    U[1] = (rho * s * zc)[:, None]
    U[3] = rho[:, None] * 300.0
    V = lev._viscous(U)
    ref = ph.mu * s * (rho[2:] - rho[:-2]) / (2 * lev.Hz)
    np.testing.assert_allclose(V[1, 1:-1], np.broadcast_to(ref[:, None], V[1, 1:-1].shape), rtol=1e-10)
    assert np.abs(V[2]).max() < 1e-15 and np.abs(V[3]).max() < 1e-10


# ---- pins of the W cycle (Sec. 3.4: the coarse correction applied twice) ----

def test_w_cycle_visits_level_l_two_to_the_l_times():
    # MG_l calls MG_{l+1} `cycles` times: one cycle from the finest level visits
    # level l once (V) or 2^l times (W)
    w, dg, Up = _mg_case()
    w4 = synth.scaled(w, 16, 8, k=1, fv_levels=4)
    dg4 = DG(w4.nx, w4.nz, w4.x0, w4.x1, w4.z0, w4.z1, w4.k, ROBERT)
    U4 = dg4.init_state(w4.theta_pert(dg4.X, dg4.Z))
    for key, expect in (("mg001111V", [1, 1, 1, 1]), ("mg001111W", [1, 2, 4, 8])):
        mg = Multigrid(dg4, 4, key)
        assert len(mg.levels) == 4
        mg.linearize(U4, 0.1 * w4.dt)
        b = np.random.default_rng(1).standard_normal(mg.levels[0].shape)
        mg.mg(0, np.zeros_like(b), b, True)
        assert mg.stats['visits'] == expect


def test_w_cycle_converges_at_least_as_fast_as_v_per_cycle():
    # the W cycle solves the coarse-grid problems more accurately, so as a stand-
    # alone solver on the moderate pseudo-CFL problem it contracts monotonically
    # and per cycle at least as fast as the V cycle
    w, dg, Up = _mg_case()
    b = np.random.default_rng(0).standard_normal((4, 30, 60))
    hist = {}
    for key in ("mg001111V", "mg001111W"):
        mg = Multigrid(dg, w.fv_levels, key)
        mg.linearize(Up, 0.1 * w.dt)
        x = np.zeros_like(b)
        res = [norm(b)]
        for _ in range(5):
            x = x + mg.mg(0, np.zeros_like(b), b - mg.gprime(0, x), True)
            res.append(norm(b - mg.gprime(0, x)))
        hist[key] = res
    rv, rw = hist["mg001111V"], hist["mg001111W"]
    assert all(r1 < r0 for r0, r1 in zip(rw, rw[1:]))
    assert rw[-1] <= rv[-1] * 1.000001


# ---- pin of the multi-stage pseudo-time smoother (Sec. 3.5) ----

@pytest.mark.parametrize("alpha,coef", [
    ((1.0,), [1, 1]),                                            # explicit Euler: R(z) = 1 + z
    ((0.25, 1 / 3, 0.5, 1.0), [1, 1, 1 / 2, 1 / 6, 1 / 24]),     # Jameson-Schmidt-Turkel 4 stages
    ((0.5, 1.0), [1, 1, 1 / 2]),                                 # 2 stages: R(z) = 1 + z + z^2/2
])
def test_rk_smoother_amplification_is_the_stability_polynomial(alpha, coef):
    # on a linear system A x = b the low-storage scheme x_k = x_0 + a_k dtau (b - A x_{k-1})
    # maps the error e_0 = x_0 - x* to R(-dtau A) e_0, R the stability polynomial fixed
    # by the stage coefficients (a_s ... a_{s-j+1} for the z^j term); from x_0 = 0 the same
    # holds with e_0 = -x*
    rng = np.random.default_rng(3)
    n = 6
    A = rng.standard_normal((n, n)) + 4.0 * np.eye(n)
    b = rng.standard_normal(n)
    xs = np.linalg.solve(A, b)
    dtau = 0.07 + 0.02 * rng.random(n)          # a local step per unknown, as per cell
    mg = Multigrid.__new__(Multigrid)
    mg.rk_alpha = alpha
    Z = -dtau[:, None] * A
    R = sum(c * np.linalg.matrix_power(Z, j) for j, c in enumerate(coef))
    x0 = rng.standard_normal(n)
    got = mg.rk_step(x0, False, dtau, b, lambda v: A @ v)
    np.testing.assert_allclose(got - xs, R @ (x0 - xs), rtol=1e-12, atol=1e-13)
    got0 = mg.rk_step(np.zeros(n), True, dtau, b, lambda v: A @ v)
    np.testing.assert_allclose(got0 - xs, R @ (-xs), rtol=1e-12, atol=1e-13)
