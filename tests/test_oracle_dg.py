"""Pins of the oracle DG operator f = M^-1 L_h (Sec. 2.1, Sec. 4) and of the
FD Jacobian-vector product (Sec. 3.1)."""
import numpy as np
import pytest

import synth
from oracle.dg import DG
from oracle.physics import Physics, UNIFORM
from oracle.solver import implicit_step

ROBERT = Physics(cp=1005.0, cv=717.95, g=9.80665, p0=1e5, theta0=300.0)
STRAKA_VISC = Physics(cp=1004.0, cv=717.0, g=9.81, p0=1e5, theta0=300.0, mu=75.0)
# dimensionless ideal gas (gamma = 1.4, R = 1) for exact-solution tests
UNIT = Physics(cp=3.5, cv=2.5, g=0.0, p0=1.0, theta0=1.0, background=UNIFORM)


def _atm(k, ph=ROBERT, nx=6, nz=4):
    return DG(nx, nz, 0.0, 6000.0, 0.0, 4000.0, k, ph)


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_well_balanced_bitwise_euler(k):
    # U' = 0 stays 0 exactly: every term is X(Ubar) - X(Ubar) (Sec. 4, perturbed-euler)
    dg = _atm(k)
    assert np.all(dg.rhs(dg.zeros()) == 0.0)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_well_balanced_viscous_to_roundoff(k):
    dg = _atm(k, STRAKA_VISC)
    f = dg.rhs(dg.zeros())
    # F_v(Ubar) = mu rho grad(theta0) vanishes up to the rounding of theta = E/rho
    assert np.abs(f).max() <= 1e-14 * STRAKA_VISC.mu * 1.2 * 300 / 100.0 ** 2 * 100


@pytest.mark.parametrize("k", [1, 2, 3])
def test_free_stream_preserved(k):
    ph = Physics(cp=3.5, cv=2.5, g=0.0, p0=1.0, theta0=1.0, background=UNIFORM, ubg=0.3, wbg=-0.2)
    dg = DG(4, 3, 0, 1, 0, 1, k, ph, periodic_x=True, periodic_z=True)
    Up = dg.zeros()
    Up[0] += 0.1
    Up[1] += 0.08
    Up[2] += 0.02
    Up[3] += 0.2
    assert np.abs(dg.rhs(Up)).max() < 1e-13


def _rand_state(dg, seed):
    return synth.random_perturbation(dg.shape[1:], seed, scales=(1e-2, 2.0, 2.0, 1.0))


@pytest.mark.parametrize("k", [1, 2, 3])
def test_conservation_walls(k):
    # slip walls: no mass or rho theta crosses the boundary (PAPER Sec. 4.1/4.3 setups)
    dg = _atm(k, STRAKA_VISC)
    f = dg.rhs(_rand_state(dg, 11))
    mw = dg.mass_weights()
    for v in (0, 3):
        tot = np.sum(mw * f[v])
        scale = np.sum(np.abs(mw * f[v]))
        assert abs(tot) <= 1e-12 * scale


@pytest.mark.parametrize("k", [1, 2, 3])
def test_conservation_periodic_all_components(k):
    ph = Physics(cp=3.5, cv=2.5, g=0.0, p0=1.0, theta0=1.0, mu=0.01, background=UNIFORM)
    dg = DG(4, 3, 0, 1, 0, 1, k, ph, periodic_x=True, periodic_z=True)
    Up = synth.random_perturbation(dg.shape[1:], 5, scales=(0.05, 0.05, 0.05, 0.05))
    f = dg.rhs(Up)
    mw = dg.mass_weights()
    for v in range(4):
        assert abs(np.sum(mw * f[v])) <= 1e-12 * np.sum(np.abs(mw * f[v]))


@pytest.mark.parametrize("k", [1, 2, 3])
def test_other_hydrostatic_state_converges_to_balance(k):
    # U' = Ubar(theta0=305) - Ubar(theta0=300): U'+Ubar is hydrostatic, so f -> 0
    # under refinement.  A wrong sign or weight of the gravity source or of the
    # pressure gradient leaves an O(1) residual.
    hot = Physics(cp=1005.0, cv=717.95, g=9.80665, p0=1e5, theta0=305.0)
    res = []
    for n in (2, 4):
        dg = DG(n, n, 0.0, 4000.0, 0.0, 4000.0, k, ROBERT)
        from oracle.physics import background
        Uh, _ = background(dg.Z, hot)
        f = dg.rhs(Uh - dg.Ub)
        res.append(np.sqrt(np.sum(dg.mass_weights() * f[2] ** 2)))
    scale = ROBERT.g * 0.017 * 2000.0        # g |rho'| |Omega|^(1/2)
    assert res[0] < 0.2 * scale
    assert np.log2(res[0] / res[1]) > k - 0.3


def _wave(dg, t, d):
    coord = dg.X if d == 0 else dg.Z
    rho = 1 + 0.2 * np.sin(2 * np.pi * (coord - t))
    E = np.full_like(rho, UNIT.p0 / UNIT.R)
    U = np.stack([rho, rho * (d == 0), rho * (d == 1), E])
    return U - dg.Ub


@pytest.mark.parametrize("k,ns,order", [(1, (16, 32), 1.8), (2, (8, 16), 2.8), (3, (4, 8), 3.5)])
@pytest.mark.parametrize("d", [0, 1])
def test_design_order_advected_density_wave(k, ns, order, d):
    # rho = 1 + 0.2 sin(2 pi (x - t)), unit velocity, constant p: exact Euler solution
    errs = []
    for n in ns:
        nx, nz = (n, 1) if d == 0 else (1, n)
        dg = DG(nx, nz, 0, 1, 0, 1, k, UNIT, periodic_x=True, periodic_z=True)
        U = _wave(dg, 0.0, d)
        for _ in range(40):
            U = implicit_step(dg, U, 0.001, scheme=1, tol=1e-11)
        e = U - _wave(dg, 0.04, d)
        errs.append(np.sqrt(np.sum(dg.mass_weights() * e[0] ** 2)))
    assert np.log2(errs[0] / errs[1]) > order


@pytest.mark.parametrize("k", [1, 2, 3])
def test_fd_jv_matches_complex_step_jacobian(k):
    dg = DG(2, 2, 0.0, 2000.0, 0.0, 2000.0, k, STRAKA_VISC)
    rng = np.random.default_rng(k)
    Up = dg.init_state(synth.Bubble(-15.0, 1000.0, 1000.0, 800.0, 800.0).theta(dg.X, dg.Z))
    Up = Up + _rand_state(dg, 3) * 0.1
    fU = dg.rhs(Up)
    for s in range(3):
        y = rng.standard_normal(dg.shape)
        ex = dg.jv_exact(Up, y, 2.0)
        # a step balancing truncation and rounding recovers the derivative to 1e-6
        fd = dg.jv(Up, fU, y, 2.0, eps=1e-7)
        assert np.linalg.norm(fd - ex) <= 1e-6 * np.linalg.norm(ex)
        # the paper's eps = sqrt(eps_mach)/|y| is rounding-limited: the perturbed
        # state carries rho theta ~ 300, so |error| ~ ulp(300)/(eps |y_i|) ~ 1e-5
        fd = dg.jv(Up, fU, y, 2.0)
        assert np.linalg.norm(fd - ex) <= 1e-4 * np.linalg.norm(ex)


def _assemble(dg, Up, rows_var, cols_var, convective=True):
    n = dg.shape
    cols = []
    idx = np.argwhere(np.ones(n[1:], dtype=bool))
    for e in idx:
        y = np.zeros(n)
        y[(cols_var,) + tuple(e)] = 1.0
        col = np.imag(dg.rhs(Up + 1e-30j * y)) / 1e-30
        cols.append(col[rows_var].ravel())
    return np.array(cols).T


@pytest.mark.parametrize("k", [1, 2])
def test_sipg_operator_symmetric_negative_semidefinite(k):
    # convection off, constant density: the viscous operator on rho theta is the
    # SIPG Laplacian, M J symmetric and negative semi-definite (A3 reading)
    ph = Physics(cp=3.5, cv=2.5, g=0.0, p0=1.0, theta0=1.0, mu=0.3, background=UNIFORM,
                 convective=False)
    dg = DG(3, 3, 0, 1, 0, 1.5, k, ph, periodic_x=True)
    J = _assemble(dg, dg.zeros(), 3, 3)
    mw = np.broadcast_to(dg.mass_weights(), dg.shape[1:]).ravel()
    MJ = mw[:, None] * J
    assert np.abs(MJ - MJ.T).max() <= 1e-12 * np.abs(MJ).max()
    ev = np.linalg.eigvalsh(0.5 * (MJ + MJ.T))
    assert ev.max() <= 1e-12 * np.abs(ev).max()
    # constants are in the kernel (no flux through walls / periodic)
    assert np.abs(J @ np.ones(J.shape[1])).max() <= 1e-11 * np.abs(J).max()


@pytest.mark.parametrize("k", [1, 2, 3])
@pytest.mark.parametrize("periodic", [True, False])
def test_viscous_operator_blind_to_density_at_fixed_velocity_and_theta(k, periodic):
    # F_v = mu rho (0, grad u, grad w, grad theta) (Sec. 4) sees U only through the
    # gradients of u, w and theta, so a perturbation of rho alone at fixed u = w = 0 and
    # fixed theta (rho theta' = theta rho') gives f = 0 even when it jumps between
    # elements: the interior penalty acts on the jumps of u, w, theta (weighted by
    # mu rho), not on those of the conserved rho u, rho w, rho theta
    ph = Physics(cp=3.5, cv=2.5, g=0.0, p0=1.0, theta0=1.3, mu=0.3, background=UNIFORM,
                 convective=False)
    dg = DG(4, 3, 0, 1, 0, 1.5, k, ph, periodic_x=periodic)
    rng = np.random.Generator(np.random.Philox(11))
    U = dg.zeros()
    U[0] = 0.2 * rng.standard_normal(U[0].shape)
    U[3] = (dg.Ub[3] / dg.Ub[0]) * U[0]
    f = dg.rhs(U)
    assert np.abs(f).max() <= 1e-11
    # a theta jump at fixed rho is damped: the same test with rho theta' alone is not blind
    V = dg.zeros()
    V[3] = U[0]
    assert np.abs(dg.rhs(V)).max() > 1e-2


@pytest.mark.parametrize("k,order", [(1, 1.8), (2, 2.8)])
def test_sipg_heat_equation_order(k, order):
    # rho = 1, no convection: d_t (rho theta) = mu Laplacian(rho theta), exact decay
    mu = 0.05
    ph = Physics(cp=3.5, cv=2.5, g=0.0, p0=1.0, theta0=1.0, mu=mu, background=UNIFORM,
                 convective=False)
    T, nt = 0.05, 25
    errs = []
    for n in (8, 16):
        dg = DG(n, 1, 0, 1, 0, 1, k, ph, periodic_x=True, periodic_z=True)
        E = lambda t: 0.1 * np.cos(2 * np.pi * dg.X) * np.exp(-4 * np.pi ** 2 * mu * t)
        U = dg.zeros()
        U[3] = E(0.0)
        for _ in range(nt):
            U = implicit_step(dg, U, T / nt, scheme=1, tol=1e-12)
        errs.append(np.sqrt(np.sum(dg.mass_weights() * (U[3] - E(T)) ** 2)))
    assert np.log2(errs[0] / errs[1]) > order


@pytest.mark.parametrize("k", [1, 3])
def test_well_balanced_bitwise_constant_n_with_wind(k):
    # Sec. 4.1 environment: constant N, mean flow 20 m/s, periodic in x
    from oracle.physics import CONST_N
    ph = Physics(cp=1005.0, cv=717.95, g=9.80665, p0=1e5, theta0=250.0, background=CONST_N, ubg=20.0, N_bv=0.01)
    dg = DG(6, 3, 0.0, 30000.0, 0.0, 10000.0, k, ph, periodic_x=True)
    assert np.all(dg.rhs(dg.zeros()) == 0.0)
