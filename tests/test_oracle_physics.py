"""Pins of the oracle's model functions (Sec. 4: eq. compressible-euler,
eq. add-perturbation, environmental atmospheres; HLLC of Sec. 2.1)."""
import numpy as np
import pytest

from oracle.physics import (Physics, UNIFORM, background, background_pressure_theta, flux_n,
                            hllc, insert_perturbation, mirror, pressure, viscous_flux)

PH = Physics(cp=1005.0, cv=717.95, g=9.80665, p0=1e5, theta0=300.0)


def _states(n, seed):
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.5, 1.3, n)
    u = rng.uniform(-30, 30, n)
    w = rng.uniform(-30, 30, n)
    th = rng.uniform(280, 320, n)
    return np.stack([rho, rho * u, rho * w, rho * th])


def test_insertion_preserves_pressure_and_velocity():
    z = np.linspace(0, 10000, 41)
    thp = np.random.default_rng(3).uniform(-15, 15, z.shape)
    U = insert_perturbation(z, thp, PH)
    p_bg, th_bg, _, _ = background_pressure_theta(z, PH)
    np.testing.assert_allclose(pressure(U[3], PH), p_bg, rtol=1e-13)
    np.testing.assert_allclose(U[3] / U[0], th_bg + thp, rtol=1e-14)
    assert np.all(U[1] == 0) and np.all(U[2] == 0)


def test_isentropic_background_is_hydrostatic():
    z = np.linspace(100, 9900, 50)
    U, dU = background(z, PH)
    h = 1e-2
    Up, _ = background(z + h, PH)
    Um, _ = background(z - h, PH)
    dpdz = (pressure(Up[3], PH) - pressure(Um[3], PH)) / (2 * h)
    np.testing.assert_allclose(dpdz, -U[0] * PH.g, rtol=1e-7)
    np.testing.assert_allclose(U[3] / U[0], PH.theta0, rtol=1e-15)
    # temperature T = p/(rho R) = theta0 - g z / c_p  (Sec. 4.2)
    T = pressure(U[3], PH) / (U[0] * PH.R)
    np.testing.assert_allclose(T, PH.theta0 - PH.g * z / PH.cp, rtol=1e-13)
    np.testing.assert_allclose(dU, (Up - Um) / (2 * h), rtol=1e-7, atol=1e-12)


@pytest.mark.parametrize("d", [0, 1])
def test_hllc_consistent(d):
    U = _states(200, 1)
    np.testing.assert_allclose(hllc(U, U, d, PH), flux_n(U, d, PH), rtol=1e-13, atol=1e-9)


@pytest.mark.parametrize("d", [0, 1])
def test_hllc_reflection_symmetry(d):
    UL, UR = _states(300, 2), _states(300, 3)
    H = hllc(UL, UR, d, PH)
    Hm = hllc(mirror(UR, d), mirror(UL, d), d, PH)
    sign = -np.ones((4, 1))
    sign[1 + d] = 1.0
    np.testing.assert_allclose(Hm, sign * H, rtol=1e-12, atol=1e-8)


@pytest.mark.parametrize("d", [0, 1])
def test_hllc_resolves_isolated_contact(d):
    # equal normal velocity and pressure, different density: exact upwind flux
    rng = np.random.default_rng(5)
    n = 100
    un = rng.uniform(-20, 20, n)
    ut = rng.uniform(-5, 5, n)
    rL, rR = rng.uniform(0.6, 1.2, n), rng.uniform(0.6, 1.2, n)
    E = np.full(n, 250.0)          # same rho theta => same pressure
    def st(r):
        U = np.zeros((4, n))
        U[0] = r
        U[1 + d] = r * un
        U[2 - d] = r * ut
        U[3] = E
        return U
    UL, UR = st(rL), st(rR)
    expect = np.where(un[None] >= 0, flux_n(UL, d, PH), flux_n(UR, d, PH))
    np.testing.assert_allclose(hllc(UL, UR, d, PH), expect, rtol=1e-12, atol=1e-9)


@pytest.mark.parametrize("d", [0, 1])
def test_hllc_wall_flux(d):
    U = _states(100, 7)
    H = hllc(U, mirror(U, d), d, PH)
    # contact speed S* = 0: no mass, rho theta or tangential momentum through the wall
    c = np.sqrt(PH.gamma * pressure(U[3], PH) / U[0])
    assert np.all(np.abs(H[0]) <= 1e-13 * U[0] * c)
    assert np.all(np.abs(H[3]) <= 1e-13 * U[3] * c)
    assert np.all(np.abs(H[2 - d]) <= 1e-13 * U[0] * c * (1 + np.abs(U[2 - d] / U[0])))
    # normal momentum flux is the star pressure, above p when flow goes into the wall
    p = pressure(U[3], PH)
    into = U[1 + d] > 0
    assert np.all(H[1 + d][into] > p[into]) and np.all(H[1 + d][~into] <= p[~into])


def test_viscous_flux_is_mu_rho_grad_primitive():
    ph = Physics(mu=75.0)
    x = np.linspace(0, 1, 11)
    rho, drho = 1 + 0.1 * x, 0.1 + 0 * x
    u, du = np.sin(x), np.cos(x)
    w, dw = x ** 2, 2 * x
    th, dth = 300 + x, 1 + 0 * x
    U = np.stack([rho, rho * u, rho * w, rho * th])
    dU = np.stack([drho, drho * u + rho * du, drho * w + rho * dw, drho * th + rho * dth])
    Fv = viscous_flux(U, dU, ph)
    np.testing.assert_allclose(Fv[0], 0)
    np.testing.assert_allclose(Fv[1], 75 * rho * du, rtol=1e-13)
    np.testing.assert_allclose(Fv[2], 75 * rho * dw, rtol=1e-13, atol=1e-12)
    np.testing.assert_allclose(Fv[3], 75 * rho * dth, rtol=1e-13)


def test_uniform_background_constant():
    ph = Physics(cp=3.5, cv=2.5, g=0.0, p0=1.0, theta0=2.0, background=UNIFORM, ubg=0.5)
    U, dU = background(np.linspace(0, 1, 5), ph)
    assert np.all(dU == 0)
    np.testing.assert_allclose(U[1] / U[0], 0.5)
    np.testing.assert_allclose(pressure(U[3], ph), 1.0, rtol=1e-15)


def test_constant_n_background_hydrostatic_and_stratified():
    from oracle.physics import CONST_N
    ph = Physics(cp=1005.0, cv=717.95, g=9.80665, p0=1e5, theta0=250.0, background=CONST_N, ubg=20.0, N_bv=0.01)
    z = np.linspace(100, 9900, 40)
    U, dU = background(z, ph)
    h = 1e-2
    Up, _ = background(z + h, ph)
    Um, _ = background(z - h, ph)
    dpdz = (pressure(Up[3], ph) - pressure(Um[3], ph)) / (2 * h)
    np.testing.assert_allclose(dpdz, -U[0] * ph.g, rtol=1e-7)
    H = ph.g / ph.N_bv ** 2
    np.testing.assert_allclose(U[3] / U[0], 250.0 * np.exp(z / H), rtol=1e-13)
    # N^2 = g dln(theta)/dz
    th = lambda zz: background(zz, ph)[0][3] / background(zz, ph)[0][0]
    np.testing.assert_allclose(ph.g * (np.log(th(z + h)) - np.log(th(z - h))) / (2 * h), 1e-4, rtol=1e-6)
    np.testing.assert_allclose(U[1] / U[0], 20.0)
    np.testing.assert_allclose(dU, (Up - Um) / (2 * h), rtol=1e-6, atol=1e-12)
