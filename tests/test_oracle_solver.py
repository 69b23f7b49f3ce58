"""Pins of the oracle solvers: FGMRES, Eisenstat-Walker Newton, SDIRK2 / BE (Sec. 2.2, 3.1)."""
import math

import numpy as np
import pytest

import synth
from oracle.dg import DG
from oracle.fv import Multigrid
from oracle.physics import Physics, UNIFORM
from oracle.solver import SDIRK2_ALPHA, NewtonStats, fgmres, implicit_step, newton, norm

ROBERT = Physics(cp=1005.0, cv=717.95, g=9.80665, p0=1e5, theta0=300.0)
UNIT = Physics(cp=3.5, cv=2.5, g=0.0, p0=1.0, theta0=1.0, background=UNIFORM)


def test_sdirk2_coefficient():
    # Sec. 2.2: alpha = 1 - sqrt(2)/2, the root of alpha^2 - 2 alpha + 1/2 = 0 in (0,1)
    assert abs(SDIRK2_ALPHA - (2 - math.sqrt(2)) / 2) <= 1e-16
    assert abs(SDIRK2_ALPHA ** 2 - 2 * SDIRK2_ALPHA + 0.5) <= 1e-16


@pytest.mark.parametrize("m", [5, 30])
def test_fgmres_matches_dense_solve(m):
    rng = np.random.default_rng(0)
    n = 60
    A = np.eye(n) * 4 + rng.standard_normal((n, n)) / np.sqrt(n)
    b = rng.standard_normal(n)
    Minv = np.linalg.inv(np.diag(np.diag(A)) + 0.1 * np.triu(A, 1))
    x, its, est = fgmres(lambda v: A @ v, b, lambda v: Minv @ v, tol_abs=1e-13 * norm(b), m=m, maxit=500)
    xe = np.linalg.solve(A, b)
    assert norm(x - xe) <= 1e-10 * norm(xe)
    # estimate equals the true residual
    assert abs(norm(b - A @ x) - est) <= 1e-10 * norm(b)


def test_fgmres_on_the_dg_jacobian_matches_dense_lu():
    dg = DG(2, 2, 0.0, 2000.0, 0.0, 2000.0, 2, ROBERT)
    Up = dg.init_state(synth.Bubble(2.0, 1000.0, 800.0, 700.0, 700.0).theta(dg.X, dg.Z))
    adt = 3.0
    N = dg.N
    J = np.empty((N, N))
    for i in range(N):
        e = np.zeros(N)
        e[i] = 1.0
        J[:, i] = dg.jv_exact(Up, e.reshape(dg.shape), adt).ravel()
    b = synth.random_perturbation(dg.shape[1:], 1).ravel()
    xe = np.linalg.solve(J, b)
    x, _, _ = fgmres(lambda v: (J @ v.ravel()).reshape(dg.shape), b.reshape(dg.shape),
                     tol_abs=1e-14 * norm(b), m=30, maxit=2000)
    assert norm(x.ravel() - xe) <= 1e-10 * norm(xe)
    fU = dg.rhs(Up)
    x, _, _ = fgmres(lambda v: dg.jv(Up, fU, v, adt, eps=1e-7), b.reshape(dg.shape),
                     tol_abs=1e-12 * norm(b), m=30, maxit=2000)
    # FD products carry ~1e-7 relative error, amplified by the conditioning of G'
    assert norm(x.ravel() - xe) <= 1e-4 * norm(xe)


def _bubble_case(nx=8, nz=4, k=2):
    w = synth.scaled(synth.BUBBLE_Q2_20x10, nx, nz, k=k)
    dg = DG(w.nx, w.nz, w.x0, w.x1, w.z0, w.z1, w.k, ROBERT)
    Up = dg.init_state(w.theta_pert(dg.X, dg.Z))
    return w, dg, Up


def test_newton_reaches_tolerance_and_ew_forcing():
    w, dg, Up = _bubble_case()
    st = NewtonStats()
    tol = 1e-8
    U, fU = newton(dg, Up, w.dt, tol, stats=st)
    G, _ = dg.G(U, w.dt, Up, fU)
    assert st.converged and norm(G) < tol * st.res_history[0]
    # Eisenstat-Walker choice 2 with gamma=0.1, alpha=1: GMRES reduces by ~eta,
    # so each Newton step shrinks |G| by at least ~1/(2 eta) until the floor
    h = st.res_history
    assert all(h[i + 1] < 0.5 * h[i] for i in range(len(h) - 1))


def test_preconditioned_and_plain_newton_agree():
    w, dg, Up = _bubble_case(10, 5, 2)
    U0 = implicit_step(dg, Up, w.dt, scheme=0, tol=1e-8)
    mg = Multigrid(dg, 3, "mg111111V")
    U1 = implicit_step(dg, Up, w.dt, scheme=0, tol=1e-8, precond=mg)
    assert norm(U1 - U0) <= 1e-8 * norm(U0 - Up) * 10
    assert norm(U1 - U0) <= 1e-8 * norm(U0)


@pytest.mark.parametrize("scheme,order", [(0, 0.9), (1, 1.85)])
def test_time_order(scheme, order):
    # smooth advected density wave on a fixed grid; error vs a fine-step solution
    dg = DG(6, 1, 0, 1, 0, 1, 2, UNIT, periodic_x=True, periodic_z=True)
    rho = 1 + 0.2 * np.sin(2 * np.pi * dg.X)
    U0 = np.stack([rho, rho, 0 * rho, np.full_like(rho, 1 / UNIT.R)]) - dg.Ub
    T = 0.08

    def run(nt):
        U = U0
        for _ in range(nt):
            U = implicit_step(dg, U, T / nt, scheme=scheme, tol=1e-12)
        return U
    ref = run(64)
    e = [norm(run(n) - ref) for n in (4, 8)]
    assert np.log2(e[0] / e[1]) > order
