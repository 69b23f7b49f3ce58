"""Inexact Jacobian-free Newton-GMRES and SDIRK time stepping (oracle).

Sec. 2.2: SDIRK2 of Ellsiepen, alpha = 1 - sqrt(2)/2, tableau
[[alpha, 0], [1-alpha, alpha]], b = (1-alpha, alpha) (stiffly accurate);
backward Euler is the one-stage case alpha = 1.  Each stage solves
G(U_s) = U_s - alpha dt f(U_s) - Ubar_s = 0 (eq. newton).
Sec. 3.1: Newton from U_s^0 = Ubar_s, G'(U^k) dU = -G(U^k), stop when
|G(U^k)| < TOL |G(U^0)|; GMRES tolerance from Eisenstat-Walker choice 2
with gamma = 0.1, alpha = 1; G'y by the finite difference with
eps = sqrt(eps_mach)/|y|.  GMRES is right preconditioned and flexible
(the preconditioner is nonlinear), restarted every m iterations,
orthogonalised by modified Gram-Schmidt, least squares by Givens rotations.
"""
from __future__ import annotations

import math

import numpy as np


def norm(x):
    return float(np.sqrt(np.sum(x * x)))


def fgmres(A, b, M=None, tol_abs=0.0, m=30, maxit=300):
    """Solve A x = b from x = 0; stop when the residual estimate |g_{j+1}| <= tol_abs.
    Returns (x, iterations, final residual estimate)."""
    x = np.zeros_like(b)
    r = b.copy()
    beta = norm(r)
    its = 0
    if beta <= tol_abs or beta == 0.0:
        return x, 0, beta
    while its < maxit:
        V = [r / beta]
        Z = []
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        j_done = 0
        conv = False
        for j in range(m):
            z = V[j] if M is None else M(V[j])
            Z.append(z)
            w = A(z)
            for i in range(j + 1):
                H[i, j] = float(np.sum(w * V[i]))
                w = w - H[i, j] * V[i]
            H[j + 1, j] = norm(w)
            V.append(w / H[j + 1, j] if H[j + 1, j] != 0.0 else w * 0.0)
            for i in range(j):
                a, c = H[i, j], H[i + 1, j]
                H[i, j] = cs[i] * a + sn[i] * c
                H[i + 1, j] = -sn[i] * a + cs[i] * c
            den = math.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = (1.0, 0.0) if den == 0.0 else (H[j, j] / den, H[j + 1, j] / den)
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            j_done = j + 1
            if abs(g[j + 1]) <= tol_abs or H[j, j] == 0.0 or its >= maxit:
                conv = abs(g[j + 1]) <= tol_abs
                break
        y = np.zeros(j_done)
        for i in range(j_done - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:j_done] @ y[i + 1:]) / H[i, i]
        for i in range(j_done):
            x = x + y[i] * Z[i]
        est = abs(g[j_done])
        if conv or its >= maxit:
            return x, its, est
        r = b - A(x)
        beta = norm(r)
        if beta <= tol_abs:
            return x, its, beta
    return x, its, beta


class NewtonStats:
    def __init__(self):
        self.newton_its = 0
        self.gmres_its = 0
        self.gmres_per_newton = []   # GMRES iterations of each Newton iteration, in order
        self.res_history = []
        self.converged = True


def newton(dg, Ubar_s, alpha_dt, tol, precond=None, ew_gamma=0.1, ew_alpha=1.0,
           eta0=0.1, eta_max=0.9, newton_max=20, gmres_m=30, gmres_max=300, stats=None):
    """Solve G(U) = U - alpha dt f(U) - Ubar_s = 0 from U^0 = Ubar_s.

    Eisenstat-Walker choice 2: eta_k = gamma (|G_k|/|G_{k-1}|)^alpha, safeguard
    eta_k >= gamma eta_{k-1}^alpha when that exceeds 0.1, eta_k <= eta_max, and
    eta_k >= 0.5 TOL |G_0| / |G_k| so GMRES does not solve beyond the Newton target.
    Returns (U, f(U))."""
    st = stats if stats is not None else NewtonStats()
    U = Ubar_s.copy()
    G, fU = dg.G(U, alpha_dt, Ubar_s)
    n0 = norm(G)
    st.res_history.append(n0)
    if n0 == 0.0:
        return U, fU
    nk_prev, eta_prev = None, None
    nk = n0
    for k in range(newton_max + 1):
        if k > 0 and nk < tol * n0:
            return U, fU
        if k == newton_max:
            break
        if k == 0:
            eta = eta0
        else:
            eta = ew_gamma * (nk / nk_prev) ** ew_alpha
            sg = ew_gamma * eta_prev ** ew_alpha
            if sg > 0.1:
                eta = max(eta, sg)
            eta = min(eta, eta_max)
            eta = max(eta, 0.5 * tol * n0 / nk)
        if precond is not None:
            precond.linearize(U, alpha_dt, fU)
            M = precond.apply
        else:
            M = None
        A = lambda y, U=U, fU=fU: dg.jv(U, fU, y, alpha_dt)
        dU, its, _ = fgmres(A, -G, M, tol_abs=eta * nk, m=gmres_m, maxit=gmres_max)
        st.gmres_its += its
        st.gmres_per_newton.append(its)
        st.newton_its += 1
        U = U + dU
        G, fU = dg.G(U, alpha_dt, Ubar_s)
        nk_prev, eta_prev = nk, eta
        nk = norm(G)
        st.res_history.append(nk)
    st.converged = False
    return U, fU


SDIRK2_ALPHA = 1.0 - math.sqrt(2.0) / 2.0


def implicit_step(dg, Un, dt, scheme=1, tol=1e-8, precond=None, stats=None, **kw):
    """One step of backward Euler (scheme 0) or SDIRK2 (scheme 1) for U' = f(U)."""
    st = stats if stats is not None else NewtonStats()
    if scheme == 0:
        U1, _ = newton(dg, Un, dt, tol, precond, stats=st, **kw)
        return U1
    a = SDIRK2_ALPHA
    U1, f1 = newton(dg, Un, a * dt, tol, precond, stats=st, **kw)
    Ubar2 = Un + (1.0 - a) * dt * f1
    U2, _ = newton(dg, Ubar2, a * dt, tol, precond, stats=st, **kw)
    return U2
