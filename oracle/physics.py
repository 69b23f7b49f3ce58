"""Model of Sec. 4 (oracle): 2D viscous compressible flow with gravity in
(rho, rho u, rho w, rho theta) variables, eq. (compressible-euler).

State arrays have the 4 components on axis 0.  Every function accepts
float64 or complex128 arrays; branch decisions use real parts only.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

ISENTROPIC, UNIFORM, CONST_N = 0, 1, 2


@dataclass
class Physics:
    cp: float = 1005.0
    cv: float = 717.95
    g: float = 9.80665
    p0: float = 1.0e5
    theta0: float = 300.0
    mu: float = 0.0            # kinematic viscosity, F_v = mu rho (0, grad u, grad w, grad theta)
    background: int = ISENTROPIC
    ubg: float = 0.0           # background wind: UNIFORM (ubg, wbg); CONST_N mean flow ubg
    wbg: float = 0.0
    N_bv: float = 0.01         # Brunt-Vaisala frequency (CONST_N)
    convective: bool = True    # test aid: False drops F_c and H_c (pure SIPG diffusion)

    @property
    def R(self):
        return self.cp - self.cv

    @property
    def gamma(self):
        return self.cp / self.cv


def pressure(E, ph: Physics):
    """EOS in theta form, p = p0 (R rho theta / p0)^gamma (inverse of eq. add-perturbation)."""
    return ph.p0 * (ph.R * E / ph.p0) ** ph.gamma


def background(z, ph: Physics):
    """Environmental atmosphere Ubar(z) and dUbar/dz, each of shape (4,)+z.shape.

    ISENTROPIC (Sec. 4.2/4.3): theta = theta0, T = theta0 - g z / c_p,
    p = p0 (T/theta0)^(c_p/R), rho = p / (R T), no wind.
    UNIFORM: rho = p0/(R theta0), theta = theta0, wind (ubg, wbg); meant for g = 0.
    """
    z = np.asarray(z, dtype=np.float64)
    U = np.zeros((4,) + z.shape)
    dU = np.zeros((4,) + z.shape)
    R = ph.R
    if ph.background == ISENTROPIC:
        T = ph.theta0 - z * ph.g / ph.cp
        Tz = -ph.g / ph.cp
        p = ph.p0 * (T / ph.theta0) ** (ph.cp / R)
        pz = ph.p0 * (ph.cp / R) * (T / ph.theta0) ** (ph.cp / R - 1.0) * Tz / ph.theta0
        rho = p / (R * T)
        rhoz = (pz * T - p * Tz) / (R * T * T)
        U[0] = rho
        U[3] = rho * ph.theta0
        dU[0] = rhoz
        dU[3] = rhoz * ph.theta0
    elif ph.background == UNIFORM:
        rho = ph.p0 / (R * ph.theta0)
        U[0] = rho
        U[1] = rho * ph.ubg
        U[2] = rho * ph.wbg
        U[3] = rho * ph.theta0
    elif ph.background == CONST_N:
        # Sec. 4.1: theta = T0 exp(z/H), T = T0 (alpha - (alpha-1) exp(z/H)),
        # p = p0 exp(c_p/R (ln(T/T0) - z/H)), H = g/N^2, alpha = g H / (c_p T0); wind ubg
        p, th, T, H, alpha = _const_n(z, ph)
        rho = p / (R * T)
        ez = np.exp(z / H)
        dT = -ph.theta0 * (alpha - 1.0) * ez / H
        dp = -rho * ph.g
        drho = (dp * T - p * dT) / (R * T * T)
        dth = th / H
        U[0] = rho
        U[1] = rho * ph.ubg
        U[3] = rho * th
        dU[0] = drho
        dU[1] = drho * ph.ubg
        dU[3] = drho * th + rho * dth
    else:
        raise ValueError("unknown background")
    return U, dU


def _const_n(z, ph: Physics):
    H = ph.g / ph.N_bv ** 2
    alpha = ph.g * H / (ph.cp * ph.theta0)
    ez = np.exp(z / H)
    th = ph.theta0 * ez
    T = ph.theta0 * (alpha - (alpha - 1.0) * ez)
    p = ph.p0 * np.exp(ph.cp / ph.R * (np.log(T / ph.theta0) - z / H))
    return p, th, T, H, alpha


def background_pressure_theta(z, ph: Physics):
    """(p~, theta~, u~, w~) of the environmental atmosphere at height z."""
    z = np.asarray(z, dtype=np.float64)
    R = ph.R
    if ph.background == ISENTROPIC:
        T = ph.theta0 - z * ph.g / ph.cp
        p = ph.p0 * (T / ph.theta0) ** (ph.cp / R)
        return p, np.full_like(z, ph.theta0), np.zeros_like(z), np.zeros_like(z)
    if ph.background == CONST_N:
        p, th, _, _, _ = _const_n(z, ph)
        return p, th, np.full_like(z, ph.ubg), np.zeros_like(z)
    rho = ph.p0 / (R * ph.theta0)
    p = pressure(rho * ph.theta0 * np.ones_like(z), ph)
    return p, np.full_like(z, ph.theta0), np.full_like(z, ph.ubg), np.full_like(z, ph.wbg)


def insert_perturbation(z, theta_p, ph: Physics):
    """eq. (add-perturbation): keep p~ and v~, theta = theta~ + theta',
    rho = p0^(R/c_p) p~^(1/gamma) / (R (theta~ + theta')).  Returns the full state U."""
    p, th, u, w = background_pressure_theta(z, ph)
    theta = th + theta_p
    rho = ph.p0 ** (ph.R / ph.cp) * p ** (1.0 / ph.gamma) / (ph.R * theta)
    return np.stack([rho, rho * u, rho * w, rho * theta])


def flux_n(U, d: int, ph: Physics):
    """Convective flux F_c(U) . e_d for d = 0 (x) or 1 (z)."""
    rho = U[0]
    un = U[1 + d] / rho
    p = pressure(U[3], ph)
    F = np.stack([U[1 + d], U[1] * un, U[2] * un, U[3] * un])
    F[1 + d] = F[1 + d] + p
    return F


def mirror(U, d: int):
    """Slip-wall ghost state: normal momentum reversed."""
    G = U.copy()
    G[1 + d] = -G[1 + d]
    return G


def _pick(cond, a, b):
    return np.where(cond, a, b)


def hllc(UL, UR, d: int, ph: Physics):
    """HLLC flux (Toro) for the theta system in direction e_d, n from L to R.

    Davis wave speeds S_L = min(u_L - c_L, u_R - c_R), S_R = max(u_L + c_L, u_R + c_R),
    c = sqrt(gamma p / rho); contact speed S* from the pressure balance; star
    states rho*_K = rho_K (S_K - u_K)/(S_K - S*) carrying (1, S* n + tangential v_K,
    theta_K); F*_K = F_K + S_K (U*_K - U_K).  Branches: 0 <= S_L -> F_L,
    0 <= S* -> F*_L, 0 <= S_R -> F*_R, else F_R.
    """
    iN, iT = 1 + d, 2 - d
    rL, rR = UL[0], UR[0]
    uL, uR = UL[iN] / rL, UR[iN] / rR
    pL, pR = pressure(UL[3], ph), pressure(UR[3], ph)
    cL = np.sqrt(ph.gamma * pL / rL)
    cR = np.sqrt(ph.gamma * pR / rR)
    a1, a2 = uL - cL, uR - cR
    SL = _pick(np.real(a1) <= np.real(a2), a1, a2)
    b1, b2 = uL + cL, uR + cR
    SR = _pick(np.real(b1) >= np.real(b2), b1, b2)
    Sst = (pR - pL + rL * uL * (SL - uL) - rR * uR * (SR - uR)) / (rL * (SL - uL) - rR * (SR - uR))
    FL = flux_n(UL, d, ph)
    FR = flux_n(UR, d, ph)

    def star(U, r, un, S):
        fac = r * (S - un) / (S - Sst)
        Us = np.empty_like(U * fac)
        Us[0] = fac
        Us[iN] = fac * Sst
        Us[iT] = fac * (U[iT] / r)
        Us[3] = fac * (U[3] / r)
        return Us

    FsL = FL + SL * (star(UL, rL, uL, SL) - UL)
    FsR = FR + SR * (star(UR, rR, uR, SR) - UR)
    zero = 0.0
    out = _pick(zero <= np.real(SR), FsR, FR)
    out = _pick(zero <= np.real(Sst), FsL, out)
    out = _pick(zero <= np.real(SL), FL, out)
    return out


def viscous_flux(U, dU, ph: Physics):
    """F_v . e_d = mu rho (0, d u, d w, d theta) written as A(U) dU with
    A = mu [[0,0,0,0], [-u,1,0,0], [-w,0,1,0], [-theta,0,0,1]] (dU = d/dx_d of U)."""
    rho = U[0]
    u, w, th = U[1] / rho, U[2] / rho, U[3] / rho
    Z = np.zeros_like(dU[0] * u)
    return ph.mu * np.stack([Z, dU[1] - u * dU[0], dU[2] - w * dU[0], dU[3] - th * dU[0]])


def sound_speed(U, ph: Physics):
    return np.sqrt(ph.gamma * pressure(U[3], ph) / U[0])
