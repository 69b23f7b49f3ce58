"""Low-order-approximation preconditioner Q^-1 = T^-1 q^-1 T (oracle), Sec. 3.2-3.5.

* FV operator f_low: the DG method with k = 0 on the subgrid with (k+1)x(k+1)
  equal subcells per element (same number of unknowns), and on every coarser
  agglomerated level (Sec. 3.2, 3.4).  Perturbation form with the background
  at the cell centres: H(u'+ubar_L, u'+ubar_R) - H(ubar_L, ubar_R); two-point
  viscous flux mu {rho} (phi_R - phi_L)/d for phi = u, w, theta.
* Transfer T: interpolation of the DG polynomial at the subcell centres with the
  mass fix of eq. (transfer-mass-fix); m_E(u) is the exact integral of the DG
  polynomial (GL quadrature).  T^-1: inverse tensor interpolation followed by
  the same mass fix in the other direction.
* Hierarchy: subgrid, then one (k+1)x(k+1) agglomeration to the DG grid (or
  2x2 steps when k+1 is a power of two), then 2x2 agglomeration while both
  counts are even.  R = volume-weighted agglomeration, P = injection (Sec. 3.4).
* MG_l(x, b; u): pre-smooth, restrict the residual R(g'x - b), recurse once (V)
  or twice (W) from v = 0 on the restricted state R u, correct x -= P v,
  post-smooth; zero-initial-guess flag skips products with x = 0 (Sec. 3.4).
* Smoother: explicit Runge-Kutta in pseudo time for dw/dtau = -(g'(u) w - b) with
  the local step dtau = sigma / (1 + alpha dt lambda_c) (Sec. 3.5), in the
  low-storage form w_k = w_0 + a_k dtau (b - g'(u) w_{k-1}), k = 1..s; the
  default s = 1, a_1 = 1 is the explicit Euler smoother of the paper's runs.
* g'(u) x by the finite difference of Sec. 3.1 applied to g(u) = u - alpha dt
  f_low(u) - ubar_s, with eps = sqrt(eps_mach)/|x| over the level's vector
  (`fd_eps` replaces the numerator sqrt(eps_mach) for the preconditioner's FD
  products, FV and DG smoothing alike; the paper's value is the default).
"""
from __future__ import annotations

import numpy as np

from .dg import DG, EPS_MACH
from .physics import Physics, background, hllc, mirror, sound_speed


def parse_mg_key(key: str):
    """'mg a b c d e f G' (Sec. 4): DG pre/post, finest FV pre/post,
    intermediate FV pre/post, cycle V or W."""
    s = key.strip()
    if not s.startswith("mg") or len(s) != 9 or s[8] not in "VW":
        raise ValueError(f"bad mg key {key!r}")
    a, b, c, d, e, f = (int(ch) for ch in s[2:8])
    return dict(dg_pre=a, dg_post=b, fine_pre=c, fine_post=d, mid_pre=e, mid_post=f,
                cycles=1 if s[8] == "V" else 2)


def hierarchy(nx, nz, k, levels):
    """Grid sizes finest -> coarsest and the agglomeration factor between
    consecutive levels."""
    n1 = k + 1
    sizes = [(nx * n1, nz * n1)]
    facs = []
    if n1 & (n1 - 1) == 0:
        r = n1
        while r > 1 and len(sizes) < levels:
            X, Z = sizes[-1]
            sizes.append((X // 2, Z // 2))
            facs.append(2)
            r //= 2
    elif len(sizes) < levels:
        sizes.append((nx, nz))
        facs.append(n1)
    while len(sizes) < levels:
        X, Z = sizes[-1]
        if X % 2 or Z % 2 or X < 2 or Z < 2:
            break
        sizes.append((X // 2, Z // 2))
        facs.append(2)
    return sizes, facs


class FVLevel:
    """k = 0 discretisation on an NX x NZ Cartesian grid."""

    def __init__(self, NX, NZ, x0, x1, z0, z1, ph: Physics, periodic_x=False):
        self.NX, self.NZ = NX, NZ
        self.Hx, self.Hz = (x1 - x0) / NX, (z1 - z0) / NZ
        self.ph = ph
        self.px = periodic_x
        self.zc = z0 + (np.arange(NZ) + 0.5) * self.Hz
        Ub, _ = background(self.zc, ph)
        self.ub = Ub[:, :, None]                # (4, NZ, 1) point values at centres

    @property
    def shape(self):
        return (4, self.NZ, self.NX)

    def rhs(self, up):
        """f_low(u') = -(1/|c|) sum_faces |e| H^pert . nu + S^pert (+ viscous)."""
        ph = self.ph
        NX, NZ, Hx, Hz = self.NX, self.NZ, self.Hx, self.Hz
        ub = np.broadcast_to(self.ub, up.shape)
        U = up + ub
        f = np.zeros_like(up * 1.0)
        # vertical faces I = 0..NX between cells I-1 and I
        Fx = np.zeros((4, NZ, NX + 1), dtype=f.dtype)
        Fx[:, :, 1:NX] = hllc(U[:, :, :-1], U[:, :, 1:], 0, ph) - hllc(ub[:, :, :-1], ub[:, :, 1:], 0, ph)
        if self.px:
            Hp = hllc(U[:, :, -1:], U[:, :, :1], 0, ph) - hllc(ub[:, :, -1:], ub[:, :, :1], 0, ph)
            Fx[:, :, :1] = Hp
            Fx[:, :, NX:] = Hp
        else:
            Ui, ui = U[:, :, :1], ub[:, :, :1]
            Fx[:, :, :1] = hllc(mirror(Ui, 0), Ui, 0, ph) - hllc(mirror(ui, 0), ui, 0, ph)
            Ui, ui = U[:, :, -1:], ub[:, :, -1:]
            Fx[:, :, NX:] = hllc(Ui, mirror(Ui, 0), 0, ph) - hllc(ui, mirror(ui, 0), 0, ph)
        # horizontal faces J = 0..NZ between cells J-1 and J
        Fz = np.zeros((4, NZ + 1, NX), dtype=f.dtype)
        Fz[:, 1:NZ] = hllc(U[:, :-1], U[:, 1:], 1, ph) - hllc(ub[:, :-1], ub[:, 1:], 1, ph)
        Ui, ui = U[:, :1], ub[:, :1]
        Fz[:, :1] = hllc(mirror(Ui, 1), Ui, 1, ph) - hllc(mirror(ui, 1), ui, 1, ph)
        Ui, ui = U[:, -1:], ub[:, -1:]
        Fz[:, NZ:] = hllc(Ui, mirror(Ui, 1), 1, ph) - hllc(ui, mirror(ui, 1), 1, ph)
        f -= (Fx[:, :, 1:] - Fx[:, :, :-1]) / Hx + (Fz[:, 1:] - Fz[:, :-1]) / Hz
        f[2] += -ph.g * up[0]
        if ph.mu != 0.0:
            f += self._viscous(U)
        return f

    def _viscous(self, U):
        ph = self.ph
        NX, NZ = self.NX, self.NZ
        rho = U[0]
        phi = np.stack([U[1] / rho, U[2] / rho, U[3] / rho])     # u, w, theta
        Vx = np.zeros((4, NZ, NX + 1), dtype=U.dtype)
        Vx[1:, :, 1:NX] = ph.mu * 0.5 * (rho[None, :, :-1] + rho[None, :, 1:]) * (phi[:, :, 1:] - phi[:, :, :-1]) / self.Hx
        if self.px:
            Vp = ph.mu * 0.5 * (rho[None, :, -1:] + rho[None, :, :1]) * (phi[:, :, :1] - phi[:, :, -1:]) / self.Hx
            Vx[1:, :, :1] = Vp
            Vx[1:, :, NX:] = Vp
        Vz = np.zeros((4, NZ + 1, NX), dtype=U.dtype)
        Vz[1:, 1:NZ] = ph.mu * 0.5 * (rho[None, :-1] + rho[None, 1:]) * (phi[:, 1:] - phi[:, :-1]) / self.Hz
        return (Vx[:, :, 1:] - Vx[:, :, :-1]) / self.Hx + (Vz[:, 1:] - Vz[:, :-1]) / self.Hz

    def dtau(self, up, alpha_dt, sigma=1.0):
        """dtau_c = sigma / (1 + alpha dt lambda_c), lambda_c = sum_faces 1/2 s_e |e|/|c|
        (+ 2 mu (1/Hx^2 + 1/Hz^2)), s_e = max over the two sides of |v.n| + c."""
        U = up + self.ub
        c = sound_speed(U, self.ph)
        sx = np.abs(U[1] / U[0]) + c
        sz = np.abs(U[2] / U[0]) + c
        ex = np.empty((self.NZ, self.NX + 1))
        ex[:, 1:-1] = np.maximum(sx[:, :-1], sx[:, 1:])
        if self.px:
            ex[:, 0] = ex[:, -1] = np.maximum(sx[:, -1], sx[:, 0])
        else:
            ex[:, 0], ex[:, -1] = sx[:, 0], sx[:, -1]
        ez = np.empty((self.NZ + 1, self.NX))
        ez[1:-1] = np.maximum(sz[:-1], sz[1:])
        ez[0], ez[-1] = sz[0], sz[-1]
        lam = 0.5 * (ex[:, :-1] + ex[:, 1:]) / self.Hx + 0.5 * (ez[:-1] + ez[1:]) / self.Hz
        lam = lam + 2.0 * self.ph.mu * (1.0 / self.Hx ** 2 + 1.0 / self.Hz ** 2)
        return sigma / (1.0 + alpha_dt * lam)


def restrict(u, fac):
    """(R u)_E = (1/|E|) sum_{q in C(E)} |q| u_q with fac x fac equal children."""
    V, NZ, NX = u.shape
    return u.reshape(V, NZ // fac, fac, NX // fac, fac).mean(axis=(2, 4))


def prolong(v, fac):
    """(P v)_q = v_E for q in C(E) (injection)."""
    return np.repeat(np.repeat(v, fac, axis=1), fac, axis=2)


class Transfer:
    """T^mf (DG -> FV subgrid) and its inverse with mass fix; with l2=True the L2
    projection onto the subcells (mass conservative, no mass fix) and its inverse."""

    def __init__(self, dg: DG, l2=False):
        self.dg = dg
        self.t = dg.t
        self.area = dg.hx * dg.hz
        self.l2 = l2

    def _mass_dg(self, u):
        # exact integral of the DG polynomial per element and variable
        return np.einsum('ba,vzxba->vzx', self.dg.mass_weights(), u)

    def _mass_fv(self, v):
        n1 = self.dg.k + 1
        return self.area / n1 ** 2 * v.sum(axis=(3, 4))

    def to_fv(self, u, massfix=True):
        """T^mf_E u = T_E u - (m_E(T_E u) - m_E(u))/|E| (eq. transfer-mass-fix), as an
        FV array (4, nz(k+1), nx(k+1)) with subcell (j, i) of element (ez, ex) at
        row ez(k+1)+j, column ex(k+1)+i."""
        V = self.t.P if self.l2 else self.t.V
        Tu = np.einsum('jb,ia,vzxba->vzxji', V, V, u)
        if massfix and not self.l2:
            Tu = Tu - ((self._mass_fv(Tu) - self._mass_dg(u)) / self.area)[..., None, None]
        return self._blocks_to_grid(Tu)

    def to_dg(self, v, massfix=True):
        """Inverse interpolation then mass fix: T^-1 v - (m_E(T^-1 v) - m_E(v))/|E|."""
        Vi = self.t.Pinv if self.l2 else self.t.Vinv
        vb = self._grid_to_blocks(v)
        u = np.einsum('bj,ai,vzxji->vzxba', Vi, Vi, vb)
        if massfix and not self.l2:
            u = u - ((self._mass_dg(u) - self._mass_fv(vb)) / self.area)[..., None, None]
        return u

    def _blocks_to_grid(self, b):
        V, nz, nx, n1, _ = b.shape
        return b.transpose(0, 1, 3, 2, 4).reshape(V, nz * n1, nx * n1)

    def _grid_to_blocks(self, v):
        V, NZ, NX = v.shape
        n1 = self.dg.k + 1
        return v.reshape(V, NZ // n1, n1, NX // n1, n1).transpose(0, 1, 3, 2, 4)


class Multigrid:
    """Q^-1 = T^-1 q^-1 T with DG pre/post smoothing (Sec. 3.2-3.5)."""

    def __init__(self, dg: DG, levels: int, mg_key="mg111111V", sigma_fv=1.0, sigma_dg=1.0,
                 massfix=True, l2=False, fd_eps=None, rk_alpha=(1.0,)):
        self.dg = dg
        self.key = parse_mg_key(mg_key)
        sizes, facs = hierarchy(dg.nx, dg.nz, dg.k, levels)
        self.sizes, self.facs = sizes, facs
        # self.levels[0] is the finest grid
        self.levels = [FVLevel(X, Z, dg.x0, dg.x1, dg.z0, dg.z1, dg.ph, dg.px) for X, Z in sizes]
        self.T = Transfer(dg, l2=l2)
        self.sigma_fv, self.sigma_dg = sigma_fv, sigma_dg
        self.massfix = massfix
        # numerator of eps = c / |x| in the preconditioner's FD products (Sec. 3.1: c = sqrt(eps_mach))
        self.fd_c = np.sqrt(EPS_MACH) if fd_eps is None else float(fd_eps)
        # stage coefficients a_1..a_s of the pseudo-time smoother (Sec. 3.5)
        self.rk_alpha = tuple(float(a) for a in rk_alpha)
        self.stats = dict(dg_calls=0, fv_calls=[0] * len(sizes), visits=[0] * len(sizes))

    # -- linearisation at the Newton iterate U^k ----------------------------
    def linearize(self, Up, alpha_dt, fU=None):
        self.Up = Up
        self.alpha_dt = alpha_dt
        self.fU = self.dg.rhs(Up) if fU is None else fU
        self.dtau_dg = self.dg.smoother_dtau(Up, alpha_dt, self.sigma_dg)
        u = self.T.to_fv(Up, self.massfix)
        self.u, self.fu, self.dtau = [], [], []
        for l, lev in enumerate(self.levels):
            if l > 0:
                u = restrict(u, self.facs[l - 1])
            self.u.append(u)
            self.fu.append(lev.rhs(u))
            self.dtau.append(lev.dtau(u, alpha_dt, self.sigma_fv))

    # -- FV level operators -------------------------------------------------
    def gprime(self, l, x):
        """g'(u_l) x ~ x - alpha dt (f_low(u_l + eps x) - f_low(u_l))/eps."""
        nx_ = np.sqrt(np.sum(x * x))
        if nx_ == 0.0:
            return np.zeros_like(x)
        eps = self.fd_c / nx_
        self.stats['fv_calls'][l] += 1
        return x - self.alpha_dt * (self.levels[l].rhs(self.u[l] + eps * x) - self.fu[l]) / eps

    def rk_step(self, x, zero, dtau, b, gprime):
        """One pseudo-time step of the low-storage explicit RK smoother:
        x_k = x_0 + a_k dtau (b - g' x_{k-1}), k = 1..s, from x_0 = x (x_0 = 0 when
        `zero`, whose first stage needs no product).  s = 1, a_1 = 1: explicit Euler."""
        x0, xk = x, x
        for k, a in enumerate(self.rk_alpha):
            if zero and k == 0:
                xk = (a * dtau) * b
            elif zero:
                xk = (a * dtau) * (b - gprime(xk))
            else:
                xk = x0 + (a * dtau) * (b - gprime(xk))
        return xk

    def smooth(self, l, x, b, zero, steps):
        """Pseudo-time smoothing steps on FV level l (explicit Euler by default)."""
        for _ in range(steps):
            x = self.rk_step(x, zero, self.dtau[l][None], b, lambda v: self.gprime(l, v))
            zero = False
        return x, zero

    def mg(self, l, x, b, zero):
        """MG_l(x, b; u_l), level index l counted from the finest (0)."""
        nl = len(self.levels)
        self.stats['visits'][l] += 1
        if l == 0:
            pre, post = self.key['fine_pre'], self.key['fine_post']
        else:
            pre, post = self.key['mid_pre'], self.key['mid_post']
        x, zero = self.smooth(l, x, b, zero, pre)
        if l < nl - 1:
            res = -b if zero else self.gprime(l, x) - b
            r = restrict(res, self.facs[l])
            v = np.zeros_like(r)
            vz = True
            for _ in range(self.key['cycles']):
                v = self.mg(l + 1, v, r, vz)
                vz = False
            x = (0.0 * b if zero else x) - prolong(v, self.facs[l])
            zero = False
        x, zero = self.smooth(l, x, b, zero, post)
        if zero:
            x = np.zeros_like(b)
        return x

    # -- DG level --------------------------------------------------------------
    def dg_gprime(self, z):
        self.stats['dg_calls'] += 1
        nz_ = np.sqrt(np.sum(z * z))
        if nz_ == 0.0:
            return np.zeros_like(z)
        return self.dg.jv(self.Up, self.fU, z, self.alpha_dt, eps=self.fd_c / nz_)

    def apply(self, r):
        """z = Q^-1 r: DG pre-smoothing, transfer of the DG residual, FV multigrid
        from zero, transfer back and correction, DG post-smoothing."""
        dtau = self.dtau_dg[None, :, :, None, None]
        z = np.zeros_like(r)
        zero = True
        for _ in range(self.key['dg_pre']):
            z = self.rk_step(z, zero, dtau, r, self.dg_gprime)
            zero = False
        d = r if zero else r - self.dg_gprime(z)
        b = self.T.to_fv(d, self.massfix)
        x = self.mg(0, np.zeros_like(b), b, True)
        z = z + self.T.to_dg(x, self.massfix)
        for _ in range(self.key['dg_post']):
            z = self.rk_step(z, False, dtau, r, self.dg_gprime)
        return z
