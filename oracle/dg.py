"""Well-balanced DG operator f = M^-1 L_h(U') (oracle), Sec. 2.1 and Sec. 4.

Unknowns are the perturbations U' = U - Ubar of the nodal values on the
tensor Gauss-Legendre nodes (eq. perturbed-euler).  Array layout
(4, nz, nx, k+1, k+1) = [variable, element row ez, element column ex,
node index b along z, node index a along x].

<psi, L_h> = <psi, K_h> + <psi, I_h>           (eq. convDiscr)
K_h: int_E (F_c^pert - F_v) : grad psi + S^pert . psi      (eq. elementint)
I_h: interior faces: {F_v(U,[[U]])^T : grad psi} + {F_v} : [[psi]]
     all faces:     -(H_c^pert - H_v) : [[psi]]               (eq. surfaceint)
with H_c = HLLC, the viscous numerical flux read as symmetric interior
penalty on the variables F_v differentiates: the penalty term is
C_IP (k+1)^2 / h {A(U)} [[U]] = C_IP (k+1)^2 / h mu {rho} ([[u]], [[w]], [[theta]])
to first order (A(U) dU = mu (0, d(rho u) - u d rho, d(rho w) - w d rho,
d(rho theta) - theta d rho), {.} the mean of the two sides), slip walls with a
mirrored ghost state and no viscous wall flux.
Volume and face integrals use the collocated GL nodes, so the mass matrix is
diagonal (Sec. 2.2) and f = M^-1 L_h is a per-node division.
"""
from __future__ import annotations

import numpy as np

from .physics import Physics, background, flux_n, hllc, mirror, viscous_flux, sound_speed
from .tables import Tables

EPS_MACH = 2.0 ** -52


class DG:
    def __init__(self, nx, nz, x0, x1, z0, z1, k, ph: Physics, periodic_x=False,
                 periodic_z=False, c_ip=2.0):
        self.nx, self.nz, self.k = nx, nz, k
        self.x0, self.x1, self.z0, self.z1 = x0, x1, z0, z1
        self.hx, self.hz = (x1 - x0) / nx, (z1 - z0) / nz
        self.ph = ph
        self.px, self.pz = periodic_x, periodic_z
        self.c_ip = c_ip
        self.t = t = Tables(k)
        n1 = k + 1
        ex = np.arange(nx)[None, :, None, None]
        ez = np.arange(nz)[:, None, None, None]
        # node coordinates [ez, ex, b, a]
        self.X = np.broadcast_to(x0 + (ex + (1 + t.xi[None, None, None, :]) / 2) * self.hx, (nz, nx, n1, n1)).copy()
        self.Z = np.broadcast_to(z0 + (ez + (1 + t.xi[None, None, :, None]) / 2) * self.hz, (nz, nx, n1, n1)).copy()
        self.shape = (4, nz, nx, n1, n1)
        self.N = 4 * nz * nx * n1 * n1
        # background at volume nodes, vertical-face points (z of node rows) and
        # horizontal faces (z = z0 + j hz, j = 0..nz)
        self.Ub, self.dUb = background(self.Z, ph)
        zrow = self.Z[:, 0, :, 0]                      # (nz, b)
        self.Ubv, self.dUbv = background(zrow, ph)      # (4, nz, b)
        zf = z0 + np.arange(nz + 1) * self.hz
        self.Ubh, self.dUbh = background(zf, ph)        # (4, nz+1)

    # -- helpers -------------------------------------------------------------
    def zeros(self, dtype=np.float64):
        return np.zeros(self.shape, dtype=dtype)

    def mass_weights(self):
        """Diagonal of M per node: w_a w_b hx hz / 4."""
        w = self.t.w
        return (w[None, :] * w[:, None]) * self.hx * self.hz / 4.0   # [b, a]

    # -- operator ------------------------------------------------------------
    def rhs(self, Up):
        """f = M^-1 L_h(U') for perturbation nodal values Up of shape (4,nz,nx,k+1,k+1)."""
        t, ph = self.t, self.ph
        hx, hz = self.hx, self.hz
        w, D = t.w, t.D
        U = Up + self.Ub
        f = np.zeros_like(Up * 1.0)

        # ---- element integrals (eq. elementint) ----
        Gx = np.zeros_like(f)
        Gz = np.zeros_like(f)
        if ph.convective:
            Gx = Gx + (flux_n(U, 0, ph) - flux_n(self.Ub, 0, ph))
            Gz = Gz + (flux_n(U, 1, ph) - flux_n(self.Ub, 1, ph))
        if ph.mu != 0.0:
            # grad U at the nodes: DG derivative of U' plus analytic dUbar/dz
            dUx = (2.0 / hx) * np.einsum('qa,vzxba->vzxbq', D, Up)
            dUz = (2.0 / hz) * np.einsum('br,vzxra->vzxba', D, Up) + self.dUb
            Gx = Gx - viscous_flux(U, dUx, ph)
            Gz = Gz - viscous_flux(U, dUz, ph)
        # int_E G : grad psi_ab / (w_a w_b |J|)
        f += (2.0 / hx) * np.einsum('q,qa,vzxbq->vzxba', w, D, Gx) / w[None, None, None, None, :]
        f += (2.0 / hz) * np.einsum('r,rb,vzxra->vzxba', w, D, Gz) / w[None, None, None, :, None]
        # gravity source S^pert = S(U'+Ubar) - S(Ubar) = (0, 0, -rho' g, 0)
        f[2] += -ph.g * Up[0]

        # ---- face integrals (eq. surfaceint) ----
        self._faces_x(Up, U, f)
        self._faces_z(Up, U, f)
        return f

    def _faces_x(self, Up, U, f):
        """Vertical faces, normal +x; face points are the node rows b."""
        t, ph = self.t, self.ph
        nx, hx, hz = self.nx, self.hx, self.hz
        lp, lm = t.lp, t.lm
        trR = np.einsum('a,vzxba->vzxb', lp, Up)     # trace at xi=+1 of each element
        trL = np.einsum('a,vzxba->vzxb', lm, Up)     # trace at xi=-1
        Ubf = self.Ubv[:, :, None, :]                # (4, nz, 1, b)
        # face fx sits between elements fx-1 and fx (fx = 0..nx)
        H = np.zeros(trR.shape[:2] + (nx + 1,) + trR.shape[3:], dtype=(Up * 1.0).dtype)
        if ph.convective:
            # interior faces
            UL = trR[:, :, :-1] + Ubf
            UR = trL[:, :, 1:] + Ubf
            H[:, :, 1:nx] = hllc(UL, UR, 0, ph) - hllc(Ubf + 0 * UL, Ubf + 0 * UR, 0, ph)
            if self.px:
                UL = trR[:, :, -1:] + Ubf
                UR = trL[:, :, :1] + Ubf
                Hp = hllc(UL, UR, 0, ph) - hllc(Ubf + 0 * UL, Ubf + 0 * UR, 0, ph)
                H[:, :, :1] = Hp
                H[:, :, nx:] = Hp
            else:
                Ui = trL[:, :, :1] + Ubf
                H[:, :, :1] = hllc(mirror(Ui, 0), Ui, 0, ph) - hllc(mirror(Ubf + 0 * Ui, 0), Ubf + 0 * Ui, 0, ph)
                Ui = trR[:, :, -1:] + Ubf
                H[:, :, nx:] = hllc(Ui, mirror(Ui, 0), 0, ph) - hllc(Ubf + 0 * Ui, mirror(Ubf + 0 * Ui, 0), 0, ph)
        # -int H.nu psi: left face of an element adds +l_a(-1) H, right face -l_a(+1) H
        sc = (2.0 / hx) / t.w                                  # [a]
        f += sc[None, None, None, None, :] * (
            lm[None, None, None, None, :] * H[:, :, :-1, :, None]
            - lp[None, None, None, None, :] * H[:, :, 1:, :, None])

        if self.ph.mu != 0.0:
            self._viscous_faces_x(Up, f, trR, trL)

    def _viscous_faces_x(self, Up, f, trR, trL):
        t, ph = self.t, self.ph
        nx, hx = self.nx, self.hx
        Ubf = self.Ubv[:, :, None, :]
        # normal-gradient traces of U' at xi = +1 and xi = -1 (dUbar/dx = 0)
        gxR = (2.0 / hx) * np.einsum('a,vzxba->vzxb', t.dlp, Up)
        gxL = (2.0 / hx) * np.einsum('a,vzxba->vzxb', t.dlm, Up)
        # interior face pairs (L = element ex, R = element ex+1)
        pairs = [(np.arange(nx - 1), np.arange(1, nx))]
        if self.px:
            pairs.append((np.array([nx - 1]), np.array([0])))
        eta = self.c_ip * (t.k + 1) ** 2 * ph.mu / hx
        sc = (2.0 / hx) / t.w
        for iL, iR in pairs:
            ULp, URp = trR[:, :, iL], trL[:, :, iR]
            UL, UR = ULp + Ubf, URp + Ubf
            FvL = viscous_flux(UL, gxR[:, :, iL], ph)
            FvR = viscous_flux(UR, gxL[:, :, iR], ph)
            avg = 0.5 * (FvL + FvR)
            J = ULp - URp
            symL = 0.5 * viscous_flux(UL, J, ph)       # 1/2 A(U_L) [U]
            symR = 0.5 * viscous_flux(UR, J, ph)
            # penalty on the jumps of u, w, theta: (eta / mu) {A(U)} [U]
            pen = (eta / ph.mu) * (symL + symR)
            # element L (outward +x, trace at +1)
            f[:, :, iL] += sc[None, None, None, None, :] * (
                t.lp[None, None, None, None, :] * (avg - pen)[..., None]
                + (2.0 / hx) * t.dlp[None, None, None, None, :] * symL[..., None])
            # element R (outward -x, trace at -1)
            f[:, :, iR] += sc[None, None, None, None, :] * (
                t.lm[None, None, None, None, :] * (-avg + pen)[..., None]
                + (2.0 / hx) * t.dlm[None, None, None, None, :] * symR[..., None])

    def _faces_z(self, Up, U, f):
        """Horizontal faces, normal +z; face points are the node columns a."""
        t, ph = self.t, self.ph
        nz, hx, hz = self.nz, self.hx, self.hz
        lp, lm = t.lp, t.lm
        trT = np.einsum('b,vzxba->vzxa', lp, Up)     # trace at eta=+1
        trB = np.einsum('b,vzxba->vzxa', lm, Up)     # trace at eta=-1
        Ubh = self.Ubh                                # (4, nz+1)
        H = np.zeros((4, nz + 1) + trT.shape[2:], dtype=(Up * 1.0).dtype)
        if ph.convective:
            Uf = Ubh[:, 1:nz, None, None]
            UB = trT[:, :-1] + Uf
            UT = trB[:, 1:] + Uf
            H[:, 1:nz] = hllc(UB, UT, 1, ph) - hllc(Uf + 0 * UB, Uf + 0 * UT, 1, ph)
            if self.pz:
                Uf = Ubh[:, :1, None, None]
                UB = trT[:, -1:] + Uf
                UT = trB[:, :1] + Uf
                Hp = hllc(UB, UT, 1, ph) - hllc(Uf + 0 * UB, Uf + 0 * UT, 1, ph)
                H[:, :1] = Hp
                H[:, nz:] = Hp
            else:
                Uf = Ubh[:, :1, None, None]
                Ui = trB[:, :1] + Uf
                H[:, :1] = hllc(mirror(Ui, 1), Ui, 1, ph) - hllc(mirror(Uf + 0 * Ui, 1), Uf + 0 * Ui, 1, ph)
                Uf = Ubh[:, nz:, None, None]
                Ui = trT[:, -1:] + Uf
                H[:, nz:] = hllc(Ui, mirror(Ui, 1), 1, ph) - hllc(Uf + 0 * Ui, mirror(Uf + 0 * Ui, 1), 1, ph)
        sc = (2.0 / hz) / t.w                                   # [b]
        f += sc[None, None, None, :, None] * (
            lm[None, None, None, :, None] * H[:, :-1, :, None, :]
            - lp[None, None, None, :, None] * H[:, 1:, :, None, :])
        if self.ph.mu != 0.0:
            self._viscous_faces_z(Up, f, trT, trB)

    def _viscous_faces_z(self, Up, f, trT, trB):
        t, ph = self.t, self.ph
        nz, hx, hz = self.nz, self.hx, self.hz
        # normal-gradient traces of U' at eta = +1 and eta = -1
        gzT = (2.0 / hz) * np.einsum('b,vzxba->vzxa', t.dlp, Up)
        gzB = (2.0 / hz) * np.einsum('b,vzxba->vzxa', t.dlm, Up)
        pairs = [(np.arange(nz - 1), np.arange(1, nz), np.arange(1, nz))]
        if self.pz:
            pairs.append((np.array([nz - 1]), np.array([0]), np.array([0])))
        eta = self.c_ip * (t.k + 1) ** 2 * ph.mu / hz
        sc = (2.0 / hz) / t.w
        for iB, iT, jf in pairs:
            Uf = self.Ubh[:, jf, None, None]
            dUf = self.dUbh[:, jf, None, None]
            UBp, UTp = trT[:, iB], trB[:, iT]
            UB, UT = UBp + Uf, UTp + Uf
            FvB = viscous_flux(UB, gzT[:, iB] + dUf, ph)
            FvT = viscous_flux(UT, gzB[:, iT] + dUf, ph)
            avg = 0.5 * (FvB + FvT)
            J = UBp - UTp
            symB = 0.5 * viscous_flux(UB, J, ph)
            symT = 0.5 * viscous_flux(UT, J, ph)
            pen = (eta / ph.mu) * (symB + symT)
            f[:, iB] += sc[None, None, None, :, None] * (
                t.lp[None, None, None, :, None] * (avg - pen)[:, :, :, None, :]
                + (2.0 / hz) * t.dlp[None, None, None, :, None] * symB[:, :, :, None, :])
            f[:, iT] += sc[None, None, None, :, None] * (
                t.lm[None, None, None, :, None] * (-avg + pen)[:, :, :, None, :]
                + (2.0 / hz) * t.dlm[None, None, None, :, None] * symT[:, :, :, None, :])

    # -- nonlinear system and FD Jacobian-vector product (Sec. 2.2, 3.1) -------
    def G(self, Up, alpha_dt, Ubar_s, fU=None):
        """G(U) = U - alpha dt f(U) - Ubar_s (eq. newton), in perturbation variables."""
        if fU is None:
            fU = self.rhs(Up)
        return Up - alpha_dt * fU - Ubar_s, fU

    def jv(self, Up, fU, y, alpha_dt, eps=None):
        """G'(U) y ~ [G(U + eps y) - G(U)] / eps with eps = sqrt(eps_mach)/|y| (Sec. 3.1).

        The identity part of G is linear, so it contributes y exactly:
        G'(U) y ~ y - alpha dt (f(U + eps y) - f(U)) / eps."""
        if eps is None:
            ny = np.sqrt(np.sum(y * y))
            if ny == 0.0:
                return np.zeros_like(y)
            eps = np.sqrt(EPS_MACH) / ny
        return y - alpha_dt * (self.rhs(Up + eps * y) - fU) / eps

    def jv_exact(self, Up, y, alpha_dt, h=1e-30):
        """Complex-step derivative: G'(U) y = y - alpha dt Im f(U + i h y)/h (test aid)."""
        return y - alpha_dt * np.imag(self.rhs(Up + 1j * h * y)) / h

    # -- DG smoother step size (pseudo-time, Sec. 3.5) -------------------------
    def smoother_dtau(self, Up, alpha_dt, sigma=1.0):
        """Per-element pseudo-time step dtau_E = sigma / (1 + alpha dt lambda_E),
        lambda_E = (k+1)^2 max_nodes(|v| + c) (1/hx + 1/hz) + 2 mu (k+1)^4 (1/hx^2 + 1/hz^2)."""
        U = Up + self.Ub
        v = np.sqrt((U[1] / U[0]) ** 2 + (U[2] / U[0]) ** 2) + sound_speed(U, self.ph)
        vmax = v.max(axis=(2, 3))                   # (nz, nx)
        n1 = self.k + 1
        lam = n1 ** 2 * vmax * (1.0 / self.hx + 1.0 / self.hz)
        lam = lam + 2.0 * self.ph.mu * n1 ** 4 * (1.0 / self.hx ** 2 + 1.0 / self.hz ** 2)
        return sigma / (1.0 + alpha_dt * lam)

    # -- initial data (Sec. 2.2: L2 projection = nodal interpolation on GL) ----
    def init_state(self, theta_p):
        from .physics import insert_perturbation
        U = insert_perturbation(self.Z, theta_p, self.ph)
        return U - self.Ub
