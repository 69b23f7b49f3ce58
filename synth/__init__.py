"""Seeded synthetic workloads shaped like the paper's atmospheric test cases.

This module holds no arithmetic of the method (no EOS, no background
atmosphere, no basis, no operator).  It only fixes workload parameters
(grids, orders, physical constants, time steps, solver keys), the
analytic potential-temperature perturbations that the test cases
prescribe (Sec. 4.3 cosine cold bubble, reused with other centres and
signs for the warm-bubble workloads), seeded noise, seeded random
perturbation states for parity tests, ensemble draws and Poisson request
streams.  Both the CUDA path and the oracle take their inputs from here;
neither imports the other.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import Optional

import numpy as np

# Physical constant sets quoted by the paper.
# Rising bubble / inertia gravity: c_p, c_v, g of Sec. 4.2 (c_p=1005 J/(kg K)).
PHYS_ROBERT = dict(cp=1005.0, cv=717.95, g=9.80665, p0=1.0e5)
# Density current: c_p, c_v, g of Sec. 4.3.
PHYS_STRAKA = dict(cp=1004.0, cv=717.0, g=9.81, p0=1.0e5)


@dataclass(frozen=True)
class Bubble:
    """theta'(x,z) = A/2 (1 + cos(pi r)) for r<1, r^2 = ((x-xc)/xr)^2 + ((z-zc)/zr)^2."""
    amp: float
    xc: float
    zc: float
    xr: float
    zr: float

    def theta(self, x, z):
        x = np.asarray(x, dtype=np.float64)
        z = np.asarray(z, dtype=np.float64)
        r = np.sqrt(((x - self.xc) / self.xr) ** 2 + ((z - self.zc) / self.zr) ** 2)
        return np.where(r < 1.0, 0.5 * self.amp * (1.0 + np.cos(np.pi * np.minimum(r, 1.0))), 0.0)


@dataclass(frozen=True)
class FlattenedGaussian:
    """theta'(x,z) = A for r < a, A exp(-(r-a)^2/s^2) for 0 <= r-a <= 3s, else 0,
    r = |(x,z) - (xc,zc)|  (the rising-bubble perturbation of Sec. 4.2)."""
    amp: float
    xc: float
    zc: float
    a: float
    s: float

    def theta(self, x, z):
        x = np.asarray(x, dtype=np.float64)
        z = np.asarray(z, dtype=np.float64)
        d = np.sqrt((x - self.xc) ** 2 + (z - self.zc) ** 2) - self.a
        g = np.exp(-np.maximum(d, 0.0) ** 2 / self.s ** 2)
        return self.amp * np.where(d < 0.0, 1.0, np.where(d <= 3.0 * self.s, g, 0.0))


@dataclass(frozen=True)
class Wave:
    """theta'(x,z) = theta_c sin(pi z/Z) / (1 + ((x-xc)/a)^2)  (Sec. 4.1 perturbation)."""
    theta_c: float
    xc: float
    a: float
    Z: float

    def theta(self, x, z):
        x = np.asarray(x, dtype=np.float64)
        z = np.asarray(z, dtype=np.float64)
        return self.theta_c * np.sin(np.pi * z / self.Z) / (1.0 + ((x - self.xc) / self.a) ** 2)


@dataclass(frozen=True)
class Workload:
    name: str
    nx: int
    nz: int
    x0: float
    x1: float
    z0: float
    z1: float
    k: int
    cp: float
    cv: float
    g: float
    p0: float
    theta0: float
    mu: float
    bubble: object               # Bubble or Wave: theta'(x, z)
    noise_amp: float = 0.0
    noise_seed: int = 0
    scheme: int = 1              # 0 backward Euler, 1 SDIRK2
    cfl_mult: float = 10.0       # dt = cfl_mult * dt_acoustic (unless dt given)
    dt_fixed: Optional[float] = None
    steps: int = 1
    fv_levels: int = 3
    mg_key: str = "mg111111V"
    newton_tol: float = 1e-8
    periodic_x: bool = False
    background: int = 0          # 0 isentropic, 1 uniform, 2 constant Brunt-Vaisala frequency
    ubg: float = 0.0             # mean flow of the environmental atmosphere (background 1, 2)
    N_bv: float = 0.01           # Brunt-Vaisala frequency (background 2)

    @property
    def n_el(self) -> int:
        return self.nx * self.nz

    @property
    def n_unknowns(self) -> int:
        return 4 * self.n_el * (self.k + 1) ** 2

    @property
    def hx(self) -> float:
        return (self.x1 - self.x0) / self.nx

    @property
    def hz(self) -> float:
        return (self.z1 - self.z0) / self.nz

    def dt_acoustic(self) -> float:
        """h_min / ((2k+1) c_max) with c_max the surface sound speed sqrt(gamma R theta0)."""
        R = self.cp - self.cv
        c = math.sqrt(self.cp / self.cv * R * self.theta0)
        return min(self.hx, self.hz) / ((2 * self.k + 1) * c)

    @property
    def dt(self) -> float:
        return self.dt_fixed if self.dt_fixed is not None else self.cfl_mult * self.dt_acoustic()

    def theta_pert(self, x, z):
        """Perturbation theta' at the given node coordinates, plus seeded nodal noise.

        x, z have the DG node shape (nz, nx, k+1, k+1) = [ez, ex, b, a]."""
        th = self.bubble.theta(x, z)
        if self.noise_amp > 0.0:
            th = th + self.noise(th.shape)
        return th

    def noise(self, shape):
        rng = np.random.Generator(np.random.Philox(self.noise_seed))
        return rng.uniform(-self.noise_amp, self.noise_amp, size=shape)


# Workload 1: Q2 on 20x10 quads over [0,20km]x[0,10km], +2K cosine warm bubble
# (r=2km, centre (10km, 2km)), one backward-Euler step at dt = 10x acoustic CFL,
# 3x3 FV subcells per element, 3 multigrid levels.
BUBBLE_Q2_20x10 = Workload(
    name="warm-bubble Q2 20x10 (7,200 DOF), 1 BE step, dt=10x acoustic",
    nx=20, nz=10, x0=0.0, x1=20000.0, z0=0.0, z1=10000.0, k=2,
    theta0=300.0, mu=0.0, bubble=Bubble(2.0, 10000.0, 2000.0, 2000.0, 2000.0),
    scheme=0, cfl_mult=10.0, steps=1, fv_levels=3, **PHYS_ROBERT)

# Workload 2: same state on Q3 160x80 plus seeded +-0.1K white noise on theta,
# 10 SDIRK2 steps at dt = 20x acoustic CFL, 4x4 subcells, 5 MG levels.
BUBBLE_Q3_160x80 = Workload(
    name="warm-bubble Q3 160x80 (819,200 DOF), SDIRK2, dt=20x acoustic",
    nx=160, nz=80, x0=0.0, x1=20000.0, z0=0.0, z1=10000.0, k=3,
    theta0=300.0, mu=0.0, bubble=Bubble(2.0, 10000.0, 2000.0, 2000.0, 2000.0),
    noise_amp=0.1, noise_seed=2505,
    scheme=1, cfl_mult=20.0, steps=10, fv_levels=5, **PHYS_ROBERT)

# Workload 3: viscous density current, mu = 75 m^2/s, Q2 on 256x32 over
# [0,51.2km]x[0,6.4km], -15K cosine cold bubble (xr=4km, zr=2km, centre (0,3km)),
# SDIRK2 at dt = 1 s, 20 steps, 4 MG levels.
DENSITY_CURRENT_Q2_256x32 = Workload(
    name="viscous density current Q2 256x32 (294,912 DOF), SDIRK2, dt=1s",
    nx=256, nz=32, x0=0.0, x1=51200.0, z0=0.0, z1=6400.0, k=2,
    theta0=300.0, mu=75.0, bubble=Bubble(-15.0, 0.0, 3000.0, 4000.0, 2000.0),
    scheme=1, dt_fixed=1.0, steps=20, fv_levels=4, **PHYS_STRAKA)


# Workload 4: non-hydrostatic inertia gravity wave (Sec. 4.1): [0,300km]x[0,10km],
# periodic in x, constant N = 0.01/s, T0 = 250 K, mean flow 20 m/s,
# theta' = 0.01 K sin(pi z/10km) / (1 + ((x-100km)/5km)^2); Q3 on 80x3 quads
# (node spacing ~940 m in x), SDIRK2 at dt = 25 s, 3 MG levels.
INERTIA_GRAVITY_Q3_80x3 = Workload(
    name="inertia gravity Q3 80x3 (15,360 DOF), SDIRK2, dt=25s",
    nx=80, nz=3, x0=0.0, x1=300000.0, z0=0.0, z1=10000.0, k=3,
    theta0=250.0, mu=0.0, bubble=Wave(0.01, 100000.0, 5000.0, 10000.0),
    scheme=1, dt_fixed=25.0, steps=120, fv_levels=3, periodic_x=True,
    background=2, ubg=20.0, N_bv=0.01, **PHYS_ROBERT)


# Workload 5: rising bubble (Sec. 4.2): [0,1000m]x[0,2000m], neutral atmosphere
# theta0 = 303.15 K, flattened Gaussian theta' (A = 0.5 K, centre (500 m, 520 m),
# a = 50 m, s = 100 m), slip walls; DG Q3 on 40 x 80 quads (25 m elements),
# 5 FV levels, SDIRK2 at the paper's dt = 10 s.
RISING_BUBBLE_Q3_40x80 = Workload(
    name="rising bubble Q3 40x80 (204,800 DOF), SDIRK2, dt=10s",
    nx=40, nz=80, x0=0.0, x1=1000.0, z0=0.0, z1=2000.0, k=3,
    theta0=303.15, mu=0.0, bubble=FlattenedGaussian(0.5, 500.0, 520.0, 50.0, 100.0),
    scheme=1, dt_fixed=10.0, steps=120, fv_levels=5, **PHYS_ROBERT)


def scaled(w: Workload, nx: int, nz: int, **kw) -> Workload:
    """The same workload on another grid (for oracle-sized parity cases)."""
    return replace(w, nx=nx, nz=nz, **kw)


def ensemble_member(m: int) -> Workload:
    """Member m of the 64-member uneven ensemble (seed 1000+m).

    Level a in {0..3} gives (40*2^a) x (20*2^a) quads; k in {1..4};
    bubble amplitude ~ U(1,4) K; centre ~ U([6,14] km x [1.5,3] km); r = 2 km;
    dt = 10x acoustic CFL; SDIRK2.  Number of MG levels: subgrid + agglomeration
    down to a 40x20-or-coarser grid."""
    rng = np.random.Generator(np.random.Philox(1000 + m))
    a = int(rng.integers(0, 4))
    k = int(rng.integers(1, 5))
    amp = float(rng.uniform(1.0, 4.0))
    xc = float(rng.uniform(6000.0, 14000.0))
    zc = float(rng.uniform(1500.0, 3000.0))
    nx, nz = 40 * 2 ** a, 20 * 2 ** a
    return Workload(
        name=f"ensemble member {m}: Q{k} {nx}x{nz}",
        nx=nx, nz=nz, x0=0.0, x1=20000.0, z0=0.0, z1=10000.0, k=k,
        theta0=300.0, mu=0.0, bubble=Bubble(amp, xc, zc, 2000.0, 2000.0),
        scheme=1, cfl_mult=10.0, steps=1, fv_levels=3, **PHYS_ROBERT)


def ensemble(n: int = 64):
    return [ensemble_member(m) for m in range(n)]


def poisson_arrivals(rate: float, horizon: float, seed: int = 7):
    """Arrival times of a Poisson stream (exponential gaps) over [0, horizon)."""
    rng = np.random.Generator(np.random.Philox(seed))
    t, out = 0.0, []
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t >= horizon:
            return np.asarray(out)
        out.append(t)


def random_perturbation(shape, seed: int, scales=(1e-3, 1.0, 1.0, 0.3)):
    """Seeded random perturbation state U' = (rho', (rho u)', (rho w)', (rho theta)').

    `shape` is the per-variable shape; scales are absolute magnitudes of each
    component (kg/m^3, kg/(m^2 s), kg/(m^2 s), K kg/m^3)."""
    rng = np.random.Generator(np.random.Philox(seed))
    out = np.empty((4,) + tuple(shape))
    for v in range(4):
        out[v] = scales[v] * rng.standard_normal(shape)
    return out


def random_vector(n: int, seed: int):
    rng = np.random.Generator(np.random.Philox(seed))
    return rng.standard_normal(n)
