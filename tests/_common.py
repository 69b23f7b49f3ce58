"""Shared helpers of the tests: one workload -> (CUDA context, oracle operator)."""
from __future__ import annotations

import numpy as np

import synth
from oracle.dg import DG
from oracle.physics import Physics as OPhys


def oracle_physics(w: synth.Workload, **kw):
    return OPhys(cp=w.cp, cv=w.cv, g=w.g, p0=w.p0, theta0=w.theta0, mu=w.mu,
                 background=w.background, ubg=w.ubg, N_bv=w.N_bv, **kw)


def oracle_dg(w: synth.Workload, c_ip=2.0):
    return DG(w.nx, w.nz, w.x0, w.x1, w.z0, w.z1, w.k, oracle_physics(w), periodic_x=w.periodic_x, c_ip=c_ip)


def gpu_context(w: synth.Workload, **opt):
    import paper_2505_24504_gb300 as P
    g = P.Grid(w.nx, w.nz, w.x0, w.x1, w.z0, w.z1, int(w.periodic_x))
    ph = P.Physics(w.cp, w.cv, w.g, w.p0, w.theta0, w.mu, w.background, w.ubg, 0.0, w.N_bv)
    kw = dict(fv_levels=w.fv_levels, mg_key=w.mg_key, newton_tol=w.newton_tol)
    kw.update(opt)
    return P.Context(g, w.k, ph, P.Opts.defaults(**kw))


def to_gpu(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def to_cpu(t, shape=None):
    a = t.detach().cpu().numpy()
    return a.reshape(shape) if shape is not None else a


def initial_state(w: synth.Workload, dg: DG):
    """Oracle initial state of the workload (bubble + optional noise)."""
    return dg.init_state(w.theta_pert(dg.X, dg.Z))


def perturbed_state(w, dg, seed=7, scale=1.0):
    """Bubble state plus a seeded random perturbation of all four components, shaped
    like a state some steps into the run (|rho'| ~ 1e-3, |m| ~ 1, |(rho theta)'| ~ 0.3)."""
    U = initial_state(w, dg)
    return U + scale * synth.random_perturbation(dg.shape[1:], seed)


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))
