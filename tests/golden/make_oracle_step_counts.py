"""Writes oracle_step_counts.json: the iteration counts of one implicit step of
the FP64 oracle on each measured workload (Newton iterations per stage, GMRES
iterations of every Newton iteration), with the schedule it ran.

The CPU reference leg of bench.py times bounded samples of the oracle (a
Newton residual, a linearisation of the preconditioner, preconditioned FGMRES
iterations) and scales them to whole steps with these counts.  Calls only the
oracle and the seeded input generators:

    python tests/golden/make_oracle_step_counts.py
"""
from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle.dg import DG  # noqa: E402
from oracle.fv import Multigrid  # noqa: E402
from oracle.physics import Physics  # noqa: E402
from oracle.solver import NewtonStats, implicit_step  # noqa: E402

# the schedules the benchmark runs (mg key of Sec. 4, pseudo-time factors of Sec. 3.5)
RUNS = {
    "warm_bubble_q3_160x80": (synth.BUBBLE_Q3_160x80, dict(mg_key="mg131211V", sigma_fv=1.0, sigma_dg=0.9)),
    "warm_bubble_q2_20x10": (synth.BUBBLE_Q2_20x10, dict(mg_key="mg111111V", sigma_fv=1.0, sigma_dg=1.0)),
}


def run(w, sched):
    ph = Physics(cp=w.cp, cv=w.cv, g=w.g, p0=w.p0, theta0=w.theta0, mu=w.mu, background=w.background,
                 ubg=w.ubg, N_bv=w.N_bv)
    dg = DG(w.nx, w.nz, w.x0, w.x1, w.z0, w.z1, w.k, ph, periodic_x=w.periodic_x)
    U0 = dg.init_state(w.theta_pert(dg.X, dg.Z))
    st = NewtonStats()
    t0 = time.perf_counter()
    implicit_step(dg, U0, w.dt, scheme=w.scheme, tol=w.newton_tol,
                  precond=Multigrid(dg, w.fv_levels, **sched), stats=st)
    return {"workload": w.name, "scheme": w.scheme, "dt": w.dt, "newton_tol": w.newton_tol,
            "fv_levels": w.fv_levels, "schedule": sched, "newton_its": st.newton_its,
            "gmres_its": st.gmres_its, "gmres_per_newton": st.gmres_per_newton,
            "stages": 1 if w.scheme == 0 else 2, "converged": st.converged,
            "host_seconds_one_thread": round(time.perf_counter() - t0, 1)}


if __name__ == "__main__":
    out = {name: run(w, sched) for name, (w, sched) in RUNS.items()}
    with open(os.path.join(HERE, "oracle_step_counts.json"), "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")
    print(json.dumps(out, indent=1))
