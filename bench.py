#!/usr/bin/env python
"""Throughput of implicit SDIRK2 steps of the JFNK-GMRES solver with the DG->FV
multigrid preconditioner on one GB300, as one JSON line.

Workload: warm bubble on DG Q3, 160 x 80 quads over [0,20 km] x [0,10 km]
(819,200 unknowns), isentropic atmosphere theta0 = 300 K, +2 K cosine bubble
plus seeded +-0.1 K white noise in theta, SDIRK2 at dt = 20x the acoustic CFL
step, Newton TOL 1e-8, 5 FV levels, the recorded schedule and launch shapes of
presets.WARM_BUBBLE_Q3_160x80.  A step is one SDIRK2 step (two Newton solves,
every kernel of the path).  `value` is the FP32-preconditioner form (the
preconditioner in FP32, residual / FD products / Arnoldi in FP64); the plain
FP64 form is timed beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun: every rank steps its own replica of the workload
(members are independent, no collective on the data path); the timed region is
bracketed by barriers and the max over ranks is taken.  `--impl reference`
times the FP64 CPU oracle on the host cores (rank 0 only).
"""
from __future__ import annotations

import os
import sys

if "--impl" in sys.argv and "reference" in sys.argv:
    # the CPU reference is single-threaded numpy: keep any math library on one thread
    for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(_v, "1")

import argparse  # noqa: E402
import json  # noqa: E402
import statistics  # noqa: E402
import subprocess  # noqa: E402
import tempfile  # noqa: E402
import time  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from paper_2505_24504_gb300 import presets  # noqa: E402

WORKLOAD = synth.BUBBLE_Q3_160x80
PRESET = presets.WARM_BUBBLE_Q3_160x80
METRIC = "implicit steps/s & DOF/s at 1e-8 Newton tol (batched mixed vs plain FP64); p50/p99"
L2_FLUSH_BYTES = 512 << 20
COUNTS_FILE = os.path.join(ROOT, "tests", "golden", "oracle_step_counts.json")
COUNTS_KEY = "warm_bubble_q3_160x80"
# nvidia-smi-free fallback of the roofline denominators (MEASURED_PEAKS.json absent)
FALLBACK_HBM_GBS = 6800.0
# FP64 arithmetic per SM and clock: the nominal 1.25 TFLOP/s of a 152-SM GB300 at
# 2.07 GHz is 2 DFMA (4 flops) per SM and clock
FP64_FLOP_PER_SM_CLK = 4.0
# DRAM bytes (read + write) of one FP64 FD-product face launch on this workload,
# ncu, cold L2 (writes stay in L2)
TRAFFIC_FACE = 13_339_136


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--plain-steps", type=int, default=None)
    p.add_argument("--form", default="both", choices=["both", "fp32"],
                   help="fp32: time only the FP32-preconditioner steps (for profiler runs)")
    p.add_argument("--tune", action="store_true",
                   help="run the autotuner (schedule and launch shapes) instead of the recorded preset")
    p.add_argument("--ensemble", type=int, default=64, help="members of the batched ensemble (0: skip)")
    p.add_argument("--ensemble-steps", type=int, default=2)
    p.add_argument("--ensemble-threads", type=int, default=16, help="host threads / streams of the batched ensemble")
    p.add_argument("--serve-seconds", type=float, default=60.0, help="Poisson horizon below capacity (0: skip)")
    p.add_argument("--serve-rate", type=float, default=40.0, help="arrival rate of the below-capacity run (1/s)")
    p.add_argument("--overload-seconds", type=float, default=2.0, help="horizon of the 200/s overload run")
    p.add_argument("--secondary-steps", type=int, default=3,
                   help="timed steps of the viscous, inertia-gravity and rising-bubble workloads (0: skip)")
    p.add_argument("--no-sweep", action="store_true", help="skip the mg-key sweep and the dt trends")
    p.add_argument("--no-long", action="store_true",
                   help="skip the test cases run to their end times (density current 900 s, "
                        "inertia gravity 3000 s, rising bubble 300 s)")
    p.add_argument("--schedule", default=None, metavar="KEY", help="override the preset's mg key")
    p.add_argument("--profile-dg", type=int, default=0, metavar="REPS",
                   help="only run REPS FP64 FD products (face + volume kernels) of the workload "
                        "and print their CUDA-event times (small profiler captures)")
    p.add_argument("--profile-ensemble", type=int, default=-1, metavar="MODE",
                   help="only run one batched step of the ensemble in batch MODE (0 streams, 1 lock-step, "
                        "2 lock-step without grouping) inside the NVTX range timed_step, after one "
                        "untimed step (profiler captures)")
    p.add_argument("--ensemble-order", type=int, default=0, metavar="K",
                   help="with --profile-ensemble: only the members of order K (0: all)")
    return p.parse_args()


# ---------------------------------------------------------------------------
class Clocks:
    """nvidia-smi samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for ln in fh:
                parts = [x.strip() for x in ln.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def config_of(w, world: int, preset=PRESET) -> dict:
    """The `config` object of both arms (the same workload, schedule and tolerance)."""
    return {"workload": w.name, "unknowns": w.n_unknowns, "scheme": "SDIRK2", "dt": w.dt,
            "newton_tol": w.newton_tol, "fv_levels": w.fv_levels, "mg_key": preset["mg_key"],
            "sigma_fv": preset["sigma_fv"], "sigma_dg": preset["sigma_dg"],
            "l2": "GPU arm: flushed between timed steps (512 MiB write); CPU arm: host caches",
            "parallelism": f"replicas x{world}"}


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


# ---------------------------------------------------------------------------
def make_args(w, prec, **kw):
    import paper_2505_24504_gb300 as P
    g = P.Grid(w.nx, w.nz, w.x0, w.x1, w.z0, w.z1, int(w.periodic_x))
    ph = P.Physics(w.cp, w.cv, w.g, w.p0, w.theta0, w.mu, w.background, w.ubg, 0.0, w.N_bv)
    kwargs = dict(fv_levels=w.fv_levels, mg_key=w.mg_key, newton_tol=w.newton_tol, precond_prec=prec)
    kwargs.update(kw)
    return g, w.k, ph, P.Opts.defaults(**kwargs)


def make_context(w, prec, **kw):
    import paper_2505_24504_gb300 as P
    return P.Context(*make_args(w, prec, **kw))


def initial_state(ctx, w):
    import torch
    x, z = ctx.node_coords()
    sh = (w.nz, w.nx, w.k + 1, w.k + 1)
    th = w.theta_pert(x.reshape(sh), z.reshape(sh))
    U = torch.empty(ctx.N, dtype=torch.float64, device="cuda")
    ctx.jfnk_init_state(torch.from_numpy(th.ravel().copy()).cuda(), U)
    return U


def time_steps(ctx, U, w, steps, warmup, dist, flush):
    """Device time of `steps` SDIRK2 steps (CUDA events on the launching stream),
    L2 flushed between steps outside the events."""
    import torch
    s = torch.cuda.current_stream()
    for _ in range(warmup):
        ctx.implicit_step(U, w.dt, scheme=w.scheme)
    stats = []
    ms = 0.0
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    from paper_2505_24504_gb300 import jfnk
    n0 = jfnk.launch_count()
    for _ in range(steps):
        flush.add_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("timed_step")   # lets a profiler select the timed launches
        e0.record(s)
        st = ctx.implicit_step(U, w.dt, scheme=w.scheme)
        e1.record(s)
        torch.cuda.nvtx.range_pop()
        e1.synchronize()
        ms += e0.elapsed_time(e1)
        stats.append(st.as_dict())
    torch.cuda.synchronize()
    time_steps.launches = jfnk.launch_count() - n0   # this library's kernels in the timed steps
    if dist:
        dist.barrier()
    return ms, stats


def timed_once(ctx, U, w, **kw):
    """(ms, stats) of one implicit step after one untimed step."""
    import torch
    ctx.implicit_step(U, w.dt, scheme=w.scheme, raise_on_error=False)
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s)
    st = ctx.implicit_step(U, w.dt, scheme=w.scheme, raise_on_error=False)
    e1.record(s)
    e1.synchronize()
    return e0.elapsed_time(e1), st


# ---------------------------------------------------------------------------
# Algorithmic FP64 flops of the FD product, from the formulas (a divide, square
# root or x^gamma counts one flop, an FMA two, compares and selects none):
#  face point, stored traces of U plus eps times the traces of y:
#    traces of y: 2 sides x 4 variables x (k+1) FMA; tr(U) + eps tr(y): 8 FMA;
#    + background: 8; HLLC: 1/rho 2, velocities 2, pressures 2 x 3, sound speeds
#    2 x 3, wave-speed bounds 4, S - u 2, contact speed numerator 7, denominator
#    3, quotient 1, star factor 4, star state 5, side flux 4, F + S (U* - U) 12
#    (58); minus the background flux: 4
#  node, volume term: U + eps y 4 FMA; + background 4; 1/rho 1; pressure 3;
#    velocities 2; two convective fluxes 8; minus the background fluxes 8;
#    sum factorisation 4 variables x 2 directions x (k+1) FMA; gravity 2; lift of
#    the four face terms 4 x 4 FMA; FD quotient and update 3 per variable
HLLC_FLOPS = 58


def alg_flops_face_point(k):
    return 2 * (2 * 4 * (k + 1)) + 2 * 8 + 8 + HLLC_FLOPS + 4


def alg_flops_node(k):
    return 2 * 4 + 4 + 1 + 3 + 2 + 8 + 8 + 2 * (4 * 2 * (k + 1)) + 2 + 2 * 16 + 3 * 4


def fp64_peak_tflops(sm_mhz):
    import torch
    nsm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    return nsm * FP64_FLOP_PER_SM_CLK * sm_mhz * 1e6 / 1e12, nsm


def kernel_bandwidths(w, preset, hbm_peak, peak_note, flush, U0):
    """Live CUDA-event times of the FP32 preconditioner kernels and the CGS2
    passes on this workload (L2 flushed before every timed launch) with their
    algorithmic bytes per launch and the fraction of the HBM peak."""
    import torch
    n1 = w.k + 1
    cells = w.n_el * n1 * n1            # finest FV level: one cell per DG node
    nodes = cells
    ctx = make_context(w, 32, **preset)
    y = torch.randn(ctx.N, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(7))

    def avg(which, reps=6):
        a, b = [], []
        ctx.time_operator(which, U0, y, 1)   # warm
        for _ in range(reps):
            flush.add_(1.0)
            torch.cuda.synchronize()
            m0, m1 = ctx.time_operator(which, U0, y, 1)
            a.append(m0)
            b.append(m1)
        return statistics.median(a), statistics.median(b)

    def entry(ms, nbytes, what):
        gbs = nbytes / (ms * 1e-3) / 1e9
        return {"ms": ms, "bytes": nbytes, "gbs": gbs, "frac": gbs / hbm_peak, "algorithmic_bytes": what}

    fv_s, fv_d = avg(3)
    dg_f, dg_v = avg(2)
    gs1, gs23 = avg(4)
    out = {
        "peak_gbs": hbm_peak, "peak": peak_note,
        "fv_smooth_fp32_finest": entry(fv_s, 68 * cells, "read u, x, b (16 B each) and dtau (4 B), write x (16 B) per cell"),
        "fv_defect_restrict_fp32_finest": entry(fv_d, 56 * cells, "read u, x, b per cell, write b_c and x_c (4 B per fine cell)"),
        "dg_tangent_fp32": entry(dg_f + dg_v, 64 * nodes, "read U, z, r (16 B each), write the defect (16 B) per node"),
        "cgs2_nv8": entry(gs1 + gs23, (20 * 8 + 44) * ctx.N, "(20 NV + 44) B per element: V32 and w, then V, w in and out twice"),
        "cgs2_pass1_fp32": entry(gs1, (4 * 8 + 8) * ctx.N, "V32 (4 NV B) and w (8 B) per element"),
    }
    ctx.close()
    return out


def run_ensemble(n, steps, warmup, threads, hbm_peak):
    """64-member uneven ensemble (Q1..Q4, 40x20 .. 320x160), one batched SDIRK2 step
    per timed iteration, FP32 preconditioner, in both batch modes: member streams
    (host thread pool, tuned launch shapes, graphs) and lock-step (one grouped
    launch per operator across the members that reach it together, the library's
    default launch shapes so that same-order members share kernels); returns a
    dict for the JSON line."""
    import torch

    import paper_2505_24504_gb300 as P
    from paper_2505_24504_gb300 import autotune
    members = synth.ensemble(n)
    dof = sum(m.n_unknowns for m in members)
    dts = [m.dt for m in members]
    sch = [m.scheme for m in members]

    def timed(batch, Us):
        for _ in range(warmup):
            batch.jfnk_batch_step(Us, dts, sch)
        torch.cuda.synchronize()
        t, its, status, lls = 0.0, [], [], []
        n0 = P.jfnk.launch_count()
        for _ in range(steps):
            t0 = time.perf_counter()
            status, stats = batch.jfnk_batch_step(Us, dts, sch, raise_on_error=False)
            torch.cuda.synchronize()
            t += time.perf_counter() - t0
            its.append(sum(s.gmres_its for s in stats))
            lls.append(batch.last_launches())
        launches = (P.jfnk.launch_count() - n0) / steps
        return {"ensemble_steps_per_s": steps / t, "member_steps_per_s": n * steps / t,
                "dof_per_s": dof * steps / t, "ms_per_ensemble_step": 1e3 * t / steps,
                "failed_members": sum(1 for x in status if x != 0),
                "gmres_its_per_ensemble_step": sum(its) / len(its),
                "launches_per_ensemble_step": launches}, lls

    # member streams
    ctxs, Us = [], []
    for m in members:
        c0 = make_context(m, 32)
        U = initial_state(c0, m)
        c, _ = autotune.tuned_context(c0.grid, c0.k, c0.phys, c0.opts, U)
        c0.close()
        ctxs.append(c)
        Us.append(U)
    U0 = [u.clone() for u in Us]
    batch = P.Batch(ctxs, max_threads=threads)
    streams, _ = timed(batch, Us)
    streams["timing"] = f"wall clock of jfnk_batch_step (host-driven members on {threads} threads / streams)"
    grouped = time_grouped_residual(batch, ctxs, Us, dof, hbm_peak)
    batch.close()
    for c in ctxs:
        c.close()
    # lock-step
    ctxs = [make_context(m, 32) for m in members]
    Us = [u.clone() for u in U0]
    batch = P.Batch(ctxs, mode=P.jfnk.BATCH_LOCKSTEP)
    lock, lls = timed(batch, Us)
    ll = lls[-1]
    lock.update({"kernel_launches_per_ensemble_step": ll["launches"], "grouped_launches": ll["grouped"],
                 "launches_if_members_alone": ll["member_launches"], "replay_rounds": ll["rounds"],
                 "host_ms": {"members_to_sync": ll["ms_members"], "issue": ll["ms_issue"],
                             "device_wait": ll["ms_device"]},
                 "launch_reduction": ll["member_launches"] / max(1, ll["launches"]),
                 "timing": "wall clock of jfnk_batch_step (members recorded on their own host threads, "
                           "replayed on one stream with grouped launches)"})
    batch.close()
    for c in ctxs:
        c.close()
    # the same members and step sizes, plain FP64 (FP64 preconditioner with FD products
    # in the FV levels), one member at a time on one stream: the single-instance form
    # the batched mixed form is compared with
    plain_s, plain_its, plain_fail = 0.0, 0, 0
    for m, u in zip(members, U0):
        c = make_context(m, 64)
        U = u.clone()
        c.implicit_step(U, m.dt, scheme=m.scheme, raise_on_error=False)   # warm (graphs)
        U.copy_(u)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = c.implicit_step(U, m.dt, scheme=m.scheme, raise_on_error=False)
        torch.cuda.synchronize()
        plain_s += time.perf_counter() - t0
        plain_its += st.gmres_its
        plain_fail += st.status != 0
        c.close()
        del U
    plain = {"ensemble_steps_per_s": 1.0 / plain_s, "member_steps_per_s": n / plain_s, "dof_per_s": dof / plain_s,
             "ms_per_ensemble_step": 1e3 * plain_s, "gmres_its_per_ensemble_step": plain_its,
             "failed_members": plain_fail,
             "timing": "wall clock of each member's first implicit step, one member at a time"}
    del Us, U0
    torch.cuda.empty_cache()
    best = lock if lock["dof_per_s"] > streams["dof_per_s"] else streams
    return {"members": n, "unknowns_total": dof, "grouped_residual": grouped,
            "ensemble_steps_per_s": best["ensemble_steps_per_s"], "member_steps_per_s": best["member_steps_per_s"],
            "dof_per_s": best["dof_per_s"], "mode": "lockstep" if best is lock else "streams",
            "streams": streams, "lockstep": lock, "plain_fp64_serial": plain,
            "batched_vs_plain_fp64": best["dof_per_s"] / plain["dof_per_s"],
            "precond": "fp32", "dt": "10x acoustic CFL per member"}


def time_grouped_residual(batch, ctxs, Us, dof, hbm_peak, reps=10):
    """FP64 residual of every member: one face + one volume launch per (order,
    viscous) group (jfnk_batch_dg_residual) against one launch pair per member,
    both on one stream, CUDA events.  The 64 members' states (470 MB) exceed
    the L2, so the residual's algorithmic 16 B per unknown (read U', write f) is
    also quoted as a fraction of the HBM peak."""
    import torch
    outs = [torch.empty(c.N, dtype=torch.float64, device="cuda") for c in ctxs]
    s = torch.cuda.current_stream()

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(reps):
            fn()
        e1.record(s)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    def per_member():
        for c, u, f in zip(ctxs, Us, outs):
            c.dg_residual(u, f)

    g = timed(lambda: batch.jfnk_batch_dg_residual(Us, outs))
    m = timed(per_member)
    del outs
    gbs = 16.0 * dof / (g * 1e-3) / 1e9
    return {"ms_grouped": g, "ms_per_member_launches": m, "dof_per_s_grouped": dof / (g / 1e3),
            "dof_per_s_per_member": dof / (m / 1e3), "launches_grouped": 2 * len({(c.k, c.phys.mu != 0.0) for c in ctxs}),
            "launches_per_member": 2 * len(ctxs), "hbm_gbs": gbs, "hbm_frac": gbs / hbm_peak,
            "note": "16 B per unknown algorithmic; FP64-ALU bound, so far below the HBM roof"}


def run_serving(seconds, rate, overload_seconds, rank=0, world=1, dist=None):
    """Poisson arrivals of implicit-step requests on resident states: 16 ensemble
    members (80 %) and 4 viscous density-current states (20 %).  The HBM budget
    is what the device has free, so every state keeps its context (Krylov basis,
    FV levels, graphs) resident across requests.  One run below capacity over the
    full horizon, one short overload run at 200/s, and the same request list
    stepped serially with plain FP64 contexts for comparison.  With several
    ranks each GPU serves the states it owns (sid % world == rank) and the
    ranks pool their latencies at the end (no exchange while serving)."""
    import numpy as np
    import torch

    from paper_2505_24504_gb300 import jfnk
    from paper_2505_24504_gb300.serve import Server, StateSpec, pooled_summary, shard_requests, shard_states
    ens = synth.ensemble(16)
    visc = [synth.DENSITY_CURRENT_Q2_256x32] * 4
    work = ens + visc

    def specs_for(prec):
        specs = {}
        for sid, m in enumerate(work):
            if sid % world != rank:
                continue
            c = make_context(m, prec)
            specs[sid] = StateSpec(grid=c.grid, k=c.k, phys=c.phys, opts=c.opts, dt=m.dt, scheme=m.scheme,
                                   U=initial_state(c, m))
            c.close()
        return specs

    def requests(r, horizon, seed):
        arr = synth.poisson_arrivals(r, horizon, seed=seed)
        rng = np.random.Generator(np.random.Philox(seed + 4))
        reqs = [(float(t), int(rng.integers(0, 16)) if rng.random() < 0.8 else 16 + int(rng.integers(0, 4)))
                for t in arr]
        return shard_requests(reqs, rank, world)

    free, _ = torch.cuda.mem_get_info()
    budget = int(0.5 * free)
    out = {"states": len(work), "hbm_budget_bytes": budget, "ranks": world,
           "sharding": "state sid served by rank sid % world" if world > 1 else "one GPU"}
    for name, r, horizon in (("below_capacity", rate, seconds), ("overload", 200.0, overload_seconds)):
        if horizon <= 0:
            continue
        specs = specs_for(32)
        reqs = requests(r, horizon, 7)
        srv = Server(specs, hbm_budget=budget, workers=16)
        rep = srv.run(reqs, timeout_s=max(600.0, 20 * horizon))
        srv.close()
        s = rep.summary()
        if world > 1:
            s["pooled_over_ranks"] = pooled_summary(rep, dist)
        s.update({"arrival_rate_per_s": r, "horizon_s": horizon,
                  "basis_rebuilds": rep.contexts_created - len({q[1] for q in reqs}),
                  "footprint_total_bytes": sum(sp.footprint for sp in specs.values())})
        out[name] = s
        del specs
        torch.cuda.empty_cache()
    # the same request list (first 200 requests of the below-capacity run) stepped
    # one at a time with plain FP64 contexts, one context per state
    reqs = requests(rate, seconds if seconds > 0 else 5.0, 7)[:200]
    specs = specs_for(64)
    ctxs = {}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _, sid in reqs:
        sp = specs[sid]
        if sid not in ctxs:
            ctxs[sid] = jfnk.Context(sp.grid, sp.k, sp.phys, sp.opts)
        ctxs[sid].implicit_step(sp.U, sp.dt, scheme=sp.scheme)
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    for c in ctxs.values():
        c.close()
    del specs
    torch.cuda.empty_cache()
    out["plain_fp64_serial"] = {"requests": len(reqs), "steps_per_s": len(reqs) / t, "wall_s": t,
                                "note": "same requests, one at a time, FP64 preconditioner, contexts kept"}
    # capacity: the overload run keeps every worker busy, the below-capacity run only
    # follows its arrivals (its rate is the arrival rate)
    if "overload" in out:
        out["served_vs_plain_fp64_serial"] = out["overload"]["steps_per_s"] / out["plain_fp64_serial"]["steps_per_s"]
        out["served_vs_plain_note"] = "overload (capacity) steps/s over the plain FP64 serial steps/s"
    return out


def run_case(w, steps, preset=None, **opt):
    """Timed SDIRK2 steps of a secondary workload (FP32 preconditioner)."""
    import torch
    from paper_2505_24504_gb300 import autotune
    o = dict(preset or {})
    o.update(opt)
    c0 = make_context(w, 32, **o)
    U = initial_state(c0, w)
    if preset is None:
        ctx, _ = autotune.tuned_context(c0.grid, c0.k, c0.phys, c0.opts, U)
        c0.close()
    else:
        ctx = c0
    ctx.implicit_step(U, w.dt, scheme=w.scheme)
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    ms, its = 0.0, []
    for _ in range(steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        st = ctx.implicit_step(U, w.dt, scheme=w.scheme)
        e1.record(s)
        e1.synchronize()
        ms += e0.elapsed_time(e1)
        its.append((st.newton_its, st.gmres_its))
    ctx.close()
    return {"workload": w.name, "steps_per_s": steps / (ms / 1e3), "dof_per_s": w.n_unknowns * steps / (ms / 1e3),
            "ms_per_step": ms / steps, "newton_gmres_per_step": its[-1], "precond": "fp32",
            "mg_key": o.get("mg_key", w.mg_key)}


def _node_xz(w):
    """Node coordinates (nz, nx, k+1, k+1) in the library's layout [ez][ex][b][a] of one variable."""
    import numpy as np
    xi = np.polynomial.legendre.leggauss(w.k + 1)[0]
    hx, hz = (w.x1 - w.x0) / w.nx, (w.z1 - w.z0) / w.nz
    ex = np.arange(w.nx)[None, :, None, None]
    ez = np.arange(w.nz)[:, None, None, None]
    X = w.x0 + (ex + (1 + xi[None, None, None, :]) / 2) * hx
    Z = w.z0 + (ez + (1 + xi[None, None, :, None]) / 2) * hz
    shape = (w.nz, w.nx, w.k + 1, w.k + 1)
    return np.broadcast_to(X, shape), np.broadcast_to(Z, shape)


def run_long_runs():
    """The paper's test cases run to their end times (Sec. 4.1-4.3) with the FP32
    preconditioner: SDIRK2 steps at the workload's dt, every step's status, Newton
    and GMRES counts, device time, and a transport check of the final state taken
    from the perturbation variables: the density current's front (largest x at
    the lowest node row where rho' exceeds rho_surface / 300, i.e. theta' below
    about -1 K at near-constant pressure), the inertia-gravity packet's centre (the
    mean flow of 20 m/s carries it from 100 km to 160 km in 3000 s: the centroid
    of (rho theta)'^2 along the node row nearest mid height), the rising bubble's
    height (z of the most negative rho')."""
    import numpy as np
    import torch
    cases = ((synth.DENSITY_CURRENT_Q2_256x32, 900.0), (synth.INERTIA_GRAVITY_Q3_80x3, 3000.0),
             (synth.RISING_BUBBLE_Q3_40x80, 300.0))
    out = {}
    for w, T in cases:
        ctx = make_context(w, 32)
        U = initial_state(ctx, w)
        n = int(round(T / w.dt))
        s = torch.cuda.current_stream()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        failed, newton, gmres = 0, 0, 0
        e0.record(s)
        for _ in range(n):
            st = ctx.implicit_step(U, w.dt, scheme=w.scheme, raise_on_error=False)
            failed += st.status != 0
            newton += st.newton_its
            gmres += st.gmres_its
        e1.record(s)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        a = U.detach().cpu().numpy().reshape((4, w.nz, w.nx, w.k + 1, w.k + 1))
        X, Z = _node_xz(w)
        row = {"workload": w.name, "end_time_s": n * w.dt, "steps": n, "failed_steps": failed,
               "newton_per_step": newton / n, "gmres_per_step": gmres / n, "seconds": ms / 1e3,
               "steps_per_s": n / (ms / 1e3)}
        if w is synth.DENSITY_CURRENT_Q2_256x32:
            cold = a[0, 0, :, 0, :] > 1.161 / 300.0
            row["front_km"] = float(X[0, :, 0, :][cold].max() / 1e3) if cold.any() else 0.0
        elif w is synth.INERTIA_GRAVITY_Q3_80x3:
            mid = np.abs(Z - 0.5 * (w.z0 + w.z1))
            sel = mid == mid.min()
            wgt = np.where(sel, a[3] ** 2, 0.0)
            row["packet_centre_km"] = float((wgt * X).sum() / wgt.sum() / 1e3)
        else:
            i = np.argmin(a[0])
            row["bubble_height_m"] = float(Z.ravel()[i])
        out[w.name] = row
        ctx.close()
    return out


def run_mg_sweep():
    """GMRES iterations, operator calls and time of one SDIRK2 (or BE) step for the
    paper's schedule variants (Sec. 4.2): none, mg001111V, mg111111V, mg111111W and
    the tuned key, on the three measured workloads (FP32 preconditioner)."""
    out = {}
    cases = ((synth.BUBBLE_Q2_20x10, {}), (WORKLOAD, PRESET), (synth.DENSITY_CURRENT_Q2_256x32, {}))
    for w, pre in cases:
        rows = {}
        keys = ["", "mg001111V", "mg111111V", "mg111111W"]
        if pre and pre["mg_key"] not in keys:
            keys.append(pre["mg_key"])
        for key in keys:
            o = dict(pre)
            o.update(mg_key=key, gmres_max=3000)
            ctx = make_context(w, 32, **o)
            U = initial_state(ctx, w)
            ms, st = timed_once(ctx, U, w)
            rows[key or "none"] = {"ms": ms, "status": st.status, "newton": st.newton_its, "gmres": st.gmres_its,
                                   "dg_calls": st.dg_calls, "fv_calls": st.fv_calls}
            ctx.close()
        out[w.name] = rows
    return out


def run_dt_trends():
    """Newton / GMRES iterations per step against the time step, with the
    preconditioner (mg111111V) and without, on the paper's three test cases at
    reduced grids (Sec. 4.1-4.3: the preconditioner's iteration counts grow
    slowly with dt, the unpreconditioned ones fast)."""
    cases = (synth.scaled(synth.INERTIA_GRAVITY_Q3_80x3, 40, 3),
             synth.scaled(synth.RISING_BUBBLE_Q3_40x80, 10, 20, fv_levels=4),
             synth.scaled(synth.DENSITY_CURRENT_Q2_256x32, 64, 32, x1=12800.0, fv_levels=4))
    out = {}
    for w in cases:
        rows = []
        for f in (0.25, 0.5, 1.0, 2.0):
            wd = synth.replace(w, dt_fixed=f * w.dt)
            row = {"dt": wd.dt}
            for key in ("mg111111V", ""):
                ctx = make_context(wd, 32, mg_key=key, gmres_max=3000)
                U = initial_state(ctx, wd)
                st = ctx.implicit_step(U, wd.dt, scheme=1, raise_on_error=False)
                row["precond" if key else "none"] = {"status": st.status, "newton": st.newton_its,
                                                     "gmres": st.gmres_its}
                ctx.close()
            rows.append(row)
        out[w.name] = rows
    return out


def max_over_ranks(x, dist, device="cuda"):
    """Max of x over the ranks (the timed region of the slowest rank)."""
    if not dist:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, ms_max, world):
    """Aggregate throughput: the units all ranks processed over the max time."""
    return world * units_per_rank / (ms_max / 1e3)


# ---------------------------------------------------------------------------
# The FP64 oracle as it stands, timed on the host cores.
def oracle_counts():
    """The oracle's own iteration counts of one step of the workload (written by
    tests/golden/make_oracle_step_counts.py, which runs the oracle's step)."""
    with open(COUNTS_FILE) as fh:
        rec = json.load(fh)[COUNTS_KEY]
    want = presets.schedule(PRESET)
    if rec["schedule"] != want:
        raise RuntimeError(f"{COUNTS_FILE} was made with {rec['schedule']}, the preset runs {want}")
    return rec


class OracleSampler:
    """Bounded samples of the oracle's implicit step on the workload: the Newton
    residual G(U), the preconditioner's linearisation, and preconditioned FGMRES
    iterations (each = Q^-1 v, the FD product, modified Gram-Schmidt), timed at
    the step's first Newton iterate with the workload's schedule."""

    def __init__(self, w, preset):
        from oracle.dg import DG
        from oracle.fv import Multigrid
        from oracle.physics import Physics
        from oracle.solver import SDIRK2_ALPHA
        ph = Physics(cp=w.cp, cv=w.cv, g=w.g, p0=w.p0, theta0=w.theta0, mu=w.mu)
        self.dg = DG(w.nx, w.nz, w.x0, w.x1, w.z0, w.z1, w.k, ph)
        self.U = self.dg.init_state(w.theta_pert(self.dg.X, self.dg.Z))
        self.adt = SDIRK2_ALPHA * w.dt
        self.mg = Multigrid(self.dg, w.fv_levels, **presets.schedule(preset))
        self.t_res, self.t_lin, self.t_it = [], [], []

    def sample(self, gmres_its=2):
        """One sample: residual, linearisation and `gmres_its` FGMRES iterations."""
        from oracle.solver import fgmres
        t0 = time.perf_counter()
        G, fU = self.dg.G(self.U, self.adt, self.U)
        t1 = time.perf_counter()
        self.mg.linearize(self.U, self.adt, fU)
        t2 = time.perf_counter()
        A = lambda y: self.dg.jv(self.U, fU, y, self.adt)
        _, done, _ = fgmres(A, -G, self.mg.apply, tol_abs=0.0, m=30, maxit=gmres_its)
        t3 = time.perf_counter()
        self.t_res.append(t1 - t0)
        self.t_lin.append(t2 - t1)
        self.t_it.append((t3 - t2) / max(done, 1))
        return t3 - t0

    def seconds_per_step(self, rec):
        """Whole-step time from the sampled unit times and the oracle's counts:
        per stage one initial residual, per Newton iteration one linearisation,
        its GMRES iterations and one residual."""
        r, l, it = (statistics.mean(x) for x in (self.t_res, self.t_lin, self.t_it))
        return rec["stages"] * r + rec["newton_its"] * (l + r) + rec["gmres_its"] * it


def _oracle_whole_step_seconds(w):
    """One whole oracle step of a small workload, timed (runs in a child process
    for the all-core figure)."""
    from oracle.dg import DG
    from oracle.fv import Multigrid
    from oracle.physics import Physics
    from oracle.solver import implicit_step
    ph = Physics(cp=w.cp, cv=w.cv, g=w.g, p0=w.p0, theta0=w.theta0, mu=w.mu)
    dg = DG(w.nx, w.nz, w.x0, w.x1, w.z0, w.z1, w.k, ph)
    U0 = dg.init_state(w.theta_pert(dg.X, dg.Z))
    t0 = time.perf_counter()
    implicit_step(dg, U0, w.dt, scheme=w.scheme, tol=w.newton_tol, precond=Multigrid(dg, w.fv_levels, w.mg_key))
    return time.perf_counter() - t0


def _child_whole_step(_):
    os.environ["OMP_NUM_THREADS"] = "1"
    return _oracle_whole_step_seconds(synth.BUBBLE_Q2_20x10)


def cpu_baseline(w):
    """The oracle on the host: a bounded sample of this workload's step on one
    core scaled to steps/s by the oracle's own counts, plus one whole step of the
    small warm-bubble workload on one core and on every core at once (independent
    steps in `nproc` processes), and one whole step of the viscous density
    current on one core."""
    import multiprocessing as mp
    rec = oracle_counts()
    smp = OracleSampler(w, PRESET)
    t0 = time.perf_counter()
    smp.sample(gmres_its=2)
    smp.sample(gmres_its=2)
    sampled = time.perf_counter() - t0
    sec = smp.seconds_per_step(rec)
    one = _oracle_whole_step_seconds(synth.BUBBLE_Q2_20x10)
    wv = synth.DENSITY_CURRENT_Q2_256x32
    visc = _oracle_whole_step_seconds(wv)
    ncores = min(len(os.sched_getaffinity(0)), 64)
    t1 = time.perf_counter()
    with mp.get_context("spawn").Pool(ncores) as pool:
        pool.map(_child_whole_step, range(ncores))
    wall = time.perf_counter() - t1
    return {"value": 1.0 / sec, "unit": "implicit steps/s", "cores": 1, "kind": "oracle",
            "dof_per_s": w.n_unknowns / sec, "seconds_sampled": sampled,
            "sample": (f"oracle (numpy FP64, 1 thread, {PRESET['mg_key']}): 2 samples of residual + "
                       f"linearisation + 2 preconditioned FGMRES iterations at the first Newton iterate of "
                       f"this workload, scaled to a whole SDIRK2 step by the oracle's own counts "
                       f"({rec['newton_its']} Newton, {rec['gmres_its']} GMRES; tests/golden/oracle_step_counts.json)"),
            "small_workload_whole_step": {"workload": synth.BUBBLE_Q2_20x10.name, "seconds_1_core": one,
                                          "steps_per_s_1_core": 1.0 / one, "cores_all": ncores,
                                          "steps_per_s_all_cores": ncores / wall,
                                          "note": "independent steps, one process per core"},
            "viscous_workload_whole_step": {"workload": wv.name, "seconds_1_core": visc,
                                            "steps_per_s_1_core": 1.0 / visc,
                                            "dof_per_s_1_core": wv.n_unknowns / visc}}


def run_reference(args):
    """The reference leg: the FP64 oracle on the host, each timed step one bounded
    sample (residual, linearisation, 2 preconditioned FGMRES iterations) of this
    workload's SDIRK2 step; `value` scales the sampled unit times to whole steps
    with the oracle's own iteration counts."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = WORKLOAD
    rec = oracle_counts()
    smp = OracleSampler(w, PRESET)
    for _ in range(args.warmup):
        smp.sample()
    smp.t_res, smp.t_lin, smp.t_it = [], [], []
    per = []
    for _ in range(args.steps):
        per.append(smp.sample())
    sec = smp.seconds_per_step(rec)
    value = 1.0 / sec
    world = int(os.environ.get("WORLD_SIZE", "1"))
    desc = (f"oracle (numpy FP64, 1 thread, {PRESET['mg_key']}): each timed step = residual + linearisation + "
            f"2 preconditioned FGMRES iterations at the first Newton iterate; value = whole SDIRK2 steps/s from "
            f"the mean unit times and the oracle's own counts ({rec['newton_its']} Newton, {rec['gmres_its']} "
            f"GMRES per step, tests/golden/oracle_step_counts.json)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "implicit steps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * statistics.mean(per), "ms_per_implicit_step": 1e3 * sec,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "dof_per_s": value * w.n_unknowns,
        "config": config_of(w, world),
        "cpu_baseline": {"value": value, "unit": "implicit steps/s", "cores": 1, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": "implicit steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "unit_seconds": {"residual": statistics.mean(smp.t_res), "linearise": statistics.mean(smp.t_lin),
                         "fgmres_iteration": statistics.mean(smp.t_it)},
    }
    print(json.dumps(line))


# ---------------------------------------------------------------------------
def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch

    import paper_2505_24504_gb300 as P
    from paper_2505_24504_gb300 import build as B
    B.build()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as D
        D.init_process_group("nccl")
        dist = D
    torch.cuda.set_device(local)
    w = WORKLOAD
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    preset = dict(PRESET)
    if args.schedule:
        preset["mg_key"] = args.schedule
    if args.profile_dg:
        c64 = make_context(w, 64, **preset)
        U0 = initial_state(c64, w)
        y = torch.randn(c64.N, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(5))
        fm, vm = c64.time_operator(1, U0, y, args.profile_dg)
        print(json.dumps({"profile": "FP64 FD product", "face_ms": fm, "volume_ms": vm, "reps": args.profile_dg}))
        return
    if args.profile_ensemble >= 0:
        members = [m for m in synth.ensemble(args.ensemble) if args.ensemble_order in (0, m.k)]
        ctxs = [make_context(m, 32) for m in members]
        Us = [initial_state(c, m) for c, m in zip(ctxs, members)]
        batch = P.Batch(ctxs, max_threads=args.ensemble_threads, mode=args.profile_ensemble)
        dts, sch = [m.dt for m in members], [m.scheme for m in members]
        batch.jfnk_batch_step(Us, dts, sch)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("timed_step")
        t0 = time.perf_counter()
        status, _ = batch.jfnk_batch_step(Us, dts, sch, raise_on_error=False)
        torch.cuda.synchronize()
        ms = 1e3 * (time.perf_counter() - t0)
        torch.cuda.nvtx.range_pop()
        print(json.dumps({"profile": "ensemble step", "mode": args.profile_ensemble, "members": len(members),
                          "order": args.ensemble_order, "ms": ms, "failed": sum(1 for x in status if x != 0),
                          "launches": batch.last_launches()}))
        batch.close()
        for c in ctxs:
            c.close()
        return

    # ---- the product form: FP32 preconditioner ---------------------------------
    c0 = make_context(w, 32, **preset)
    U = initial_state(c0, w)
    U0 = U.clone()
    tuning = {"source": "presets.WARM_BUBBLE_Q3_160x80 (recorded autotuner choice)"}
    if args.tune:
        from paper_2505_24504_gb300 import autotune
        c0.close()
        ctx, tiles = autotune.tuned_schedule_context(*make_args(w, 32), U0, w.dt, w.scheme)
        preset = {k: tiles[k] for k in ("mg_key", "sigma_fv", "sigma_dg", "tile_faces", "tile_volume", "tile_fv",
                                        "fv_split_cells")}
        tuning = {"source": "autotuner run in this process", "chosen": preset,
                  "schedule_trials_ms": tiles.get("schedule_trials_ms")}
    else:
        ctx = c0
    with Clocks(local) as clk:
        ms, stats = time_steps(ctx, U, w, args.steps, args.warmup, dist, flush)
    launches = time_steps.launches
    clocks = clk.summary()
    ms = max_over_ranks(ms, dist)
    value = whole_job_rate(args.steps, ms, world)
    newton = sum(s["newton_its"] for s in stats) / len(stats)
    gmres = sum(s["gmres_its"] for s in stats) / len(stats)
    if args.form == "fp32":
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "implicit steps/s", "n_gpus": world,
                              "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                              "form": "fp32 only (profiling run)", "gpu_launches": int(launches),
                              "iterations_per_step": {"newton": newton, "gmres": gmres}}))
        return

    # ---- end to end through the public API with host buffers ------------------
    Uh = U0.cpu().pin_memory()
    Uout = torch.empty_like(Uh).pin_memory()
    s = torch.cuda.current_stream()
    ctx.implicit_step(U, w.dt, scheme=w.scheme)   # warm
    e2e_ms = 0.0
    lat = []
    ne2e = max(2, args.steps // 2)
    for _ in range(ne2e):
        flush.add_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        U.copy_(Uh, non_blocking=True)
        ctx.implicit_step(U, w.dt, scheme=w.scheme)
        Uout.copy_(U, non_blocking=True)
        e1.record(s)
        e1.synchronize()
        t = e0.elapsed_time(e1)
        e2e_ms += t
        lat.append(t)
    e2e_ms = max_over_ranks(e2e_ms, dist)
    e2e = world * ne2e / (e2e_ms / 1e3)

    # ---- roofline of the dominant kernel (FP64 FD product, face kernel) --------
    peaks = measured_peaks()
    hbm_peak = peaks.get("hbm_gbs") or FALLBACK_HBM_GBS
    hbm_note = "of measured (MEASURED_PEAKS.json hbm_gbs)" if peaks.get("hbm_gbs") else "of fallback"
    sm_mhz = peaks.get("sm_max_mhz") or clocks.get("sm_max_mhz") or 2070.0
    peak64, nsm = fp64_peak_tflops(sm_mhz)
    y = torch.randn(ctx.N, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    ctx64 = make_context(w, 64, **preset)
    fm, vm = ctx64.time_operator(1, U0, y, 20)
    n1 = w.k + 1
    face_pts = (w.nz * (w.nx + 1) + (w.nz + 1) * w.nx) * n1
    nodes = w.n_el * n1 * n1
    fl_face, fl_node = alg_flops_face_point(w.k), alg_flops_node(w.k)
    ach = fl_face * face_pts / (fm * 1e-3) / 1e12
    ach_v = fl_node * nodes / (vm * 1e-3) / 1e12
    roof = {"bound": "alu", "kernel": "k_faces<D64> FP64 FD product (face points)", "achieved": ach,
            "peak": peak64, "unit": "TFLOP/s", "frac": ach / peak64, "traffic": TRAFFIC_FACE,
            "peak_source": (f"derived, not measured: {nsm} SMs (device properties) x {FP64_FLOP_PER_SM_CLK:g} FP64 "
                            f"flop/SM/clock x {sm_mhz:g} MHz"),
            "launch_ms": fm, "flop_per_unit": fl_face, "units_per_launch": face_pts,
            "flop_counting": "algorithmic, from the formulas (bench.py alg_flops_face_point); ncu counts 250 "
                             "executed FP64-pipe flops per face point (IEEE divide/sqrt sequences, table power)",
            "volume_kernel": {"achieved": ach_v, "frac": ach_v / peak64, "launch_ms": vm,
                              "flop_per_unit": fl_node, "units_per_launch": nodes},
            "hbm": kernel_bandwidths(w, preset, hbm_peak, hbm_note, flush, U0)}

    # ---- phase breakdown of one more step (events at the solver's own syncs) ----
    ctx_p = make_context(w, 32, profile=1, **preset)
    Up = U0.clone()
    ctx_p.implicit_step(Up, w.dt, scheme=w.scheme)
    stp = ctx_p.implicit_step(Up, w.dt, scheme=w.scheme)
    phases = {"precond_ms": stp.t_precond_ms, "fd_product_ms": stp.t_jv_ms, "orthogonalisation_ms": stp.t_orth_ms,
              "newton_residual_linearise_ms": stp.t_newton_ms, "gmres_its": stp.gmres_its,
              "second_gram_schmidt_passes": stp.reorth}
    ctx_p.close()

    # ---- BF16 numerics on the coarsest FV level (precond_prec = 16), same schedule ----
    c16 = make_context(w, 16, **preset)
    U16 = U0.clone()
    U32 = U0.clone()
    ms16, st16 = time_steps(c16, U16, w, 2, 1, None, flush)
    _, _ = time_steps(ctx, U32, w, 2, 1, None, flush)
    bf16 = {"steps_per_s": 2 / (ms16 / 1e3), "gmres_per_step": sum(x["gmres_its"] for x in st16) / 2,
            "rel_diff_vs_fp32_form": float(torch.linalg.norm(U16 - U32) / torch.linalg.norm(U32 - U0)),
            "note": "relative to the 3-step state change; both converge to the 1e-8 Newton tolerance"}
    c16.close()

    # ---- the plain FP64 single-instance form ----------------------------------
    U64 = U0.clone()
    kp = args.plain_steps or max(2, args.steps // 3)
    ms64, st64 = time_steps(ctx64, U64, w, kp, 1, dist, flush)
    ms64 = max_over_ranks(ms64, dist)
    plain = world * kp / (ms64 / 1e3)

    line = {
        "metric": METRIC, "value": value, "unit": "implicit steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "dof_per_s": value * w.n_unknowns,
        "precision": "FP64 residual, FD products and Arnoldi; FP32 preconditioner",
        "plain_fp64": {"value": plain, "unit": "implicit steps/s", "dof_per_s": plain * w.n_unknowns,
                       "ms_per_step": ms64 / kp,
                       "iterations_per_step": {"newton": sum(x["newton_its"] for x in st64) / kp,
                                               "gmres": sum(x["gmres_its"] for x in st64) / kp}},
        "iterations_per_step": {"newton": newton, "gmres": gmres},
        "phases_per_step": phases,
        "bf16_coarsest": bf16,
        "config": config_of(w, world, preset),
        "tuning": dict(tuning, tiles={k: preset.get(k) for k in ("tile_faces", "tile_volume", "tile_fv",
                                                                 "fv_split_cells")}),
        "clocks": clocks,
        "gpu_launches": int(launches),
        "e2e": {"value": e2e, "unit": "implicit steps/s", "h2d_bytes_per_step": 8 * ctx.N,
                "d2h_bytes_per_step": 8 * ctx.N, "p50_ms": statistics.median(lat),
                "p99_ms": sorted(lat)[min(len(lat) - 1, int(0.99 * len(lat)))]},
        "roofline": roof,
    }
    ctx.close()
    ctx64.close()
    if args.secondary_steps > 0:
        line["viscous"] = run_case(synth.DENSITY_CURRENT_Q2_256x32, args.secondary_steps)
        igw = synth.INERTIA_GRAVITY_Q3_80x3
        line["inertia_gravity"] = run_case(igw, args.secondary_steps)
        line["inertia_gravity"]["transfer_l2"] = {k: v for k, v in run_case(igw, args.secondary_steps,
                                                                            transfer_l2=1).items() if k != "workload"}
        line["rising_bubble"] = run_case(synth.RISING_BUBBLE_Q3_40x80, args.secondary_steps)
    if not args.no_long:
        line["long_runs"] = run_long_runs()
    if not args.no_sweep:
        line["mg_sweep"] = run_mg_sweep()
        line["dt_trends"] = run_dt_trends()
    if args.ensemble > 0:
        line["batched"] = run_ensemble(args.ensemble, args.ensemble_steps, 1, args.ensemble_threads, hbm_peak)
    if args.serve_seconds > 0 or args.overload_seconds > 0:
        line["serving"] = run_serving(args.serve_seconds, args.serve_rate, args.overload_seconds, rank, world, dist)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w)
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
