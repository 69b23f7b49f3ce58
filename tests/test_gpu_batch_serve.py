"""Batched ensembles and the serving loop: every member / request result is the
same bits as running that state alone (deterministic kernels, per-member
buffers), under concurrency, uneven grids and orders, and HBM-budget eviction."""
import numpy as np
import pytest

import synth
from tests._common import gpu_context, oracle_dg, to_cpu, to_gpu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _members():
    w = synth.BUBBLE_Q2_20x10
    ms = [synth.scaled(w, 16, 8, k=1, scheme=1), synth.scaled(w, 20, 10, k=2, scheme=1),
          synth.scaled(w, 12, 6, k=3, scheme=1, fv_levels=4), synth.scaled(w, 8, 4, k=4, scheme=1),
          synth.scaled(synth.DENSITY_CURRENT_Q2_256x32, 24, 6, x1=19200.0, k=2)]
    states = []
    for m in ms:
        dg = oracle_dg(m)
        states.append(dg.init_state(m.theta_pert(dg.X, dg.Z)))
    return ms, states


@pytest.mark.timeout(600)
@pytest.mark.parametrize("prec,mode", [(64, 0), (32, 0), (32, 1), (64, 1)])
def test_batch_step_bitwise_equals_alone(prec, mode):
    # mode 1: lock-step, every operator launch shared by the members that reach it
    # together (uneven grids and orders, one viscous member)
    import paper_2505_24504_gb300 as P
    ms, U0 = _members()
    alone = []
    for m, u in zip(ms, U0):
        ctx = gpu_context(m, precond_prec=prec)
        U = to_gpu(u)
        for _ in range(2):
            ctx.implicit_step(U, m.dt, scheme=m.scheme)
        alone.append(to_cpu(U))
        ctx.close()
    ctxs = [gpu_context(m, precond_prec=prec) for m in ms]
    batch = P.Batch(ctxs, max_threads=4, mode=mode)
    Us = [to_gpu(u) for u in U0]
    for _ in range(2):
        status, stats = batch.jfnk_batch_step(Us, [m.dt for m in ms], [m.scheme for m in ms])
        assert status == [0] * len(ms)
        assert all(s.newton_its > 0 for s in stats)
        if mode == 1:
            ll = batch.last_launches()
            assert ll["grouped"] > 0 and ll["launches"] < ll["member_launches"], ll
    torch.cuda.synchronize()
    for a, u in zip(alone, Us):
        assert np.array_equal(a, to_cpu(u))
    batch.close()


@pytest.mark.timeout(600)
def test_lockstep_same_shape_members_share_launches():
    # eight members of one shape (different bubbles): bitwise equal to alone, and
    # far fewer launches than the members would issue alone
    import paper_2505_24504_gb300 as P
    w = synth.BUBBLE_Q2_20x10
    ms = [synth.scaled(w, 20, 10, k=2, scheme=1,
                       bubble=synth.Bubble(1.0 + 0.4 * i, 8000.0 + 500.0 * i, 2000.0, 2000.0, 2000.0))
          for i in range(8)]
    U0 = []
    for m in ms:
        dg = oracle_dg(m)
        U0.append(dg.init_state(m.theta_pert(dg.X, dg.Z)))
    alone = []
    for m, u in zip(ms, U0):
        ctx = gpu_context(m, precond_prec=32)
        U = to_gpu(u)
        ctx.implicit_step(U, m.dt, scheme=m.scheme)
        alone.append(to_cpu(U))
        ctx.close()
    ctxs = [gpu_context(m, precond_prec=32) for m in ms]
    batch = P.Batch(ctxs, mode=P.jfnk.BATCH_LOCKSTEP)
    Us = [to_gpu(u) for u in U0]
    status, _ = batch.jfnk_batch_step(Us, [m.dt for m in ms], [m.scheme for m in ms])
    assert status == [0] * len(ms)
    ll = batch.last_launches()
    torch.cuda.synchronize()
    for a, u in zip(alone, Us):
        assert np.array_equal(a, to_cpu(u))
    assert ll["launches"] * 4 < ll["member_launches"], ll
    batch.close()


@pytest.mark.timeout(600)
def test_serving_mix_equals_alone_under_eviction():
    import paper_2505_24504_gb300 as P
    from paper_2505_24504_gb300.serve import Server, StateSpec
    ms, U0 = _members()
    specs = {}
    for sid, (m, u) in enumerate(zip(ms, U0)):
        c = gpu_context(m, precond_prec=32)
        specs[sid] = StateSpec(grid=c.grid, k=c.k, phys=c.phys, opts=c.opts, dt=m.dt, scheme=m.scheme,
                               U=to_gpu(u))
        c.close()
    # budget for the two largest contexts only: forces admission waits and evictions
    fp = sorted(s.footprint for s in specs.values())
    srv = Server(specs, hbm_budget=fp[-1] + fp[-2], workers=3)
    arr = synth.poisson_arrivals(400.0, 0.06, seed=7)
    rng = np.random.default_rng(3)
    reqs = [(float(t), int(rng.integers(0, len(ms)))) for t in arr]
    rep = srv.run(reqs, timeout_s=300.0)
    srv.close()
    summ = rep.summary()
    assert summ["requests"] == len(reqs) and summ["failed"] == 0
    assert summ["p99_ms"] >= summ["p50_ms"] > 0
    assert rep.contexts_evicted > 0 and rep.peak_bytes <= fp[-1] + fp[-2]
    # each state alone, as many steps as it was served
    for sid, (m, u) in enumerate(zip(ms, U0)):
        ctx = gpu_context(m, precond_prec=32)
        U = to_gpu(u)
        for _ in range(specs[sid].steps_done):
            ctx.implicit_step(U, m.dt, scheme=m.scheme)
        torch.cuda.synchronize()
        assert np.array_equal(to_cpu(U), to_cpu(specs[sid].U)), sid
        ctx.close()


@pytest.mark.timeout(300)
def test_grouped_residual_bitwise_equals_per_member():
    # one face + one volume launch per (order, viscous) group must give each
    # member exactly its own dg_residual; two members share order k = 2 so a
    # group holds more than one member
    import paper_2505_24504_gb300 as P
    ms, _ = _members()
    w = synth.BUBBLE_Q2_20x10
    ms = ms + [synth.scaled(w, 10, 6, k=2, scheme=1), synth.scaled(w, 6, 3, k=1, scheme=1)]
    ctxs = [gpu_context(m) for m in ms]
    states, alone = [], []
    for i, (m, c) in enumerate(zip(ms, ctxs)):
        dg = oracle_dg(m)
        u = to_gpu(synth.random_perturbation(dg.shape[1:], 40 + i))
        f = torch.empty(c.N, dtype=torch.float64, device="cuda")
        c.dg_residual(u, f)
        states.append(u)
        alone.append(to_cpu(f))
    batch = P.Batch(ctxs)
    outs = [torch.full((c.N,), float("nan"), dtype=torch.float64, device="cuda") for c in ctxs]
    for _ in range(2):   # twice: the descriptors are rewritten in place
        batch.jfnk_batch_dg_residual(states, outs)
        torch.cuda.synchronize()
        for a, o in zip(alone, outs):
            assert np.array_equal(a, to_cpu(o))
    batch.close()
