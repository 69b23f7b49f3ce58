"""Failure paths of the implicit step, made on the host side (no GPU fault):
an iteration cap that cannot be met, a non-finite state in one ensemble member,
a wall-clock budget that runs out.  Each returns its error code, leaves the
failing state at U^n and leaves every other state untouched."""
import numpy as np
import pytest

import synth
from tests._common import gpu_context, initial_state, oracle_dg, to_cpu, to_gpu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

JFNK_ENOTCONV, JFNK_ETIMEOUT, JFNK_ENAN = -4, -5, -6


def _case(k=2, nx=12, nz=6):
    w = synth.scaled(synth.BUBBLE_Q2_20x10, nx, nz, k=k, scheme=1)
    dg = oracle_dg(w)
    return w, initial_state(w, dg)


@pytest.mark.parametrize("prec", [64, 32])
def test_gmres_cap_gives_enotconv_and_restores_the_state(prec):
    # one GMRES iteration per Newton step and two Newton steps cannot reach the
    # 1e-8 Newton tolerance: ENOTCONV, and U is put back to U^n bit for bit
    w, U0 = _case()
    ctx = gpu_context(w, precond_prec=prec, gmres_max=1, newton_max=2)
    U = to_gpu(U0)
    st = ctx.implicit_step(U, w.dt, scheme=1, raise_on_error=False)
    assert st.status == JFNK_ENOTCONV
    assert np.array_equal(to_cpu(U).ravel(), U0.ravel())
    # the context stays usable: the same state steps normally afterwards
    ok = gpu_context(w, precond_prec=prec)
    st2 = ok.implicit_step(U, w.dt, scheme=1, raise_on_error=False)
    assert st2.status == 0


def test_time_budget_gives_etimeout_and_restores_the_state():
    w, U0 = _case(k=3, nx=24, nz=12)
    ctx = gpu_context(w, time_budget_ms=1e-3)      # 1 us: over after the first Arnoldi step
    U = to_gpu(U0)
    st = ctx.implicit_step(U, w.dt, scheme=1, raise_on_error=False)
    assert st.status == JFNK_ETIMEOUT
    assert np.array_equal(to_cpu(U).ravel(), U0.ravel())
    roomy = gpu_context(w, time_budget_ms=60_000.0)
    st2 = roomy.implicit_step(U, w.dt, scheme=1, raise_on_error=False)
    assert st2.status == 0


@pytest.mark.timeout(600)
@pytest.mark.parametrize("mode", [0, 1])
def test_nan_in_one_batch_member_fails_only_that_member(mode):
    # a NaN written into member 1's state: its residual norm is non-finite, so it
    # returns ENAN with its state restored (NaN included, bit for bit); the other
    # members' results are the bits they get when stepped alone
    import paper_2505_24504_gb300 as P
    w = synth.BUBBLE_Q2_20x10
    ms = [synth.scaled(w, 12, 6, k=1, scheme=1), synth.scaled(w, 10, 5, k=2, scheme=1),
          synth.scaled(w, 8, 4, k=3, scheme=1, fv_levels=4)]
    U0 = [initial_state(m, oracle_dg(m)) for m in ms]
    alone = []
    for m, u in zip(ms, U0):
        c = gpu_context(m, precond_prec=32)
        U = to_gpu(u)
        c.implicit_step(U, m.dt, scheme=1)
        alone.append(to_cpu(U))
        c.close()
    ctxs = [gpu_context(m, precond_prec=32) for m in ms]
    batch = P.Batch(ctxs, max_threads=3, mode=mode)
    Us = [to_gpu(u) for u in U0]
    Us[1].view(-1)[17] = float("nan")
    bad = to_cpu(Us[1])
    status, stats = batch.jfnk_batch_step(Us, [m.dt for m in ms], [1, 1, 1], raise_on_error=False)
    torch.cuda.synchronize()
    assert status[1] == JFNK_ENAN and stats[1].status == JFNK_ENAN
    assert status[0] == 0 and status[2] == 0
    got1 = to_cpu(Us[1])
    assert np.array_equal(np.isnan(got1), np.isnan(bad))
    assert np.array_equal(got1[~np.isnan(bad)], bad[~np.isnan(bad)])
    assert np.array_equal(to_cpu(Us[0]), alone[0])
    assert np.array_equal(to_cpu(Us[2]), alone[2])
    batch.close()
