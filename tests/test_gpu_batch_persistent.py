"""Persistent mode of the batched ensemble: a step is one cooperative kernel for the
IBM phases, one for the contact phases and the particle update, and the collide-stream
launch.  The phases run the same per-block code as the ordinary mode's fused launches,
so every member must still reproduce its run alone.  The grid barriers' waits are
bounded: a limit of one poll makes them give up, ibm_lbm_batch_sync reports TIMEOUT,
every kernel returns, and after the reset the batch steps on normally."""
import time

import numpy as np
import pytest

from paper_2002_08855_gb300 import inputs
from paper_2002_08855_gb300.inputs import Workload

from gpu_util import rel_l2, require_gpu

pytestmark = pytest.mark.gpu


def _members(storage=0):
    base = dict(dim=2, tau=0.6, delta_kind=4, drs=2.6, mdf_iters=3, density_ratio=1.5,
                gravity=(0.0, -1e-5, 0.0), pdf_storage=storage)
    ws = [
        Workload(name="m0", nx=64, ny=80, n_particles=3, n_lag=25, diameter=8.0, seed=11, **base),
        Workload(name="m1", nx=96, ny=72, n_particles=5, n_lag=39, diameter=12.5, seed=12, **base),
        Workload(name="m2", nx=70, ny=64, n_particles=2, n_lag=50, diameter=16.0, seed=13, **base),
        Workload(name="m3", nx=80, ny=90, n_particles=0, seed=14, **{**base, "tau": 0.7}),
        Workload(name="m4", nx=130, ny=66, n_particles=4, n_lag=31, diameter=10.0, seed=15, **base),
        Workload(name="m5", nx=48, ny=52, n_particles=6, n_lag=25, diameter=8.0, seed=16, **base),
    ]
    return ws, [inputs.place_particles(w) for w in ws]


@pytest.mark.parametrize("storage", [0, 1])
def test_persistent_members_match_runs_alone(storage):
    require_gpu()
    from paper_2002_08855_gb300.binding import Batch, Simulation

    ws, Xs = _members(storage)
    tol = 1e-6 if storage == 0 else 1e-3  # atomic order of the spreading only
    batch = Batch(ws, Xs)
    batch.set_persistent(True)
    assert batch.persistent()
    batch.step(40)
    batch.sync()
    for w, X, m in zip(ws, Xs, batch.members):
        alone = Simulation(w, X)
        alone.step(40)
        alone.sync()
        _, ub = m.get_fields()
        _, ua = alone.get_fields()
        assert rel_l2(ub.cpu().numpy(), ua.cpu().numpy()) < tol, w.name
        if w.n_particles:
            pb, pa = m.get_particles(), alone.get_particles()
            assert rel_l2(pb["X"] - X, pa["X"] - X) < tol, w.name
            assert rel_l2(pb["U"], pa["U"]) < 10 * tol, w.name
            if storage == 0:
                assert np.array_equal(m.get_pairs(), alone.get_pairs()), w.name
        alone.close()
    batch.close()


@pytest.mark.parametrize("mdf", [0, 1])
def test_persistent_mdf_counts(mdf):
    """No forcing iteration (one box gather, then the sums) and a single one."""
    require_gpu()
    from paper_2002_08855_gb300.binding import Batch

    ws, Xs = _members()
    ws = [w.with_(mdf_iters=mdf) for w in ws]
    out = []
    for persistent in (False, True):
        batch = Batch(ws, Xs)
        batch.set_persistent(persistent)
        batch.step(12)
        batch.sync()
        out.append([(m.get_fields()[1].cpu().numpy(), m.get_particles()["X"] if w.n_particles else None)
                    for w, m in zip(ws, batch.members)])
        batch.close()
    for w, X, (ua, xa), (ub, xb) in zip(ws, Xs, *out):
        assert rel_l2(ua, ub) < 1e-6, w.name
        if xa is not None:
            assert rel_l2(xa - X, xb - X) < 1e-6, w.name


def test_ensemble_persistent_three_launches_per_step():
    require_gpu()
    from paper_2002_08855_gb300.binding import Batch

    ws = inputs.ensemble_2d()
    Xs = [inputs.place_particles(w) for w in ws]
    runs = []
    for persistent in (False, True):
        batch = Batch(ws, Xs)
        batch.set_persistent(persistent)
        batch.step(5)
        batch.sync()
        n0 = batch.launch_count()
        batch.step(4)
        batch.sync()
        per_step = (batch.launch_count() - n0) / 4
        if persistent:
            assert per_step <= 3, per_step
        runs.append([batch.members[k].get_fields()[1].cpu().numpy() for k in (0, 17, 101, 255)])
        batch.close()
    for a, b in zip(*runs):
        assert np.isfinite(b).all()
        assert rel_l2(a, b) < 1e-6


def test_barrier_limit_runs_out_and_the_batch_recovers():
    """Batch A steps with a one-poll barrier limit (its barriers give up), batch B the
    same steps in the ordinary mode.  A's sync reports TIMEOUT once; given B's member
    states, A then steps on exactly like B."""
    require_gpu()
    from paper_2002_08855_gb300.binding import Batch, IbmLbmError

    ws, Xs = _members()
    A, B = Batch(ws, Xs), Batch(ws, Xs)
    for b in (A, B):
        b.step(2)
        b.sync()
    A.set_persistent(True, barrier_limit=1)
    t0 = time.perf_counter()
    A.step(6)
    with pytest.raises(IbmLbmError) as e:
        A.sync()
    assert e.value.name == "TIMEOUT"
    assert time.perf_counter() - t0 < 30.0  # every kernel returned
    A.sync()  # the status was cleared
    B.step(6)
    B.sync()
    for ma, mb in zip(A.members, B.members):
        ma.set_state(mb.get_state())
    A.set_persistent(True)  # the default limit
    for b in (A, B):
        b.step(10)
        b.sync()
    for w, ma, mb in zip(ws, A.members, B.members):
        assert rel_l2(ma.get_fields()[1].cpu().numpy(), mb.get_fields()[1].cpu().numpy()) < 1e-6, w.name
        if w.n_particles:
            assert np.array_equal(ma.get_pairs(), mb.get_pairs()), w.name
    A.close()
    B.close()
