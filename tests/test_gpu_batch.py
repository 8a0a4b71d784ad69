"""Batched ensemble: independent 2D cavities of different sizes, diameters, point
counts and particle counts stepped together with fused launches.  Every member must
reproduce the same cavity run alone (the kernels are the same; only the order of
floating-point atomics in the spreading may differ) and, through it, the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2002_08855_gb300 import inputs
from paper_2002_08855_gb300.inputs import Workload

from gpu_util import rel_l2, require_gpu

pytestmark = pytest.mark.gpu


def _members():
    base = dict(dim=2, tau=0.6, delta_kind=4, drs=2.6, mdf_iters=3, density_ratio=1.5,
                gravity=(0.0, -1e-5, 0.0))
    ws = [
        Workload(name="m0", nx=64, ny=80, n_particles=3, n_lag=25, diameter=8.0, seed=11, **base),
        Workload(name="m1", nx=96, ny=72, n_particles=5, n_lag=39, diameter=12.5, seed=12, **base),
        Workload(name="m2", nx=70, ny=64, n_particles=2, n_lag=50, diameter=16.0, seed=13, **base),
        Workload(name="m3", nx=80, ny=90, n_particles=0, seed=14, **{**base, "tau": 0.7}),
        Workload(name="m4", nx=130, ny=66, n_particles=4, n_lag=31, diameter=10.0, seed=15, **base),
    ]
    return ws, [inputs.place_particles(w) for w in ws]


@pytest.mark.parametrize("storage", [0, 1])
def test_members_match_runs_alone(storage):
    require_gpu()
    from paper_2002_08855_gb300.binding import Batch, Simulation

    ws, Xs = _members()
    ws = [w.with_(pdf_storage=storage) for w in ws]
    # FP32: rounding of the atomic order only.  FP16: that difference can flip a
    # 16-bit rounding of a stored PDF, so the bound is at the FP16 rounding level.
    tol = 1e-6 if storage == 0 else 1e-3
    batch = Batch(ws, Xs)
    batch.step(40)
    batch.sync()
    for w, X, m in zip(ws, Xs, batch.members):
        alone = Simulation(w, X)
        alone.step(40)
        alone.sync()
        _, ub = m.get_fields()
        _, ua = alone.get_fields()
        e_u = rel_l2(ub.cpu().numpy(), ua.cpu().numpy())
        print(f"{w.name} storage {storage}: velocity {e_u:.2e}")
        assert e_u < tol, w.name
        if w.n_particles:
            pb, pa = m.get_particles(), alone.get_particles()
            assert rel_l2(pb["X"] - X, pa["X"] - X) < tol, w.name
            if storage == 0:
                assert np.array_equal(m.get_pairs(), alone.get_pairs())
        alone.close()
    assert batch.launch_count() > 0
    batch.close()


def test_member_matches_oracle():
    require_gpu()
    from paper_2002_08855_gb300.binding import Batch

    ws, Xs = _members()
    batch = Batch(ws, Xs)
    batch.step(60)
    batch.sync()
    for k in (1, 3):  # a member with particles and one without
        ref = oracle.Sim(ws[k].as_dict(), Xs[k])
        ref.step(60)
        _, ug = batch.members[k].get_fields()
        _, uo = ref.get_fields()
        assert rel_l2(ug.cpu().numpy(), uo) < 1e-5
        if ws[k].n_particles:
            pg, po = batch.members[k].get_particles(), ref.get_particles()
            assert rel_l2(pg["X"] - Xs[k], po["X"] - Xs[k]) < 1e-5
    batch.close()


def test_ensemble_256_cavities_steps():
    require_gpu()
    from paper_2002_08855_gb300.binding import Batch

    ws = inputs.ensemble_2d()
    Xs = [inputs.place_particles(w) for w in ws]
    batch = Batch(ws, Xs)
    batch.step(5)
    batch.sync()
    n0 = batch.launch_count()
    batch.step(4)
    batch.sync()
    # fused launches whatever the number of members: one per kernel, and the
    # interpolation and spreading once per box-size class (5 here: d = 8..16)
    assert (batch.launch_count() - n0) / 4 <= 8 + 6 * 5
    p, u = batch.members[17].get_fields()
    assert np.isfinite(u.cpu().numpy()).all()
    batch.close()


def _flow_members(storage):
    """Particle-free members of assorted shapes (short rows, a single row, a one-node
    cavity, periodic axes) with random PDFs and a body force: the collide-stream
    launch alone decides their state, and it has no atomics, so it is deterministic."""
    from paper_2002_08855_gb300.inputs import random_pdfs

    shapes = [(64, 64, (0, 0, 0)), (65, 3, (1, 0, 0)), (1, 1, (0, 0, 0)), (2, 7, (0, 1, 0)),
              (130, 90, (0, 0, 0)), (512, 33, (1, 1, 0)), (33, 1, (1, 0, 0)), (97, 101, (0, 0, 0))]
    ws = [Workload(name=f"f{i}", dim=2, nx=nx, ny=ny, periodic=per, tau=0.55 + 0.05 * (i % 3),
                   body_force=(1e-5, -2e-5, 0.0), pdf_storage=storage, seed=40 + i)
          for i, (nx, ny, per) in enumerate(shapes)]
    f0 = [random_pdfs(9, w.n_grid, seed=70 + i, scale=1e-2) for i, w in enumerate(ws)]
    return ws, f0


@pytest.mark.parametrize("storage", [0, 1])
def test_tile_shapes_update_every_node_identically(storage):
    """Every collide-stream tile shape (flat tiles of K x 128 consecutive nodes, warp
    tiles of 32 K nodes, W warps per block, persistent or not) gives the same PDFs bit
    for bit, over both AA parities."""
    require_gpu()
    from paper_2002_08855_gb300.binding import Batch, tile_shapes

    ws, f0 = _flow_members(storage)
    out = []
    for sh in range(len(tile_shapes(storage))):
        batch = Batch(ws, [None] * len(ws))
        for m, f in zip(batch.members, f0):
            m.set_pdfs(f)
        batch.set_tile_shape(sh)
        batch.step(7)
        batch.sync()
        assert batch.tile_shape() == sh
        out.append([m.get_pdfs().cpu().numpy() for m in batch.members])
        batch.close()
    for sh in range(1, len(out)):
        for i, (a, b) in enumerate(zip(out[0], out[sh])):
            assert np.array_equal(a, b), (sh, ws[i].name)


def test_autotune_picks_the_fastest_shape_and_keeps_the_results():
    """The autotuner's steps are real steps: after tuning and ten more steps every
    member equals its run alone after the same number of steps."""
    require_gpu()
    from paper_2002_08855_gb300.binding import Batch, Simulation, tile_shapes

    ws, Xs = _members()
    batch = Batch(ws, Xs)
    batch.step(2)
    chosen, ms = batch.autotune(4)
    assert len(ms) == len(tile_shapes(0)) and min(ms) > 0.0
    assert chosen == int(np.argmin(ms))
    batch.step(10)
    batch.sync()
    steps = 2 + 4 * len(ms) + 10
    for w, X, m in zip(ws, Xs, batch.members):
        alone = Simulation(w, X)
        alone.step(steps)
        alone.sync()
        _, ub = m.get_fields()
        _, ua = alone.get_fields()
        assert rel_l2(ub.cpu().numpy(), ua.cpu().numpy()) < 1e-6, w.name
        alone.close()
    batch.close()
