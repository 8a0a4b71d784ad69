"""GPU pair search against the oracle's brute-force half search (Table 4): the pair
list must be identical, bit for bit, for the same positions."""
import numpy as np
import pytest

import oracle
from paper_2002_08855_gb300 import inputs

from gpu_util import require_gpu

pytestmark = pytest.mark.gpu


def _cfg(dim, shape, per=(0, 0, 0), D=10.0, zeta=2.0):
    return inputs.Workload(name="p", dim=dim, nx=shape[0], ny=shape[1],
                           nz=shape[2] if dim == 3 else 1, periodic=per, diameter=D,
                           zeta=zeta).as_dict()


def _gpu(dim, shape, per, X, D=10.0, zeta=2.0, kmax=0):
    from paper_2002_08855_gb300.binding import pair_search
    return pair_search(dim, shape, per, D, zeta, X, max_neighbors=kmax)


@pytest.mark.parametrize("dim,shape,per,n,seed", [
    (2, (200, 150, 1), (0, 0, 0), 1000, 1),
    (2, (97, 61, 1), (1, 0, 0), 200, 2),
    (2, (64, 64, 1), (1, 1, 0), 150, 3),
    (3, (50, 40, 60), (0, 0, 0), 400, 4),
    (3, (30, 33, 36), (1, 1, 1), 120, 5),
    (2, (30, 30, 1), (0, 0, 0), 1, 6),
])
def test_random_positions_match_brute_force(dim, shape, per, n, seed):
    """Uniform random centres, overlaps allowed (about 15-30 partners each), so the
    list capacity is raised to its maximum of 64."""
    require_gpu()
    X = inputs.random_points(n, dim, [-0.5] * dim, [s - 0.5 - 1e-9 for s in shape[:dim]], seed)
    ref = oracle.pairs_bruteforce(_cfg(dim, shape, per), X)
    got = _gpu(dim, shape, per, X, kmax=64)
    assert np.array_equal(got, ref)


def test_capacity_overflow_is_reported():
    """More partners than max_neighbors: CAPACITY, never a silent truncation."""
    require_gpu()
    from paper_2002_08855_gb300.binding import IbmLbmError
    X = inputs.random_points(400, 2, [0, 0], [40, 40], seed=8)
    with pytest.raises(IbmLbmError) as e:
        _gpu(2, (40, 40, 1), (0, 0, 0), X, kmax=8)
    assert e.value.name == "CAPACITY"


def test_exact_threshold_ties_and_cell_faces():
    """Spacing exactly D + zeta gives no pairs (strict rule); a hair closer gives all;
    centres sit exactly on cell faces of the GPU grid (cell side 12 here)."""
    require_gpu()
    shape = (144, 144, 1)
    g = np.arange(0, 144, 12.0) - 0.5
    X = np.array([(x, y) for x in g for y in g])
    assert len(_gpu(2, shape, (0, 0, 0), X)) == 0
    assert len(oracle.pairs_bruteforce(_cfg(2, shape), X)) == 0
    Y = X * (11.999 / 12.0)
    ref = oracle.pairs_bruteforce(_cfg(2, shape), Y)
    assert len(ref) > 0
    assert np.array_equal(_gpu(2, shape, (0, 0, 0), Y), ref)


def test_dense_packing_at_full_size():
    """2048 x 4096 cavity, 42723 particles (solid fraction 0.4) with a contact gap of
    0.3 lattice units, so that neighbours fall inside D + zeta."""
    require_gpu()
    X = inputs.place_hex((2048, 4096), 42723, 10.0, seed=inputs.SEED_BASE + 203, gap=0.3)
    ref = oracle.pairs_bruteforce(_cfg(2, (2048, 4096, 1)), X)
    got = _gpu(2, (2048, 4096, 1), (0, 0, 0), X)
    assert len(ref) > 1000
    assert np.array_equal(got, ref)


def test_handle_pairs_and_contact_forces():
    """The pair list and Eq. 16 forces of a step (particles held fixed) against the
    oracle on the same positions."""
    require_gpu()
    from paper_2002_08855_gb300.binding import Simulation

    w = inputs.Workload(name="c", dim=2, nx=120, ny=100, n_particles=40, n_lag=25, diameter=8.0,
                        zeta=2.0, gravity=(0, -1e-5, 0), density_ratio=1.5, fixed_particles=1,
                        mdf_iters=0)
    X = inputs.place_rsa(2, (120, 100), 40, 8.0, seed=9, gap=0.2, wall_gap=0.1)
    sim = Simulation(w, X)
    sim.step(1)
    pairs = sim.get_pairs()
    ref = oracle.pairs_bruteforce(w.as_dict(), X)
    assert len(ref) > 0
    assert np.array_equal(pairs, ref)
    Fc = sim.get_particles()["F_c"]
    Fo = oracle.contact_forces(w.as_dict(), X)
    assert np.abs(Fc - Fo).max() <= 1e-12 * max(np.abs(Fo).max(), 1e-30)
    sim.close()


@pytest.mark.parametrize("dim,shape,per", [
    (2, (120, 100, 1), (0, 0, 0)),
    (2, (90, 70, 1), (1, 1, 0)),
    (3, (40, 36, 34), (0, 0, 0)),
    (3, (34, 30, 32), (1, 0, 1)),
])
def test_grid_search_pairs_and_forces(dim, shape, per):
    """The grid search of Table 5 (one particle per cell of side < D_p / sqrt(dim)) on
    held particles, some pairs overlapping so that two centres share a grid cell (the
    overflow list): the pair list equals the brute-force half search and the Eq. 16
    forces equal the oracle's."""
    require_gpu()
    from paper_2002_08855_gb300.binding import Simulation

    D = 8.0
    n0 = 30 if dim == 2 else 20
    X = inputs.place_rsa(dim, shape[:dim], n0, D, seed=31 + dim, gap=0.2, wall_gap=0.5)
    # overlapping partners: 1.5 lattice units from a placed centre (same or next cell)
    extra = X[:3] + np.array([1.5] + [0.3] * (dim - 1))
    X = np.vstack([X, extra])
    w = inputs.Workload(name="g", dim=dim, nx=shape[0], ny=shape[1], nz=shape[2] if dim == 3 else 1,
                        periodic=per, n_particles=len(X), n_lag=25 if dim == 2 else 100, diameter=D,
                        zeta=2.0, gravity=(0, -1e-5, 0), density_ratio=1.5, fixed_particles=1,
                        mdf_iters=0, pair_search=1)
    sim = Simulation(w, X, max_neighbors=64)
    sim.step(1)
    ref = oracle.pairs_bruteforce(w.as_dict(), X)
    assert len(ref) > 3
    assert np.array_equal(sim.get_pairs(), ref)
    Fc = sim.get_particles()["F_c"]
    Fo = oracle.contact_forces(w.as_dict(), X)
    assert np.abs(Fc - Fo).max() <= 1e-12 * max(np.abs(Fo).max(), 1e-30)
    sim.close()


def test_grid_search_whole_steps_match_oracle():
    """The 128 x 256 cavity (12 circles, 200 steps) with the grid search: the same
    trajectory as the oracle, and the in-run pair list of step 200 equals the
    brute-force list of the centres it was built from."""
    require_gpu()
    from paper_2002_08855_gb300.binding import Simulation

    from gpu_util import rel_l2

    w = inputs.cavity_2d_small().with_(pair_search=1)
    X0 = inputs.place_particles(w)
    sim = Simulation(w, X0)
    ref = oracle.Sim(w.as_dict(), X0)
    sim.step(199)
    X199 = sim.get_particles()["X"]
    sim.step(1)
    sim.sync()
    ref.step(200)
    _, ug = sim.get_fields()
    _, uo = ref.get_fields()
    assert rel_l2(ug.cpu().numpy(), uo) < 1e-5
    pg, po = sim.get_particles(), ref.get_particles()
    assert rel_l2(pg["X"] - X0, po["X"] - X0) < 1e-5
    assert np.array_equal(sim.get_pairs(), oracle.pairs_bruteforce(w.as_dict(), X199))
    sim.close()
