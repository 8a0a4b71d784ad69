"""Oracle pins: pair search (Tables 4-5), pair force (Eq. 16), particle motion.

- The half search of Table 4 and the grid search of Table 5 are different
  algorithms; on non-overlapping particles (the grid search's precondition,
  Eq. 49) they must produce the same pair set.  Exact ties at D + zeta are
  excluded by the strict rule.
- Eq. 16 is continuous at d = D + zeta (zero) and at d = D, repulsive, and
  obeys Newton's third law, so contact forces sum to zero without walls.
- With no hydrodynamic force a particle accelerates at (1 - rho_f/rho_p) g.
- Fluid plus particle momentum balances exactly in a periodic box.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2002_08855_gb300.inputs import Workload, place_rsa, random_points


def _cfg(dim, shape, periodic=(0, 0, 0), D=10.0, zeta=2.0, **kw):
    return Workload(name="p", dim=dim, nx=shape[0], ny=shape[1],
                    nz=shape[2] if dim == 3 else 1, periodic=periodic, diameter=D,
                    zeta=zeta, **kw).as_dict()


@pytest.mark.parametrize("dim,shape,n,seed,zeta", [
    (2, (300, 260, 1), 300, 1, 2.0), (2, (128, 256, 1), 90, 2, 2.0),
    (3, (90, 80, 100), 250, 3, 1.0)])
def test_half_search_equals_grid_search(dim, shape, n, seed, zeta):
    """In 3D, Eq. 49-50 leave a cell size only when (D + zeta)/2 < D/sqrt(3)."""
    X = place_rsa(dim, shape[:dim], n, 10.0, seed=seed, gap=0.3)
    cfg = _cfg(dim, shape, zeta=zeta)
    a = oracle.pairs_bruteforce(cfg, X)
    b = oracle.pairs_gridsearch(cfg, X)
    assert len(a) > 10
    assert np.array_equal(a, b)


def test_pair_rule_is_strict_at_threshold():
    cfg = _cfg(2, (100, 100, 1))
    X = np.array([[10.0, 10.0], [22.0, 10.0], [10.0, 21.75], [40.0, 40.0], [40.0, 52.0]])
    got = oracle.pairs_bruteforce(cfg, X)
    # |0-1| = 12 = D + zeta exactly (no pair); |0-2| = 11.75 (pair); |3-4| = 12 (no pair)
    assert got.tolist() == [[0, 2]]


def test_grid_search_rejects_overlap():
    cfg = _cfg(2, (100, 100, 1))
    X = np.array([[10.0, 10.0], [10.5, 10.2]])
    with pytest.raises(ValueError):
        oracle.pairs_gridsearch(cfg, X)


def test_periodic_pairs_use_nearest_image():
    cfg = _cfg(2, (50, 40, 1), periodic=(1, 0, 0))
    X = np.array([[1.0, 20.0], [47.5, 20.0], [25.0, 20.0]])
    assert oracle.pairs_bruteforce(cfg, X).tolist() == [[0, 1]]


def test_pair_force_eq16_shape():
    D, z = 10.0, 2.0
    cfg = _cfg(2, (100, 100, 1), D=D, zeta=z)
    c = 0.37
    f = lambda d: oracle.pair_force(cfg, c, (50.0 + d, 50.0), (50.0, 50.0))
    assert np.abs(f(D + z)).max() == 0.0
    assert np.abs(f(D + z - 1e-9)).max() < 1e-12
    eps = 1e-9
    assert abs(f(D - eps)[0] - f(D + eps)[0]) < 1e-5
    # within range the force pushes i away from j and grows as they approach
    mags = [f(d)[0] for d in (11.9, 11.0, 10.0, 9.5, 9.0)]
    assert all(m > 0 for m in mags)
    assert all(b > a for a, b in zip(mags, mags[1:]))
    # value of the middle case of Eq. 16 at d = D: (c / eps_pp) * 1
    assert f(D)[0] == pytest.approx(c / 1e-2, rel=1e-12)


def test_contact_forces_newton_third_law_and_walls():
    cfg = _cfg(2, (60, 50, 1), periodic=(1, 1, 0), gravity=(0, -1e-5, 0), density_ratio=1.5)
    X = random_points(40, 2, [0, 0], [60, 50], seed=4)
    Fc = oracle.contact_forces(cfg, X)
    assert np.abs(Fc).max() > 0
    assert np.abs(Fc.sum(0)).max() < 1e-12 * np.abs(Fc).max() * len(X)
    # near the lower wall (at -1/2) the mirror image pushes the particle up
    cfg_w = _cfg(2, (60, 50, 1), gravity=(0, -1e-5, 0), density_ratio=1.5)
    Fw = oracle.contact_forces(cfg_w, np.array([[30.0, 4.8]]))  # gap to wall 5.3, image at 10.6
    c = abs(0.5 * math.pi * 25.0 * 1e-5)
    t = (10.6 - 10.0 - 2.0) / 2.0
    assert Fw[0, 0] == 0.0
    assert Fw[0, 1] == pytest.approx(c / 1e-2 * t * t, rel=1e-12)


@pytest.mark.parametrize("dim", [2, 3])
def test_free_fall_reaches_reduced_gravity(dim):
    """With no fluid coupling (no MDF iteration, fluid at rest) the only force is the
    weight less buoyancy (M_p - rho_f V_p) g acting on M_p: the acceleration settles
    at (1 - rho_f/rho_p) g, the stabilising K terms only delay the start by a bounded
    number of steps, and nothing rotates."""
    g = (0.0, -1e-5, 0.0) if dim == 2 else (0.0, 0.0, -1e-5)
    shape = (40, 60, 1) if dim == 2 else (30, 30, 40)
    rho = 1.5
    w = Workload(name="ff", dim=dim, nx=shape[0], ny=shape[1], nz=shape[2], tau=0.7,
                 n_particles=1, n_lag=30 if dim == 2 else 100, diameter=8.0, mdf_iters=0,
                 gravity=g, density_ratio=rho)
    x0 = np.array([[20.0, 30.0]]) if dim == 2 else np.array([[15.0, 15.0, 20.0]])
    S = oracle.Sim(w.as_dict(), x0)
    a_inf = (1.0 - 1.0 / rho) * np.array(g[:dim])
    S.step(299)
    u1 = S.get_particles()["U"][0]
    S.step(1)
    st = S.get_particles()
    assert np.abs((st["U"][0] - u1) - a_inf).max() < 1e-15
    lag = (300 * a_inf - st["U"][0])[dim - 1] / a_inf[dim - 1]
    assert 0.0 < lag < 2.0
    assert np.abs(st["Omega"]).max() == 0.0
    assert np.abs(st["F_h"]).max() == 0.0


@pytest.mark.parametrize("dim", [2, 3])
def test_fluid_particle_momentum_balance(dim):
    """Fully periodic box: the collision adds sum_x f_IB = sum_b F_b dV to the fluid
    momentum (Eq. 8 moments, Eq. 48 partition of unity) and each particle receives the
    two-step mean of F_h = -sum_b F_b dV plus the change of its interior fluid
    momentum.  The stabilised update telescopes, so
      Q(t) = sum_x u*(t) + sum_p [M_p U^t + K a^{t-1} + F_h^{t-1}/2 - P_int^{t-1}]
             - t N_p (M_p - rho_f V_p) g
    is conserved up to round-off (contact forces cancel by Newton's third law)."""
    if dim == 2:
        w = Workload(name="mb", dim=2, nx=48, ny=40, periodic=(1, 1, 0), tau=0.7, n_particles=3,
                     n_lag=30, diameter=9.0, density_ratio=1.8, gravity=(2e-6, -1e-5, 0))
        xc = np.array([[12.0, 10.0], [30.0, 22.0], [20.5, 30.0]])
    else:
        w = Workload(name="mb3", dim=3, nx=20, ny=18, nz=22, periodic=(1, 1, 1), tau=0.7,
                     n_particles=2, n_lag=150, diameter=7.0, density_ratio=1.8,
                     gravity=(0, 2e-6, -1e-5))
        xc = np.array([[6.0, 6.0, 7.0], [13.0, 12.5, 15.0]])
    S = oracle.Sim(w.as_dict(), xc)
    D = w.diameter
    V = math.pi * D * D / 4 if dim == 2 else math.pi * D ** 3 / 6
    Mp = w.density_ratio * V
    meff = Mp - V
    K = w.n_lag * oracle.point_volume(w.as_dict())
    g = np.array(w.gravity[:dim])

    def Q(t, u_prev):
        _, u = S.get_fields()
        st = S.get_particles()
        P, _ = S.get_interior_momentum()
        part = Mp * st["U"] + K * (st["U"] - u_prev) + 0.5 * st["F_h"] - P
        return u.sum(1) + part.sum(0) - t * len(xc) * meff * g

    u0 = S.get_particles()["U"].copy()
    S.step(1)
    q1 = Q(1, u0)
    S.step(58)
    u59 = S.get_particles()["U"].copy()
    S.step(1)
    q60 = Q(60, u59)
    scale = Mp * np.abs(S.get_particles()["U"]).sum()
    assert scale > 0
    assert np.abs(q60 - q1).max() < 1e-10 * scale
