"""GPU parity of the non-equilibrium extrapolation boundaries (the method Sec. 6.1-6.2
apply) against the FP64 oracle: the Poiseuille channel with a parabolic inlet and a
pressure outlet (Sec. 6.1's particle-free flows, 2D and 3D), body-force Poiseuille
flow between extrapolation walls, and the settling particles of Sec. 6.2 (closed
cavity with extrapolation walls, 3-point delta, drs = 1.9, density ratio 1.01).  Both
step parities are checked (odd and even step counts), since the boundary kernel writes
the layout of the next step."""
import numpy as np
import pytest

import oracle
from paper_2002_08855_gb300 import inputs
from paper_2002_08855_gb300.inputs import Workload

from gpu_util import rel_l2, require_gpu

pytestmark = pytest.mark.gpu


def _compare(w, X, steps, tol=1e-5, tol_p=3e-5):
    """Velocity within tol (relative L2); pressure within tol_p relative to the larger of
    |p| and |u| (L2 over the nodes).  p (Eq. 6) is a sum of PDFs whose size is set by
    the velocity (|f| ~ |u| / 3), so FP32 rounding puts an error of about 1e-7 |u| on p
    per node and step, whatever p is: in a channel p ~ 1e-4 against u ~ 1e-2, and in a
    body-force flow with a periodic axis p is near zero."""
    from paper_2002_08855_gb300.binding import Simulation

    sim = Simulation(w, X)
    ref = oracle.Sim(w.as_dict(), X)
    sim.step(steps)
    ref.step(steps)
    pg, ug = sim.get_fields()
    po, uo = ref.get_fields()
    e_u = rel_l2(ug.cpu().numpy(), uo)
    pgn = pg.cpu().numpy()
    e_p = np.linalg.norm(pgn - po) / max(np.linalg.norm(po), np.linalg.norm(uo))
    print(f"{w.name} {steps} steps: velocity {e_u:.2e}, pressure {e_p:.2e}")
    assert e_u < tol and e_p < tol_p
    if w.n_particles:
        a, b = sim.get_particles(), ref.get_particles()
        assert rel_l2(a["X"] - X, b["X"] - X) < tol
    sim.close()


@pytest.mark.parametrize("steps", [300, 301])
def test_channel_2d(steps):
    require_gpu()
    w = Workload(name="chan2", dim=2, nx=33, ny=40, tau=0.8, boundary=2, u_inlet=0.02)
    _compare(w, np.zeros((0, 2)), steps)


@pytest.mark.parametrize("steps", [60, 61])
def test_channel_3d(steps):
    require_gpu()
    w = Workload(name="chan3", dim=3, nx=17, ny=20, nz=15, tau=0.7, boundary=2, u_inlet=0.02)
    _compare(w, np.zeros((0, 3)), steps)


@pytest.mark.parametrize("dim", [2, 3])
def test_body_force_poiseuille_between_extrapolation_walls(dim):
    require_gpu()
    w = Workload(name=f"pois{dim}", dim=dim, nx=21, ny=6, nz=5 if dim == 3 else 1, periodic=(0, 1, 1),
                 tau=0.9, body_force=(0.0, 1e-5, 0.0), boundary=1)
    _compare(w, np.zeros((0, dim)), 401)


def test_closed_cavity_settling_with_extrapolation_walls():
    """Sec. 6.2: settling circles (rho_p / rho_f = 1.01) in a closed cavity whose walls
    are extrapolation boundaries, 3-point delta with drs = 1.9."""
    require_gpu()
    w = Workload(name="settle", dim=2, nx=96, ny=128, tau=0.6, n_particles=10, n_lag=31,
                 diameter=10.0, delta_kind=3, drs=1.9, density_ratio=1.01,
                 gravity=(0.0, -1e-3, 0.0), boundary=1, seed=21)
    X = inputs.place_particles(w)
    _compare(w, X, 151)


def test_smallest_domain_and_mixed_axes():
    """Three nodes across each wall axis (the smallest the method allows), a periodic
    x axis beside a channel along y, and a z wall pair in 3D."""
    require_gpu()
    w = Workload(name="tiny", dim=3, nx=5, ny=3, nz=3, periodic=(1, 0, 0), tau=0.75,
                 body_force=(2e-5, 0.0, 0.0), boundary=2, u_inlet=0.01)
    _compare(w, np.zeros((0, 3)), 41)


def test_closed_cavity_3d_settling_with_extrapolation_walls():
    """The 3D form of Sec. 6.2's setting: spheres (d = 10, density ratio 1.01, 3-point
    delta, drs = 1.9) settling in a closed cube whose walls are extrapolation
    boundaries, with the grid search of Table 5 for the contacts."""
    require_gpu()
    w = Workload(name="settle3", dim=3, nx=40, ny=40, nz=48, tau=0.6, n_particles=6, n_lag=314,
                 diameter=10.0, delta_kind=3, drs=1.9, density_ratio=1.01,
                 gravity=(0.0, 0.0, -1e-3), boundary=1, pair_search=1, seed=23)
    X = inputs.place_particles(w)
    _compare(w, X, 41)
