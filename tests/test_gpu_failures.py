"""Failure detection: the device status word, reported by ibm_lbm_sync.

Every failure is injected from the host through the public calls; nothing here faults,
traps or hangs the GPU:
- NONFINITE: a NaN spin set on bodies held in place (their centres stay put, so no
  kernel ever sees a non-finite position); the update flags the non-finite state.
- CAPACITY: contact lists of one slot for three bodies in mutual range; the search
  writes the first entry only and flags the overflow.
- OUT_OF_DOMAIN: with no IB forcing, a body is given a velocity that carries its
  centre through a wall within one step.  Within that step the IBM and the contact
  search use the centre it had before (inside); only the point regeneration sees the
  new one, and it clips its node marks at every wall.  The run is not stepped again.
After each failure sync clears the word, and the handle keeps working.
"""
import numpy as np
import pytest

from paper_2002_08855_gb300.inputs import Workload

from gpu_util import require_gpu

pytestmark = pytest.mark.gpu


def _sim(dim=2, **kw):
    from paper_2002_08855_gb300.binding import Simulation

    base = dict(name="fail", dim=dim, nx=48, ny=40, nz=36 if dim == 3 else 1, tau=0.7,
                n_particles=1, n_lag=31 if dim == 2 else 201, diameter=10.0 if dim == 2 else 8.0,
                density_ratio=1.5, gravity=(0.0, -1e-5, 0.0))
    base.update(kw)
    return Workload(**base)


def _code(sim):
    from paper_2002_08855_gb300.binding import IbmLbmError

    try:
        sim.sync()
        return "OK"
    except IbmLbmError as e:
        return e.name


@pytest.mark.parametrize("dim", [2, 3])
def test_nonfinite_spin_is_reported_and_cleared(dim):
    require_gpu()
    from paper_2002_08855_gb300.binding import Simulation

    w = _sim(dim, fixed_particles=1)
    X = np.array([[24.3, 20.1]]) if dim == 2 else np.array([[24.3, 20.1, 17.6]])
    sim = Simulation(w, X)
    sim.step(2)
    assert _code(sim) == "OK"
    sim.set_particles(X, Omega=np.full((1, 1 if dim == 2 else 3), np.nan))
    sim.step(1)
    assert _code(sim) == "NONFINITE"
    # the word was cleared; with a finite state and fresh PDFs the run continues
    sim.set_particles(X, Omega=np.zeros((1, 1 if dim == 2 else 3)))
    sim.set_pdfs(np.zeros((9 if dim == 2 else 19, w.n_grid), dtype=np.float32))
    sim.step(3)
    assert _code(sim) == "OK"
    p, u = sim.get_fields()
    assert bool(u.isfinite().all())
    sim.close()


def test_contact_list_overflow_is_reported():
    require_gpu()
    from paper_2002_08855_gb300.binding import Simulation

    w = _sim(2, n_particles=3, nx=64, ny=64)
    X = np.array([[30.0, 30.0], [41.0, 30.5], [35.5, 40.0]])  # pairwise within D + zeta = 12
    sim = Simulation(w, X, max_neighbors=1)
    sim.step(1)
    assert _code(sim) == "CAPACITY"
    sim.close()
    ok = Simulation(w, X, max_neighbors=2)
    ok.step(2)
    assert _code(ok) == "OK"
    ok.close()


@pytest.mark.parametrize("dim", [2, 3])
def test_centre_leaving_through_a_wall_is_reported(dim):
    require_gpu()
    from paper_2002_08855_gb300.binding import Simulation

    w = _sim(dim, mdf_iters=0, gravity=(0.0, 0.0, 0.0))
    X = np.array([[24.0, 8.0]]) if dim == 2 else np.array([[24.0, 8.0, 17.0]])
    U = np.zeros_like(X)
    U[0, 1] = -9.0  # through the wall at y = -1/2 within the step
    sim = Simulation(w, X)
    sim.set_particles(X, U=U)
    sim.step(1)
    assert _code(sim) == "OUT_OF_DOMAIN"
    assert sim.get_particles()["X"][0, 1] < -0.5
    # the run is put back inside and continues
    sim.set_particles(X, U=np.zeros_like(X))
    sim.step(2)
    assert _code(sim) == "OK"
    sim.close()
