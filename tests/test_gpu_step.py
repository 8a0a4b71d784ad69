"""Whole-step parity: the 128 x 256 D2Q9 cavity with 12 settling circles (d = 16,
50 points, 4-point delta, drs = 2.6, M = 3, density ratio 1.5, gravity 1e-5)
after 200 steps, FP32 GPU against the FP64 oracle: 1e-5 relative L2 on the
velocity field and on the particle displacement."""
import numpy as np
import pytest

import oracle
from paper_2002_08855_gb300 import inputs

from gpu_util import rel_l2, require_gpu

pytestmark = pytest.mark.gpu


def test_cavity_128x256_200_steps():
    require_gpu()
    from paper_2002_08855_gb300.binding import Simulation

    w = inputs.cavity_2d_small()
    X0 = inputs.place_particles(w)
    sim = Simulation(w, X0)
    ref = oracle.Sim(w.as_dict(), X0)
    sim.step(199)
    X199 = sim.get_particles()["X"]
    sim.step(1)  # its contact list is built from the centres of step 199
    sim.sync()
    ref.step(200)
    _, ug = sim.get_fields()
    _, uo = ref.get_fields()
    e_u = rel_l2(ug.cpu().numpy(), uo)
    pg, po = sim.get_particles(), ref.get_particles()
    e_x = rel_l2(pg["X"] - X0, po["X"] - X0)
    e_X = rel_l2(pg["X"], po["X"])
    print(f"velocity rel L2 {e_u:.3e}, displacement {e_x:.3e}, position {e_X:.3e}")
    assert e_u < 1e-5
    assert e_X < 1e-5
    assert e_x < 1e-5
    assert np.array_equal(sim.get_pairs(), oracle.pairs_bruteforce(w.as_dict(), X199))
    sim.close()


def test_cavity_3d_small():
    require_gpu()
    from paper_2002_08855_gb300.binding import Simulation

    w = inputs.Workload(name="c3", dim=3, nx=32, ny=32, nz=48, tau=0.6, n_particles=4,
                        n_lag=452, diameter=12.0, density_ratio=1.5, gravity=(0, 0, -1e-5),
                        seed=77)
    X0 = inputs.place_particles(w)
    sim = Simulation(w, X0)
    ref = oracle.Sim(w.as_dict(), X0)
    sim.step(40)
    ref.step(40)
    _, ug = sim.get_fields()
    _, uo = ref.get_fields()
    assert rel_l2(ug.cpu().numpy(), uo) < 1e-5
    pg, po = sim.get_particles(), ref.get_particles()
    assert rel_l2(pg["X"] - X0, po["X"] - X0) < 1e-5
    sim.close()


def test_cavity_128x256_3_point_delta():
    """The same cavity with the 3-point delta function and drs = 1.9 (the paper's
    experiments, Sec. 2.2 and 6.2), 100 steps."""
    require_gpu()
    from paper_2002_08855_gb300.binding import Simulation

    w = inputs.cavity_2d_small().with_(delta_kind=3, drs=1.9)
    X0 = inputs.place_particles(w)
    sim = Simulation(w, X0)
    ref = oracle.Sim(w.as_dict(), X0)
    sim.step(100)
    ref.step(100)
    _, ug = sim.get_fields()
    _, uo = ref.get_fields()
    assert rel_l2(ug.cpu().numpy(), uo) < 1e-5
    pg, po = sim.get_particles(), ref.get_particles()
    assert rel_l2(pg["X"] - X0, po["X"] - X0) < 1e-5
    sim.close()


def test_periodic_box_particles_crossing_the_edges():
    """A 64 x 72 box periodic on both axes, three circles (d = 10, 31 points) whose
    node boxes wrap around the edges and that move across them within 120 steps: the
    IB force the spreading of one step leaves on the grid, wrapped nodes included, must
    be gone before the step after next spreads into the same buffer."""
    require_gpu()
    from paper_2002_08855_gb300.binding import Simulation

    w = inputs.Workload(name="per", dim=2, nx=64, ny=72, periodic=(1, 1, 0), tau=0.7,
                        n_particles=3, n_lag=31, diameter=10.0, density_ratio=1.5,
                        gravity=(0.0, -1e-5, 0.0), mdf_iters=3)
    X0 = np.array([[62.9, 20.4], [30.2, 0.6], [0.8, 71.0]])
    U0 = np.array([[0.04, 0.01], [-0.01, -0.05], [-0.03, 0.035]])
    Om0 = np.array([[1e-3], [-2e-3], [5e-4]])
    sim = Simulation(w, X0)
    sim.set_particles(X0, U=U0, Omega=Om0)
    ref = oracle.Sim(w.as_dict(), X0)
    ref.set_particles(X0, U=U0, Omega=Om0)
    sim.step(120)
    ref.step(120)
    _, ug = sim.get_fields()
    _, uo = ref.get_fields()
    pg, po = sim.get_particles(), ref.get_particles()
    # each circle crossed an edge (its centre wrapped)
    assert pg["X"][0, 0] < 10.0 and pg["X"][2, 1] < 10.0 and pg["X"][1, 1] > 60.0
    assert rel_l2(ug.cpu().numpy(), uo) < 1e-5
    assert rel_l2(pg["X"], po["X"]) < 1e-6
    assert rel_l2(pg["U"], po["U"]) < 1e-5
    sim.close()
