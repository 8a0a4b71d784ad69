"""Long-run statistics of the CUDA path against the FP64 oracle: the 128 x 256 cavity
with 12 circles (d = 16, density ratio 1.5) at ten times its default gravity, 3000
steps, by which the circles settle at close to their terminal velocity.  The mean
settling velocity, the mean vertical hydrodynamic force and the mean height of the
circles over the last 1000 steps (samples every 100 steps) agree within 1 %."""
import numpy as np
import pytest

import oracle
from paper_2002_08855_gb300 import inputs

from gpu_util import require_gpu

pytestmark = pytest.mark.gpu


def _series(sim, steps, every=100):
    U, F, Y = [], [], []
    for _ in range(steps // every):
        sim.step(every)
        P = sim.get_particles()
        U.append(P["U"][:, 1].mean())
        F.append(P["F_h"][:, 1].mean())
        Y.append(P["X"][:, 1].mean())
    return np.array(U), np.array(F), np.array(Y)


def test_settling_statistics_over_3000_steps():
    require_gpu()
    from paper_2002_08855_gb300.binding import Simulation

    w = inputs.cavity_2d_small().with_(gravity=(0.0, -1e-4, 0.0))
    X0 = inputs.place_particles(w)
    sim = Simulation(w, X0)
    ref = oracle.Sim(w.as_dict(), X0)
    g = _series(sim, 3000)
    o = _series(ref, 3000)
    sim.close()
    ref.close()
    for name, a, b in zip(("settling velocity", "force", "height"), g, o):
        ma, mb = a[-10:].mean(), b[-10:].mean()
        print(f"{name}: GPU {ma:.6e}, oracle {mb:.6e}")
        assert abs(ma - mb) <= 0.01 * abs(mb), name
    # the circles are settling: velocity downward and close to steady over the window
    assert g[0][-1] < 0.0 and abs(g[0][-1] - g[0][-10]) < 0.1 * abs(g[0][-1])
