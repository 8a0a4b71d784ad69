"""Checkpoint and resume: a run restored from a state continues as the run that saved
it (2D and 3D, FP32 and FP16 storage, extrapolation walls, the learned initializer),
whatever state the restoring handle was in; states of another configuration and
buffers that are not states are rejected."""
import numpy as np
import pytest

from paper_2002_08855_gb300 import inputs
from paper_2002_08855_gb300.inputs import Workload

from gpu_util import rel_l2, require_gpu

pytestmark = pytest.mark.gpu


def _cases():
    base2 = inputs.cavity_2d_small()
    return [
        ("2d", base2),
        ("2d_fp16", base2.with_(pdf_storage=1)),
        ("2d_walls", base2.with_(boundary=1, delta_kind=3, drs=1.9, density_ratio=1.01, gravity=(0.0, -1e-3, 0.0))),
        ("3d", Workload(name="c3", dim=3, nx=32, ny=32, nz=48, tau=0.6, n_particles=4, n_lag=452,
                        diameter=12.0, density_ratio=1.5, gravity=(0, 0, -1e-5), seed=77)),
    ]


@pytest.mark.parametrize("name,w", _cases(), ids=[c[0] for c in _cases()])
def test_resume_continues_the_saved_run(name, w):
    """Steps 1..40, save, 25 more (A); a second handle that ran other steps from other
    centres restores the state and runs the 25 (B): A and B agree to the rounding of
    the spreading's atomic order, and with the saved run's step parity."""
    require_gpu()
    from paper_2002_08855_gb300.binding import Simulation

    X0 = inputs.place_particles(w)
    a = Simulation(w, X0)
    a.step(41)  # odd: the state is saved in the layout of an odd step counter
    state = a.get_state()
    a.step(25)
    pa, ua = a.get_particles(), a.get_fields()[1].cpu().numpy()
    b = Simulation(w, inputs.place_particles(w.with_(seed=w.seed + 9)))
    b.step(6)
    b.set_state(state)
    b.step(25)
    pb, ub = b.get_particles(), b.get_fields()[1].cpu().numpy()
    tol = 1e-6 if w.pdf_storage == 0 else 1e-3
    assert rel_l2(ub, ua) < tol
    assert rel_l2(pb["X"] - X0, pa["X"] - X0) < tol
    assert rel_l2(pb["U"], pa["U"]) < tol * 10
    a.close()
    b.close()


def test_resume_keeps_the_learned_initializer():
    require_gpu()
    from paper_2002_08855_gb300 import mlp
    from paper_2002_08855_gb300.binding import Simulation

    w = inputs.cavity_2d_small().with_(mlp_init=1, mdf_iters=2)
    X0 = inputs.place_particles(w)
    p = mlp.init_params(11)
    p[-2], p[-1] = 1e3, 1e-4
    a = Simulation(w, X0)
    a.set_mlp(p)
    a.step(10)
    state = a.get_state()
    a.step(10)
    b = Simulation(w, X0)  # no set_mlp: the parameters come with the state
    b.set_state(state)
    b.step(10)
    assert rel_l2(b.get_fields()[1].cpu().numpy(), a.get_fields()[1].cpu().numpy()) < 1e-6
    a.close()
    b.close()


def test_foreign_states_are_rejected():
    require_gpu()
    from paper_2002_08855_gb300.binding import IbmLbmError, Simulation

    w = inputs.cavity_2d_small()
    a = Simulation(w, inputs.place_particles(w))
    a.step(2)
    state = a.get_state()
    w2 = w.with_(nx=w.nx + 2)
    b = Simulation(w2, inputs.place_particles(w2))
    with pytest.raises(IbmLbmError):
        b.set_state(state)
    bad = state.copy()
    bad[:8] = 0
    with pytest.raises(IbmLbmError):
        a.set_state(bad)
    a.close()
    b.close()
