"""Reduced-precision PDF storage (FP16 / BF16 holding h_a = f_a / w_a, FP32 arithmetic).

- Streaming stays a permutation: values representable in the storage type come back
  unchanged after any number of pure streaming steps (tau = 1e30, no force).
- Error against the FP64 oracle on the 128 x 256 cavity with 12 settling circles after
  200 steps, stated per field: velocity, pressure and particle displacement.  The
  bounds are about twice the errors measured on a GB300; FP32 storage meets 1e-5
  on the same case (test_gpu_step).
"""
import numpy as np
import pytest

import oracle
from paper_2002_08855_gb300 import inputs
from paper_2002_08855_gb300.inputs import Workload

from gpu_util import rel_l2, require_gpu

pytestmark = pytest.mark.gpu

W2 = np.array([4 / 9] + [1 / 9, 1 / 36] * 4)


def _weights(q):
    if q == 9:
        return W2
    w = np.full(19, 1 / 36)
    w[0] = 1 / 3
    w[[1, 2, 3, 10, 11, 12]] = 1 / 18
    return w


@pytest.mark.parametrize("storage,dtype", [(1, np.float16), (2, "bf16")])
@pytest.mark.parametrize("dim,shape,per", [
    (2, (37, 29, 1), (0, 0, 0)), (3, (19, 13, 11), (1, 0, 1)),
    # 2D rows whose length is a multiple of 8: the vector kernel, with several warps per
    # row and a last warp holding one lane (the 3D shapes take the row kernel)
    (2, (264, 21, 1), (0, 0, 0)), (2, (512, 9, 1), (1, 1, 0)),
    (3, (388, 5, 6), (0, 1, 0)), (3, (128, 7, 6), (1, 0, 1))])
def test_streaming_permutes_stored_values(storage, dtype, dim, shape, per):
    torch = require_gpu()
    from paper_2002_08855_gb300.binding import Simulation

    w = Workload(name="st", dim=dim, nx=shape[0], ny=shape[1], nz=shape[2] if dim == 3 else 1,
                 periodic=per, tau=1e30, pdf_storage=storage)
    q = 9 if dim == 2 else 19
    rng = np.random.Generator(np.random.PCG64(5))
    h = rng.uniform(-1e-2, 1e-2, (q, w.n_grid))
    if dtype == "bf16":
        h = torch.from_numpy(h).to(torch.bfloat16).double().numpy()
    else:
        h = h.astype(np.float16).astype(np.float64)
    f0 = h * _weights(q)[:, None]
    sim = Simulation(w)
    sim.set_pdfs(f0.astype(np.float32))
    ref = oracle.Sim(w.as_dict())
    ref.set_pdfs(f0)
    for _ in range(4):
        sim.step(1)
        ref.step(1)
    got = sim.get_pdfs().cpu().numpy().astype(np.float64) / _weights(q)[:, None]
    want = ref.get_pdfs() / _weights(q)[:, None]
    # every stored value is a permuted input value (to FP32 rounding of w h)
    assert np.abs(got - want).max() <= 1e-6 * np.abs(want).max()
    sim.close()


# stated bounds (relative L2 against the FP64 oracle after 200 steps)
# measured on a GB300: FP16 velocity 3.0e-4, pressure 5.0e-4, displacement 2.0e-5;
# BF16 2.4e-3, 3.9e-3, 1.8e-4
BOUNDS = {1: {"u": 6e-4, "p": 1e-3, "x": 5e-5}, 2: {"u": 5e-3, "p": 8e-3, "x": 4e-4}}


@pytest.mark.parametrize("storage", [1, 2])
def test_cavity_error_against_oracle(storage):
    require_gpu()
    from paper_2002_08855_gb300.binding import Simulation

    w = inputs.cavity_2d_small().with_(pdf_storage=storage)
    X0 = inputs.place_particles(w)
    sim = Simulation(w, X0)
    ref = oracle.Sim(w.as_dict(), X0)
    sim.step(200)
    sim.sync()
    ref.step(200)
    pg_, ug = sim.get_fields()
    po_, uo = ref.get_fields()
    e_u = rel_l2(ug.cpu().numpy(), uo)
    e_p = rel_l2(pg_.cpu().numpy(), po_)
    pg, po = sim.get_particles(), ref.get_particles()
    e_x = rel_l2(pg["X"] - X0, po["X"] - X0)
    print(f"storage {storage}: velocity {e_u:.3e}, pressure {e_p:.3e}, displacement {e_x:.3e}")
    b = BOUNDS[storage]
    assert e_u < b["u"] and e_p < b["p"] and e_x < b["x"]
    sim.close()


# 3D (the 384 x 384 x 768 cavity scaled to 48 x 48 x 96 with 30 spheres of d = 12,
# solid fraction 0.12: random placement with the contact gap stalls before the full
# cavity's 0.16 in this small box), relative L2 against the FP64 oracle after 60 steps
# measured on a GB300: FP32 velocity 1.2e-6, pressure 4.8e-6, displacement 5.0e-7, F_h
# 3.1e-6; FP16 1.9e-4, 2.3e-4, 5.9e-6, 2.6e-4; BF16 1.3e-3, 1.5e-3, 5.4e-5, 2.2e-3
BOUNDS3 = {0: {"u": 1e-5, "p": 1e-5, "x": 1e-5, "f": 1e-5},
           1: {"u": 4e-4, "p": 5e-4, "x": 2e-5, "f": 6e-4},
           2: {"u": 3e-3, "p": 4e-3, "x": 2e-4, "f": 5e-3}}


@pytest.mark.parametrize("storage", [0, 1, 2])
def test_cavity_3d_error_per_field(storage):
    """Velocity, pressure, particle displacement and hydrodynamic force of the 3D
    cavity per PDF storage against the FP64 oracle."""
    require_gpu()
    from paper_2002_08855_gb300.binding import Simulation

    w = inputs.cavity_3d(8).with_(n_particles=30, pdf_storage=storage)
    X0 = inputs.place_particles(w)
    sim = Simulation(w, X0)
    ref = oracle.Sim(w.as_dict(), X0)
    sim.step(60)
    sim.sync()
    ref.step(60)
    pg_, ug = sim.get_fields()
    po_, uo = ref.get_fields()
    e_u = rel_l2(ug.cpu().numpy(), uo)
    e_p = rel_l2(pg_.cpu().numpy(), po_)
    pg, po = sim.get_particles(), ref.get_particles()
    e_x = rel_l2(pg["X"] - X0, po["X"] - X0)
    e_f = rel_l2(pg["F_h"], po["F_h"])
    print(f"3D storage {storage}: velocity {e_u:.3e}, pressure {e_p:.3e}, displacement {e_x:.3e}, "
          f"F_h {e_f:.3e}")
    b = BOUNDS3[storage]
    assert e_u < b["u"] and e_p < b["p"] and e_x < b["x"] and e_f < b["f"]
    sim.close()
