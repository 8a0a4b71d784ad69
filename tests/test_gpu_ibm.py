"""GPU parity of the immersed-boundary kernels (interpolation, spreading, MDF, interior
momentum) and the particle update against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2002_08855_gb300 import inputs
from paper_2002_08855_gb300.inputs import Workload, random_pdfs

from gpu_util import rel_l2, require_gpu

pytestmark = pytest.mark.gpu


def _pair(w, X, U, Om=None, f0=None):
    from paper_2002_08855_gb300.binding import Simulation

    sim = Simulation(w, X)
    sim.set_particles(X, U=U, Omega=Om)
    ref = oracle.Sim(w.as_dict(), X)
    ref.set_particles(X, U=U, Omega=Om)
    if f0 is not None:
        sim.set_pdfs(f0)
        ref.set_pdfs(f0.astype(np.float64))
    return sim, ref


CASES = [
    # dim, shape, periodic, centres, diameter, n_lag
    (2, (64, 56, 1), (0, 0, 0), [[20.3, 25.7], [41.9, 30.2]], 12.0, 40),
    (2, (48, 40, 1), (0, 0, 0), [[6.6, 20.1]], 10.0, 31),          # support beyond a wall
    (2, (50, 44, 1), (1, 1, 0), [[1.2, 42.9], [25.0, 20.0]], 10.0, 31),  # wraps both axes
    (3, (30, 28, 26), (0, 0, 0), [[14.2, 13.6, 12.9]], 12.0, 452),
    (3, (24, 26, 28), (1, 0, 1), [[1.5, 12.2, 26.8]], 8.0, 200),
    # near contact: the supports of neighbouring particles share nodes
    (2, (64, 48, 1), (0, 0, 0), [[20.2, 23.9], [31.1, 25.3]], 10.0, 31),
    (3, (40, 36, 34), (0, 0, 0), [[12.5, 17.2, 16.9], [25.3, 17.9, 17.4], [18.9, 28.1, 16.2]], 12.0, 452),
    # large particles: 3D spheres whose box does not fit in shared memory (the IBM runs
    # from global memory), a 2D pair whose boxes take fewer warps per block
    (3, (48, 44, 46), (0, 0, 0), [[23.2, 21.7, 22.9]], 20.0, 1257),
    (3, (40, 40, 40), (1, 1, 1), [[2.5, 38.1, 20.3]], 18.0, 1018),
    (2, (120, 110, 1), (0, 0, 0), [[50.3, 55.6], [93.0, 54.2]], 40.0, 126),
]


# the 3-point delta function (drs = 1.9, Sec. 2.2) on a subset of the cases
CASES3 = [CASES[1], CASES[2], CASES[3], CASES[4], CASES[5], CASES[6], CASES[7], CASES[9]]


@pytest.mark.parametrize("dim,shape,per,xc,D,nl", CASES)
def test_one_step_lagrangian_forces(dim, shape, per, xc, D, nl):
    _one_step(dim, shape, per, xc, D, nl, 4, 2.6)


@pytest.mark.parametrize("dim,shape,per,xc,D,nl", CASES3)
def test_one_step_lagrangian_forces_3_point_delta(dim, shape, per, xc, D, nl):
    _one_step(dim, shape, per, xc, D, nl, 3, 1.9)


def _one_step(dim, shape, per, xc, D, nl, kind, drs):
    require_gpu()
    xc = np.array(xc)
    w = Workload(name="ibm", dim=dim, nx=shape[0], ny=shape[1], nz=shape[2] if dim == 3 else 1,
                 periodic=per, tau=0.7, n_particles=len(xc), n_lag=nl, diameter=D, mdf_iters=3,
                 fixed_particles=1, delta_kind=kind, drs=drs)
    rng = np.random.Generator(np.random.PCG64(3))
    U = rng.uniform(-2e-3, 2e-3, xc.shape)
    Om = rng.uniform(-1e-4, 1e-4, (len(xc), 1 if dim == 2 else 3))
    f0 = random_pdfs(9 if dim == 2 else 19, w.n_grid, seed=31, scale=1e-3)
    sim, ref = _pair(w, xc, U, Om, f0)
    sim.step(1)
    ref.step(1)
    lg, lo = sim.get_lagrangian(), ref.get_lagrangian()
    assert np.abs(lg["X_b"] - lo["X_b"]).max() < 1e-9  # 32.32 fixed point on the GPU
    assert rel_l2(lg["U_b"], lo["U_b"]) < 1e-6
    assert rel_l2(lg["u_b_star"], lo["u_b_star"]) < 1e-5
    assert rel_l2(lg["F_b"], lo["F_b"]) < 1e-5
    pg, po = sim.get_particles(), ref.get_particles()
    assert rel_l2(pg["F_h"], po["F_h"]) < 1e-5
    assert rel_l2(pg["T_h"], po["T_h"]) < 1e-4
    Pg, Lg = sim.get_interior_momentum()
    Po, Lo = ref.get_interior_momentum()
    assert rel_l2(Pg, Po) < 1e-5
    assert rel_l2(sim.get_pdfs().cpu().numpy(), ref.get_pdfs()) < 1e-5
    sim.close()


def test_moving_particles_several_steps():
    require_gpu()
    w = Workload(name="mv", dim=2, nx=80, ny=96, tau=0.65, n_particles=3, n_lag=40,
                 diameter=12.0, density_ratio=1.5, gravity=(0.0, -1e-5, 0.0))
    xc = np.array([[20.5, 60.2], [45.1, 48.9], [62.3, 70.4]])
    U = np.array([[1e-3, -2e-3], [-5e-4, 1e-3], [0.0, -1e-3]])
    sim, ref = _pair(w, xc, U)
    for n in (1, 9, 20):
        sim.step(n)
        ref.step(n)
    pg, po = sim.get_particles(), ref.get_particles()
    assert rel_l2(pg["X"] - xc, po["X"] - xc) < 1e-5
    assert rel_l2(pg["U"], po["U"]) < 1e-5
    _, ug = sim.get_fields()
    _, uo = ref.get_fields()
    assert rel_l2(ug.cpu().numpy(), uo) < 1e-5
    sim.sync()
    sim.close()


def test_mdf_iterations_are_jacobi_across_many_spheres():
    """900 spheres (d = 8, 201 points) in a 112^3 box, 99 % of them within reach of a
    neighbour's support: more blocks than the GPU holds at once, so spheres are
    processed in waves.  Every sphere's interpolation of MDF iteration m must see the
    spreading of iterations 1 .. m-1 of all spheres and none of iteration m, as in the
    oracle; one step of Lagrangian forces, hydrodynamic forces and PDFs."""
    require_gpu()
    X = inputs.place_rsa(3, (112, 112, 112), 900, 8.0, seed=41, gap=0.5, wall_gap=1.0)
    w = Workload(name="many", dim=3, nx=112, ny=112, nz=112, tau=0.7, n_particles=len(X),
                 n_lag=201, diameter=8.0, mdf_iters=3, fixed_particles=1)
    rng = np.random.Generator(np.random.PCG64(5))
    U = rng.uniform(-2e-3, 2e-3, X.shape)
    f0 = random_pdfs(19, w.n_grid, seed=33, scale=1e-3)
    sim, ref = _pair(w, X, U, None, f0)
    sim.step(1)
    ref.step(1)
    lg, lo = sim.get_lagrangian(), ref.get_lagrangian()
    assert rel_l2(lg["F_b"], lo["F_b"]) < 1e-5
    assert rel_l2(lg["u_b_star"], lo["u_b_star"]) < 1e-5
    pg, po = sim.get_particles(), ref.get_particles()
    assert rel_l2(pg["F_h"], po["F_h"]) < 1e-5
    assert rel_l2(sim.get_pdfs().cpu().numpy(), ref.get_pdfs()) < 1e-5
    sim.close()


def test_large_spheres_several_steps():
    """Four spheres of d = 18 (box beyond shared memory: the global-memory IBM) moving
    near contact for 30 steps, against the oracle."""
    require_gpu()
    w = Workload(name="big3", dim=3, nx=64, ny=60, nz=62, tau=0.7, n_particles=4, n_lag=1018,
                 diameter=18.0, density_ratio=1.5, gravity=(0.0, -1e-5, 0.0))
    xc = np.array([[18.5, 20.2, 30.1], [38.9, 21.0, 30.6], [28.4, 39.8, 29.5], [29.0, 30.1, 49.0]])
    U = np.array([[1e-3, 0.0, 0.0], [-1e-3, 5e-4, 0.0], [0.0, -1e-3, 2e-4], [0.0, 0.0, -1e-3]])
    sim, ref = _pair(w, xc, U)
    sim.step(30)
    ref.step(30)
    pg, po = sim.get_particles(), ref.get_particles()
    assert rel_l2(pg["X"] - xc, po["X"] - xc) < 1e-5
    _, ug = sim.get_fields()
    _, uo = ref.get_fields()
    assert rel_l2(ug.cpu().numpy(), uo) < 1e-5
    sim.close()


@pytest.mark.parametrize("dim", [2, 3])
def test_spin_in_a_shear_wave(dim):
    """Centres held, spins integrated (fixed_particles = 2): bodies at the zero of a
    shear wave u_x = U0 sin(k y) and one off it, so the torque, the rotational closure
    (interior angular momentum, K_r) and Omega x r in the boundary velocity carry the
    whole coupling; spin and field against the oracle."""
    require_gpu()
    if dim == 2:
        L, D, steps = 96, 8.0, 150
        w = Workload(name="spin", dim=2, nx=L, ny=L, periodic=(1, 1, 0), tau=1.0, n_particles=2,
                     n_lag=25, diameter=D, density_ratio=1.0, fixed_particles=2)
        xc = np.array([[30.3, 48.0], [70.6, 20.2]])
    else:
        L, D, steps = 36, 6.0, 60
        w = Workload(name="spin3", dim=3, nx=L, ny=L, nz=L, periodic=(1, 1, 1), tau=1.0,
                     n_particles=2, n_lag=113, diameter=D, density_ratio=1.0, fixed_particles=2)
        xc = np.array([[9.3, 18.0, 17.8], [26.4, 8.1, 20.5]])
    N = w.n_grid
    y = (np.arange(N) // L) % L
    u = np.zeros((dim, N))
    u[0] = 1e-3 * np.sin(2 * np.pi * y / L)
    sim, ref = _pair(w, xc, None)
    sim.set_fields(np.zeros(N), u)
    ref.set_fields(np.zeros(N), u)
    # during spin-up the torque is large; near the torque-free state it is a nearly
    # complete cancellation of the points' contributions, so it is compared early
    sim.step(5)
    ref.step(5)
    assert rel_l2(sim.get_particles()["T_h"], ref.get_particles()["T_h"]) < 1e-4
    sim.step(steps - 5)
    ref.step(steps - 5)
    pg, po = sim.get_particles(), ref.get_particles()
    assert np.abs(po["Omega"]).max() > 1e-5
    assert np.array_equal(pg["X"], xc) and np.abs(pg["U"]).max() == 0.0
    assert rel_l2(pg["Omega"], po["Omega"]) < 1e-5
    _, ug = sim.get_fields()
    _, uo = ref.get_fields()
    assert rel_l2(ug.cpu().numpy(), uo) < 1e-5
    sim.close()
