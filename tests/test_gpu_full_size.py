"""Whole-step parity at the benchmark sizes.

1. The 2048 x 4096 D2Q9 cavity with 10681 circles (d = 10, 31 points, solid fraction
   0.1): the launch configuration the benchmark times (every IBM kernel in many block
   waves, the full lbm_step grid).  The particles start with seeded velocities and
   spins in fluid at rest, so the IBM drives all of the flow from the first step; four
   whole steps against the FP64 oracle, element by element.

2. The 384 x 384 x 768 D3Q19 cavity: 19 x 113,246,208 PDFs, more than 2^31 elements,
   so the last direction's slots of the top planes (z >= 740) lie beyond element index
   2^31.  Only the top planes carry data: PDFs and spheres there, zero PDFs below.  In
   this model the zero state is a fixed point of the collision (every f_eq and force
   term vanishes at p = 0, u = 0, F = 0), and a population moves one plane per step,
   so for k steps the planes more than k below the data stay exactly zero and the
   cavity's floor is never reached.  The oracle therefore runs only a sub-box of the
   same x-y size holding the top planes (its own floor is never reached either), and
   the GPU's full lattice must match it there and stay zero below.
"""
import numpy as np
import pytest

import oracle
from paper_2002_08855_gb300 import inputs
from paper_2002_08855_gb300.inputs import random_pdfs

from gpu_util import rel_l2, require_gpu

pytestmark = pytest.mark.gpu


def _seeded_motion(n, dim, seed, u=2e-3, om=1e-4):
    rng = np.random.Generator(np.random.PCG64(seed))
    U = rng.uniform(-u, u, (n, dim))
    Om = rng.uniform(-om, om, (n, 1 if dim == 2 else 3))
    return U, Om


def test_headline_cavity_2048x4096_four_steps():
    require_gpu()
    from paper_2002_08855_gb300.binding import Simulation

    w = inputs.cavity_2d_large(0.1)
    X0 = inputs.place_particles(w)
    assert len(X0) == 10681
    U0, Om0 = _seeded_motion(len(X0), 2, seed=2048)
    sim = Simulation(w, X0)
    sim.set_particles(X0, U=U0, Omega=Om0)
    ref = oracle.Sim(w.as_dict(), X0)
    ref.set_particles(X0, U=U0, Omega=Om0)
    sim.step(3)
    ref.step(3)
    X3 = ref.get_particles()["X"]
    sim.step(1)  # its contact list is built from the centres after step 3
    ref.step(1)
    sim.sync()
    _, ug = sim.get_fields()
    _, uo = ref.get_fields()
    e_u = rel_l2(ug.cpu().numpy(), uo)
    pg, po = sim.get_particles(), ref.get_particles()
    lg, lo = sim.get_lagrangian(), ref.get_lagrangian()
    e = dict(u=e_u, dX=rel_l2(pg["X"] - X0, po["X"] - X0), U=rel_l2(pg["U"], po["U"]),
             Om=rel_l2(pg["Omega"], po["Omega"]), F_h=rel_l2(pg["F_h"], po["F_h"]),
             T_h=rel_l2(pg["T_h"], po["T_h"]), F_b=rel_l2(lg["F_b"], lo["F_b"]))
    print("relative L2 against the oracle:", {k: f"{v:.2e}" for k, v in e.items()})
    assert e["u"] < 1e-5 and e["dX"] < 1e-5 and e["U"] < 1e-5
    assert e["F_h"] < 1e-5 and e["F_b"] < 1e-5
    assert e["Om"] < 1e-4 and e["T_h"] < 1e-4
    assert np.array_equal(sim.get_pairs(), oracle.pairs_bruteforce(w.as_dict(), X3))
    sim.close()


def test_headline_cavity_2048x4096_fp16_storage_four_steps():
    """The same four steps with FP16 storage (h = f / w, the chosen form's storage; the
    vector lbm_step kernel): velocity and displacement within the storage's stated
    error, the Lagrangian forces within the same bound."""
    require_gpu()
    from paper_2002_08855_gb300.binding import Simulation

    w = inputs.cavity_2d_large(0.1)
    X0 = inputs.place_particles(w)
    U0, Om0 = _seeded_motion(len(X0), 2, seed=2048)
    sim = Simulation(w.with_(pdf_storage=1), X0)
    sim.set_particles(X0, U=U0, Omega=Om0)
    ref = oracle.Sim(w.as_dict(), X0)
    ref.set_particles(X0, U=U0, Omega=Om0)
    sim.step(4)
    ref.step(4)
    _, ug = sim.get_fields()
    _, uo = ref.get_fields()
    pg, po = sim.get_particles(), ref.get_particles()
    lg, lo = sim.get_lagrangian(), ref.get_lagrangian()
    e = dict(u=rel_l2(ug.cpu().numpy(), uo), dX=rel_l2(pg["X"] - X0, po["X"] - X0),
             F_b=rel_l2(lg["F_b"], lo["F_b"]), F_h=rel_l2(pg["F_h"], po["F_h"]))
    print("FP16 storage, relative L2 against the oracle:", {k: f"{v:.2e}" for k, v in e.items()})
    assert e["u"] < 2e-3 and e["dX"] < 2e-3 and e["F_b"] < 2e-3 and e["F_h"] < 2e-3
    sim.close()


NX, NY, NZ = 384, 384, 768
PLANE = NX * NY


def _top_planes_pdfs(torch, z_seed, seed, scale):
    """Full-lattice [19][N] FP32 device PDFs: seeded values on planes z >= z_seed, zero
    below; also the seeded block itself (host, planes z_seed..NZ-1)."""
    top = random_pdfs(19, (NZ - z_seed) * PLANE, seed=seed, scale=scale)
    f = torch.zeros((19, NX * NY * NZ), dtype=torch.float32, device="cuda")
    f[:, z_seed * PLANE:] = torch.from_numpy(top).to("cuda")
    return f, top


def _sub_box(z0, z_seed, top):
    """The oracle's view of planes z0..NZ-1: zeros below z_seed, then the seeded block."""
    f = np.zeros((19, (NZ - z0) * PLANE))
    f[:, (z_seed - z0) * PLANE:] = top
    return f


def test_cavity_3d_full_lattice_beyond_2_31_elements_streaming_bit_exact():
    """tau = 1e30 makes the collision the identity on every PDF much larger than 1e-30
    times its node's others: three steps (both parities of the in-place streaming) move
    the seeded top planes exactly as the oracle's push streaming does, walls included.
    The one exception is a zero-valued direction at a node that has just received data
    (the planes below the seeded block): the collision leaves (f_eq - 0) / tau, about
    1e-32 there, which FP32 and FP64 round differently, so those residues are held to
    an absolute 1e-28 instead."""
    torch = require_gpu()
    from paper_2002_08855_gb300.binding import Simulation

    q, z0, z_seed = 19, 736, 744
    assert (q - 1) * NX * NY * NZ + z_seed * PLANE > 2 ** 31  # direction 18, top planes
    w = inputs.Workload(name="c3full", dim=3, nx=NX, ny=NY, nz=NZ, tau=1e30)
    sim = Simulation(w)
    f, top = _top_planes_pdfs(torch, z_seed, seed=7681, scale=1e-2)
    sim.set_pdfs(f)
    del f
    ref = oracle.Sim(w.with_(nz=NZ - z0).as_dict())
    ref.set_pdfs(_sub_box(z0, z_seed, top))
    for k in range(3):
        sim.step(1)
        ref.step(1)
        g = sim.get_pdfs()
        assert int(torch.count_nonzero(g[:, : z0 * PLANE])) == 0
        gt = g[:, z0 * PLANE:].cpu().numpy().astype(np.float64)
        del g
        fo = ref.get_pdfs()
        big = np.abs(fo) > 1e-20
        assert big.sum() >= 19 * (NZ - z_seed - k - 1) * PLANE
        assert np.array_equal(gt[big], fo[big]), f"step {k + 1}"
        assert np.abs(gt[~big] - fo[~big]).max() < 1e-28, f"step {k + 1}"
    sim.close()


def test_cavity_3d_full_lattice_beyond_2_31_elements_spheres():
    """The 384 x 384 x 768 cavity's own sphere positions (20000 spheres, d = 12, 452
    points), keeping those in the top planes (975 of them), with seeded PDFs there and
    seeded sphere velocities and spins: four whole steps (MDF, collision, streaming,
    contacts, Newton-Euler update) against the oracle's sub-box."""
    torch = require_gpu()
    from paper_2002_08855_gb300.binding import Simulation

    k, z0, z_seed = 4, 712, 720
    w3 = inputs.cavity_3d()
    R = 0.5 * w3.diameter
    Xall = inputs.place_particles(w3)
    X = Xall[Xall[:, 2] >= z0 + R + 2 + k + 2]  # supports stay k + 2 planes above z0
    assert len(X) > 900
    U0, Om0 = _seeded_motion(len(X), 3, seed=3841, u=1e-3)
    w = w3.with_(n_particles=len(X))
    sim = Simulation(w, X)
    sim.set_particles(X, U=U0, Omega=Om0)
    f, top = _top_planes_pdfs(torch, z_seed, seed=7682, scale=1e-3)
    sim.set_pdfs(f)
    del f
    shift = np.array([0.0, 0.0, float(z0)])
    ref = oracle.Sim(w.with_(nz=NZ - z0).as_dict(), X - shift)
    ref.set_particles(X - shift, U=U0, Omega=Om0)
    ref.set_pdfs(_sub_box(z0, z_seed, top))
    sim.step(k)
    ref.step(k)
    sim.sync()
    g = sim.get_pdfs()
    assert int(torch.count_nonzero(g[:, : z0 * PLANE])) == 0
    del g
    _, ug = sim.get_fields()
    assert int(torch.count_nonzero(ug[:, : z0 * PLANE])) == 0
    ut = ug[:, z0 * PLANE:].cpu().numpy()
    del ug
    _, uo = ref.get_fields()
    pg, po = sim.get_particles(), ref.get_particles()
    e = dict(u=rel_l2(ut, uo), dX=rel_l2(pg["X"] - X, po["X"] + shift - X),
             U=rel_l2(pg["U"], po["U"]), Om=rel_l2(pg["Omega"], po["Omega"]),
             F_h=rel_l2(pg["F_h"], po["F_h"]), T_h=rel_l2(pg["T_h"], po["T_h"]))
    print("relative L2 against the oracle:", {kk: f"{v:.2e}" for kk, v in e.items()})
    assert e["u"] < 1e-5 and e["dX"] < 1e-5 and e["U"] < 1e-5 and e["F_h"] < 1e-5
    assert e["Om"] < 1e-4 and e["T_h"] < 1e-4
    sim.close()
