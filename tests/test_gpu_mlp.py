"""Learned MDF initializer on the GPU: training kernels against the FP64 reference,
tensor-core inference, the sample features, and what the trained network gains over
the plain multi-direct forcing (boundary-velocity residual after the same number of
iterations)."""
import ctypes as C

import numpy as np
import pytest

from oracle import mlp_ref
from paper_2002_08855_gb300.inputs import Workload, place_particles

from gpu_util import rel_l2, require_gpu

pytestmark = pytest.mark.gpu


def _random(seed, B):
    rng = np.random.Generator(np.random.PCG64(seed))
    p = rng.normal(0.0, 0.2, mlp_ref.N_PARAMS).astype(np.float32)
    p[-2:] = (1.0, 1.0)
    X = rng.normal(0.0, 1.0, (B, mlp_ref.N_IN)).astype(np.float32)
    T = rng.normal(0.0, 1.0, (B, mlp_ref.N_OUT)).astype(np.float32)
    return p, X, T


def test_gradient_matches_reference():
    torch = require_gpu()
    from paper_2002_08855_gb300.binding import _check, lib

    B = 512
    p, X, T = _random(5, B)
    dev = torch.device("cuda")
    P, Xd, Td = (torch.from_numpy(a).to(dev) for a in (p, X, T))
    G = torch.zeros_like(P)
    sz = C.c_size_t(0)
    _check(lib().ibm_lbm_mlp_scratch_size(B, C.byref(sz)), "scratch")
    scratch = torch.empty(sz.value, dtype=torch.uint8, device=dev)
    loss = C.c_double(0)
    s = torch.cuda.current_stream()
    _check(lib().ibm_lbm_mlp_grad(C.c_void_p(P.data_ptr()), C.c_void_p(Xd.data_ptr()), C.c_void_p(Td.data_ptr()),
                                  B, C.c_void_p(G.data_ptr()), C.byref(loss), C.c_void_p(scratch.data_ptr()),
                                  sz.value, C.c_void_p(s.cuda_stream)), "grad")
    lr, gr = mlp_ref.loss_and_grad(p.astype(np.float64), X.astype(np.float64), T.astype(np.float64))
    assert abs(loss.value - lr) < 1e-5 * lr
    assert rel_l2(G.cpu().numpy(), gr) < 1e-5


def test_tensor_core_inference_matches_reference():
    torch = require_gpu()
    from paper_2002_08855_gb300 import mlp

    p, X, _ = _random(6, 1000)  # 1000 rows: 62 full warps of 16 and a ragged tail
    p[-2:] = (0.5, 3.0)
    Y = mlp.infer(p, torch.from_numpy(X).cuda()).cpu().numpy()
    Yr = mlp_ref.predict(p.astype(np.float64), X.astype(np.float64))
    assert rel_l2(Y, Yr) < 1e-2  # FP16 operands, FP32 accumulation


def _workload(seed, n=24, nx=160, ny=192, **kw):
    return Workload(name="mlp", dim=2, nx=nx, ny=ny, tau=0.6, n_particles=n, n_lag=31, diameter=10.0,
                    mdf_iters=3, density_ratio=1.5, gravity=(0.0, -1e-4, 0.0), seed=seed, **kw)


def test_samples_are_the_stencils_of_the_last_step():
    require_gpu()
    from paper_2002_08855_gb300.binding import Simulation

    w = _workload(31)
    sim = Simulation(w, place_particles(w))
    sim.step(6)
    X, Y = sim.mdf_samples()
    lg = sim.get_lagrangian()
    Xr = mlp_ref.features_2d(lg["U_b"], lg["u_b_star"], w.n_lag)
    assert rel_l2(X.cpu().numpy(), Xr) < 1e-5
    k = np.arange(len(Xr)) % w.n_lag
    th = 2 * np.pi * k / w.n_lag
    F = lg["F_b"].astype(np.float64)
    Yr = np.stack([F[:, 0] * np.cos(th) + F[:, 1] * np.sin(th), -F[:, 0] * np.sin(th) + F[:, 1] * np.cos(th)], 1)
    assert rel_l2(Y.cpu().numpy()[:, :2], Yr) < 1e-5
    sim.close()


def test_initializer_lowers_the_mdf_residual():
    require_gpu()
    from paper_2002_08855_gb300 import mlp
    from paper_2002_08855_gb300.binding import Simulation

    train = [_workload(40 + s, n=60, nx=256, ny=256) for s in range(3)]
    X, Y = mlp.collect_samples(train, [place_particles(w) for w in train], steps=40, every=2)
    params, losses = mlp.train(X, Y, epochs=25, batch=4096, lr=2e-3, seed=3)
    assert losses[-1] < 0.5 * losses[0]
    w = _workload(77, n=60, nx=256, ny=256)  # held out
    X0 = place_particles(w)
    res = {}
    for init in (0, 1):
        sim = Simulation(w.with_(mlp_init=init), X0)
        if init:
            sim.set_mlp(params)
        sim.set_residual_tracking(True)
        r = []
        for _ in range(40):
            sim.step(1)
            r.append(sim.mdf_residual()[0])
        res[init] = float(np.mean(r[-20:]))
        sim.close()
    print(f"training loss {losses[0]:.3e} -> {losses[-1]:.3e}; residual after 3 MDF iterations "
          f"plain {res[0]:.3e}, learned first force {res[1]:.3e} ({res[1] / res[0]:.2f}x)")
    assert res[1] < res[0]


@pytest.mark.parametrize("n_lag", [31, 50, 12])
def test_step_2d_starts_from_the_network_prediction(n_lag):
    """With mdf_iters = 1 and the learned start, F_b of the step is the prediction of the
    tensor-core network (FP16 operands) from the step's stencils, rotated from each
    point's (normal, tangent) frame: 31 points fill the two 16-row tiles of a pass but
    one row, 50 take a second, ragged pass, 12 leave most rows empty."""
    require_gpu()
    from paper_2002_08855_gb300 import mlp
    from paper_2002_08855_gb300.binding import Simulation

    w = _workload(33, n=20, mlp_init=1, fixed_particles=1).with_(n_lag=n_lag, mdf_iters=1)
    p = mlp.init_params(7)
    p[-2], p[-1] = 200.0, 1e-3  # in_scale, out_scale of the deficits' size
    sim = Simulation(w, place_particles(w))
    sim.set_mlp(p)
    sim.step(2)
    lg = sim.get_lagrangian()
    Fl = mlp_ref.predict(p, mlp_ref.features_2d(lg["U_b"], lg["u_b_star"], w.n_lag))
    th = 2 * np.pi * (np.arange(len(Fl)) % w.n_lag) / w.n_lag
    F = np.stack([Fl[:, 0] * np.cos(th) - Fl[:, 1] * np.sin(th), Fl[:, 0] * np.sin(th) + Fl[:, 1] * np.cos(th)], 1)
    assert rel_l2(lg["F_b"], F) < 2e-2
    sim.close()


# ---------------------------------------------------------------- spheres (3D)
def _workload3(seed, n=12, side=56, **kw):
    kw = {"mdf_iters": 3, **kw}
    return Workload(name="mlp3", dim=3, nx=side, ny=side, nz=side, tau=0.6, n_particles=n, n_lag=452,
                    diameter=12.0, density_ratio=1.5, gravity=(0.0, -1e-4, 0.0), seed=seed, **kw)


def _sphere_ref(w, X0, sim=None):
    """The oracle's reference offsets of the spheres' points (its own Fibonacci lattice)."""
    import oracle

    ref = oracle.Sim(w.as_dict(), X0)
    ref.step(1)  # the points of a step are placed from the centres at its start
    lg = ref.get_lagrangian()
    return lg["X_b"][: w.n_lag] - X0[0]


def test_samples_3d_are_the_stencils_of_the_last_step():
    """GPU stencil table (built by the library's host code) and features against the FP64
    reference built from the oracle's own sphere points."""
    require_gpu()
    from paper_2002_08855_gb300.binding import Simulation

    w = _workload3(31)
    X0 = place_particles(w)
    sim = Simulation(w, X0)
    sim.step(3)
    X, Y = sim.mdf_samples()
    lg = sim.get_lagrangian()
    ref = _sphere_ref(w, X0, sim)
    Xr = mlp_ref.features_3d(lg["U_b"], lg["u_b_star"], ref)
    assert rel_l2(X.cpu().numpy(), Xr) < 1e-5
    Yr = mlp_ref.to_frame_3d(lg["F_b"], ref)
    assert rel_l2(Y.cpu().numpy(), Yr) < 1e-5
    sim.close()


def test_step_3d_starts_from_the_network_prediction():
    """With mdf_iters = 1 and the learned start, F_b of the step is the prediction of the
    tensor-core network (FP16 operands) from the step's stencils."""
    require_gpu()
    from paper_2002_08855_gb300 import mlp
    from paper_2002_08855_gb300.binding import Simulation

    w = _workload3(32, mdf_iters=1, mlp_init=1, fixed_particles=1)
    X0 = place_particles(w)
    p = mlp.init_params(5)
    p[-2], p[-1] = 200.0, 1e-3  # in_scale, out_scale of the deficits' size
    sim = Simulation(w, X0)
    sim.set_mlp(p)
    sim.step(2)
    lg = sim.get_lagrangian()
    ref = _sphere_ref(w, X0, sim)
    frames, _ = mlp_ref.sphere_stencil(ref)
    Fl = mlp_ref.predict(p, mlp_ref.features_3d(lg["U_b"], lg["u_b_star"], ref))
    k = np.arange(len(Fl)) % w.n_lag
    F = np.einsum("pa,pac->pc", Fl, frames[k])
    assert rel_l2(lg["F_b"], F) < 2e-2
    sim.close()


def test_residual_tracking_3d_matches_oracle():
    require_gpu()
    import oracle
    from paper_2002_08855_gb300.binding import Simulation

    w = _workload3(33, n=6, side=44)
    X0 = place_particles(w)
    sim = Simulation(w, X0)
    ref = oracle.Sim(w.as_dict(), X0)
    sim.set_residual_tracking(True)
    sim.step(4)
    ref.step(4)
    rg, ro = sim.mdf_residual()[0], ref.get_mdf_residual()[0]
    assert abs(rg - ro) < 1e-3 * ro
    sim.close()


def test_initializer_3d_lowers_the_mdf_residual():
    """Trained on spheres of other seeds (converged forces, 10 iterations); on a held-out
    box the learned start with M = 2 beats the plain M = 2."""
    require_gpu()
    from paper_2002_08855_gb300 import mlp
    from paper_2002_08855_gb300.binding import Simulation

    train = [_workload3(50 + s, n=20, side=64) for s in range(3)]
    X, Y = mlp.collect_samples(train, [place_particles(w) for w in train], steps=30, every=3)
    params, losses = mlp.train(X, Y, epochs=25, batch=4096, lr=2e-3, seed=3)
    assert losses[-1] < 0.5 * losses[0]
    w = _workload3(88, n=20, side=64, mdf_iters=2)  # held out
    X0 = place_particles(w)
    res = {}
    for init in (0, 1):
        sim = Simulation(w.with_(mlp_init=init), X0)
        if init:
            sim.set_mlp(params)
        sim.set_residual_tracking(True)
        r = []
        for _ in range(20):
            sim.step(1)
            r.append(sim.mdf_residual()[0])
        res[init] = float(np.mean(r[-10:]))
        sim.close()
    print(f"3D training loss {losses[0]:.3e} -> {losses[-1]:.3e}; residual after 2 MDF iterations "
          f"plain {res[0]:.3e}, learned first force {res[1]:.3e} ({res[1] / res[0]:.2f}x)")
    assert res[1] < res[0]
