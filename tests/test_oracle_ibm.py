"""Oracle pins: regularised delta functions, interpolation / spreading and MDF.

- The 4-point and 3-point functions are defined by moment conditions: the
  partition of unity, a zero first moment (hence exact interpolation of linear
  fields) and a fixed sum of squares (3/8 and 1/2).
- D_I and D_E (Eq. 12-13) are built as dense matrices by brute force on tiny
  grids: D_E must equal D_I^T diag(dV), and the point-to-node sums (Eq. 47-48)
  must equal the all-node sums (Eq. 43-44).
- Multi-direct forcing: one pass is the BTDF scheme of Eq. 9-11; the thickened
  shell (drs = 2.6 for the 4-point function, Sec. 2.2) leaves a smaller slip
  than drs = 1, and extra iterations keep reducing it.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2002_08855_gb300.inputs import Workload, random_points

RNG = np.random.Generator(np.random.PCG64(21))


@pytest.mark.parametrize("kind,width,sumsq", [(4, 4, 3.0 / 8.0), (3, 3, 0.5)])
def test_delta_moment_conditions(kind, width, sumsq):
    for X in RNG.uniform(-5, 5, 200):
        j = np.arange(math.floor(X) - 3, math.floor(X) + 4)
        phi = oracle.delta(kind, j - X)
        assert abs(phi.sum() - 1.0) < 1e-14
        assert abs(((j - X) * phi).sum()) < 1e-14
        assert abs((phi * phi).sum() - sumsq) < 1e-14
        assert (phi >= 0).all()
        assert (phi > 0).sum() <= width
        if kind == 4:
            assert abs(phi[j % 2 == 0].sum() - 0.5) < 1e-14


def test_delta_values_and_continuity():
    assert oracle.delta(4, 0.0)[0] == pytest.approx(0.5, abs=1e-16)
    assert oracle.delta(3, 0.0)[0] == pytest.approx(2.0 / 3.0, abs=1e-16)
    for kind, breaks in ((4, (1.0, 2.0)), (3, (0.5, 1.5))):
        for b in breaks:
            lo, hi = oracle.delta(kind, [b - 1e-12, b + 1e-12])
            assert abs(lo - hi) < 1e-5
        assert oracle.delta(kind, breaks[-1] + 1e-9)[0] == 0.0
        r = np.linspace(-2.5, 2.5, 101)
        assert np.array_equal(oracle.delta(kind, r), oracle.delta(kind, -r))


def test_point_to_node_support_ratio_fig5():
    """The point-to-node box has (2r)^d = 3^d nodes for the 3-point function; the
    standard box around a particle has about (D + 2r)^d.  Their ratio matches the
    values printed with Fig. 5 within 10 percent."""
    rows = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "fig5_ratios.txt"))
    for dim, D, printed in rows:
        X = 0.37
        j = np.arange(-4, 5)
        width = int((oracle.delta(3, j - X) > 0).sum())
        assert width == 3
        ratio = ((D + width) / width) ** dim
        assert abs(ratio / printed - 1) < 0.1


def _cfg(dim, shape, periodic=(0, 0, 0), kind=4):
    return Workload(name="ibm", dim=dim, nx=shape[0], ny=shape[1],
                    nz=shape[2] if dim == 3 else 1, periodic=periodic, delta_kind=kind).as_dict()


@pytest.mark.parametrize("dim,kind", [(2, 4), (3, 4), (2, 3)])
def test_interpolation_is_exact_for_linear_fields(dim, kind):
    shape = (12, 11, 10)
    cfg = _cfg(dim, shape, kind=kind)
    N = int(np.prod(shape[:dim]))
    coords = np.stack(np.meshgrid(*[np.arange(s) for s in shape[:dim]], indexing="ij"), -1)
    coords = coords.transpose(*reversed(range(dim)), dim).reshape(N, dim)  # x fastest
    A = RNG.normal(size=(dim, dim))
    c = RNG.normal(size=dim)
    g = (coords @ A.T + c).T  # [dim][N]
    X = random_points(40, dim, [3.0] * dim, [s - 4.0 for s in shape[:dim]], seed=5)
    ub = oracle.interp(cfg, g, X)
    assert np.abs(ub - (X @ A.T + c)).max() < 1e-12


@pytest.mark.parametrize("dim,shape,periodic,kind", [
    (2, (8, 7, 1), (0, 0, 0), 4),
    (2, (8, 7, 1), (1, 0, 0), 4),
    (2, (9, 8, 1), (0, 0, 0), 3),
    (3, (6, 5, 6), (0, 1, 0), 4),
])
def test_spread_is_adjoint_of_interp_dense(dim, shape, periodic, kind):
    """D_E = D_I^T diag(dV) as dense matrices (Eq. 12-13), points anywhere including
    near walls (support nodes outside the domain are dropped on both sides)."""
    cfg = _cfg(dim, shape, periodic, kind)
    N = int(np.prod(shape[:dim]))
    X = random_points(5, dim, [-0.4] * dim, [s - 0.6 for s in shape[:dim]], seed=9)
    dV = 2.6
    DI = np.zeros((dim, X.shape[0], N))
    for n in range(N):
        for c in range(dim):
            g = np.zeros((dim, N))
            g[c, n] = 1.0
            DI[c, :, n] = oracle.interp(cfg, g, X)[:, c]
    DE = np.zeros((dim, N, X.shape[0]))
    for b in range(X.shape[0]):
        for c in range(dim):
            F = np.zeros((X.shape[0], dim))
            F[b, c] = 1.0
            DE[c, :, b] = oracle.spread(cfg, X, F, dV)[c]
    for c in range(dim):
        assert np.abs(DE[c] - DI[c].T * dV).max() < 1e-15
        assert np.abs(DI[c] - DI[0]).max() == 0.0  # same operator for every component


def test_point_to_node_equals_all_node_sums():
    """Eq. 47 (support box only) equals Eq. 43 (all nodes) because delta vanishes
    outside the box; likewise Eq. 48 vs Eq. 44."""
    shape = (14, 12)
    cfg = _cfg(2, shape)
    N = shape[0] * shape[1]
    X = random_points(7, 2, [1.5, 1.5], [11.5, 9.5], seed=13)
    g = RNG.normal(size=(2, N))
    F = RNG.normal(size=(7, 2))
    dV = 1.7
    xs, ys = np.meshgrid(np.arange(shape[0]), np.arange(shape[1]), indexing="xy")
    xs, ys = xs.ravel(), ys.ravel()
    naive_u = np.zeros((7, 2))
    naive_f = np.zeros((2, N))
    for b in range(7):
        w = oracle.delta(4, xs - X[b, 0]) * oracle.delta(4, ys - X[b, 1])
        naive_u[b] = g @ w
        naive_f += F[b][:, None] * w[None, :] * dV
    assert np.abs(oracle.interp(cfg, g, X) - naive_u).max() < 1e-14
    assert np.abs(oracle.spread(cfg, X, F, dV) - naive_f).max() < 1e-14


@pytest.mark.parametrize("dim", [2, 3])
def test_total_force_conserved(dim):
    shape = (16, 15, 14)
    cfg = _cfg(dim, shape)
    X = random_points(30, dim, [2.5] * dim, [s - 3.5 for s in shape[:dim]], seed=17)
    F = RNG.normal(size=(30, dim))
    dV = 2.3
    f = oracle.spread(cfg, X, F, dV)
    assert np.abs(f.sum(1) - F.sum(0) * dV).max() < 1e-12


def _moving_cylinder(M, drs, U=(2e-3, -1e-3)):
    w = Workload(name="cyl", dim=2, nx=48, ny=44, tau=0.8, n_particles=1, n_lag=60,
                 diameter=18.0, drs=drs, mdf_iters=M, fixed_particles=1)
    xc = np.array([[23.3, 21.6]])
    S = oracle.Sim(w.as_dict(), xc)
    S.set_particles(xc, U=np.array([U]))
    S.step(1)
    return S


def test_single_pass_is_btdf_eq9_11():
    """From rest (u* = 0), one pass gives F_b = 2 rho_f (U_b - 0) / dt (Eq. 10)."""
    S = _moving_cylinder(1, 2.6)
    lag = S.get_lagrangian()
    assert np.abs(lag["u_b_star"]).max() == 0.0
    assert np.abs(lag["F_b"] - 2.0 * lag["U_b"]).max() < 1e-18


def test_thickened_shell_and_iterations_reduce_slip():
    res = {M: _moving_cylinder(M, 2.6).get_mdf_residual()[0] for M in (1, 2, 3, 5)}
    assert res[1] > res[2] > res[3] > res[5]
    df = _moving_cylinder(1, 1.0).get_mdf_residual()[0]
    # Sec. 2.2: with drs = dh (conventional DF) the slip after one pass is much larger
    assert res[1] < 0.25 * df


def test_drag_converges_with_mdf_iterations():
    """A fixed cylinder in a periodic box of fluid started at a uniform velocity: the
    hydrodynamic force after 30 steps converges as the number of MDF iterations grows
    (each difference to M = 10 smaller than the last, below 0.2 % from M = 3), and the
    boundary residual after the last iteration does not grow with M."""
    N = 96 * 64
    res = {}
    for M in (1, 2, 3, 4, 10):
        w = Workload(name="drag", dim=2, nx=96, ny=64, periodic=(1, 1, 0), tau=0.8, n_particles=1,
                     n_lag=50, diameter=16.0, delta_kind=4, drs=2.6, mdf_iters=M, fixed_particles=1,
                     density_ratio=1.5)
        S = oracle.Sim(w.as_dict(), np.array([[40.3, 31.7]]))
        u = np.zeros((2, N))
        u[0] = 0.01
        S.set_fields(np.zeros(N), u)
        S.step(30)
        res[M] = (S.get_particles()["F_h"][0], S.get_mdf_residual()[0])
        S.close()
    ref = res[10][0]
    gap = [np.linalg.norm(res[M][0] - ref) / np.linalg.norm(ref) for M in (1, 2, 3, 4)]
    assert gap[0] > gap[1] > gap[2] > gap[3]
    assert gap[2] < 2e-3
    rms = [res[M][1] for M in (1, 2, 3, 4, 10)]
    assert all(a >= b for a, b in zip(rms, rms[1:]))
