"""Pins of the oracle's non-equilibrium extrapolation boundaries (Sec. 6.1 and 6.2 apply
the method of the paper's ref. [48]; the formulas used are restated at the oracle's
reading R13) against closed forms and the method's order:

* body-force Poiseuille flow between walls on the boundary nodes x = 0 and x = L
  (L = n_x - 1): u_y = g x (L - x) / (2 nu), nu = (tau - 1/2) / 3;
* a channel along y with the same parabola imposed on the inlet nodes and p = 0 on
  the outlet nodes: the developed profile and the pressure gradient dp/dy = -8 nu U / L^2.

The steady bulk satisfies the discrete momentum balance nu (u_{x+1} - 2 u_x + u_{x-1})
+ g = 0 (exact for the lattice equations of a unidirectional steady flow), the boundary
nodes carry the prescribed velocity exactly (u* = u_b - F/2 by construction), and the
extrapolation error is second order: halving the spacing relative to L divides the
error by four."""
import numpy as np
import pytest

import oracle
from paper_2002_08855_gb300.inputs import Workload

TAU = 1.0
NU = (TAU - 0.5) / 3.0
G = 1e-6


def _poiseuille(dim, nx, steps):
    w = Workload(name="pois", dim=dim, nx=nx, ny=4, nz=4 if dim == 3 else 1, periodic=(0, 1, 1),
                 tau=TAU, body_force=(0.0, G, 0.0), boundary=1)
    S = oracle.Sim(w.as_dict(), np.zeros((0, dim)))
    S.step(steps)
    _, u = S.get_fields()  # u* (Eq. 5): the force half is not added
    uy = u[1].reshape(-1, nx)[1]  # one line of nodes across the channel
    ux = u[0].reshape(-1, nx)
    L = nx - 1
    x = np.arange(nx)
    exact = G / (2.0 * NU) * x * (L - x)
    err = np.abs(uy[1:-1] - exact[1:-1]).max() / exact.max()
    balance = np.abs(NU * (uy[3:-1] - 2.0 * uy[2:-2] + uy[1:-3]) + G).max() / G
    return err, balance, uy, np.abs(ux).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_body_force_poiseuille_between_extrapolation_walls(dim):
    e16, b16, u16, ux16 = _poiseuille(dim, 17, 6000)
    e32, b32, u32, _ = _poiseuille(dim, 33, 12000)
    for b in (b16, b32):
        assert b < 1e-5  # steady discrete momentum balance in the bulk
    for u in (u16, u32):  # boundary nodes: corrected velocity u* + g/2 = 0
        assert abs(u[0] + 0.5 * G) < 1e-18 and abs(u[-1] + 0.5 * G) < 1e-18
    assert ux16 < 1e-5 * u16.max()  # no cross flow beyond compressibility effects
    assert e16 < 0.01
    assert 3.8 < e16 / e32 < 4.2  # second order


def _channel(nx, ny, steps, U=0.01):
    w = Workload(name="chan", dim=2, nx=nx, ny=ny, tau=TAU, boundary=2, u_inlet=U)
    S = oracle.Sim(w.as_dict(), np.zeros((0, 2)))
    S.step(steps)
    p, u = S.get_fields()
    uy, ux, P = u[1].reshape(ny, nx), u[0].reshape(ny, nx), p.reshape(ny, nx)
    L = nx - 1
    x = np.arange(nx)
    exact = 4.0 * U * x * (L - x) / L**2
    j0, j1 = ny // 6, ny - ny // 6  # away from the inlet and outlet rows
    prof = max(float(np.abs(uy[j] - exact).max()) for j in range(j0, j1)) / U
    slope = np.polyfit(np.arange(j0, j1), P[j0:j1, nx // 2], 1)[0]
    dp = slope / (-8.0 * NU * U / L**2) - 1.0
    return prof, dp, uy[0] - exact, ux[0]


def test_channel_with_parabolic_inlet_and_pressure_outlet():
    p16, d16, inlet16, inx16 = _channel(17, 24, 3000)
    p32, d32, _, _ = _channel(33, 48, 9000)
    assert np.abs(inlet16).max() < 1e-15 and np.abs(inx16).max() < 1e-15  # inlet nodes exact
    assert p16 < 0.01 and abs(d16) < 0.01
    assert 3.6 < p16 / p32 < 4.4  # developed profile: second order
    assert 3.6 < d16 / d32 < 4.4  # pressure gradient: second order


def test_channel_inlet_3d_carries_the_product_parabola():
    nx, ny, nz, U = 9, 10, 9, 0.01
    w = Workload(name="chan3", dim=3, nx=nx, ny=ny, nz=nz, tau=TAU, boundary=2, u_inlet=U)
    S = oracle.Sim(w.as_dict(), np.zeros((0, 3)))
    S.step(50)
    _, u = S.get_fields()
    uy = u[1].reshape(nz, ny, nx)
    c = np.arange(nx)
    par = 4.0 * c * (nx - 1 - c) / (nx - 1) ** 2
    assert np.abs(uy[:, 0, :] - U * np.outer(par, par)).max() < 1e-15
    assert np.abs(u[0].reshape(nz, ny, nx)[:, 0, :]).max() < 1e-15
