"""Oracle pins: streaming, conservation and closed-form flows.

- Swap streaming (Sec. 3.3) is an independent formulation of the push
  streaming of Eq. 18: the two must agree bit for bit, with walls and periodic
  axes, and the result must be a permutation of the post-collision values.
- Collision and streaming with halfway bounce-back conserve
  sum_x sum_{a>=1} f_a exactly without forcing (Eq. 6 inverts Eq. 4); a force
  adds exactly -sum_x F_0 of Eq. 8.
- Body-force Poiseuille flow has a parabolic closed form; with halfway
  bounce-back BGK it is reproduced to round-off at (tau - 1/2)^2 = 3/16 and
  converges at second order otherwise.
- Taylor-Green vortices decay at 2 nu k^2 with nu = (tau - 1/2)/3 (Sec. 2.1).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2002_08855_gb300.inputs import Workload, random_pdfs

RNG = np.random.Generator(np.random.PCG64(11))


@pytest.mark.parametrize("dim,shape,periodic", [
    (2, (7, 5), (0, 0, 0)),
    (2, (6, 9), (1, 0, 0)),
    (2, (5, 4), (1, 1, 0)),
    (3, (5, 4, 3), (0, 0, 0)),
    (3, (4, 5, 6), (1, 0, 1)),
    (3, (3, 4, 5), (1, 1, 1)),
])
def test_swap_equals_push_streaming_bit_exact(dim, shape, periodic):
    q = 9 if dim == 2 else 19
    N = int(np.prod(shape))
    fp = RNG.normal(0, 1, (q, N))
    a = oracle.stream_push(dim, shape, periodic, fp)
    b = oracle.stream_swap(dim, shape, periodic, fp)
    assert np.array_equal(a, b)
    # streaming only moves values: the multiset of values is unchanged
    assert np.array_equal(np.sort(a.ravel()), np.sort(fp.ravel()))


def test_push_streaming_moves_each_population_one_link():
    """A single nonzero population at an interior node arrives at x + e_a; at a wall node
    pointing outward it returns to the same node in the opposite direction."""
    shape = (5, 4)
    e, _ = oracle.lattice(2)
    N = 20
    for a in range(9):
        fp = np.zeros((9, N))
        x, y = 2, 1
        fp[a, x + 5 * y] = 1.0
        f = oracle.stream_push(2, shape, (0, 0, 0), fp)
        tx, ty = x + e[a, 0], y + e[a, 1]
        assert f[a, tx + 5 * ty] == 1.0 and f.sum() == 1.0
    # wall node (0, 0), populations 5, 6, 7 leave the domain and come back reversed
    for a, back in ((5, 1), (6, 2), (7, 3)):
        fp = np.zeros((9, N))
        fp[a, 0] = 1.0
        f = oracle.stream_push(2, shape, (0, 0, 0), fp)
        assert f[back, 0] == 1.0 and f.sum() == 1.0


@pytest.mark.parametrize("dim,periodic", [(2, (0, 0, 0)), (2, (1, 0, 0)), (3, (0, 0, 0)),
                                          (3, (1, 1, 0))])
def test_pressure_moment_conserved_without_force(dim, periodic):
    """Eq. 17-18 conserve M1 = sum_x sum_{a>=1} f_a exactly when no force acts: Eq. 6
    makes sum_{a>=1} f_eq equal sum_{a>=1} f at every node, and streaming (with
    bounce-back) only permutes the a >= 1 populations.  sum_a f itself is not an
    invariant of this model, because sum_a f_eq = 0 relaxes it towards zero."""
    shape = (23, 17, 1) if dim == 2 else (11, 9, 8)
    w = Workload(name="m", dim=dim, nx=shape[0], ny=shape[1], nz=shape[2], tau=0.7,
                 periodic=periodic)
    S = oracle.Sim(w.as_dict())
    q = 9 if dim == 2 else 19
    f0 = random_pdfs(q, w.n_grid, seed=3).astype(np.float64)
    S.set_pdfs(f0)
    m0 = f0[1:].sum()
    scale = np.abs(f0).sum()
    S.step(200)
    f = S.get_pdfs()
    assert abs(f[1:].sum() - m0) <= 1e-13 * scale
    assert abs(f.sum()) < 0.5 * abs(f0.sum())  # sum_a f relaxes, as stated above


@pytest.mark.parametrize("dim", [2, 3])
def test_pressure_moment_source_is_force_term_zero(dim):
    """With a force, M1 changes each step by exactly -sum_x F_0 (Eq. 8 at a = 0),
    i.e. by 3 (1 - 1/(2 tau)) w0 sum_x u . f with u the corrected velocity of Eq. 7."""
    F = (2e-4, -1e-4, 3e-5 if dim == 3 else 0.0)
    shape = (19, 13, 1) if dim == 2 else (9, 8, 7)
    w = Workload(name="mf", dim=dim, nx=shape[0], ny=shape[1], nz=shape[2], tau=0.8,
                 body_force=F)
    S = oracle.Sim(w.as_dict())
    q = 9 if dim == 2 else 19
    S.set_pdfs(random_pdfs(q, w.n_grid, seed=5).astype(np.float64))
    _, w0 = oracle.lattice(dim)
    Fv = np.array(F[:dim])[:, None]
    for _ in range(5):
        m_before = S.get_pdfs()[1:].sum()
        _, us = S.get_fields()
        u = us + Fv / 2.0
        S.step(1)
        expect = 3.0 * (1 - 1 / (2 * 0.8)) * w0[0] * float((u * Fv).sum())
        assert S.get_pdfs()[1:].sum() - m_before == pytest.approx(expect, rel=1e-9, abs=1e-16)


def _poiseuille(tau, H, steps, g=1e-8):
    w = Workload(name="pois", dim=2, nx=1, ny=H, periodic=(1, 0, 0), tau=tau,
                 body_force=(g, 0.0, 0.0))
    S = oracle.Sim(w.as_dict())
    S.step(steps)
    _, u = S.get_fields()
    nu = (tau - 0.5) / 3.0
    y = np.arange(H)
    exact = g / (2 * nu) * (y + 0.5) * (H - 0.5 - y)
    # reported u is u* of Eq. 5; the physical velocity adds dt g / 2 (Eq. 7)
    ux = u[0] + g / 2
    return np.abs(ux - exact).max() / exact.max(), np.abs(u[1]).max()


def test_poiseuille_exact_at_magic_tau():
    """At (tau - 1/2)^2 = 3/16 halfway bounce-back BGK reproduces the parabola exactly
    in the linear (Stokes) limit; what remains is an O(u^2) relative effect of the
    quadratic terms of Eq. 4, which shrinks a hundredfold with a tenfold smaller force."""
    tau = 0.5 + math.sqrt(3.0 / 16.0)
    err, uy = _poiseuille(tau, 16, 20000, g=1e-8)
    assert err < 1e-11
    assert uy < 1e-13
    err_big, _ = _poiseuille(tau, 16, 20000, g=1e-7)
    assert 50.0 < err_big / err < 200.0


def test_poiseuille_second_order_convergence():
    # 2 H^2 / nu steps: about 20 decay times of the slowest transient, H^2 / (nu pi^2)
    errs = [_poiseuille(0.6, H, int(2 * H * H / ((0.6 - 0.5) / 3.0)))[0] for H in (8, 16, 32)]
    assert errs[0] > errs[1] > errs[2]
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.0 < r1 < 5.0 and 3.0 < r2 < 5.0


def _tgv_rate(N, tau, steps):
    k = 2 * math.pi / N
    U0 = 1e-3
    w = Workload(name="tgv", dim=2, nx=N, ny=N, periodic=(1, 1, 0), tau=tau)
    S = oracle.Sim(w.as_dict())
    x = np.arange(N)
    X, Y = np.meshgrid(x, x, indexing="xy")
    ux = -U0 * np.cos(k * X) * np.sin(k * Y)
    uy = U0 * np.sin(k * X) * np.cos(k * Y)
    p = -U0 * U0 / 4.0 * (np.cos(2 * k * X) + np.cos(2 * k * Y))
    S.set_fields(p.ravel(), np.stack([ux.ravel(), uy.ravel()]))
    mode = np.stack([ux.ravel(), uy.ravel()]) / U0

    def amp():
        _, u = S.get_fields()
        return float((u * mode).sum() / (mode * mode).sum())

    S.step(50)
    a0 = amp()
    S.step(steps)
    a1 = amp()
    return -math.log(a1 / a0) / steps, 2 * ((tau - 0.5) / 3.0) * k * k


def test_taylor_green_decay_rate():
    e32 = abs(_tgv_rate(32, 0.6, 400)[0] / _tgv_rate(32, 0.6, 400)[1] - 1)
    rate, expect = _tgv_rate(64, 0.6, 800)
    e64 = abs(rate / expect - 1)
    assert e64 < 1e-3
    assert e64 < e32
