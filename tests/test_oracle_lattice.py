"""Oracle pins: lattice, equilibrium, forcing term and macroscopic moments.

The oracle writes Eq. 4, 5, 6 and 8 in their general alpha-loop form.  These
tests hold it to things fixed independently of that form: the lattice symmetry
the paper states after Eq. 3, the paper's own unrolled D2Q9 forms (Eq. 19-36),
its symmetry identities (Eq. 38, 40), and the moment identities that make the
model recover the incompressible Navier-Stokes equations.
"""
import itertools

import numpy as np
import pytest

import oracle

RNG = np.random.Generator(np.random.PCG64(7))


@pytest.mark.parametrize("dim", [2, 3])
def test_lattice_isotropy_and_ordering(dim):
    e, w = oracle.lattice(dim)
    q = len(w)
    assert q == (9 if dim == 2 else 19)
    assert abs(w.sum() - 1.0) < 1e-15
    E = e[:, :dim].astype(float)
    assert np.abs((w[:, None] * E).sum(0)).max() < 1e-15
    M2 = np.einsum("a,ai,aj->ij", w, E, E)
    assert np.abs(M2 - np.eye(dim) / 3.0).max() < 1e-15
    M4 = np.einsum("a,ai,aj,ak,al->ijkl", w, E, E, E, E)
    d = np.eye(dim)
    iso = (np.einsum("ij,kl->ijkl", d, d) + np.einsum("ik,jl->ijkl", d, d)
           + np.einsum("il,jk->ijkl", d, d)) / 9.0
    assert np.abs(M4 - iso).max() < 1e-15
    # Sec. 2.1: e_a = -e_{a-(q-1)/2} for (q-1)/2 < a < q
    h = (q - 1) // 2
    for a in range(h + 1, q):
        assert (e[a] == -e[a - h]).all()
    assert len({tuple(v) for v in e}) == q
    # weight groups stated after Eq. 4
    if dim == 2:
        assert np.allclose(w, [4 / 9] + [1 / 9, 1 / 36] * 4)
    else:
        assert w[0] == pytest.approx(1 / 3)
        for a in list(range(1, 4)) + list(range(10, 13)):
            assert w[a] == pytest.approx(1 / 18)
            assert np.abs(e[a]).sum() == 1
        for a in list(range(4, 10)) + list(range(13, 19)):
            assert w[a] == pytest.approx(1 / 36)
            assert np.abs(e[a]).sum() == 2


def _unrolled_feq_d2q9(p, ux, uy, w):
    """Eq. 21-28 as printed (c = 1, rho_0 = 1)."""
    return {
        1: 3 * w[1] * (p + (ux + ux * ux - 0.5 * uy * uy)),
        2: 3 * w[2] * (p + (ux + uy + 3 * ux * uy + ux * ux + uy * uy)),
        3: 3 * w[3] * (p + (uy - 0.5 * ux * ux + uy * uy)),
        4: 3 * w[4] * (p + (-ux + uy - 3 * ux * uy + ux * ux + uy * uy)),
        5: 3 * w[5] * (p + (-ux + ux * ux - 0.5 * uy * uy)),
        6: 3 * w[6] * (p + (-ux - uy + 3 * ux * uy + ux * ux + uy * uy)),
        7: 3 * w[7] * (p + (-uy - 0.5 * ux * ux + uy * uy)),
        8: 3 * w[8] * (p + (ux - uy - 3 * ux * uy + ux * ux + uy * uy)),
    }


def _unrolled_force_d2q9(tau, ux, uy, fx, fy, w):
    """Eq. 29-36 as printed (c = 1)."""
    k = 3 * (1 - 1 / (2 * tau))
    uf = ux * fx + uy * fy
    cross = ux * fy + uy * fx
    return {
        1: k * w[1] * (fx + 3 * ux * fx - uf),
        2: k * w[2] * ((fx + fy) + 3 * cross + 2 * uf),
        3: k * w[3] * (fy + 3 * uy * fy - uf),
        4: k * w[4] * ((-fx + fy) - 3 * cross + 2 * uf),
        5: k * w[5] * (-fx + 3 * ux * fx - uf),
        6: k * w[6] * (-(fx + fy) + 3 * cross + 2 * uf),
        7: k * w[7] * (-fy + 3 * uy * fy - uf),
        8: k * w[8] * ((fx - fy) - 3 * cross + 2 * uf),
    }


def test_equilibrium_matches_unrolled_eq21_28():
    _, w = oracle.lattice(2)
    for _ in range(50):
        p, ux, uy = RNG.normal(0, 1e-2), RNG.normal(0, 0.05), RNG.normal(0, 0.05)
        feq = oracle.feq(2, p, (ux, uy))
        ref = _unrolled_feq_d2q9(p, ux, uy, w)
        for a, v in ref.items():
            assert feq[a] == pytest.approx(v, rel=1e-13, abs=1e-17)


def test_force_term_matches_unrolled_eq29_36():
    _, w = oracle.lattice(2)
    for _ in range(50):
        tau = RNG.uniform(0.52, 2.0)
        ux, uy, fx, fy = RNG.normal(0, 0.05, 4)
        Fa = oracle.force_term(2, tau, (ux, uy), (fx, fy))
        ref = _unrolled_force_d2q9(tau, ux, uy, fx, fy, w)
        for a, v in ref.items():
            assert Fa[a] == pytest.approx(v, rel=1e-12, abs=1e-17)


def test_velocity_matches_unrolled_eq19_20():
    for _ in range(20):
        f = RNG.normal(0, 1e-2, 9)
        us, _, _ = oracle.macro(2, f)
        assert us[0] == pytest.approx(f[1] + f[2] - f[4] - f[5] - f[6] + f[8], abs=1e-16)
        assert us[1] == pytest.approx(f[2] + f[3] + f[4] - f[6] - f[7] - f[8], abs=1e-16)


@pytest.mark.parametrize("dim", [2, 3])
def test_symmetry_identities_eq38_eq40(dim):
    e, w = oracle.lattice(dim)
    h = (len(w) - 1) // 2
    for _ in range(20):
        p = RNG.normal(0, 1e-2)
        u, F = RNG.normal(0, 0.05, 3), RNG.normal(0, 1e-3, 3)
        if dim == 2:
            u[2] = F[2] = 0.0
        tau = RNG.uniform(0.55, 1.5)
        feq = oracle.feq(dim, p, u)
        Fa = oracle.force_term(dim, tau, u, F)
        for a in range(h + 1, 2 * h + 1):
            b = a - h
            eu, ef = float(e[b] @ u), float(e[b] @ F)
            assert feq[a] == pytest.approx(feq[b] - 2 * w[b] * eu * 3.0, abs=1e-15)
            assert Fa[a] == pytest.approx(Fa[b] - 2 * (1 - 1 / (2 * tau)) * w[b] * ef * 3.0,
                                          abs=1e-16)


@pytest.mark.parametrize("dim", [2, 3])
def test_equilibrium_moments(dim):
    """sum f_eq = 0, sum e f_eq = rho0 u, sum e e f_eq = p I + rho0 u u."""
    e, _ = oracle.lattice(dim)
    E = e[:, :dim].astype(float)
    for _ in range(20):
        p = RNG.normal(0, 1e-2)
        u = np.zeros(3)
        u[:dim] = RNG.normal(0, 0.05, dim)
        feq = oracle.feq(dim, p, u)
        assert abs(feq.sum()) < 1e-16
        assert np.abs(E.T @ feq - u[:dim]).max() < 1e-16
        P2 = np.einsum("a,ai,aj->ij", feq, E, E)
        expect = p * np.eye(dim) + np.outer(u[:dim], u[:dim])
        assert np.abs(P2 - expect).max() < 1e-16


@pytest.mark.parametrize("dim", [2, 3])
def test_pressure_eq6_inverts_eq4(dim):
    for _ in range(20):
        p = RNG.normal(0, 1e-2)
        u = np.zeros(3)
        u[:dim] = RNG.normal(0, 0.05, dim)
        us, uu, pp = oracle.macro(dim, oracle.feq(dim, p, u))
        assert pp == pytest.approx(p, abs=1e-17)
        assert np.abs(us - u).max() < 1e-16
        assert np.abs(uu - u).max() < 1e-16


@pytest.mark.parametrize("dim", [2, 3])
def test_force_term_moments(dim):
    """sum F_a = 0, sum e F_a = (1 - 1/2tau) f, sum e e F_a = (1 - 1/2tau)(u f + f u)."""
    e, _ = oracle.lattice(dim)
    E = e[:, :dim].astype(float)
    for _ in range(20):
        tau = RNG.uniform(0.55, 2.0)
        u, F = np.zeros(3), np.zeros(3)
        u[:dim], F[:dim] = RNG.normal(0, 0.05, dim), RNG.normal(0, 1e-3, dim)
        Fa = oracle.force_term(dim, tau, u, F)
        k = 1 - 1 / (2 * tau)
        assert abs(Fa.sum()) < 1e-18
        assert np.abs(E.T @ Fa - k * F[:dim]).max() < 1e-18
        M2 = np.einsum("a,ai,aj->ij", Fa, E, E)
        expect = k * (np.outer(u[:dim], F[:dim]) + np.outer(F[:dim], u[:dim]))
        assert np.abs(M2 - expect).max() < 1e-18


def test_corrected_velocity_eq7():
    f = RNG.normal(0, 1e-2, 9)
    F = np.array([3e-4, -2e-4, 0.0])
    us, u, _ = oracle.macro(2, f, F)
    assert np.abs(u - (us + F / 2)).max() < 1e-18
