"""Input-generator checks: workload sizes against Table 7 and valid placements."""
import math
import os

import numpy as np
import pytest

from paper_2002_08855_gb300 import inputs


def test_solid_fraction_matches_table7():
    """Table 7 prints the solid fraction V_p = N_p * (particle volume) / N_grid."""
    rows = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "table7_2d_3d.txt"))
    for dim, side, n, pct, D in rows:
        dim, side, n = int(dim), int(side), int(n)
        ngrid = side ** dim
        # the printed percentage has two significant digits
        assert inputs.n_particles_for_fraction(dim, ngrid, D, pct / 100.0) == pytest.approx(n, rel=0.02)
        vp = math.pi * D ** 2 / 4 if dim == 2 else math.pi * D ** 3 / 6
        assert n * vp / ngrid * 100 == pytest.approx(pct, rel=0.02)


def test_cavity_sizes():
    w = inputs.cavity_2d_large(0.1)
    assert (w.nx, w.ny, w.n_particles, w.n_lag) == (2048, 4096, 10681, 31)
    assert [inputs.cavity_2d_large(p).n_particles for p in (0.0, 0.2, 0.4)] == [0, 21361, 42723]
    w3 = inputs.cavity_3d()
    assert (w3.n_grid, w3.n_particles, w3.n_lag) == (384 * 384 * 768, 20000, 452)


@pytest.mark.parametrize("dim,shape,n,D", [(2, (128, 256), 12, 16.0), (3, (48, 48, 96), 20, 12.0)])
def test_rsa_placement_valid_and_seeded(dim, shape, n, D):
    X = inputs.place_rsa(dim, shape, n, D, seed=99)
    Y = inputs.place_rsa(dim, shape, n, D, seed=99)
    assert np.array_equal(X, Y)
    d = np.sqrt(((X[:, None] - X[None]) ** 2).sum(-1)) + np.eye(n) * 1e9
    assert d.min() >= D + 2.0
    for k in range(dim):
        assert X[:, k].min() >= -0.5 + D / 2 + 2.0 - 1e-12
        assert X[:, k].max() <= shape[k] - 0.5 - D / 2 - 2.0 + 1e-12


def test_hex_placement_dense_fraction():
    X = inputs.place_hex((400, 300), 700, 10.0, seed=5)
    assert len(X) == 700
    d = np.sqrt(((X[:, None] - X[None]) ** 2).sum(-1)) + np.eye(len(X)) * 1e9
    assert d.min() >= 12.0 - 1e-9


def test_splitmix64_reference_values():
    """First outputs of SplitMix64 seeded with 0 (published test vector)."""
    r = inputs.SplitMix64(0)
    assert [r.next_u64() for _ in range(3)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
