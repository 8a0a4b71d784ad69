"""The oracle built with OpenMP (its node, point, particle and boundary loops on all
host cores) gives the same bits as the single-threaded build: no loop it runs in
parallel sums across iterations."""
import numpy as np
import pytest

import oracle
from paper_2002_08855_gb300 import inputs
from paper_2002_08855_gb300.inputs import Workload


@pytest.mark.parametrize("case", ["cavity2d", "channel3d"])
def test_openmp_build_is_bit_identical(case):
    try:
        oracle.build(omp=True)
    except Exception as e:  # a host without OpenMP support
        pytest.skip(f"no OpenMP build: {e}")
    if case == "cavity2d":
        w = inputs.cavity_2d_small()
        X = inputs.place_particles(w)
        steps = 15
    else:
        w = Workload(name="ch3", dim=3, nx=20, ny=24, nz=18, boundary=2, u_inlet=0.01, tau=0.7,
                     n_particles=3, n_lag=201, diameter=8.0, density_ratio=1.5,
                     gravity=(0.0, 0.0, -1e-5))
        X = np.array([[6.2, 8.1, 5.5], [13.9, 15.3, 9.8], [9.7, 12.0, 13.4]])
        steps = 8
    out = []
    for omp in (False, True):
        S = oracle.Sim(w.as_dict(), X, omp=omp)
        S.step(steps)
        st = S.get_particles()
        out.append([S.get_pdfs(), st["X"], st["U"], st["Omega"], st["F_h"],
                    S.get_lagrangian()["F_b"]])
        S.close()
    for a, b in zip(*out):
        assert np.array_equal(a, b)
    assert np.abs(out[0][4]).max() > 0
