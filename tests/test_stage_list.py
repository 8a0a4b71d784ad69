"""CPU pin of the 3D staging list (host code of the C ABI, no GPU): the cells of a
sphere's node box the interpolation stages and the spreading flushes must include
every support node (Eq. 47-48) of every Lagrangian point, whatever the position of
the centre within its anchor cell.  The points come from the FP64 oracle (its own
sphere layout), the supports from the delta functions' definitions: 4-point nodes
floor(X) - 1 .. floor(X) + 2, 3-point nodes with non-zero weight round(X) - 1 ..
round(X) + 1."""
import math

import numpy as np
import pytest

import oracle
from paper_2002_08855_gb300 import binding, build
from paper_2002_08855_gb300.inputs import Workload


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()
    oracle.build()


def _workload(d, kind, n=6):
    return Workload(name="sl", dim=3, nx=4 * int(d) + 16, ny=4 * int(d) + 16, nz=4 * int(d) + 16, tau=0.6,
                    n_particles=n, n_lag=int(round(math.pi * d * d)), diameter=float(d), delta_kind=kind,
                    drs=1.9 if kind == 3 else 2.6, fixed_particles=1)


@pytest.mark.parametrize("d", [7.3, 10.0, 12.0, 16.0])
@pytest.mark.parametrize("kind", [4, 3])
def test_every_support_node_is_listed(d, kind):
    w = _workload(d, kind)
    cells = binding.stage_list(w)
    rcell = math.ceil(d / 2)
    S = 2 * rcell + 6
    lx, ly, lz = cells & 31, (cells >> 5) & 31, (cells >> 10) & 31
    assert lx.max() < S and ly.max() < S and lz.max() < S
    listed = set(zip(lx.tolist(), ly.tolist(), lz.tolist()))
    assert len(listed) == len(cells) < S ** 3  # distinct cells, fewer than the box
    rng = np.random.default_rng(int(10 * d) + kind)
    L = w.nx
    for trial in range(3):
        # centres well apart and inside, fractional parts spread over the cell
        base = np.array([[0.25, 0.25, 0.25], [0.75, 0.25, 0.25], [0.25, 0.75, 0.25],
                         [0.25, 0.25, 0.75], [0.75, 0.75, 0.25], [0.75, 0.25, 0.75]]) * L
        xc = np.floor(base) + rng.random((6, 3))
        sim = oracle.Sim(w.as_dict(), xc)
        sim.step(1)
        Xb = sim.get_lagrangian()["X_b"].reshape(6, w.n_lag, 3)
        sim.close()
        for i in range(6):
            org = np.floor(xc[i]).astype(int) - rcell - 2
            first = (np.floor(Xb[i]) if kind == 4 else np.floor(Xb[i] + 0.5)).astype(int) - 1
            span = range(4) if kind == 4 else range(3)
            for t in np.array(np.meshgrid(span, span, span, indexing="ij")).reshape(3, -1).T:
                need = first + t - org
                missing = [tuple(c) for c in need.tolist() if tuple(c) not in listed]
                assert not missing, (d, kind, trial, i, missing[:3])


def test_no_list_in_2d_or_without_particles():
    w2 = Workload(name="sl2", dim=2, nx=64, ny=64, n_particles=2, n_lag=31, diameter=10.0)
    assert binding.stage_list(w2).size == 0
    w0 = _workload(12.0, 4).with_(n_particles=0)
    assert binding.stage_list(w0).size == 0


def test_query_errors():
    import ctypes as C

    lib = binding.lib()
    cfg = binding.make_config(_workload(12.0, 4))
    n = C.c_int64(0)
    assert lib.ibm_lbm_stage_list(C.byref(cfg), None, 0, C.byref(n)) == 0 and n.value > 0
    small = (C.c_int32 * 8)()
    assert lib.ibm_lbm_stage_list(C.byref(cfg), small, 8, C.byref(n)) == -7  # IBMLBM_ERR_CAPACITY
    assert lib.ibm_lbm_stage_list(C.byref(cfg), None, 0, None) == -1  # IBMLBM_ERR_INVALID_ARG
