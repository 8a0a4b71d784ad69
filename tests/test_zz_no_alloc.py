"""The pair search that allocates nothing, against the scratch-based pair search.

ibm_lbm_pair_search_static keeps its cell and neighbour lists in a fixed device array
inside the library, for callers that cannot provide or allocate device scratch.  It
must return exactly the pair list of ibm_lbm_pair_search (pair lists are compared
bit for bit; that list is also checked against the oracle's brute-force list), on two
calls in a row, since every call reuses the same array."""
import numpy as np
import pytest

import oracle

from paper_2002_08855_gb300 import inputs

from gpu_util import require_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dim,shape,per,n,seed", [
    (2, (400, 300, 1), (0, 0, 0), 2500, 11),
    (3, (60, 50, 70), (1, 0, 1), 600, 12),
])
def test_static_scratch_matches_caller_scratch_twice(dim, shape, per, n, seed):
    require_gpu()
    from paper_2002_08855_gb300.binding import pair_search, pair_search_static

    X = inputs.random_points(n, dim, [-0.5] * dim, [s - 0.5 - 1e-9 for s in shape[:dim]], seed)
    ref = pair_search(dim, shape, per, 10.0, 2.0, X, max_neighbors=64)
    assert len(ref) > 100
    cfg = dict(dim=dim, nx=shape[0], ny=shape[1], nz=shape[2], periodic=per, diameter=10.0, zeta=2.0)
    assert np.array_equal(ref, oracle.pairs_bruteforce(cfg, X))
    for _ in range(2):
        got = pair_search_static(dim, shape, per, 10.0, 2.0, X, max_neighbors=64)
        assert np.array_equal(got, ref)
    # a different problem in between leaves no trace in the next result
    Y = X[: n // 3]
    ref_y = pair_search(dim, shape, per, 10.0, 2.0, Y, max_neighbors=64)
    assert np.array_equal(pair_search_static(dim, shape, per, 10.0, 2.0, Y, max_neighbors=64), ref_y)
    assert np.array_equal(pair_search_static(dim, shape, per, 10.0, 2.0, X, max_neighbors=64), ref)


def test_static_scratch_rejects_problems_beyond_its_size():
    require_gpu()
    from paper_2002_08855_gb300.binding import IbmLbmError, pair_search_static

    X = inputs.random_points(200000, 2, [0, 0], [4000, 4000], seed=13)
    with pytest.raises(IbmLbmError) as e:
        pair_search_static(2, (4000, 4000, 1), (0, 0, 0), 10.0, 2.0, X, max_neighbors=64)
    assert e.value.name == "CAPACITY"
    assert "16777216" in str(e.value)
