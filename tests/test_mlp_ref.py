"""Pins of the FP64 reference of the learned MDF initializer (CPU): the backward pass
against central finite differences, the parameter layout, the scales, and the frame of
the deficit features."""
import numpy as np

from oracle import mlp_ref


def _random(seed, B=7):
    rng = np.random.Generator(np.random.PCG64(seed))
    p = rng.normal(0.0, 0.3, mlp_ref.N_PARAMS)
    X = rng.normal(0.0, 1.0, (B, mlp_ref.N_IN))
    T = rng.normal(0.0, 1.0, (B, mlp_ref.N_OUT))
    return p, X, T


def test_layout_has_6149_parameters():
    assert mlp_ref.N_PARAMS == 27 * 64 + 64 + 64 * 64 + 64 + 64 * 3 + 3 + 2 == 6149
    p, _, _ = _random(1)
    assert np.array_equal(mlp_ref.pack(mlp_ref.unpack(p)), p)


def test_gradient_matches_central_differences():
    p, X, T = _random(2)
    _, g = mlp_ref.loss_and_grad(p, X, T)
    rng = np.random.Generator(np.random.PCG64(3))
    idx = np.concatenate([rng.choice(mlp_ref.N_PARAMS - 2, 60, replace=False),
                          [0, 27 * 64, 27 * 64 + 64, mlp_ref.N_PARAMS - 3]])
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        lp, _ = mlp_ref.loss_and_grad(p + e, X, T)
        lm, _ = mlp_ref.loss_and_grad(p - e, X, T)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])
    assert g[-1] == 0.0 and g[-2] == 0.0  # the scales are not trained


def test_scales_act_on_input_and_output():
    p, X, _ = _random(4)
    q = mlp_ref.unpack(p)
    q["in_scale"], q["out_scale"] = 2.0, 3.0
    p2 = mlp_ref.pack(q)
    Y, _, _ = mlp_ref.forward(p2, 2.0 * X)
    assert np.allclose(mlp_ref.predict(p2, X), 3.0 * Y)


def test_features_are_frame_components_of_the_stencil():
    nl = 12
    th = 2 * np.pi * np.arange(nl) / nl
    # a deficit field that is purely normal with unit size at every point of one circle
    d = np.stack([np.cos(th), np.sin(th)], axis=1)
    X = mlp_ref.features_2d(d, np.zeros_like(d), nl)
    assert np.allclose(X[:, 3 * 4], 1.0) and np.allclose(X[:, 3 * 4 + 1], 0.0)  # the point itself
    # neighbour j of point k is rotated by (j - 4) 2 pi / nl in the frame of k
    for j in range(9):
        a = (j - 4) * 2 * np.pi / nl
        assert np.allclose(X[:, 3 * j], np.cos(a)) and np.allclose(X[:, 3 * j + 1], np.sin(a))
    assert np.all(X[:, 2::3] == 0.0)


def _sphere_ref(nl=452, d=12.0):
    """Point offsets of the oracle's reference sphere (Fibonacci lattice, Sec. 2.2)."""
    import oracle

    w = dict(dim=3, nx=24, ny=24, nz=24, n_particles=1, n_lag=nl, diameter=d, mdf_iters=1)
    S = oracle.Sim(w, np.array([[11.5, 11.5, 11.5]]))
    S.step(1)
    return S.get_lagrangian()["X_b"] - np.array([11.5, 11.5, 11.5])


def test_sphere_stencil_frames_and_neighbours():
    from scipy.spatial import cKDTree

    ref = _sphere_ref()
    frames, nbr = mlp_ref.sphere_stencil(ref)
    n, t1, t2 = frames[:, 0], frames[:, 1], frames[:, 2]
    assert np.allclose(np.einsum("kij,klj->kil", frames, frames), np.eye(3)[None], atol=1e-12)
    assert np.allclose(np.linalg.det(frames), 1.0)  # right-handed (n, t1, t2)
    assert np.allclose(n, ref / np.linalg.norm(ref, axis=1, keepdims=True))  # outward normal
    dist, idx = cKDTree(ref).query(ref, k=9)  # the point itself and its 8 nearest
    for k in range(len(ref)):
        assert set(nbr[k]) == set(idx[k, 1:]) or np.isclose(dist[k, 8], np.sort(
            np.linalg.norm(ref[nbr[k]] - ref[k], axis=1))[-1])
        rel = ref[nbr[k]] - ref[k]
        az = np.mod(np.arctan2(rel @ t2[k], rel @ t1[k]), 2 * np.pi)
        assert np.all(np.diff(az) >= -1e-9)  # azimuth order


def test_sphere_features_are_frame_components_of_the_stencil():
    ref = _sphere_ref()
    frames, nbr = mlp_ref.sphere_stencil(ref)
    nl = len(ref)
    unit = ref / np.linalg.norm(ref, axis=1, keepdims=True)
    # purely radial unit deficits: the point's own triple is (1, 0, 0)
    X = mlp_ref.features_3d(unit, np.zeros_like(unit), ref)
    assert np.allclose(X[:, 0:3], [1.0, 0.0, 0.0])
    # one uniform deficit e everywhere: the nine triples of point k all equal e in k's frame
    e = np.array([0.3, -1.2, 0.7])
    X = mlp_ref.features_3d(np.tile(e, (2 * nl, 1)), np.zeros((2 * nl, 3)), ref)  # two spheres
    want = np.einsum("c,kac->ka", e, frames)
    for j in range(9):
        assert np.allclose(X[:nl, 3 * j:3 * j + 3], want) and np.allclose(X[nl:, 3 * j:3 * j + 3], want)
    # neighbour triples come from the neighbour's deficit: a field that is zero except at
    # point 5 shows up at (k, j) exactly where nbr[k][j - 1] == 5
    d = np.zeros((nl, 3))
    d[5] = e
    X = mlp_ref.features_3d(d, np.zeros_like(d), ref)
    for k in range(nl):
        for j in range(1, 9):
            hit = nbr[k][j - 1] == 5
            assert np.allclose(X[k, 3 * j:3 * j + 3], frames[k] @ e if hit else 0.0)
    # the output frame is orthonormal: back-transforming recovers the vectors
    F = np.random.default_rng(1).normal(size=(nl, 3))
    Fl = mlp_ref.to_frame_3d(F, ref)
    assert np.allclose(np.einsum("ka,kac->kc", Fl, frames), F)
