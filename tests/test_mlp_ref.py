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
