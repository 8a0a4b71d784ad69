"""FP64 CPU reference of the learned MDF initializer — TEST INFRASTRUCTURE ONLY.

Only the test suite may import this module.  It restates, in plain numpy double
precision, what the GPU computes for the initializer: the velocity-deficit stencil
features of a Lagrangian point and the perceptron 27 -> 64 -> 64 -> 3 (ReLU) with its
mean-squared-error loss and the gradient of that loss (the backward pass written out
by the chain rule).  The gradient is pinned by central finite differences in
tests/test_mlp_ref.py.  There is no counterpart in the paper (which iterates the plain
multi-direct forcing); the layout follows include/ibmlbm.h.
"""
from __future__ import annotations

import numpy as np

N_IN, N_H, N_OUT = 27, 64, 3
SHAPES = [("W1", (N_IN, N_H)), ("b1", (N_H,)), ("W2", (N_H, N_H)), ("b2", (N_H,)),
          ("W3", (N_H, N_OUT)), ("b3", (N_OUT,)), ("in_scale", ()), ("out_scale", ())]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = p[o:o + n].reshape(shape) if shape else p[o]
        o += n
    return out


def pack(d) -> np.ndarray:
    return np.concatenate([np.asarray(d[name], dtype=np.float64).reshape(-1) for name, _ in SHAPES])


def forward(p, X):
    """Network output (before out_scale) for feature rows X (already scaled), and the
    hidden activations."""
    q = unpack(p)
    h1 = np.maximum(X @ q["W1"] + q["b1"], 0.0)
    h2 = np.maximum(h1 @ q["W2"] + q["b2"], 0.0)
    return h2 @ q["W3"] + q["b3"], h1, h2


def loss_and_grad(p, X, T):
    """Mean over the rows of the squared error summed over the outputs, and its gradient
    with respect to every parameter (zero for the two scales)."""
    q = unpack(p)
    B = X.shape[0]
    Y, h1, h2 = forward(p, X)
    E = Y - T
    loss = float(np.sum(E * E) / B)
    dY = 2.0 * E / B
    g = {"W3": h2.T @ dY, "b3": dY.sum(0)}
    dh2 = (dY @ q["W3"].T) * (h2 > 0)
    g["W2"], g["b2"] = h1.T @ dh2, dh2.sum(0)
    dh1 = (dh2 @ q["W2"].T) * (h1 > 0)
    g["W1"], g["b1"] = X.T @ dh1, dh1.sum(0)
    g["in_scale"] = 0.0
    g["out_scale"] = 0.0
    return loss, pack(g)


def predict(p, X_raw):
    """Force in the point's frame for raw features (the network sees X * in_scale)."""
    q = unpack(p)
    Y, _, _ = forward(p, np.asarray(X_raw, dtype=np.float64) * q["in_scale"])
    return Y * q["out_scale"]


def features_2d(U_b, u_b_star, n_lag):
    """[npts][27] deficit stencils: for point k of each circle, U_b - u_b* at points
    k-4 .. k+4 (cyclic), as (normal, tangent, 0) in the frame of point k, whose normal
    is the direction of the point's angle 2 pi k / N_L."""
    d = np.asarray(U_b, dtype=np.float64) - np.asarray(u_b_star, dtype=np.float64)
    npts = d.shape[0]
    k = np.arange(npts) % n_lag
    base = np.arange(npts) - k
    th = 2.0 * np.pi * k / n_lag
    nx, ny = np.cos(th), np.sin(th)
    X = np.zeros((npts, N_IN))
    for j in range(9):
        kk = (k + j - 4) % n_lag
        dj = d[base + kk]
        X[:, 3 * j] = dj[:, 0] * nx + dj[:, 1] * ny
        X[:, 3 * j + 1] = -dj[:, 0] * ny + dj[:, 1] * nx
    return X


def sphere_stencil(ref):
    """Frame and neighbour order of every point of a sphere (3D reading of the learned
    initializer's stencil), from the point offsets ref [N_L][3] of the reference sphere:
      n = r_k / |r_k|;  t1 = (a x n) / |a x n| with a = e_z, or e_x where |n_z| >= 0.9;
      t2 = n x t1;
      neighbours: the 8 other points nearest to point k (distance |r_j - r_k|, ties by
      index), ordered by their azimuth atan2((r_j - r_k).t2, (r_j - r_k).t1) in [0, 2 pi)
      (ties by index).
    Distances and azimuths are compared after rounding to 1e-9, so ties resolve by index
    alike on any machine.  Returns (frames [N_L][3][3] rows n, t1, t2; nbr [N_L][8])."""
    r = np.asarray(ref, dtype=np.float64)
    nl = r.shape[0]
    n = r / np.linalg.norm(r, axis=1, keepdims=True)
    a = np.where(np.abs(n[:, 2:3]) < 0.9, np.array([[0.0, 0.0, 1.0]]), np.array([[1.0, 0.0, 0.0]]))
    t1 = np.cross(a, n)
    t1 /= np.linalg.norm(t1, axis=1, keepdims=True)
    t2 = np.cross(n, t1)
    frames = np.stack([n, t1, t2], axis=1)
    nbr = np.zeros((nl, 8), dtype=np.int64)
    idx = np.arange(nl)
    for k in range(nl):
        dist = np.round(np.linalg.norm(r - r[k], axis=1), 9)
        cand = [j for j in np.lexsort((idx, dist)) if j != k][:8]
        rel = r[cand] - r[k]
        az = np.mod(np.arctan2(rel @ t2[k], rel @ t1[k]), 2.0 * np.pi)
        order = np.lexsort((np.asarray(cand), np.round(az, 9)))
        nbr[k] = np.asarray(cand)[order]
    return frames, nbr


def features_3d(U_b, u_b_star, ref):
    """[npts][27] deficit stencils of spheres: for point k, U_b - u_b* at point k and at
    its 8 stencil neighbours (sphere_stencil order), each as (normal, t1, t2) components
    in the frame of point k."""
    d = np.asarray(U_b, dtype=np.float64) - np.asarray(u_b_star, dtype=np.float64)
    frames, nbr = sphere_stencil(ref)
    nl = frames.shape[0]
    npts = d.shape[0]
    k = np.arange(npts) % nl
    base = np.arange(npts) - k
    X = np.zeros((npts, N_IN))
    pts = np.concatenate([k[:, None], nbr[k]], axis=1)  # [npts][9]
    for j in range(9):
        dj = d[base + pts[:, j]]
        X[:, 3 * j:3 * j + 3] = np.einsum("pc,pac->pa", dj, frames[k])
    return X


def to_frame_3d(F, ref):
    """Per-point vectors F [npts][3] in the frame of their point (normal, t1, t2)."""
    frames, _ = sphere_stencil(ref)
    nl = frames.shape[0]
    k = np.arange(F.shape[0]) % nl
    return np.einsum("pc,pac->pa", np.asarray(F, dtype=np.float64), frames[k])
