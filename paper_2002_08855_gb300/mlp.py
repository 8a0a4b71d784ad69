"""Training of the learned MDF initializer on the GPU (argument marshalling and the
optimisation loop; every forward, backward and update runs in the library's kernels).

The samples come from the method itself: runs with many MDF iterations give, per
Lagrangian point, the deficit stencil of the first iteration and the converged total
force (ibm_lbm_mdf_samples)."""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import binding
from .binding import _check, lib
from .inputs import SplitMix64

N_IN, N_H, N_OUT = 27, 64, 3


def init_params(seed: int) -> np.ndarray:
    """He-normal weights (Box-Muller on a SplitMix64 stream), zero biases, unit scales."""
    rng = SplitMix64(seed)

    def normal(n):
        u = np.array([rng.uniform() for _ in range(2 * ((n + 1) // 2))])
        u1, u2 = np.maximum(u[0::2], 1e-300), u[1::2]
        z = np.sqrt(-2.0 * np.log(u1))
        return np.concatenate([z * np.cos(2 * np.pi * u2), z * np.sin(2 * np.pi * u2)])[:n]

    parts = [normal(N_IN * N_H) * np.sqrt(2.0 / N_IN), np.zeros(N_H),
             normal(N_H * N_H) * np.sqrt(2.0 / N_H), np.zeros(N_H),
             normal(N_H * N_OUT) * np.sqrt(2.0 / N_H), np.zeros(N_OUT), [1.0], [1.0]]
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == lib().ibm_lbm_mlp_param_count()
    return p


def collect_samples(workloads, centres, steps, every: int = 1, mdf_iters: int = 10):
    """Run each workload with mdf_iters iterations (converged forces) and gather the
    samples of every `every`-th step; returns CUDA tensors (X [n][27], Y [n][3])."""
    import torch

    Xs, Ys = [], []
    for w, X0 in zip(workloads, centres):
        sim = binding.Simulation(w.with_(mdf_iters=mdf_iters, mlp_init=0), X0)
        for t in range(steps):
            sim.step(1)
            if (t + 1) % every == 0:
                X, Y = sim.mdf_samples()
                Xs.append(X)
                Ys.append(Y)
        sim.close()
    return torch.cat(Xs), torch.cat(Ys)


def train(X, Y, epochs: int = 20, batch: int = 4096, lr: float = 2e-3, seed: int = 7, stream=None,
          params=None):
    """Adam on the mean squared error of the scaled targets.  X, Y: CUDA float tensors.
    Sets in_scale = 1 / RMS(X) and out_scale = RMS(Y).  Returns (params, losses per
    epoch)."""
    import torch

    dev = X.device
    s = stream if stream is not None else torch.cuda.Stream(dev)
    p = init_params(seed) if params is None else np.asarray(params, dtype=np.float32).copy()
    in_scale = float(1.0 / max(X.pow(2).mean().sqrt().item(), 1e-30))
    out_scale = float(max(Y.pow(2).mean().sqrt().item(), 1e-30))
    p[-2], p[-1] = in_scale, out_scale
    Xs = (X * in_scale).contiguous()
    Ys = (Y / out_scale).contiguous()
    P = torch.from_numpy(p).to(dev)
    G, M, V = (torch.zeros_like(P) for _ in range(3))
    sz = C.c_size_t(0)
    _check(lib().ibm_lbm_mlp_scratch_size(batch, C.byref(sz)), "mlp_scratch_size")
    scratch = torch.empty(sz.value, dtype=torch.uint8, device=dev)
    n = Xs.shape[0]
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    losses, t = [], 0
    s.wait_stream(torch.cuda.current_stream(dev))
    for ep in range(epochs):
        perm = torch.from_numpy(rng.permutation(n)).to(dev)
        Xp, Yp = Xs[perm].contiguous(), Ys[perm].contiguous()
        s.wait_stream(torch.cuda.current_stream(dev))
        tot, nb = 0.0, 0
        for b0 in range(0, n - batch + 1, batch):
            loss = C.c_double(0)
            _check(lib().ibm_lbm_mlp_grad(C.c_void_p(P.data_ptr()), C.c_void_p(Xp[b0:].data_ptr()),
                                          C.c_void_p(Yp[b0:].data_ptr()), batch, C.c_void_p(G.data_ptr()),
                                          C.byref(loss), C.c_void_p(scratch.data_ptr()), sz.value,
                                          C.c_void_p(s.cuda_stream)), "mlp_grad")
            t += 1
            _check(lib().ibm_lbm_mlp_adam(C.c_void_p(P.data_ptr()), C.c_void_p(G.data_ptr()),
                                          C.c_void_p(M.data_ptr()), C.c_void_p(V.data_ptr()), t, lr,
                                          C.c_void_p(s.cuda_stream)), "mlp_adam")
            tot += loss.value
            nb += 1
        losses.append(tot / max(nb, 1))
    s.synchronize()
    return P.cpu().numpy(), losses


def infer(params, X):
    """Tensor-core inference of raw feature rows (CUDA tensor) -> [n][3] CUDA tensor."""
    import torch

    P = torch.from_numpy(np.asarray(params, dtype=np.float32)).to(X.device)
    Xc = X.contiguous()
    Y = torch.empty((Xc.shape[0], N_OUT), dtype=torch.float32, device=X.device)
    s = torch.cuda.current_stream(X.device)
    _check(lib().ibm_lbm_mlp_infer(C.c_void_p(P.data_ptr()), C.c_void_p(Xc.data_ptr()), Xc.shape[0],
                                   C.c_void_p(Y.data_ptr()), C.c_void_p(s.cuda_stream)), "mlp_infer")
    s.synchronize()
    return Y
