"""Benchmark: whole IB-LBM time steps on the 2048 x 4096 D2Q9 cavity.

Workload: D2Q9 closed cavity 2048 x 4096, 10681 circles d = 10 (31 points each,
solid fraction 0.1), 4-point delta, drs = 2.6, 3 MDF iterations, density ratio 1.2,
gravity 1e-5, FP32 PDFs, FP64 particles; seeded synthetic placement (no dataset).
A step is one pass of the whole hot path: moments, MDF interpolation/spreading,
interior momentum, fused collide+stream, pair search + contacts, particle update.

Metric: MLUPS = N_grid * steps / (1e6 * seconds) (Eq. 52), whole job over all ranks,
for plain FP32 PDF storage with 3 MDF iterations (the headline) and for the chosen
form, FP16 storage of h = f / w with the learned first MDF force and 2 iterations, at
its stated error and its boundary-velocity residual (against the plain form's).  Also reported: the roofline of
the dominant kernel (lbm_step) against the measured HBM copy bandwidth, an
end-to-end number through the C ABI with host buffers, the FP64 CPU oracle timed
on a bounded sample on the host cores, the batched ensemble of 256 independent
cavities (aggregate MLUPS) and the 384 x 384 x 768 D3Q19 cavity with 20000 spheres.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
(N > 1: launch with torchrun; each rank runs an independent replica.)
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PHI = 0.1
WORKLOAD = "cavity2d_2048x4096_phi0.1"
METRIC = "MLUPS"


def _workload():
    from paper_2002_08855_gb300 import inputs
    return inputs.cavity_2d_large(PHI)


NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e, the vendor figure (context beside the measured peak)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _forced_nodes(w, Xb):
    """Nodes in the 4-point support of some Lagrangian point: the nodes where the IB
    force can be non-zero (Eq. 48), from the points' positions."""
    Xb = np.asarray(Xb)
    base = np.floor(Xb).astype(np.int64) - 1
    mask = np.zeros((w.ny, w.nx), dtype=bool)
    for sy in range(4):
        for sx in range(4):
            gx, gy = base[:, 0] + sx, base[:, 1] + sy
            ok = (gx >= 0) & (gx < w.nx) & (gy >= 0) & (gy < w.ny)
            mask[gy[ok], gx[ok]] = True
    return int(mask.sum())


def _kernel_hash():
    h = hashlib.sha256()
    for f in ("lbm.cu", "common.cuh", "pdf_access.cuh"):
        with open(os.path.join(ROOT, "paper_2002_08855_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _traffic(n_grid):
    """DRAM bytes per lbm_step launch from the committed ncu summary, scaled to this
    lattice, or None when the kernel changed since the counters were taken."""
    try:
        with open(os.path.join(ROOT, "profiles", "lbm_step_traffic.json")) as fh:
            d = json.load(fh)
        if d.get("kernel_hash") != _kernel_hash():
            return None
        return float(d["dram_bytes_per_node"]) * n_grid
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            with open(self.path) as fh:
                for line in fh:
                    p = [s.strip() for s in line.split(",")]
                    if len(p) >= 9 and p[1].replace(".", "").isdigit():
                        rows.append(p)
        except Exception:
            pass
        if self.path and os.path.exists(self.path):
            os.remove(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(rows[0][2]), "reasons": reasons,
                "samples": len(rows)}


def whole_job(ms_local, n_grid, steps, world, dist=None, device="cpu"):
    """Replicas only: every rank steps its own copy of the workload.  The job's time is
    the slowest rank's (max over ranks); its MLUPS count every rank's node updates."""
    import torch

    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    return ms_max, world * n_grid * steps / (1e3 * ms_max)


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _host_cpu():
    """(threads this process may use, the host CPU's model name)."""
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    model = "unknown"
    try:
        import subprocess
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return cores, model


def _oracle_rate(omp, seconds_target):
    """Whole-step MLUPS of the FP64 oracle on the 512 x 1024 sub-cavity at the workload's
    solid fraction, timed until about seconds_target have passed."""
    import oracle
    from paper_2002_08855_gb300 import inputs

    w = _workload()
    sw = w.with_(nx=512, ny=1024, n_particles=inputs.n_particles_for_fraction(2, 512 * 1024, w.diameter, PHI),
                 seed=w.seed + 50)
    X = inputs.place_particles(sw)
    sim = oracle.Sim(sw.as_dict(), X, omp=omp)
    sim.step(1)
    steps, t0 = 0, time.perf_counter()
    while True:
        sim.step(1)
        steps += 1
        el = time.perf_counter() - t0
        if el >= seconds_target or steps >= 400:
            break
    sim.close()
    sample = (f"{steps} whole steps of a 512x1024 sub-cavity, {sw.n_particles} particles "
              f"(same solid fraction and particle parameters), FP64, {el:.1f} s")
    return sw.n_grid * steps / (1e6 * el), sample


def cpu_baseline(seconds_target=12.0):
    """The FP64 oracle, as it stands, on a bounded sample of the workload (one 512 x 1024
    sub-cavity at the same solid fraction), single threaded; beside it the same oracle
    built with OpenMP on every host core (its parallel loops write disjoint data, so the
    two builds give identical bits)."""
    cores, model = _host_cpu()
    v1, sample1 = _oracle_rate(False, seconds_target)
    out = {"value": v1, "unit": METRIC, "cores": 1, "kind": "oracle", "sample": sample1,
           "host_cpu": model, "host_threads": cores}
    try:
        vn, samplen = _oracle_rate(True, 0.6 * seconds_target)
        out["all_cores"] = {"value": vn, "unit": METRIC, "cores": cores, "kind": "oracle (OpenMP build)",
                            "sample": samplen}
    except Exception as e:  # no OpenMP on the host
        out["all_cores"] = {"unavailable": str(e)[:200]}
    return out


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    from paper_2002_08855_gb300 import inputs

    w = _workload()
    sw = w.with_(nx=512, ny=1024, n_particles=inputs.n_particles_for_fraction(2, 512 * 1024, w.diameter, PHI),
                 seed=w.seed + 50)
    X = inputs.place_particles(sw)
    sim = oracle.Sim(sw.as_dict(), X)
    for _ in range(args.warmup):
        sim.step(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sim.step(1)
    el = time.perf_counter() - t0
    v = sw.n_grid * args.steps / (1e6 * el)
    cores, model = _host_cpu()
    sample = (f"{args.steps} whole FP64 oracle steps of a 512x1024 sub-cavity at the workload's "
              f"density, single threaded on {model} ({cores} threads available)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": METRIC, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "sample": "512x1024 sub-cavity"},
        "cpu_baseline": {"value": v, "unit": METRIC, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# Error of each PDF storage against the FP64 oracle on the 128 x 256 cavity with 12
# circles after 200 steps, as measured by tests/test_gpu_precision.py and
# tests/test_gpu_step.py on a GB300 (relative L2: velocity, pressure, displacement).
STATED_ERROR = {
    "fp32": {"velocity": 4.4e-6, "displacement": 2.7e-6},
    "fp16": {"velocity": 3.0e-4, "pressure": 5.0e-4, "displacement": 2.0e-5},
    "bf16": {"velocity": 2.4e-3, "pressure": 3.9e-3, "displacement": 1.8e-4},
}
# 3D cavity copy (48 x 48 x 96, 30 spheres of d = 12), relative L2 against the FP64
# oracle after 60 steps (tests/test_gpu_precision.py)
STATED_ERROR_3D = {
    "fp32": {"velocity": 1.2e-6, "pressure": 4.8e-6, "displacement": 5.0e-7, "F_h": 3.1e-6},
    "fp16": {"velocity": 1.9e-4, "pressure": 2.3e-4, "displacement": 5.9e-6, "F_h": 2.6e-4},
    "bf16": {"velocity": 1.3e-3, "pressure": 1.5e-3, "displacement": 5.4e-5, "F_h": 2.2e-3},
}


def _deviation_from_fp32(storage, dev):
    """Relative L2 difference between the FP32 path and the given storage after 200
    steps of the 128 x 256 cavity (measured live; the FP32 path itself is held to 1e-5
    against the FP64 oracle by the parity tests)."""
    from paper_2002_08855_gb300 import binding, inputs

    w = inputs.cavity_2d_small()
    X0 = inputs.place_particles(w)
    out = {}
    for st in (0, storage):
        sim = binding.Simulation(w.with_(pdf_storage=st), X0, device=str(dev))
        sim.step(200)
        sim.sync()
        p, u = sim.get_fields()
        out[st] = (p.cpu().numpy(), u.cpu().numpy(), sim.get_particles()["X"] - X0)
        sim.close()
    rel = lambda a, b: float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
    return {"velocity": rel(out[storage][1], out[0][1]), "pressure": rel(out[storage][0], out[0][0]),
            "displacement": rel(out[storage][2], out[0][2]), "case": "128x256 cavity, 12 circles, 200 steps"}


def _train_initializer(w, dev, steps=120, every=40):
    """The learned MDF initializer, trained on samples of the configuration w with
    another seed: 10 MDF iterations (converged forces), samples every `every` steps
    (2D headline: steps 40, 80, 120, about 1e6 points), 20 epochs of Adam on the GPU
    kernels."""
    import torch

    from paper_2002_08855_gb300 import binding, inputs, mlp

    t0 = time.perf_counter()
    wt = w.with_(seed=w.seed + 1000, mdf_iters=10)
    sim = binding.Simulation(wt, inputs.place_particles(wt), device=str(dev))
    Xs, Ys = [], []
    for t in range(steps):
        sim.step(1)
        if (t + 1) % every == 0:
            Xf, Yf = sim.mdf_samples()
            Xs.append(Xf)
            Ys.append(Yf)
    sim.close()
    Xf, Yf = torch.cat(Xs), torch.cat(Ys)
    t1 = time.perf_counter()
    params, losses = mlp.train(Xf, Yf, epochs=20, batch=4096, lr=2e-3, seed=3)
    info = {"samples": int(Xf.shape[0]), "collect_s": t1 - t0, "train_s": time.perf_counter() - t1,
            "loss_first_last_epoch": [losses[0], losses[-1]],
            "network": "27-64-64-3 ReLU, FP16 tensor-core inference (mma.sync), FP32 training kernels"}
    return params, info


def _form(args, w, X, dev, peak, peak_kind, local, name, storage=0, mdf_iters=3, params=None):
    """One form of the method on the workload: MLUPS, the lbm_step roofline and the
    boundary-velocity residual |U_b - D_I u^(M)| after the MDF (mean of 20 steps)."""
    import torch

    from paper_2002_08855_gb300 import binding

    wf = w.with_(pdf_storage=storage, mdf_iters=mdf_iters, mlp_init=1 if params is not None else 0)
    sim = binding.Simulation(wf, X, device=str(dev))
    if params is not None:
        sim.set_mlp(params)
    sim.step(args.warmup)
    sim.sync()
    torch.cuda.synchronize(dev)
    n0 = sim.launch_count()
    with ClockSampler(local) as clk:
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(sim.stream)
        sim.step(args.steps)
        ev1.record(sim.stream)
        ev1.synchronize()
        sim.sync()
    ms = ev0.elapsed_time(ev1) / args.steps
    launches = sim.launch_count() - n0
    nparts = max(3, min(args.steps, 50))
    parts = sim.time_parts(nparts)
    t_lbm = parts["collide_stream"] / nparts * 1e-3
    nforced = _forced_nodes(wf, sim.get_lagrangian()["X_b"])
    sim.set_residual_tracking(True)
    res = []
    for _ in range(20):
        sim.step(1)
        res.append(sim.mdf_residual()[0])
    sim.close()
    bytes_lbm = (72.0 if storage == 0 else 36.0) * wf.n_grid + 8.0 * nforced  # + f_IB read
    achieved = bytes_lbm / t_lbm / 1e9
    return {
        "form": name, "value": wf.n_grid / (ms * 1e3), "unit": METRIC, "ms_per_step": ms,
        "gpu_launches": launches, "mdf_iters": mdf_iters,
        "mdf_residual_rms": float(np.mean(res)),
        "roofline": {"bound": "hbm", "kernel": "lbm_step", "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                     "algorithmic_bytes": bytes_lbm, "ms_per_launch": t_lbm * 1e3},
        "parts_ms_per_step": {k: v / nparts for k, v in parts.items()},
        "clocks": clk.summary(),
    }


def _forms(args, w, X, dev, peak, peak_kind, local):
    """The plain FP32 form's residual (for comparison), FP16 storage, the learned first
    MDF force with one iteration fewer, and both together (the chosen form)."""
    params, info = _train_initializer(w, dev)
    plain = _form(args, w, X, dev, peak, peak_kind, local, "fp32, plain MDF, 3 iterations")
    fp16 = _form(args, w, X, dev, peak, peak_kind, local, "fp16 storage, plain MDF, 3 iterations", storage=1)
    fp16["stated_error_vs_oracle"] = STATED_ERROR["fp16"]
    fp16["deviation_from_fp32"] = _deviation_from_fp32(1, dev)
    learned = _form(args, w, X, dev, peak, peak_kind, local, "fp32, learned first force + 2 iterations",
                    mdf_iters=2, params=params)
    chosen = _form(args, w, X, dev, peak, peak_kind, local,
                   "fp16 storage, learned first force + 2 iterations", storage=1, mdf_iters=2, params=params)
    chosen["stated_error_vs_oracle"] = STATED_ERROR["fp16"]
    chosen["residual_vs_plain_fp32"] = chosen["mdf_residual_rms"] / plain["mdf_residual_rms"]
    chosen["learned_initializer"] = info
    return chosen, {"plain_fp32": plain, "fp16_storage": fp16, "learned_init": learned}


def _ensemble(args, dev, local):
    """The batched ensemble: 256 independent D2Q9 cavities (sides 64..512, 1..200
    circles of one diameter 8..16 per cavity, N_L = round(pi d)) stepped together with
    fused launches; aggregate MLUPS over all members."""
    import torch

    from paper_2002_08855_gb300 import binding, inputs

    ws = inputs.ensemble_2d()
    Xs = [inputs.place_particles(w) for w in ws]
    b = binding.Batch(ws, Xs, device=str(dev))
    b.step(args.warmup)
    # the autotuner picks the collide-stream tile shape on real steps (untimed), then
    # the steps after it capture new graphs
    chosen, shape_ms = b.autotune(4)
    b.step(3)
    b.sync()
    n0 = b.launch_count()
    with ClockSampler(local) as clk:
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(b.stream)
        b.step(args.steps)
        ev1.record(b.stream)
        ev1.synchronize()
        b.sync()
    ms = ev0.elapsed_time(ev1) / args.steps
    out = {"workload": "ensemble2d_256_cavities", "members": len(ws), "nodes": b.n_grid,
           "particles": int(sum(w.n_particles for w in ws)), "value": b.n_grid / (ms * 1e3),
           "unit": METRIC, "ms_per_step": ms, "gpu_launches_per_step": (b.launch_count() - n0) / args.steps,
           "pdf_storage": "fp32", "clocks": clk.summary(),
           "tile_shape": {"chosen": chosen, "nodes_per_thread_warps_persistent": binding.tile_shapes(0)[chosen],
                          "collide_stream_ms_per_shape": shape_ms}}
    b.close()
    return out


def _cavity3d(args, dev, local):
    """The D3Q19 cavity 384 x 384 x 768 with 20000 spheres (d = 12, 452 points), FP32
    and FP16 storage: MLUPS over min(steps, 20) timed steps."""
    import torch

    from paper_2002_08855_gb300 import binding, inputs

    w = inputs.cavity_3d(1)
    X = inputs.place_particles(w)
    steps = max(3, min(args.steps, 20))
    out = {"workload": w.name, "lattice": "D3Q19 384x384x768", "particles": w.n_particles,
           "points_per_particle": w.n_lag, "steps": steps}
    # learned initializer for spheres: trained on the 96 x 96 x 192 copy (same solid
    # fraction, another seed), 10 MDF iterations for converged forces
    wt = inputs.cavity_3d(4)
    params, info = _train_initializer(wt, dev, steps=60, every=20)
    out["learned_initializer"] = info
    forms = ((0, "fp32", 3, None), (1, "fp16", 3, None), (0, "fp32_learned_m2", 2, params),
             (1, "fp16_learned_m2", 2, params))
    for st, name, M, p in forms:
        sim = binding.Simulation(w.with_(pdf_storage=st, mdf_iters=M, mlp_init=int(p is not None)), X,
                                 device=str(dev))
        if p is not None:
            sim.set_mlp(p)
        sim.step(3)
        sim.sync()
        with ClockSampler(local) as clk:
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(sim.stream)
            sim.step(steps)
            ev1.record(sim.stream)
            ev1.synchronize()
            sim.sync()
        ms = ev0.elapsed_time(ev1) / steps
        parts = sim.time_parts(3)
        sim.set_residual_tracking(True)
        res = []
        for _ in range(3):
            sim.step(1)
            res.append(sim.mdf_residual()[0])
        sim.close()
        out[name] = {"value": w.n_grid / (ms * 1e3), "unit": METRIC, "ms_per_step": ms, "mdf_iters": M,
                     "mdf_residual_rms": float(np.mean(res)),
                     "parts_ms_per_step": {k: v / 3 for k, v in parts.items()}, "clocks": clk.summary()}
    out["learned_m2_residual_vs_plain_m3"] = out["fp32_learned_m2"]["mdf_residual_rms"] / out["fp32"]["mdf_residual_rms"]
    out["stated_error_vs_oracle"] = STATED_ERROR_3D
    return out


def _sec62_point(dev, w, steps=20, reps=5):
    """One point of the Sec. 6.2 sweeps: MLUPS over `steps` graph-replayed steps, the
    part times per step, mesh ratio eta = N_p N_L / N_grid and solid fraction."""
    import torch

    from paper_2002_08855_gb300 import binding, inputs

    X = inputs.place_particles(w)
    sim = binding.Simulation(w, X, device=str(dev))
    sim.step(3)
    sim.sync()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(sim.stream)
    sim.step(steps)
    ev1.record(sim.stream)
    ev1.synchronize()
    sim.sync()
    ms = ev0.elapsed_time(ev1) / steps
    parts = sim.time_parts(reps)
    sim.close()
    vp = math.pi * w.diameter ** 2 / 4.0 if w.dim == 2 else math.pi * w.diameter ** 3 / 6.0
    return {"n_grid": w.n_grid, "n_particles": w.n_particles, "diameter": w.diameter, "n_lag": w.n_lag,
            "eta": w.n_particles * w.n_lag / w.n_grid, "solid_fraction": w.n_particles * vp / w.n_grid,
            "mlups": w.n_grid / (ms * 1e3), "ms_per_step": ms,
            "parts_ms_per_step": {k: v / reps for k, v in parts.items()}}


SEED_SWEEP = 2002085500 + 7000  # seeds of the sweep workloads (input-generator base + 7000)


def sweep(args):
    """The two series of Sec. 6.2 (settling particles, density ratio 1.01, 3-point
    delta with drs = 1.9, walls by non-equilibrium extrapolation): particle count at a
    fixed lattice (6.2.1, Table 7: 2048^2 with d = 16, 150^3 with d = 12) and particle
    resolution at fixed solid fraction (6.2.2: 40 d x 40 d with d = 12..48, (5 d)^3 with
    d = 12..30); N_L = round(pi d) in 2D and round(pi d^2) in 3D (point spacing about
    one lattice unit).  Prints one JSON line."""
    import torch

    from paper_2002_08855_gb300 import build
    from paper_2002_08855_gb300.inputs import Workload

    build.build()
    dev = torch.device("cuda", 0)
    base = dict(tau=0.6, delta_kind=3, drs=1.9, density_ratio=1.01, boundary=1, mdf_iters=3)
    out = {"settings": "Sec. 6.2: density ratio 1.01, 3-point delta, drs 1.9, extrapolation walls, M = 3, tau 0.6",
           "count_2d": [], "count_3d": [], "resolution_2d": [], "resolution_3d": []}
    for n in (1, 10, 100, 1000, 4000, 10000):
        w = Workload(name=f"c2_{n}", dim=2, nx=2048, ny=2048, n_particles=n, n_lag=50, diameter=16.0,
                     gravity=(0.0, -1e-4, 0.0), seed=SEED_SWEEP + n, **base)
        out["count_2d"].append(_sec62_point(dev, w))
    for n in (1, 10, 100, 300, 500):
        w = Workload(name=f"c3_{n}", dim=3, nx=150, ny=150, nz=150, n_particles=n, n_lag=452, diameter=12.0,
                     gravity=(0.0, -1e-4, 0.0), seed=SEED_SWEEP + 100 + n, **base)
        out["count_3d"].append(_sec62_point(dev, w))
    for d in (12, 18, 24, 36, 48):
        w = Workload(name=f"r2_{d}", dim=2, nx=40 * d, ny=40 * d, n_particles=400, n_lag=int(round(math.pi * d)),
                     diameter=float(d), gravity=(0.0, -1e-4, 0.0), seed=SEED_SWEEP + 200 + d, **base)
        out["resolution_2d"].append(_sec62_point(dev, w))
    for d in (12, 18, 24, 30):
        w = Workload(name=f"r3_{d}", dim=3, nx=5 * d, ny=5 * d, nz=5 * d, n_particles=20,
                     n_lag=int(round(math.pi * d * d)), diameter=float(d), gravity=(0.0, -1e-4, 0.0),
                     seed=SEED_SWEEP + 300 + d, **base)
        out["resolution_3d"].append(_sec62_point(dev, w, steps=10, reps=3))
    print(json.dumps({"sweep": out}))


def _pair_search_modes(dev, w2, X2):
    """Pair search and contact part (cell lists against the grid search of Table 5) of
    the headline workload and of the 3D cavity, as the part timer measures it (the
    contact search, Eq. 16 forces and the particle update, run on their own)."""
    from paper_2002_08855_gb300 import binding, inputs

    w3 = inputs.cavity_3d(1)
    X3 = inputs.place_particles(w3)
    out = {}
    for name, w, X, reps in (("2d_headline", w2, X2, 20), ("3d_cavity", w3, X3, 3)):
        out[name] = {}
        for mode, mname in ((0, "cell_lists"), (1, "grid_search")):
            sim = binding.Simulation(w.with_(pair_search=mode), X, device=str(dev))
            sim.step(3)
            sim.sync()
            parts = sim.time_parts(reps)
            n_pairs = len(sim.get_pairs())
            sim.close()
            out[name][mname] = {"pairs_ms_per_step": parts["pairs"] / reps, "pairs": n_pairs}
    return out


def _cavity2d_series(args, dev, local):
    """The other configurations of the 2048 x 4096 cavity (solid fraction 0, 0.2, 0.4:
    0, 21361, 42723 circles; FP32 and FP16 storage) and the 128 x 256 cavity (12
    circles of d = 16, a latency case that fits in L2): ms and MLUPS per step over
    min(steps, 100) graph-replayed steps."""
    import torch

    from paper_2002_08855_gb300 import binding, inputs

    steps = max(3, min(args.steps, 100))
    out = {"steps": steps}
    cases = [(f"2048x4096_phi{phi}", inputs.cavity_2d_large(phi)) for phi in (0.0, 0.2, 0.4)]
    cases.append(("128x256_12_circles", inputs.cavity_2d_small()))
    for name, w in cases:
        X = inputs.place_particles(w)
        out[name] = {"particles": w.n_particles}
        for st, sname in ((0, "fp32"), (1, "fp16")):
            sim = binding.Simulation(w.with_(pdf_storage=st), X, device=str(dev))
            sim.step(3)
            sim.sync()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(sim.stream)
            sim.step(steps)
            ev1.record(sim.stream)
            ev1.synchronize()
            sim.sync()
            sim.close()
            ms = ev0.elapsed_time(ev1) / steps
            out[name][sname] = {"value": w.n_grid / (ms * 1e3), "unit": METRIC, "ms_per_step": ms}
    return out


def run(args):
    import torch

    from paper_2002_08855_gb300 import binding, build

    world, rank, local = _dist()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    w = _workload()
    X = None
    from paper_2002_08855_gb300 import inputs
    X = inputs.place_particles(w)
    base = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        base = cpu_baseline()

    sim = binding.Simulation(w, X, device=str(dev))
    stream = sim.stream

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    # warm-up (the first step is eager; graphs are captured on the next two)
    sim.step(args.warmup)
    sim.sync()

    # timed region: K whole steps, device time with events on the run's stream
    launches0 = sim.launch_count()
    barrier()
    with ClockSampler(local) as clk:
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        sim.step(args.steps)
        ev1.record(stream)
        ev1.synchronize()
        sim.sync()
    barrier()
    ms = ev0.elapsed_time(ev1)
    launches = sim.launch_count() - launches0
    clocks = clk.summary()
    ms_max, mlups = whole_job(ms, w.n_grid, args.steps, world, dist, dev)

    # per-part device times (eager launches, CUDA events on the same stream)
    parts = sim.time_parts(max(3, min(args.steps, 50)))
    nparts = max(3, min(args.steps, 50))
    t_lbm = parts["collide_stream"] / nparts * 1e-3
    nforced = _forced_nodes(w, sim.get_lagrangian()["X_b"])
    # the method's bytes: PDFs read + written, the IB force read on the forced nodes
    # (its clear, and the read of zeros elsewhere, are traffic beyond them)
    bytes_lbm = 72.0 * w.n_grid + 8.0 * nforced
    peak, peak_kind = _peaks()
    achieved = bytes_lbm / t_lbm / 1e9
    traffic = _traffic(w.n_grid)

    # the other forms of the method on the same workload and the chosen one
    chosen, forms = _forms(args, w, X, dev, peak, peak_kind, local)
    # the batched ensemble of independent cavities, and the 3D cavity
    ensemble = _ensemble(args, dev, local)
    cavity3d = _cavity3d(args, dev, local)
    pair_modes = _pair_search_modes(dev, w, X)
    series2d = _cavity2d_series(args, dev, local)

    # end to end through the C ABI with host buffers: init from host centres, then per
    # step one ibm_lbm_step and a read of the particle state into pinned host memory
    sim.close()
    del sim
    torch.cuda.synchronize(dev)
    pin_x = torch.empty((w.n_particles, 2), dtype=torch.float64, pin_memory=True).numpy()
    pin_u = torch.empty((w.n_particles, 2), dtype=torch.float64, pin_memory=True).numpy()
    centres = torch.from_numpy(np.ascontiguousarray(X)).pin_memory().numpy()
    e2e_steps = max(args.steps // 2, 3)
    barrier()
    t0 = time.perf_counter()
    sim2 = binding.Simulation(w, centres, device=str(dev))
    for _ in range(e2e_steps):
        sim2.step(1)
        import ctypes as C
        binding._check(binding.lib().ibm_lbm_get_particles(
            sim2.h, binding._ptr(pin_x, C.c_double), binding._ptr(pin_u, C.c_double), None, None,
            None, None), "get_particles")
    sim2.sync()
    barrier()
    e2e_s = time.perf_counter() - t0
    sim2.close()
    e2e = world * w.n_grid * e2e_steps / (1e6 * e2e_s)

    if rank == 0:
        line = {
            "metric": METRIC, "value": mlups, "unit": METRIC, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "lattice": "D2Q9 2048x4096", "particles": w.n_particles,
                       "points_per_particle": w.n_lag, "mdf_iters": w.mdf_iters,
                       "pdf_storage": "fp32", "parallelism": f"replicas{world}" if world > 1 else "single",
                       "l2": "inputs larger than L2 (302 MB of PDFs per step)"},
            "roofline": {"bound": "hbm", "kernel": "lbm_step", "achieved": achieved, "peak": peak,
                         "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": traffic, "algorithmic_bytes": bytes_lbm,
                         "forced_nodes": nforced, "ms_per_launch": t_lbm * 1e3,
                         "peak_nominal": NOMINAL_HBM_GBS, "frac_nominal": achieved / NOMINAL_HBM_GBS},
            "parts_ms_per_step": {k: v / nparts for k, v in parts.items()},
            "clocks": clocks, "gpu_launches": launches,
            "e2e": {"value": e2e, "unit": METRIC, "h2d_bytes_per_step": int(X.nbytes / e2e_steps),
                    "d2h_bytes_per_step": int(pin_x.nbytes + pin_u.nbytes)},
            "cpu_baseline": base,
            "chosen_form": chosen,
            "forms": forms,
            "ensemble": ensemble,
            "cavity3d": cavity3d,
            "pair_search": pair_modes,
            "cavity2d_series": series2d,
        }
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sweep", action="store_true",
                    help="run the Sec. 6.2 particle-count and resolution sweeps instead")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.sweep:
        sweep(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run(args)


if __name__ == "__main__":
    main()
