"""Seeded synthetic inputs shared by the CUDA path and the oracle.

This module holds none of the method's arithmetic: it only draws numbers
(SplitMix64 streams), places non-overlapping particle centres and describes the
workloads (lattice sizes, fluid and particle parameters).  Both sides receive
the same arrays from here and compute everything else on their own.

The paper has no public dataset: its particle-laden runs place particles at
random non-overlapping positions in closed cavities of rest fluid (Sec. 6.2,
Table 7).  The workloads below follow that recipe at the sizes of the
benchmark configurations.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

_MASK64 = (1 << 64) - 1
SEED_BASE = 2002085500


class SplitMix64:
    """SplitMix64 (Steele, Lea & Flood 2014): counter-based 64-bit generator."""

    def __init__(self, seed: int):
        self.state = seed & _MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def randint(self, n: int) -> int:
        return self.next_u64() % n


@dataclass
class Workload:
    """Problem statement of one run (all lengths in lattice units, dh = dt = 1)."""

    name: str
    dim: int
    nx: int
    ny: int
    nz: int = 1
    periodic: tuple = (0, 0, 0)
    tau: float = 0.6
    body_force: tuple = (0.0, 0.0, 0.0)
    n_particles: int = 0
    n_lag: int = 0
    diameter: float = 0.0
    delta_kind: int = 4
    drs: float = 2.6
    mdf_iters: int = 3
    density_ratio: float = 1.5
    gravity: tuple = (0.0, 0.0, 0.0)
    zeta: float = 2.0
    eps_pp: float = 1e-2
    E_pp: float = 1e-4
    fixed_particles: int = 0
    boundary: int = 0     # 0 halfway bounce-back, 1 extrapolation walls, 2 extrapolation channel
    u_inlet: float = 0.0  # peak inlet velocity of the channel (boundary 2)
    pair_search: int = 0  # 0 cell lists, 1 grid search (Table 5) (GPU; same pairs)
    pdf_storage: int = 0  # 0 FP32, 1 FP16, 2 BF16 (GPU storage of the PDFs only)
    mlp_init: int = 0     # 1: learned first MDF force (GPU, 2D)
    steps: int = 100
    seed: int = SEED_BASE
    centres: np.ndarray | None = field(default=None, repr=False)

    @property
    def n_grid(self) -> int:
        return self.nx * self.ny * (self.nz if self.dim == 3 else 1)

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k in (
            "dim", "nx", "ny", "nz", "periodic", "tau", "body_force", "n_particles", "n_lag",
            "diameter", "delta_kind", "drs", "mdf_iters", "density_ratio", "gravity", "zeta",
            "eps_pp", "E_pp", "fixed_particles", "boundary", "u_inlet", "pair_search", "pdf_storage", "mlp_init")}
        if self.dim == 2:
            d["nz"] = 1
        return d


def place_rsa(dim: int, shape, n: int, diameter: float, seed: int, gap: float = 2.0,
              wall_gap: float = 2.0, max_tries: int = 2000) -> np.ndarray:
    """Random sequential addition of n centres, pairwise distance >= D + gap and at
    least wall_gap between a surface and a wall (walls at -1/2 and n-1/2)."""
    rng = SplitMix64(seed)
    R = 0.5 * diameter
    lo = [-0.5 + R + wall_gap for _ in range(dim)]
    hi = [float(shape[k]) - 0.5 - R - wall_gap for k in range(dim)]
    if any(h <= l for l, h in zip(lo, hi)) and n > 0:
        raise ValueError("domain too small for the particle size")
    dmin = diameter + gap
    cell = dmin
    ncell = [max(1, int(math.ceil((hi[k] - lo[k]) / cell)) + 1) for k in range(dim)]
    grid: dict = {}
    out = np.zeros((n, dim))
    for i in range(n):
        for _ in range(max_tries):
            p = [lo[k] + (hi[k] - lo[k]) * rng.uniform() for k in range(dim)]
            c = tuple(int((p[k] - lo[k]) / cell) for k in range(dim))
            ok = True
            rngs = [range(max(0, c[k] - 1), min(ncell[k], c[k] + 2)) for k in range(dim)]
            for cc in np.ndindex(*[len(r) for r in rngs]):
                key = tuple(rngs[k][cc[k]] for k in range(dim))
                for j in grid.get(key, ()):
                    d2 = sum((p[k] - out[j, k]) ** 2 for k in range(dim))
                    if d2 < dmin * dmin:
                        ok = False
                        break
                if not ok:
                    break
            if ok:
                out[i] = p
                grid.setdefault(c, []).append(i)
                break
        else:
            raise RuntimeError(f"random sequential addition stalled at particle {i} of {n}")
    return out


def place_hex(shape, n: int, diameter: float, seed: int, gap: float = 2.0,
              wall_gap: float = 2.0) -> np.ndarray:
    """2D dense packing: a jittered hexagonal lattice thinned at random to n sites.
    Pairwise distance stays >= D + gap (jitter radius is half the spare spacing)."""
    rng = SplitMix64(seed)
    R = 0.5 * diameter
    lo = [-0.5 + R + wall_gap] * 2
    hi = [float(shape[k]) - 0.5 - R - wall_gap for k in range(2)]
    dmin = diameter + gap

    def sites(a):
        pts = []
        dy = a * math.sqrt(3.0) / 2.0
        j = 0
        y = lo[1]
        while y <= hi[1]:
            x = lo[0] + (0.5 * a if j % 2 else 0.0)
            while x <= hi[0]:
                pts.append((x, y))
                x += a
            y += dy
            j += 1
        return pts

    area = (hi[0] - lo[0]) * (hi[1] - lo[1])
    a = 1.05 * math.sqrt(2.0 * area / (math.sqrt(3.0) * max(n, 1)))  # spacing for n sites
    while len(sites(a)) < n:
        a *= 0.995
        if a < dmin:
            raise ValueError("solid fraction too high for the hexagonal packing")
    pts = sites(a)
    jitter = 0.5 * (a - dmin)
    order = list(range(len(pts)))
    for i in range(len(order) - 1, 0, -1):  # Fisher-Yates with the seeded stream
        j = rng.randint(i + 1)
        order[i], order[j] = order[j], order[i]
    out = np.zeros((n, 2))
    for t, s in enumerate(sorted(order[:n])):
        r = jitter * math.sqrt(rng.uniform())
        th = 2.0 * math.pi * rng.uniform()
        x = min(max(pts[s][0] + r * math.cos(th), lo[0]), hi[0])
        y = min(max(pts[s][1] + r * math.sin(th), lo[1]), hi[1])
        out[t] = (x, y)
    return out


def place_particles(w: Workload) -> np.ndarray:
    """Seeded non-overlapping centres for a workload (RSA below 0.3 solid fraction,
    jittered hexagonal packing above, as RSA cannot reach 0.4 with the contact gap)."""
    if w.n_particles == 0:
        return np.zeros((0, w.dim))
    shape = (w.nx, w.ny, w.nz)[: w.dim]
    vp = math.pi * w.diameter ** 2 / 4.0 if w.dim == 2 else math.pi * w.diameter ** 3 / 6.0
    phi = w.n_particles * vp / w.n_grid
    if w.dim == 2 and phi >= 0.3:
        return place_hex(shape, w.n_particles, w.diameter, w.seed)
    return place_rsa(w.dim, shape, w.n_particles, w.diameter, w.seed)


def with_centres(w: Workload) -> Workload:
    return w.with_(centres=place_particles(w))


def n_particles_for_fraction(dim: int, n_grid: int, diameter: float, phi: float) -> int:
    vp = math.pi * diameter ** 2 / 4.0 if dim == 2 else math.pi * diameter ** 3 / 6.0
    return int(round(phi * n_grid / vp))


# ---------------------------------------------------------------- workloads
def cavity_2d_small() -> Workload:
    """D2Q9 closed cavity 128 x 256, 12 circles d = 16 (50 points), 4-point delta,
    drs = 2.6, 3 MDF iterations, density ratio 1.5, gravity 1e-5, 500 steps."""
    return Workload(name="cavity2d_128x256_np12", dim=2, nx=128, ny=256, tau=0.6,
                    n_particles=12, n_lag=50, diameter=16.0, delta_kind=4, drs=2.6,
                    mdf_iters=3, density_ratio=1.5, gravity=(0.0, -1e-5, 0.0), steps=500,
                    seed=SEED_BASE + 100)


def cavity_2d_large(phi: float = 0.1) -> Workload:
    """D2Q9 closed cavity 2048 x 4096, circles d = 10 (31 points), density ratio 1.2,
    solid fraction phi in {0, 0.1, 0.2, 0.4}, 2000 steps."""
    nx, ny, d = 2048, 4096, 10.0
    n = n_particles_for_fraction(2, nx * ny, d, phi)
    sweep = {0.0: 0, 0.1: 1, 0.2: 2, 0.4: 3}.get(round(phi, 3), 9)
    return Workload(name=f"cavity2d_2048x4096_phi{phi:g}", dim=2, nx=nx, ny=ny, tau=0.6,
                    n_particles=n, n_lag=31, diameter=d, delta_kind=4, drs=2.6, mdf_iters=3,
                    density_ratio=1.2, gravity=(0.0, -1e-5, 0.0), steps=2000,
                    seed=SEED_BASE + 200 + sweep)


def cavity_3d(scale: int = 1) -> Workload:
    """D3Q19 closed cavity 384 x 384 x 768 (z vertical), 20000 spheres d = 12 with 452
    Fibonacci points, density ratio 1.5, gravity along -z, 1000 steps.  scale = 4 gives
    the 96 x 96 x 192 copy with the same solid fraction."""
    nx, ny, nz = 384 // scale, 384 // scale, 768 // scale
    n = int(round(20000 / scale ** 3))
    return Workload(name=f"cavity3d_{nx}x{ny}x{nz}_np{n}", dim=3, nx=nx, ny=ny, nz=nz,
                    tau=0.6, n_particles=n, n_lag=452, diameter=12.0, delta_kind=4, drs=2.6,
                    mdf_iters=3, density_ratio=1.5, gravity=(0.0, 0.0, -1e-5), steps=1000,
                    seed=SEED_BASE + 300 + scale)


def ensemble_2d(n: int = 256, seed: int = SEED_BASE + 500, side=(64, 512), diam=(8.0, 16.0),
                max_particles: int = 200, phi_max: float = 0.3) -> list:
    """Batched ensemble: n independent D2Q9 closed cavities, sides uniform integers in
    [side], per cavity one diameter uniform in [diam] with N_L = round(pi d) points and
    a particle count uniform in 1..max_particles, capped at solid fraction phi_max;
    density ratio 1.5, tau = 0.6, gravity 1e-5, 3 MDF iterations, 1000 steps."""
    rng = SplitMix64(seed)
    out = []
    for c in range(n):
        nx = side[0] + rng.randint(side[1] - side[0] + 1)
        ny = side[0] + rng.randint(side[1] - side[0] + 1)
        d = diam[0] + (diam[1] - diam[0]) * rng.uniform()
        cap = int(phi_max * nx * ny / (math.pi * d * d / 4.0))
        npart = max(1, min(1 + rng.randint(max_particles), cap))
        out.append(Workload(name=f"ens{c}_{nx}x{ny}_np{npart}", dim=2, nx=nx, ny=ny, tau=0.6,
                            n_particles=npart, n_lag=int(round(math.pi * d)), diameter=d,
                            delta_kind=4, drs=2.6, mdf_iters=3, density_ratio=1.5,
                            gravity=(0.0, -1e-5, 0.0), steps=1000, seed=seed + 1 + c))
    return out


def random_pdfs(q: int, n: int, seed: int, scale: float = 1e-2) -> np.ndarray:
    """[q][n] float32 PDFs drawn uniformly in [-scale, scale) (deviation gauge)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return (scale * (2.0 * rng.random((q, n)) - 1.0)).astype(np.float32)


def random_points(n: int, dim: int, lo, hi, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    lo, hi = np.asarray(lo, float), np.asarray(hi, float)
    return lo + (hi - lo) * rng.random((n, dim))
