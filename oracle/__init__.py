"""FP64 CPU oracle for the IB-LBM hot path — TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its binding) never does: the two share no code, and they meet only through the
seeded inputs of ``paper_2002_08855_gb300.inputs``.

The arithmetic lives in ``ibmlbm_oracle.c`` (plain C, double precision, general
loops in the paper's order and notation; see the header of that file for the
readings of the paper it uses).  This module compiles it with gcc and exposes
numpy-friendly wrappers through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ibmlbm_oracle.c")
_HDR = os.path.join(_HERE, "ibmlbm_oracle.h")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_OUT_OMP = os.path.join(_HERE, "_build", "liboracle_omp.so")
_lock = threading.Lock()
_libs = {}


def build(force: bool = False, omp: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (no fused multiply-add);
    omp: the same source with -fopenmp (``liboracle_omp.so``), whose parallel loops
    write disjoint data, so it gives the same bits on all host cores."""
    out = _OUT_OMP if omp else _OUT
    os.makedirs(os.path.dirname(out), exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(out) or os.path.getmtime(out) < newest:
        tmp = out + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               *(["-fopenmp"] if omp else []), "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)
    return out


class Params(C.Structure):
    """Mirror of ``or_params`` (problem statement: lattice, fluid, particles)."""

    _fields_ = [
        ("dim", C.c_int32), ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
        ("periodic", C.c_int32 * 3), ("tau", C.c_double), ("body_force", C.c_double * 3),
        ("n_particles", C.c_int32), ("n_lag", C.c_int32), ("diameter", C.c_double),
        ("delta_kind", C.c_int32), ("drs", C.c_double), ("mdf_iters", C.c_int32),
        ("density_ratio", C.c_double), ("gravity", C.c_double * 3),
        ("zeta", C.c_double), ("eps_pp", C.c_double), ("E_pp", C.c_double),
        ("fixed_particles", C.c_int32), ("boundary", C.c_int32), ("u_inlet", C.c_double),
    ]


def make_params(cfg) -> Params:
    """Build ``or_params`` from a workload description (dict or object with attributes)."""
    get = cfg.get if isinstance(cfg, dict) else (lambda k, d=None: getattr(cfg, k, d))
    P = Params()
    P.dim = int(get("dim", 2))
    P.nx, P.ny = int(get("nx")), int(get("ny"))
    P.nz = int(get("nz", 1)) if P.dim == 3 else 1
    per = list(get("periodic", (0, 0, 0))) + [0, 0, 0]
    for k in range(3):
        P.periodic[k] = int(per[k])
    P.tau = float(get("tau", 0.6))
    bf = list(get("body_force", (0.0, 0.0, 0.0))) + [0.0, 0.0, 0.0]
    for k in range(3):
        P.body_force[k] = float(bf[k])
    P.n_particles = int(get("n_particles", 0))
    P.n_lag = int(get("n_lag", 0))
    P.diameter = float(get("diameter", 0.0))
    P.delta_kind = int(get("delta_kind", 4))
    P.drs = float(get("drs", 2.6))
    P.mdf_iters = int(get("mdf_iters", 3))
    P.density_ratio = float(get("density_ratio", 1.5))
    g = list(get("gravity", (0.0, 0.0, 0.0))) + [0.0, 0.0, 0.0]
    for k in range(3):
        P.gravity[k] = float(g[k])
    P.zeta = float(get("zeta", 2.0))
    P.eps_pp = float(get("eps_pp", 1e-2))
    P.E_pp = float(get("E_pp", 1e-4))
    P.fixed_particles = int(get("fixed_particles", 0))
    P.boundary = int(get("boundary", 0))
    P.u_inlet = float(get("u_inlet", 0.0))
    return P


_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_PP = C.POINTER(Params)


def lib(omp: bool = False):
    """Load (building first if needed) the oracle shared library (omp: the OpenMP build)."""
    with _lock:
        if omp not in _libs:
            L = C.CDLL(build(omp=omp))
            sig = {
                "or_lattice": (C.c_int, [C.c_int32, C.POINTER(C.c_int32), _ip, _dp]),
                "or_feq": (None, [C.c_int32, C.c_double, _dp, _dp]),
                "or_force_term": (None, [C.c_int32, C.c_double, _dp, _dp, _dp]),
                "or_macro": (None, [C.c_int32, _dp, _dp, _dp, _dp, C.POINTER(C.c_double)]),
                "or_delta": (C.c_double, [C.c_int32, C.c_double]),
                "or_stream_push": (None, [C.c_int32, C.c_int32, C.c_int32, C.c_int32, _ip, _dp, _dp]),
                "or_stream_swap": (None, [C.c_int32, C.c_int32, C.c_int32, C.c_int32, _ip, _dp]),
                "or_interp": (None, [_PP, _dp, C.c_int64, _dp, _dp]),
                "or_spread": (None, [_PP, C.c_int64, _dp, _dp, C.c_double, _dp]),
                "or_pairs_bruteforce": (C.c_int64, [_PP, C.c_int64, _dp, _ip, C.c_int64]),
                "or_pairs_gridsearch": (C.c_int64, [_PP, C.c_int64, _dp, _ip, C.c_int64]),
                "or_pair_force": (None, [_PP, C.c_double, _dp, _dp, _dp]),
                "or_contact_forces": (None, [_PP, C.c_int64, _dp, _dp]),
                "or_create": (C.c_void_p, [_PP, C.c_void_p]),
                "or_destroy": (None, [C.c_void_p]),
                "or_step": (None, [C.c_void_p, C.c_int32]),
                "or_get_pdfs": (None, [C.c_void_p, _dp]),
                "or_set_pdfs": (None, [C.c_void_p, _dp]),
                "or_set_fields": (None, [C.c_void_p, _dp, _dp]),
                "or_get_fields": (None, [C.c_void_p, _dp, _dp]),
                "or_get_particles": (None, [C.c_void_p] + [_dp] * 6),
                "or_set_particles": (None, [C.c_void_p, _dp, _dp, _dp]),
                "or_get_lagrangian": (None, [C.c_void_p, _dp, _dp, _dp, _dp]),
                "or_get_mdf_residual": (None, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
                "or_point_volume": (C.c_double, [_PP]),
                "or_get_interior_momentum": (None, [C.c_void_p, _dp, _dp]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _libs[omp] = L
    return _libs[omp]


def _vec3(a, n=None):
    """Pad an [n][dim] array to contiguous float64 [n][3]."""
    a = np.asarray(a, dtype=np.float64)
    if a.ndim == 1:
        a = a.reshape(-1, a.shape[0]) if n is None else a.reshape(n, -1)
    out = np.zeros((a.shape[0], 3), dtype=np.float64)
    out[:, : a.shape[1]] = a
    return out


# ------------------------------------------------------------------ node level
def lattice(dim: int):
    """(e[q][3] int32, w[q]) of D2Q9 / D3Q19 (Eq. 2-3)."""
    e = np.zeros((19, 3), dtype=np.int32)
    w = np.zeros(19)
    q = C.c_int32(0)
    if lib().or_lattice(dim, C.byref(q), e.reshape(-1), w) != 0:
        raise ValueError("dim must be 2 or 3")
    return e[: q.value].copy(), w[: q.value].copy()


def feq(dim: int, p: float, u) -> np.ndarray:
    q = 9 if dim == 2 else 19
    out = np.zeros(q)
    lib().or_feq(dim, float(p), _vec3([u])[0], out)
    return out


def force_term(dim: int, tau: float, u, F) -> np.ndarray:
    q = 9 if dim == 2 else 19
    out = np.zeros(q)
    lib().or_force_term(dim, float(tau), _vec3([u])[0], _vec3([F])[0], out)
    return out


def macro(dim: int, fnode, F=(0.0, 0.0, 0.0)):
    """(u*, u, p) of one node (Eq. 5-7)."""
    us, u = np.zeros(3), np.zeros(3)
    p = C.c_double(0.0)
    lib().or_macro(dim, np.ascontiguousarray(fnode, dtype=np.float64), _vec3([F])[0], us, u,
                   C.byref(p))
    return us, u, p.value


def delta(kind: int, r) -> np.ndarray:
    r = np.atleast_1d(np.asarray(r, dtype=np.float64))
    f = lib().or_delta
    return np.array([f(kind, float(x)) for x in r.reshape(-1)]).reshape(r.shape)


def stream_push(dim, shape, periodic, fp):
    nx, ny, nz = (list(shape) + [1])[:3]
    f = np.zeros_like(np.ascontiguousarray(fp, dtype=np.float64))
    lib().or_stream_push(dim, nx, ny, nz, np.asarray(periodic, dtype=np.int32),
                         np.ascontiguousarray(fp, dtype=np.float64).reshape(-1), f.reshape(-1))
    return f


def stream_swap(dim, shape, periodic, fp):
    nx, ny, nz = (list(shape) + [1])[:3]
    f = np.ascontiguousarray(fp, dtype=np.float64).copy()
    lib().or_stream_swap(dim, nx, ny, nz, np.asarray(periodic, dtype=np.int32), f.reshape(-1))
    return f


# ------------------------------------------------------------------- IBM level
def interp(cfg, g, X) -> np.ndarray:
    """D_I g at points X (Eq. 47); g is [dim or 3][N]."""
    P = make_params(cfg)
    N = P.nx * P.ny * P.nz
    g3 = np.zeros((3, N))
    g = np.asarray(g, dtype=np.float64).reshape(-1, N)
    g3[: g.shape[0]] = g
    X3 = _vec3(X)
    out = np.zeros_like(X3)
    lib().or_interp(C.byref(P), g3.reshape(-1), X3.shape[0], X3.reshape(-1), out.reshape(-1))
    return out[:, : P.dim]


def spread(cfg, X, F, dV: float) -> np.ndarray:
    """D_E F on the grid (Eq. 48) as [dim][N]."""
    P = make_params(cfg)
    N = P.nx * P.ny * P.nz
    X3, F3 = _vec3(X), _vec3(F)
    g = np.zeros((3, N))
    lib().or_spread(C.byref(P), X3.shape[0], X3.reshape(-1), F3.reshape(-1), float(dV), g.reshape(-1))
    return g[: P.dim]


def point_volume(cfg) -> float:
    P = make_params(cfg)
    return lib().or_point_volume(C.byref(P))


# ------------------------------------------------------------------ pair level
def _pairs(fn, cfg, X):
    P = make_params(cfg)
    X3 = _vec3(X)
    cap = 1024
    while True:
        out = np.zeros(2 * cap, dtype=np.int32)
        n = fn(C.byref(P), X3.shape[0], X3.reshape(-1), out, cap)
        if n < 0:
            raise ValueError(f"pair search precondition failed ({n})")
        if n <= cap:
            return out[: 2 * n].reshape(-1, 2)
        cap = int(n)


def pairs_bruteforce(cfg, X) -> np.ndarray:
    """Half-search pair list (Table 4), sorted by (i, j)."""
    return _pairs(lib().or_pairs_bruteforce, cfg, X)


def pairs_gridsearch(cfg, X) -> np.ndarray:
    """Grid-search pair list (Table 5), sorted by (i, j)."""
    return _pairs(lib().or_pairs_gridsearch, cfg, X)


def pair_force(cfg, c_ij: float, Xi, Xj) -> np.ndarray:
    P = make_params(cfg)
    out = np.zeros(3)
    lib().or_pair_force(C.byref(P), float(c_ij), _vec3([Xi])[0], _vec3([Xj])[0], out)
    return out[: P.dim]


def contact_forces(cfg, X) -> np.ndarray:
    P = make_params(cfg)
    X3 = _vec3(X)
    out = np.zeros_like(X3)
    lib().or_contact_forces(C.byref(P), X3.shape[0], X3.reshape(-1), out.reshape(-1))
    return out[:, : P.dim]


# ------------------------------------------------------------- whole simulation
class Sim:
    """The oracle's time stepper (macro -> MDF -> collide -> stream -> pairs -> update)."""

    def __init__(self, cfg, xc=None, omp: bool = False):
        self.L = lib(omp)  # omp: the same oracle on all host cores (identical bits)
        self.P = make_params(cfg)
        self.dim = self.P.dim
        self.q = 9 if self.dim == 2 else 19
        self.N = self.P.nx * self.P.ny * self.P.nz
        self.np = self.P.n_particles
        self.nl = self.P.n_lag
        xc3 = _vec3(xc) if (xc is not None and self.np > 0) else np.zeros((max(self.np, 1), 3))
        self._xc = xc3
        self.h = self.L.or_create(C.byref(self.P), xc3.ctypes.data_as(C.c_void_p))
        if not self.h:
            raise MemoryError("oracle allocation failed")

    def close(self):
        if getattr(self, "h", None):
            self.L.or_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def step(self, n: int = 1):
        self.L.or_step(self.h, int(n))

    def get_pdfs(self) -> np.ndarray:
        f = np.zeros((self.q, self.N))
        self.L.or_get_pdfs(self.h, f.reshape(-1))
        return f

    def set_pdfs(self, f):
        self.L.or_set_pdfs(self.h, np.ascontiguousarray(f, dtype=np.float64).reshape(-1))

    def set_fields(self, p, u):
        u3 = np.zeros((3, self.N))
        u = np.asarray(u, dtype=np.float64).reshape(-1, self.N)
        u3[: u.shape[0]] = u
        self.L.or_set_fields(self.h, np.ascontiguousarray(p, dtype=np.float64).reshape(-1),
                            u3.reshape(-1))

    def get_fields(self):
        p = np.zeros(self.N)
        u = np.zeros((3, self.N))
        self.L.or_get_fields(self.h, p, u.reshape(-1))
        return p, u[: self.dim]

    def get_particles(self):
        n = max(self.np, 1)
        arrs = [np.zeros((n, 3)) for _ in range(6)]
        self.L.or_get_particles(self.h, *[a.reshape(-1) for a in arrs])
        X, U, Om, Fh, Th, Fc = [a[: self.np] for a in arrs]
        d = self.dim
        om = Om[:, 2:3] if d == 2 else Om
        th = Th[:, 2:3] if d == 2 else Th
        return dict(X=X[:, :d], U=U[:, :d], Omega=om, F_h=Fh[:, :d], T_h=th, F_c=Fc[:, :d])

    def set_particles(self, X, U=None, Omega=None):
        n = max(self.np, 1)
        X3 = _vec3(X, n)
        U3 = _vec3(U, n) if U is not None else np.zeros((n, 3))
        Om3 = np.zeros((n, 3))
        if Omega is not None:
            om = np.asarray(Omega, dtype=np.float64).reshape(n, -1)
            if self.dim == 2:
                Om3[:, 2] = om[:, 0]
            else:
                Om3[:] = om
        self.L.or_set_particles(self.h, X3.reshape(-1), U3.reshape(-1), Om3.reshape(-1))

    def get_lagrangian(self):
        n = max(self.np * self.nl, 1)
        arrs = [np.zeros((n, 3)) for _ in range(4)]
        self.L.or_get_lagrangian(self.h, *[a.reshape(-1) for a in arrs])
        d = self.dim
        m = self.np * self.nl
        Xb, Ub, Fb, us = [a[:m, :d] for a in arrs]
        return dict(X_b=Xb, U_b=Ub, F_b=Fb, u_b_star=us)

    def get_interior_momentum(self):
        n = max(self.np, 1)
        P, L = np.zeros((n, 3)), np.zeros((n, 3))
        self.L.or_get_interior_momentum(self.h, P.reshape(-1), L.reshape(-1))
        return P[: self.np, : self.dim], (L[: self.np, 2:3] if self.dim == 2 else L[: self.np])

    def get_mdf_residual(self):
        r, m = C.c_double(0.0), C.c_double(0.0)
        self.L.or_get_mdf_residual(self.h, C.byref(r), C.byref(m))
        return r.value, m.value
