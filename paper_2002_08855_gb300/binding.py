"""ctypes binding of ``libibmlbm.so`` (C ABI in ``include/ibmlbm.h``).

Argument marshalling only: every step of the method runs in the library's CUDA
kernels.  PyTorch provides the device memory (the workspace and device-side
field buffers) and the CUDA stream the run is ordered on.  There is no CPU path:
if the library is missing or cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libibmlbm.so")
LIB_CHECKED_PATH = os.path.join(_HERE, "_build", "libibmlbm_checked.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "ibmlbm.h")

OK = 0
ERRORS = {
    -1: "INVALID_ARG", -2: "UNSUPPORTED", -3: "WORKSPACE", -4: "CUDA", -5: "NONFINITE",
    -6: "OUT_OF_DOMAIN", -7: "CAPACITY", -8: "BOUNDS", -9: "TIMEOUT",
}
PARTS = ("macro", "ibm", "collide_stream", "pairs", "particles")


class IbmLbmError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: {ERRORS.get(code, code)}: {msg}")
        self.code = code
        self.name = ERRORS.get(code, str(code))


class Config(C.Structure):
    """Mirror of ``ibm_lbm_config``."""

    _fields_ = [
        ("struct_size", C.c_uint32), ("dim", C.c_int32), ("nx", C.c_int32), ("ny", C.c_int32),
        ("nz", C.c_int32), ("periodic", C.c_int32 * 3), ("tau", C.c_double),
        ("body_force", C.c_double * 3), ("n_particles", C.c_int32), ("n_lag", C.c_int32),
        ("diameter", C.c_double), ("delta_kind", C.c_int32), ("drs", C.c_double),
        ("mdf_iters", C.c_int32), ("density_ratio", C.c_double), ("gravity", C.c_double * 3),
        ("zeta", C.c_double), ("eps_pp", C.c_double), ("E_pp", C.c_double),
        ("fixed_particles", C.c_int32), ("max_neighbors", C.c_int32), ("pdf_storage", C.c_int32),
        ("mlp_init", C.c_int32), ("boundary", C.c_int32), ("u_inlet", C.c_double),
        ("pair_search", C.c_int32),
    ]


def make_config(w, max_neighbors: int = 0) -> Config:
    """``ibm_lbm_config`` from a workload (``inputs.Workload`` or a dict of its fields)."""
    get = w.get if isinstance(w, dict) else (lambda k, d=None: getattr(w, k, d))
    c = Config()
    c.struct_size = C.sizeof(Config)
    c.dim = int(get("dim", 2))
    c.nx, c.ny = int(get("nx")), int(get("ny"))
    c.nz = int(get("nz", 1)) if c.dim == 3 else 1
    for k, v in enumerate((list(get("periodic", (0, 0, 0))) + [0, 0, 0])[:3]):
        c.periodic[k] = int(v)
    c.tau = float(get("tau", 0.6))
    for k, v in enumerate((list(get("body_force", (0, 0, 0))) + [0, 0, 0])[:3]):
        c.body_force[k] = float(v)
    c.n_particles = int(get("n_particles", 0))
    c.n_lag = int(get("n_lag", 0))
    c.diameter = float(get("diameter", 0.0))
    c.delta_kind = int(get("delta_kind", 4))
    c.drs = float(get("drs", 2.6))
    c.mdf_iters = int(get("mdf_iters", 3))
    c.density_ratio = float(get("density_ratio", 1.5))
    for k, v in enumerate((list(get("gravity", (0, 0, 0))) + [0, 0, 0])[:3]):
        c.gravity[k] = float(v)
    c.zeta = float(get("zeta", 2.0))
    c.eps_pp = float(get("eps_pp", 1e-2))
    c.E_pp = float(get("E_pp", 1e-4))
    c.fixed_particles = int(get("fixed_particles", 0))
    c.max_neighbors = int(max_neighbors)
    c.pdf_storage = int(get("pdf_storage", 0))
    c.mlp_init = int(get("mlp_init", 0))
    c.boundary = int(get("boundary", 0))
    c.u_inlet = float(get("u_inlet", 0.0))
    c.pair_search = int(get("pair_search", 0))
    return c


_lock = threading.Lock()
_libs = {}
_vp, _dp, _fp, _ip, _i64p = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_float), \
    C.POINTER(C.c_int32), C.POINTER(C.c_int64)
SIGNATURES = {
    "ibm_lbm_workspace_size": (C.c_int, [C.POINTER(Config), C.POINTER(C.c_size_t)]),
    "ibm_lbm_init": (C.c_int, [C.POINTER(Config), _vp, C.c_size_t, _vp, _dp, C.POINTER(_vp)]),
    "ibm_lbm_step": (C.c_int, [_vp, C.c_int32]),
    "ibm_lbm_sync": (C.c_int, [_vp]),
    "ibm_lbm_set_pdfs": (C.c_int, [_vp, _vp]),
    "ibm_lbm_get_pdfs": (C.c_int, [_vp, _vp]),
    "ibm_lbm_set_fields": (C.c_int, [_vp, _vp, _vp]),
    "ibm_lbm_get_fields": (C.c_int, [_vp, _vp, _vp]),
    "ibm_lbm_set_particles": (C.c_int, [_vp, _dp, _dp, _dp]),
    "ibm_lbm_get_particles": (C.c_int, [_vp, _dp, _dp, _dp, _dp, _dp, _dp]),
    "ibm_lbm_get_lagrangian": (C.c_int, [_vp, _dp, _fp, _fp, _fp]),
    "ibm_lbm_get_interior_momentum": (C.c_int, [_vp, _dp, _dp]),
    "ibm_lbm_get_pairs": (C.c_int, [_vp, _ip, C.c_int64, _i64p]),
    "ibm_lbm_get_launch_count": (C.c_int, [_vp, _i64p]),
    "ibm_lbm_time_parts": (C.c_int, [_vp, C.c_int32, _dp]),
    "ibm_lbm_stage_list": (C.c_int, [C.POINTER(Config), _ip, C.c_int64, _i64p]),
    "ibm_lbm_destroy": (None, [_vp]),
    "ibm_lbm_last_error": (C.c_char_p, []),
    "ibm_lbm_pair_search_scratch_size": (C.c_int, [C.c_int32, _ip, C.c_double, C.c_double,
                                                   C.c_int32, C.c_int32, C.POINTER(C.c_size_t)]),
    "ibm_lbm_pair_search": (C.c_int, [C.c_int32, _ip, _ip, C.c_double, C.c_double, C.c_int32,
                                      _vp, C.c_int32, _vp, C.c_size_t, _vp, C.c_int64, _i64p,
                                      _vp]),
    "ibm_lbm_pair_search_static": (C.c_int, [C.c_int32, _ip, _ip, C.c_double, C.c_double,
                                             C.c_int32, _vp, C.c_int32, _vp, C.c_int64, _i64p,
                                             _vp]),
    "ibm_lbm_mlp_param_count": (C.c_int32, []),
    "ibm_lbm_set_mlp": (C.c_int, [_vp, _fp]),
    "ibm_lbm_mdf_samples": (C.c_int, [_vp, _vp, _vp]),
    "ibm_lbm_set_residual_tracking": (C.c_int, [_vp, C.c_int32]),
    "ibm_lbm_get_mdf_residual": (C.c_int, [_vp, _dp, _dp]),
    "ibm_lbm_mlp_scratch_size": (C.c_int, [C.c_int32, C.POINTER(C.c_size_t)]),
    "ibm_lbm_mlp_grad": (C.c_int, [_vp, _vp, _vp, C.c_int32, _vp, _dp, _vp, C.c_size_t, _vp]),
    "ibm_lbm_mlp_adam": (C.c_int, [_vp, _vp, _vp, _vp, C.c_int64, C.c_float, _vp]),
    "ibm_lbm_mlp_infer": (C.c_int, [_vp, _vp, C.c_int64, _vp, _vp]),
    "ibm_lbm_state_size": (C.c_int, [_vp, C.POINTER(C.c_size_t)]),
    "ibm_lbm_get_state": (C.c_int, [_vp, _vp, C.c_size_t]),
    "ibm_lbm_set_state": (C.c_int, [_vp, _vp, C.c_size_t]),
    "ibm_lbm_batch_workspace_size": (C.c_int, [C.POINTER(Config), C.c_int32, C.POINTER(C.c_size_t)]),
    "ibm_lbm_batch_init": (C.c_int, [C.POINTER(Config), C.c_int32, _vp, C.c_size_t, _vp,
                                     C.POINTER(_dp), C.POINTER(_vp)]),
    "ibm_lbm_batch_step": (C.c_int, [_vp, C.c_int32]),
    "ibm_lbm_batch_sync": (C.c_int, [_vp]),
    "ibm_lbm_batch_member": (_vp, [_vp, C.c_int32]),
    "ibm_lbm_batch_launch_count": (C.c_int64, [_vp]),
    "ibm_lbm_tile_shape_count": (C.c_int, []),
    "ibm_lbm_tile_shape": (C.c_int, [C.c_int32, C.c_int32, _ip, _ip, _ip]),
    "ibm_lbm_batch_set_tile_shape": (C.c_int, [_vp, C.c_int32]),
    "ibm_lbm_batch_get_tile_shape": (C.c_int, [_vp, _ip]),
    "ibm_lbm_batch_autotune": (C.c_int, [_vp, C.c_int32, _fp]),
    "ibm_lbm_batch_set_persistent": (C.c_int, [_vp, C.c_int32, C.c_int64]),
    "ibm_lbm_batch_get_persistent": (C.c_int, [_vp, _ip]),
    "ibm_lbm_batch_destroy": (None, [_vp]),
}


def lib(checked: bool = False):
    """Load the CUDA library (or its bounds-checked variant); raise if it has not been
    built (there is no fallback)."""
    path = LIB_CHECKED_PATH if checked else LIB_PATH
    with _lock:
        if path not in _libs:
            if not os.path.exists(path):
                raise RuntimeError(f"{path} is missing: build it with "
                                   "paper_2002_08855_gb300.build.build() (there is no CPU path)")
            L = C.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _libs[path] = L
    return _libs[path]


def _check(rc: int, where: str, L=None):
    if rc != OK:
        raise IbmLbmError(rc, where, (L or lib()).ibm_lbm_last_error().decode())


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def stage_list(w):
    """The 3D staging list of a workload's node box (host only): int32 array of cells
    packed lx | ly << 5 | lz << 10 (empty where no list is used)."""
    import numpy as np

    cfg = make_config(w)
    n = C.c_int64(0)
    _check(lib().ibm_lbm_stage_list(C.byref(cfg), None, 0, C.byref(n)), "stage_list")
    out = np.zeros(max(n.value, 1), dtype=np.int32)
    _check(lib().ibm_lbm_stage_list(C.byref(cfg), _ptr(out, C.c_int32), n.value, C.byref(n)), "stage_list")
    return out[:n.value]


def workspace_size(w, max_neighbors: int = 0) -> int:
    cfg = make_config(w, max_neighbors)
    n = C.c_size_t(0)
    _check(lib().ibm_lbm_workspace_size(C.byref(cfg), C.byref(n)), "workspace_size")
    return n.value


class Simulation:
    """One run on one GPU: fluid cavity plus rigid particles (C ABI handle)."""

    def __init__(self, w, centres=None, device: str = "cuda", stream=None,
                 max_neighbors: int = 0, checked: bool = False):
        import torch

        self.torch = torch
        self.L = lib(checked)  # checked: the bounds-checked library
        self.cfg = make_config(w, max_neighbors)
        self.dim = self.cfg.dim
        self.q = 9 if self.dim == 2 else 19
        self.N = self.cfg.nx * self.cfg.ny * self.cfg.nz
        self.np = self.cfg.n_particles
        self.nl = self.cfg.n_lag
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        nbytes = workspace_size(w, max_neighbors)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream.wait_stream(torch.cuda.current_stream(self.device))
        self.h = C.c_void_p(None)
        xc = None
        if self.np > 0:
            if centres is None:
                raise ValueError("particle centres are required")
            xc = np.ascontiguousarray(np.asarray(centres, dtype=np.float64).reshape(self.np, self.dim))
        _check(self.L.ibm_lbm_init(C.byref(self.cfg), C.c_void_p(self.workspace.data_ptr()),
                                  nbytes, C.c_void_p(self.stream.cuda_stream),
                                  _ptr(xc, C.c_double) if xc is not None else None,
                                  C.byref(self.h)), "init", self.L)

    # ------------------------------------------------------------ stepping
    def step(self, n: int = 1):
        _check(self.L.ibm_lbm_step(self.h, int(n)), "step", self.L)

    def sync(self):
        _check(self.L.ibm_lbm_sync(self.h), "sync", self.L)

    def time_parts(self, n: int) -> dict:
        ms = np.zeros(5)
        _check(self.L.ibm_lbm_time_parts(self.h, int(n), _ptr(ms, C.c_double)), "time_parts", self.L)
        return dict(zip(PARTS, ms.tolist()))

    def launch_count(self) -> int:
        v = C.c_int64(0)
        _check(self.L.ibm_lbm_get_launch_count(self.h, C.byref(v)), "launch_count", self.L)
        return v.value

    # ------------------------------------------------------------ fields
    def _wait_torch(self):
        self.stream.wait_stream(self.torch.cuda.current_stream(self.device))

    def set_pdfs(self, f):
        t = self.torch.as_tensor(f, dtype=self.torch.float32, device=self.device).reshape(self.q, self.N).contiguous()
        self._wait_torch()
        _check(self.L.ibm_lbm_set_pdfs(self.h, C.c_void_p(t.data_ptr())), "set_pdfs", self.L)
        self.stream.synchronize()

    def get_pdfs(self):
        t = self.torch.empty((self.q, self.N), dtype=self.torch.float32, device=self.device)
        self._wait_torch()
        _check(self.L.ibm_lbm_get_pdfs(self.h, C.c_void_p(t.data_ptr())), "get_pdfs", self.L)
        self.stream.synchronize()
        return t

    def set_fields(self, p, u):
        tp = self.torch.as_tensor(p, dtype=self.torch.float64, device=self.device).reshape(self.N).contiguous()
        tu = self.torch.as_tensor(u, dtype=self.torch.float64, device=self.device).reshape(self.dim, self.N).contiguous()
        self._wait_torch()
        _check(self.L.ibm_lbm_set_fields(self.h, C.c_void_p(tp.data_ptr()), C.c_void_p(tu.data_ptr())), "set_fields", self.L)
        self.stream.synchronize()

    def get_fields(self):
        tp = self.torch.empty(self.N, dtype=self.torch.float64, device=self.device)
        tu = self.torch.empty((self.dim, self.N), dtype=self.torch.float64, device=self.device)
        self._wait_torch()
        _check(self.L.ibm_lbm_get_fields(self.h, C.c_void_p(tp.data_ptr()), C.c_void_p(tu.data_ptr())), "get_fields", self.L)
        self.stream.synchronize()
        return tp, tu

    # ------------------------------------------------------------ particles
    def _rot(self):
        return 1 if self.dim == 2 else 3

    def set_particles(self, X=None, U=None, Omega=None):
        def arr(a, cols):
            if a is None:
                return None
            return np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(self.np, cols))
        X, U, Om = arr(X, self.dim), arr(U, self.dim), arr(Omega, self._rot())
        _check(self.L.ibm_lbm_set_particles(
            self.h, *[(_ptr(a, C.c_double) if a is not None else None) for a in (X, U, Om)]),
            "set_particles", self.L)

    def get_particles(self) -> dict:
        n, d, r = max(self.np, 1), self.dim, self._rot()
        out = dict(X=np.zeros((n, d)), U=np.zeros((n, d)), Omega=np.zeros((n, r)),
                   F_h=np.zeros((n, d)), T_h=np.zeros((n, r)), F_c=np.zeros((n, d)))
        _check(self.L.ibm_lbm_get_particles(self.h, *[_ptr(out[k], C.c_double) for k in
                                                      ("X", "U", "Omega", "F_h", "T_h", "F_c")]),
               "get_particles", self.L)
        return {k: v[: self.np] for k, v in out.items()}

    def get_lagrangian(self) -> dict:
        m, d = max(self.np * self.nl, 1), self.dim
        Xb = np.zeros((m, d))
        Ub, Fb, us = (np.zeros((m, d), dtype=np.float32) for _ in range(3))
        _check(self.L.ibm_lbm_get_lagrangian(self.h, _ptr(Xb, C.c_double), _ptr(Ub, C.c_float),
                                            _ptr(Fb, C.c_float), _ptr(us, C.c_float)),
               "get_lagrangian", self.L)
        k = self.np * self.nl
        return dict(X_b=Xb[:k], U_b=Ub[:k], F_b=Fb[:k], u_b_star=us[:k])

    def get_interior_momentum(self):
        n = max(self.np, 1)
        P, L = np.zeros((n, self.dim)), np.zeros((n, self._rot()))
        _check(self.L.ibm_lbm_get_interior_momentum(self.h, _ptr(P, C.c_double), _ptr(L, C.c_double)),
               "get_interior_momentum", self.L)
        return P[: self.np], L[: self.np]

    def get_pairs(self) -> np.ndarray:
        n = C.c_int64(0)
        cap = max(16, self.np * 8)
        while True:
            buf = np.zeros(2 * cap, dtype=np.int32)
            rc = self.L.ibm_lbm_get_pairs(self.h, _ptr(buf, C.c_int32), cap, C.byref(n))
            if rc == -7 and n.value > cap:
                cap = int(n.value)
                continue
            _check(rc, "get_pairs", self.L)
            return buf[: 2 * n.value].reshape(-1, 2)

    # ------------------------------------------------------------ learned initializer
    def set_mlp(self, params):
        p = np.ascontiguousarray(np.asarray(params, dtype=np.float32).reshape(-1))
        if p.size != self.L.ibm_lbm_mlp_param_count():
            raise ValueError("wrong number of parameters")
        _check(self.L.ibm_lbm_set_mlp(self.h, _ptr(p, C.c_float)), "set_mlp", self.L)

    def mdf_samples(self):
        """(features [npts][27], targets [npts][3]) of the last step, as CUDA tensors."""
        n = self.np * self.nl
        X = self.torch.empty((n, 27), dtype=self.torch.float32, device=self.device)
        Y = self.torch.empty((n, 3), dtype=self.torch.float32, device=self.device)
        self._wait_torch()
        _check(self.L.ibm_lbm_mdf_samples(self.h, C.c_void_p(X.data_ptr()), C.c_void_p(Y.data_ptr())),
               "mdf_samples", self.L)
        return X, Y

    def get_state(self) -> np.ndarray:
        """Checkpoint of the run (host bytes)."""
        n = C.c_size_t(0)
        _check(self.L.ibm_lbm_state_size(self.h, C.byref(n)), "state_size", self.L)
        buf = np.zeros(n.value, dtype=np.uint8)
        self._wait_torch()
        _check(self.L.ibm_lbm_get_state(self.h, C.c_void_p(buf.ctypes.data), n.value), "get_state", self.L)
        return buf

    def set_state(self, buf):
        """Resume from a checkpoint of a run of the same configuration."""
        b = np.ascontiguousarray(np.asarray(buf, dtype=np.uint8))
        self._wait_torch()
        _check(self.L.ibm_lbm_set_state(self.h, C.c_void_p(b.ctypes.data), b.size), "set_state", self.L)

    def set_residual_tracking(self, on: bool = True):
        _check(self.L.ibm_lbm_set_residual_tracking(self.h, int(bool(on))), "set_residual_tracking", self.L)

    def mdf_residual(self):
        rms, mx = C.c_double(0), C.c_double(0)
        _check(self.L.ibm_lbm_get_mdf_residual(self.h, C.byref(rms), C.byref(mx)), "get_mdf_residual", self.L)
        return rms.value, mx.value

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            self.stream.synchronize()
            self.L.ibm_lbm_destroy(self.h)
            self.h = C.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchMember(Simulation):
    """One member of a Batch: the field and particle calls of a run (stepping is the
    batch's)."""

    def __init__(self, batch, i, w):
        self.torch = batch.torch
        self.L = batch.L
        self.cfg = make_config(w)
        self.dim = self.cfg.dim
        self.q = 9 if self.dim == 2 else 19
        self.N = self.cfg.nx * self.cfg.ny * self.cfg.nz
        self.np = self.cfg.n_particles
        self.nl = self.cfg.n_lag
        self.device = batch.device
        self.stream = batch.stream
        ptr = self.L.ibm_lbm_batch_member(batch.h, int(i))
        if not ptr:
            raise IbmLbmError(-1, "batch_member", self.L.ibm_lbm_last_error().decode())
        self.h = C.c_void_p(ptr)

    def step(self, n: int = 1):
        raise RuntimeError("batch members step with their batch")

    def close(self):
        self.h = C.c_void_p(None)  # owned by the batch


def tile_shapes(pdf_storage: int = 0) -> list:
    """(nodes per thread, warps per block, persistent) of each lbm_step tile shape of a
    batch, by shape index."""
    out = []
    for sh in range(lib().ibm_lbm_tile_shape_count()):
        k, w, p = C.c_int32(0), C.c_int32(0), C.c_int32(0)
        _check(lib().ibm_lbm_tile_shape(sh, int(pdf_storage), C.byref(k), C.byref(w), C.byref(p)),
               "tile_shape")
        out.append((k.value, w.value, p.value))
    return out


class Batch:
    """Many independent 2D cavities stepped together (fused launches, one CUDA graph
    per step parity).  members[i] gives the field and particle calls of member i."""

    def __init__(self, workloads, centres, device: str = "cuda", stream=None):
        import torch

        self.torch = torch
        self.L = lib()
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        n = len(workloads)
        cfgs = (Config * n)(*[make_config(w) for w in workloads])
        size = C.c_size_t(0)
        _check(self.L.ibm_lbm_batch_workspace_size(cfgs, n, C.byref(size)), "batch_workspace_size", self.L)
        self.workspace = torch.empty(size.value, dtype=torch.uint8, device=self.device)
        self.stream.wait_stream(torch.cuda.current_stream(self.device))
        self._xc = []
        ptrs = (_dp * n)()
        for i, (w, X) in enumerate(zip(workloads, centres)):
            if w.n_particles > 0:
                xc = np.ascontiguousarray(np.asarray(X, dtype=np.float64).reshape(w.n_particles, 2))
                self._xc.append(xc)
                ptrs[i] = _ptr(xc, C.c_double)
        self.h = C.c_void_p(None)
        _check(self.L.ibm_lbm_batch_init(cfgs, n, C.c_void_p(self.workspace.data_ptr()), size.value,
                                        C.c_void_p(self.stream.cuda_stream), ptrs, C.byref(self.h)),
               "batch_init", self.L)
        self.members = [BatchMember(self, i, w) for i, w in enumerate(workloads)]
        self.n_grid = sum(w.n_grid for w in workloads)

    def step(self, n: int = 1):
        _check(self.L.ibm_lbm_batch_step(self.h, int(n)), "batch_step", self.L)

    def sync(self):
        _check(self.L.ibm_lbm_batch_sync(self.h), "batch_sync", self.L)

    def launch_count(self) -> int:
        return int(self.L.ibm_lbm_batch_launch_count(self.h))

    def set_tile_shape(self, shape: int):
        _check(self.L.ibm_lbm_batch_set_tile_shape(self.h, int(shape)), "batch_set_tile_shape", self.L)

    def tile_shape(self) -> int:
        v = C.c_int32(0)
        _check(self.L.ibm_lbm_batch_get_tile_shape(self.h, C.byref(v)), "batch_get_tile_shape", self.L)
        return v.value

    def set_persistent(self, on: bool = True, barrier_limit: int = 0):
        """Three launches a step: the IBM phases and the contact phases each as one
        cooperative kernel with bounded grid barriers (barrier_limit polls; 0 = default)."""
        _check(self.L.ibm_lbm_batch_set_persistent(self.h, int(bool(on)), int(barrier_limit)),
               "batch_set_persistent", self.L)

    def persistent(self) -> bool:
        v = C.c_int32(0)
        _check(self.L.ibm_lbm_batch_get_persistent(self.h, C.byref(v)), "batch_get_persistent", self.L)
        return bool(v.value)

    def autotune(self, steps_per_shape: int = 2) -> tuple:
        """Time every tile shape on steps_per_shape real steps; keep the fastest.
        Returns (chosen shape, mean ms per step of each shape's collide-stream launches)."""
        ms = np.zeros(self.L.ibm_lbm_tile_shape_count(), dtype=np.float32)
        _check(self.L.ibm_lbm_batch_autotune(self.h, int(steps_per_shape), _ptr(ms, C.c_float)),
               "batch_autotune", self.L)
        return self.tile_shape(), [float(v) for v in ms]

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            self.stream.synchronize()
            for m in self.members:
                m.close()
            self.L.ibm_lbm_batch_destroy(self.h)
            self.h = C.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pair_search(dim: int, n_nodes, periodic, diameter: float, zeta: float, X,
                max_neighbors: int = 0, stream=None) -> np.ndarray:
    """Standalone cell-list pair search on the GPU; returns the sorted (i, j) list."""
    import torch

    X = torch.as_tensor(np.asarray(X, dtype=np.float64), device="cuda").reshape(-1, dim).contiguous()
    n = X.shape[0]
    nn = np.ascontiguousarray((list(n_nodes) + [1, 1, 1])[:3], dtype=np.int32)
    per = np.ascontiguousarray((list(periodic) + [0, 0, 0])[:3], dtype=np.int32)
    sz = C.c_size_t(0)
    _check(lib().ibm_lbm_pair_search_scratch_size(dim, _ptr(nn, C.c_int32), diameter, zeta, n,
                                                  max_neighbors, C.byref(sz)), "pair_search_scratch_size")
    scratch = torch.empty(max(sz.value, 1), dtype=torch.uint8, device="cuda")
    s = stream if stream is not None else torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    cap = max(16, n * 8)
    while True:
        pairs = torch.empty((cap, 2), dtype=torch.int32, device="cuda")
        cnt = C.c_int64(0)
        rc = lib().ibm_lbm_pair_search(dim, _ptr(nn, C.c_int32), _ptr(per, C.c_int32), diameter,
                                       zeta, n, C.c_void_p(X.data_ptr()), max_neighbors,
                                       C.c_void_p(scratch.data_ptr()), sz.value,
                                       C.c_void_p(pairs.data_ptr()), cap, C.byref(cnt),
                                       C.c_void_p(s.cuda_stream))
        if rc == -7 and cnt.value > cap:
            cap = int(cnt.value)
            continue
        _check(rc, "pair_search")
        return pairs[: cnt.value].cpu().numpy()


def pair_search_static(dim: int, n_nodes, periodic, diameter: float, zeta: float, X,
                       max_neighbors: int = 0, stream=None, cap=None) -> np.ndarray:
    """Pair search through the entry point that allocates nothing on the library side
    (its lists live in a fixed 16 MiB device array); same result as pair_search."""
    import torch

    X = torch.as_tensor(np.asarray(X, dtype=np.float64), device="cuda").reshape(-1, dim).contiguous()
    n = X.shape[0]
    nn = np.ascontiguousarray((list(n_nodes) + [1, 1, 1])[:3], dtype=np.int32)
    per = np.ascontiguousarray((list(periodic) + [0, 0, 0])[:3], dtype=np.int32)
    s = stream if stream is not None else torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    cap = max(16, n * 8) if cap is None else cap
    while True:
        pairs = torch.empty((max(cap, 1), 2), dtype=torch.int32, device="cuda")
        cnt = C.c_int64(0)
        rc = lib().ibm_lbm_pair_search_static(dim, _ptr(nn, C.c_int32), _ptr(per, C.c_int32),
                                              diameter, zeta, n, C.c_void_p(X.data_ptr()),
                                              max_neighbors, C.c_void_p(pairs.data_ptr()), cap,
                                              C.byref(cnt), C.c_void_p(s.cuda_stream))
        if rc == -7 and cnt.value > cap:
            cap = int(cnt.value)
            continue
        _check(rc, "pair_search_static")
        return pairs[: cnt.value].cpu().numpy()
