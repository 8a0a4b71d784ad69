"""Build ``libibmlbm.so`` in-tree with nvcc for sm_103a (no cmake, no torch).

The translation units compile in parallel; the link uses nvcc's static CUDA
runtime, so the library needs nothing at run time beyond the CUDA driver.
``build(checked=True)`` also builds ``libibmlbm_checked.so`` (``-DIBMLBM_CHECKED``:
every kernel index is checked against its array's extent and a failure is
reported by ``ibm_lbm_sync`` as IBMLBM_ERR_BOUNDS instead of an access out of
bounds), from the same sources in the same parallel compile.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libibmlbm.so")
OUT_CHECKED = os.path.join(OUT, "checked")
LIB_CHECKED = os.path.join(OUT, "libibmlbm_checked.so")
UNITS = ["lbm.cu", "ibm.cu", "pairs.cu", "api.cu", "pairs_static.cu", "mlp.cu"]
HEADERS = ["common.cuh", "launch.h", "pdf_access.cuh", "mlp.h", "pair_grid.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O3",
         "-I" + os.path.join(ROOT, "include"), "-I" + SRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA library cannot be built")


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Compile (if stale) and link the library; with checked, the bounds-checked one too."""
    os.makedirs(OUT, exist_ok=True)
    cc = nvcc()
    hdrs = [os.path.join(SRC, h) for h in HEADERS] + [os.path.join(ROOT, "include", "ibmlbm.h")]
    variants = [(OUT, LIB, [])] + ([(OUT_CHECKED, LIB_CHECKED, ["-DIBMLBM_CHECKED"])] if checked else [])
    jobs, links = [], []
    for out, lib, extra in variants:
        os.makedirs(out, exist_ok=True)
        objs = []
        for u in UNITS:
            src = os.path.join(SRC, u)
            obj = os.path.join(out, u.replace(".cu", ".o"))
            objs.append(obj)
            if force or _stale(obj, [src] + hdrs):
                cmd = [cc, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
                if verbose:
                    cmd.insert(1, "-Xptxas=-v")
                jobs.append(cmd)
        links.append((lib, objs))
    with cf.ThreadPoolExecutor(max_workers=max(1, len(jobs))) as ex:
        results = list(ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs))
    for cmd, r in zip(jobs, results):
        if verbose and r.stderr:
            print(r.stderr)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    for lib, objs in links:
        if force or _stale(lib, objs):
            tmp = lib + f".{os.getpid()}.tmp"
            r = subprocess.run([cc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
            os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
