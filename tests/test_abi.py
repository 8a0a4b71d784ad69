"""CPU checks of the C ABI: the library builds, loads and exports every function
declared in include/ibmlbm.h; configuration checks and workspace sizing (host
code only, no GPU call)."""
import ctypes as C
import re

import pytest

from paper_2002_08855_gb300 import binding, build, inputs


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.lib()


def declared_functions():
    text = open(binding.HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ibm_lbm_\w+)\s*\(", text)))


def test_every_declared_function_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    # the binding knows every declared function and nothing else
    assert sorted(binding.SIGNATURES) == names


def test_bounds_checked_library_exports_the_same_calls(lib):
    build.build(checked=True)
    L = binding.lib(checked=True)
    for name in declared_functions():
        assert hasattr(L, name), name
    assert L is not lib


def test_config_struct_matches_header(lib):
    text = open(binding.HEADER).read()
    body = text[text.index("typedef struct ibm_lbm_config"):text.index("} ibm_lbm_config;")]
    fields = re.findall(r"\b(?:uint32_t|int32_t|double)\s+([^;]+);", body)
    names = []
    for f in fields:
        for part in f.split(","):
            names.append(re.sub(r"\[.*\]", "", part).strip())
    assert names == [n for n, _ in binding.Config._fields_]


def test_workspace_size_of_the_2048x4096_cavity(lib):
    w = inputs.cavity_2d_large(0.1)
    n = binding.workspace_size(w)
    pdfs = 9 * 2048 * 4096 * 4
    fib = 2 * 2048 * 4096 * 4  # f_IB (2D keeps u* per particle box, not on the grid)
    points = w.n_particles * w.n_lag * 2 * (8 + 8 + 4 + 4 + 4 + 4 + 4)  # X_b x2, U_b x2, F_b, dF_b, D_I u*
    boxes = w.n_particles * 2 * 16 * 20 * 4  # u* of each particle's 16 x 16 node box (row pitch 20)
    need = pdfs + fib + points + boxes
    assert need < n < need * 1.05


def test_half_precision_storage_halves_the_pdf_bytes(lib):
    w = inputs.cavity_2d_large(0.1)
    n32 = binding.workspace_size(w)
    n16 = binding.workspace_size(w.with_(pdf_storage=1))
    assert n32 - n16 == 9 * 2048 * 4096 * 2
    assert binding.workspace_size(w.with_(pdf_storage=2)) == n16


@pytest.mark.parametrize("field,value,code", [
    ("dim", 4, "INVALID_ARG"), ("tau", 0.5, "INVALID_ARG"), ("nx", 0, "INVALID_ARG"),
    ("delta_kind", 5, "UNSUPPORTED"), ("n_lag", 0, "INVALID_ARG"), ("drs", 0.0, "INVALID_ARG"),
    ("pdf_storage", 3, "INVALID_ARG"),
])
def test_invalid_configurations_are_rejected(lib, field, value, code):
    w = inputs.cavity_2d_small().as_dict()
    w[field] = value
    with pytest.raises(binding.IbmLbmError) as e:
        binding.workspace_size(w)
    assert e.value.name == code
    assert lib.ibm_lbm_last_error().decode()


def test_struct_size_mismatch_rejected(lib):
    cfg = binding.make_config(inputs.cavity_2d_small())
    cfg.struct_size = 8
    n = C.c_size_t(0)
    assert lib.ibm_lbm_workspace_size(C.byref(cfg), C.byref(n)) == -1


def test_pair_scratch_size_host_only(lib):
    n = C.c_size_t(0)
    nodes = (C.c_int32 * 3)(2048, 4096, 1)
    assert lib.ibm_lbm_pair_search_scratch_size(2, nodes, 10.0, 2.0, 42723, 0, C.byref(n)) == 0
    assert n.value > 42723 * 32 * 4


def test_pair_search_sizes_stay_bounded_for_a_tiny_reach(lib):
    """A diameter and range far below one node on a 2^15 x 2^15 lattice would ask for
    2^60 cells: the cell grid merges cells down to 2^30 (a larger side keeps the search
    complete), the scratch size is finite, and the allocation-free entry point rejects
    the problem as too large for its fixed array before any device work (host only)."""
    nodes = (C.c_int32 * 3)(1 << 15, 1 << 15, 1)
    n = C.c_size_t(0)
    assert lib.ibm_lbm_pair_search_scratch_size(2, nodes, 1e-9, 1e-9, 100, 0, C.byref(n)) == 0
    assert (1 << 30) * 4 < n.value < (1 << 30) * 4 * 20
    dummy = (C.c_double * 200)()
    cnt = C.c_int64(-1)
    per = (C.c_int32 * 3)(0, 0, 0)
    rc = lib.ibm_lbm_pair_search_static(2, nodes, per, 1e-9, 1e-9, 100, C.cast(dummy, C.c_void_p),
                                        0, None, 0, C.byref(cnt), None)
    assert rc == -7 and cnt.value == 0
    assert "16777216" in lib.ibm_lbm_last_error().decode()


def _batch_sizes(ws):
    cfgs = (binding.Config * len(ws))(*[binding.make_config(w) for w in ws])
    n = C.c_size_t(0)
    rc = binding.lib().ibm_lbm_batch_workspace_size(cfgs, len(ws), C.byref(n))
    return rc, n.value


def test_batch_workspace_holds_every_member(lib):
    ws = inputs.ensemble_2d(8)
    rc, total = _batch_sizes(ws)
    assert rc == 0
    members = sum((binding.workspace_size(w) + 255) // 256 * 256 for w in ws)
    assert members < total < members + 4 * 1024 * 1024


@pytest.mark.parametrize("change,code", [
    (dict(dim=3, nz=8), -2), (dict(pdf_storage=2), -2), (dict(mdf_iters=2), -1)])
def test_batch_rejects_mixed_or_unsupported_members(lib, change, code):
    ws = inputs.ensemble_2d(3)
    ws[1] = ws[1].with_(**change)
    rc, _ = _batch_sizes(ws)
    assert rc == code
    assert lib.ibm_lbm_last_error().decode()


@pytest.mark.parametrize("changes", [
    dict(boundary=3),                                    # unknown kind
    dict(boundary=1, nx=2),                              # a wall axis needs 3 nodes
    dict(boundary=2, periodic=(0, 1, 0)),                # a channel needs walls on y
    dict(boundary=2, u_inlet=float("inf")),
])
def test_extrapolation_boundary_configurations_are_checked(lib, changes):
    w = inputs.cavity_2d_small().as_dict()
    w.update(changes)
    with pytest.raises(binding.IbmLbmError) as e:
        binding.workspace_size(w)
    assert "INVALID_ARG" in str(e.value)


def test_tile_shapes_reported_host_only(lib):
    """Shape 0 of the batch's collide-stream launch is the flat tiles (128 threads, four
    nodes a thread for FP32, two for the 16-bit storages); shapes 1.. are the warp tiles
    (K, W, persistent), the same for both storages."""
    s32, s16 = binding.tile_shapes(0), binding.tile_shapes(1)
    assert len(s32) == len(s16) == lib.ibm_lbm_tile_shape_count() >= 2
    assert s32[0] == (4, 4, 0) and s16[0] == (2, 4, 0)
    assert s32[1:] == s16[1:]
    assert all(k in (1, 2) and w in (4, 8) and p in (0, 1) for k, w, p in s32[1:])
    with pytest.raises(binding.IbmLbmError):
        binding.tile_shapes(3)  # no such storage
