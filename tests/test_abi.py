"""CPU checks of the C ABI: the library builds, loads and exports every symbol
the header declares; struct layouts agree between C and the binding; host-side
argument validation answers before any CUDA call."""
import ctypes
import os
import re
import subprocess
import sys
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sgd_tucker.h")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as ge
    ge.build()
    from paper_2012_03550_gb300 import binding
    return binding


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(std_[a-z_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for must in ["std_create", "std_sgd_epoch", "std_predict", "std_rmse", "std_get_params",
                 "std_set_params", "std_destroy", "std_last_error", "std_default_options",
                 "std_sgd_batches", "std_schedule"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    L = ctypes.CDLL(lib.library_path())
    missing = [n for n in _declared_functions() if not hasattr(L, n)]
    assert not missing, missing
    assert set(_declared_functions()) <= set(lib.SIGNATURES)


def test_struct_layouts_match_c(lib, tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "sgd_tucker.h"\n'
        "int main(void){\n"
        'printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(std_options), offsetof(std_options, stream),'
        " offsetof(std_options, watchdog_ns), offsetof(std_options, hbm_budget_bytes),"
        " sizeof(std_epoch_stats), sizeof(std_probe));\n"
        'printf("%zu %zu %zu %zu\\n", sizeof(std_batch_stats), offsetof(std_batch_stats, graph_replayed),'
        " offsetof(std_options, contraction), offsetof(std_options, momentum));\n"
        'printf("%zu\\n", offsetof(std_options, snapshot));\n'
        'printf("%d %d %d %d\\n", STD_MAX_ORDER, STD_MAX_RANK, STD_MAX_CORE, STD_MAX_MINIBATCH);\n'
        "return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    c_sizes = [int(v) for v in out[0].split()]
    py = [ctypes.sizeof(lib.std_options), lib.std_options.stream.offset, lib.std_options.watchdog_ns.offset,
          lib.std_options.hbm_budget_bytes.offset, ctypes.sizeof(lib.std_epoch_stats), ctypes.sizeof(lib.std_probe)]
    assert c_sizes == py
    b_sizes = [int(v) for v in out[1].split()]
    assert b_sizes == [ctypes.sizeof(lib.std_batch_stats), lib.std_batch_stats.graph_replayed.offset,
                       lib.std_options.contraction.offset, lib.std_options.momentum.offset]
    assert int(out[2]) == lib.std_options.snapshot.offset
    lims = [int(v) for v in out[3].split()]
    assert lims == [lib.STD_MAX_ORDER, lib.STD_MAX_RANK, lib.STD_MAX_CORE, lib.STD_MAX_MINIBATCH]


def test_default_options(lib):
    o = lib.std_default_options()
    assert (o.r_core, o.precision, o.norm_mode, o.ptr_kind, o.ctas) == (5, 0, 0, 0, 0)
    assert (o.init_mu, o.init_sigma) == (0.5, 0.1)


@pytest.mark.parametrize("order,sizes,ranks,r_core,code", [
    (1, [5], [2], 2, -1),                 # order < 2
    (7, [5] * 7, [2] * 7, 2, -6),         # order > STD_MAX_ORDER
    (3, [5, 0, 5], [2, 2, 2], 2, -1),     # empty mode
    (3, [5, 5, 5], [2, 0, 2], 2, -1),     # rank 0
    (3, [5, 5, 5], [2, 33, 2], 2, -6),    # rank > STD_MAX_RANK
    (3, [5, 5, 5], [2, 2, 2], 0, -1),     # R_core 0
    (3, [5, 5, 5], [2, 2, 2], 40, -6),    # R_core > STD_MAX_RANK
    (3, [5, 5, 5], [32, 32, 32], 2, -6),  # prod J > STD_MAX_CORE
])
def test_create_rejects_bad_shapes_on_the_host(lib, order, sizes, ranks, r_core, code):
    o = lib.std_default_options()
    o.r_core = r_core
    idx = np.zeros((1, order), np.int32)
    val = np.zeros(1, np.float32)
    with pytest.raises(lib.StdError) as ei:
        lib.std_create(order, sizes, ranks, 1, idx, val, o)
    assert ei.value.code == code


def test_create_rejects_bad_options_and_nnz(lib):
    idx = np.zeros((1, 3), np.int32)
    val = np.zeros(1, np.float32)
    for field, value in [("precision", 2), ("norm_mode", 3), ("ptr_kind", 5), ("ctas", -1), ("init_mode", 9),
                         ("contraction", 2), ("momentum", 1.0), ("momentum", -0.1), ("momentum", float("nan")),
                         ("snapshot", -1), ("tile", 3), ("tile", -1), ("tile", 8)]:
        o = lib.std_default_options()
        setattr(o, field, value)
        with pytest.raises(lib.StdError) as ei:
            lib.std_create(3, [4, 4, 4], [2, 2, 2], 1, idx, val, o)
        assert ei.value.code == lib.STD_EINVAL
    with pytest.raises(lib.StdError) as ei:
        lib.std_create(3, [4, 4, 4], [2, 2, 2], 0, idx, val, None)
    assert ei.value.code == lib.STD_EINVAL
    # the K-snapshot form: at most 64 minibatches per block, and no momentum
    o = lib.std_default_options()
    o.snapshot = 65
    with pytest.raises(lib.StdError) as ei:
        lib.std_create(3, [4, 4, 4], [2, 2, 2], 1, idx, val, o)
    assert ei.value.code == lib.STD_EUNSUPPORTED
    o.snapshot = 4
    o.momentum = 0.5
    with pytest.raises(lib.StdError) as ei:
        lib.std_create(3, [4, 4, 4], [2, 2, 2], 1, idx, val, o)
    assert ei.value.code == lib.STD_EINVAL


def test_null_context_is_rejected(lib):
    with pytest.raises(lib.StdError):
        lib.std_sgd_epoch(None, 0.1, 0.1, 0.0, 0.0, 16)
    with pytest.raises(lib.StdError):
        lib.std_rmse(None, 1, np.zeros((1, 3), np.int32), np.zeros(1, np.float32))
    with pytest.raises(lib.StdError):
        lib.std_progress(None)
    with pytest.raises(lib.StdError):
        lib.std_reserve(None, 16, 1, 0)
    with pytest.raises(lib.StdError):
        lib.std_device_bytes(None)
    with pytest.raises(lib.StdError):
        lib.std_batch_step(None, 0.1, 0.1, 0.0, 0.0, 16, 1)
    with pytest.raises(lib.StdError):
        lib.std_batch_reset(None, [])
    with pytest.raises(lib.StdError):
        lib.std_batch_set_groups(None, [4])
    with pytest.raises(lib.StdError):
        lib.std_batch_groups(None, 1)
    with pytest.raises(lib.StdError):
        lib.std_batch_tile(None)
    with pytest.raises(lib.StdError):
        lib.std_predict_many([None], [np.zeros((1, 3), np.int32)], [np.zeros(1, np.float32)])
    lib.std_destroy(None)
