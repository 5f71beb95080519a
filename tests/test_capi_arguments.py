"""Argument checks of the C ABI, on the CPU: every entry point rejects NULL
pointers, sizes out of range and bad sources with BFS_ERR_INVALID_ARG and a
message, before it touches a device; without a usable CUDA device, graph
creation answers BFS_ERR_UNSUPPORTED instead of failing later."""
import ctypes

import numpy as np
import pytest

INVALID_ARG = 1
UNSUPPORTED = 6

vp = ctypes.c_void_p
i32, i64, u32 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32


@pytest.fixture(scope="module")
def lib():
    from paper_1104_4518_gb300 import build
    lib = ctypes.CDLL(build.build())
    lib.bfs_last_error.restype = ctypes.c_char_p
    sig = {
        "bfs_graph_create": [vp, vp, i32, i64, u32, ctypes.POINTER(vp)],
        "bfs_graph_create_from_edges": [vp, vp, i64, i32, u32, vp, ctypes.POINTER(vp)],
        "bfs_graph_union": [vp, i32, vp, ctypes.POINTER(vp)],
        "bfs_graph_info": [vp, vp, vp, vp],
        "bfs_run": [vp, i32, vp, vp, vp, vp],
        "bfs_run_batch": [vp, vp, i32, vp, vp, vp, vp],
        "bfs_run_ragged": [vp, vp, vp, vp, vp, vp],
        "bfs_run_static": [vp, vp, i32, i64, i32, vp, vp, vp],
        "bfs_sync": [vp, vp],
        "bfs_set_tuning": [vp, vp],
        "bfs_get_tuning": [vp, vp],
        "bfs_autotune": [vp, vp, i32, vp, vp],
        "bfs_mlp_forward": [vp, vp, i32, vp, vp],
        "bfs_mlp_loss_grad": [vp, vp, vp, i32, vp, vp, vp],
        "bfs_selector_load": [ctypes.c_char_p],
        "bfs_level_features": [i32, i64, i32, i64, i64, i64, i64, vp, vp],
        "bfs_spmsv_sorted": [vp, vp, i32, vp, vp, vp, vp, vp],
        "bfs_run_sorted": [vp, i32, vp, vp, vp],
        "bfs_graph_half": [vp, vp, vp],
        "bfs_run_half": [vp, i32, vp, vp, vp],
    }
    for name, args in sig.items():
        getattr(lib, name).argtypes = args
    return lib


def expect(lib, rc, code, words):
    msg = lib.bfs_last_error().decode()
    assert rc == code, (rc, msg)
    assert words in msg, msg


def test_graph_creation_rejects_bad_arguments(lib):
    off = np.array([0, 1, 2], np.int64)
    adj = np.array([1, 0], np.int32)
    out = vp()
    expect(lib, lib.bfs_graph_create(off.ctypes.data, adj.ctypes.data, 2, 2, 1, None), INVALID_ARG, "NULL out")
    expect(lib, lib.bfs_graph_create(off.ctypes.data, adj.ctypes.data, 0, 2, 1, ctypes.byref(out)), INVALID_ARG,
           "n out of range")
    expect(lib, lib.bfs_graph_create(off.ctypes.data, adj.ctypes.data, 2, -1, 1, ctypes.byref(out)), INVALID_ARG,
           "nnz out of range")
    expect(lib, lib.bfs_graph_create(None, adj.ctypes.data, 2, 2, 1, ctypes.byref(out)), INVALID_ARG, "NULL array")
    expect(lib, lib.bfs_graph_create(off.ctypes.data, None, 2, 2, 1, ctypes.byref(out)), INVALID_ARG, "NULL array")
    expect(lib, lib.bfs_graph_create_from_edges(adj.ctypes.data, adj.ctypes.data, 2, 2, 1, None, None), INVALID_ARG,
           "NULL out")
    expect(lib, lib.bfs_graph_create_from_edges(adj.ctypes.data, adj.ctypes.data, -1, 2, 1, None, ctypes.byref(out)),
           INVALID_ARG, "m out of range")
    expect(lib, lib.bfs_graph_union(None, 0, None, ctypes.byref(out)), INVALID_ARG, "bad argument")
    assert out.value is None


def test_runs_reject_missing_graphs_and_bad_sources(lib):
    buf = np.zeros(8, np.int32)
    p = buf.ctypes.data
    expect(lib, lib.bfs_run(None, 0, p, p, None, None), INVALID_ARG, "NULL graph")
    expect(lib, lib.bfs_run_batch(None, p, 1, p, p, None, None), INVALID_ARG, "NULL graph")
    expect(lib, lib.bfs_run_ragged(None, p, None, None, None, None), INVALID_ARG, "NULL graph")
    expect(lib, lib.bfs_sync(None, None), INVALID_ARG, "NULL graph")
    expect(lib, lib.bfs_set_tuning(None, None), INVALID_ARG, "NULL graph")
    expect(lib, lib.bfs_get_tuning(None, None), INVALID_ARG, "NULL graph")
    expect(lib, lib.bfs_autotune(None, None, 0, None, None), INVALID_ARG, "NULL graph")
    expect(lib, lib.bfs_graph_info(None, None, None, None), INVALID_ARG, "NULL graph")
    expect(lib, lib.bfs_graph_tiles(None, 0, 0, None, None), INVALID_ARG, "NULL graph")
    cnt = ctypes.c_int32(5)
    expect(lib, lib.bfs_spmsv_sorted(None, p, 1, None, p, p, ctypes.byref(cnt), None), INVALID_ARG, "NULL graph")
    expect(lib, lib.bfs_run_sorted(None, 0, p, p, None), INVALID_ARG, "NULL graph")
    expect(lib, lib.bfs_graph_half(None, None, None), INVALID_ARG, "NULL graph")
    expect(lib, lib.bfs_run_half(None, 0, p, p, None), INVALID_ARG, "NULL graph")


def test_static_entry_point_checks_before_any_device_work(lib):
    off = np.array([0, 1, 2], np.int64)
    adj = np.array([1, 0], np.int32)
    out = np.zeros(2, np.int32)
    o, a, q = off.ctypes.data, adj.ctypes.data, out.ctypes.data
    expect(lib, lib.bfs_run_static(o, a, 1 << 21, 2, 0, q, q, None), INVALID_ARG, "n must be in")
    expect(lib, lib.bfs_run_static(o, a, 2, 1 << 27, 0, q, q, None), INVALID_ARG, "nnz must be in")
    expect(lib, lib.bfs_run_static(o, a, 2, 2, 5, q, q, None), INVALID_ARG, "source outside")
    expect(lib, lib.bfs_run_static(o, a, 2, 2, -1, q, q, None), INVALID_ARG, "source outside")
    expect(lib, lib.bfs_run_static(o, a, 2, 2, 0, None, q, None), INVALID_ARG, "NULL pointer")
    expect(lib, lib.bfs_run_static(None, a, 2, 2, 0, q, q, None), INVALID_ARG, "NULL pointer")


def test_selector_calls_check_their_arguments(lib):
    expect(lib, lib.bfs_mlp_forward(None, None, 4, None, None), INVALID_ARG, "bad argument")
    expect(lib, lib.bfs_mlp_loss_grad(None, None, None, 4, None, None, None), INVALID_ARG, "")
    expect(lib, lib.bfs_selector_load(b"/nonexistent/selector_weights.bin"), INVALID_ARG, "cannot open")
    expect(lib, lib.bfs_level_features(10, 20, 0, 1, 1, 1, 1, None, None), INVALID_ARG, "NULL pointer")


def test_graph_creation_without_a_device_is_unsupported(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    off = np.array([0, 1, 2], np.int64)
    adj = np.array([1, 0], np.int32)
    out = vp()
    rc = lib.bfs_graph_create(off.ctypes.data, adj.ctypes.data, 2, 2, 1, ctypes.byref(out))  # BFS_HOST_PTRS
    assert rc == UNSUPPORTED, lib.bfs_last_error()
    assert out.value is None
