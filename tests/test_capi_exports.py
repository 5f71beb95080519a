"""CPU checks of the C-ABI library and of the oracle's independence (no GPU needed).

- every function declared in include/bfs.h is exported by libbfs_gb300.so and
  by its bounds-checking build libbfs_gb300_checked.so, and nothing else is;
  each library says which build it is;
- the product package never imports the oracle, and the oracle never includes
  or loads the library's sources.
"""
import ctypes
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bfs.h")
PKG = os.path.join(ROOT, "paper_1104_4518_gb300")


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^BFS_API\s+[\w\s\*]*?\b(bfs_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1104_4518_gb300 import build as b
    return b.build()


@pytest.fixture(scope="module")
def checked_libpath():
    from paper_1104_4518_gb300 import build as b
    return b.build_checked()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("bfs_graph_create", "bfs_graph_create_from_edges", "bfs_run", "bfs_run_batch",
                     "bfs_run_ragged", "bfs_graph_destroy", "bfs_graph_info", "bfs_last_error",
                     "bfs_selector_train", "bfs_autotune", "bfs_mlp_forward", "bfs_mlp_loss_grad"):
        assert required in names


def test_library_loads_and_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert exported == set(declared_functions())
    lib.bfs_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.bfs_version()
    assert lib.bfs_bounds_checked() == 0


def test_bounds_checking_build_exports_the_same_symbols(checked_libpath):
    lib = ctypes.CDLL(checked_libpath)
    out = subprocess.run(["nm", "-D", "--defined-only", checked_libpath], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert exported == set(declared_functions())
    assert lib.bfs_bounds_checked() == 1
    lib.bfs_version.restype = ctypes.c_char_p
    assert b"bounds-checking" in lib.bfs_version()


def test_environment_selects_the_bounds_checking_library():
    code = "import paper_1104_4518_gb300 as b; print(b.BOUNDS_CHECKED, b.LIB_PATH)"
    for val, want in (("1", "libbfs_gb300_checked.so"), ("0", "libbfs_gb300.so")):
        env = dict(os.environ, BFS_BOUNDS_CHECK=val)
        out = subprocess.run(["python", "-c", code], cwd=ROOT, env=env, capture_output=True, text=True, check=True)
        assert out.stdout.split()[0] == str(val == "1") and out.stdout.split()[1].endswith(want)


def test_version_and_error_string_need_no_gpu(libpath):
    # a process that made no failing call has an empty message
    code = ("import ctypes, sys; l = ctypes.CDLL(sys.argv[1]); l.bfs_last_error.restype = ctypes.c_char_p; "
            "print(repr(l.bfs_last_error()))")
    fresh = subprocess.run([sys.executable, "-c", code, libpath], capture_output=True, text=True, check=True)
    assert fresh.stdout.strip() == "b''"
    lib = ctypes.CDLL(libpath)
    lib.bfs_last_error.restype = ctypes.c_char_p
    # an argument error is reported without touching a device
    lib.bfs_graph_info.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    assert lib.bfs_graph_info(None, None, None, None) == 1
    assert b"NULL graph" in lib.bfs_last_error()


def test_product_never_imports_oracle():
    for dirpath, _, files in os.walk(PKG):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".c")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", text, flags=re.M), f
                assert "bfs_oracle" not in text and "liboracle" not in text, f


def test_oracle_shares_no_code_with_cuda_path():
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c", ".h")):
            text = open(os.path.join(ROOT, "oracle", f)).read()
            assert "csrc" not in text and "libbfs_gb300" not in text and "bfs.h" not in text, f
            assert not re.search(r"paper_1104_4518_gb300\s+import\s+(?!inputs)", text), f


def test_python_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    import paper_1104_4518_gb300 as bfs
    monkeypatch.setattr(bfs, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(bfs, "_lib", None)
    with pytest.raises(ImportError):
        bfs.lib()
