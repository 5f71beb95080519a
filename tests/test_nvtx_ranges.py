"""The library's public calls open named NVTX ranges (visible on Nsight
timelines; `ncu --nvtx --nvtx-include bfs_run/` captures only one call's
kernels).  Checked on the CPU: a child process loads the library with a
recording NVTX tool (tests/nvtx/nvtx_recorder.c) and makes calls that fail
their argument checks inside the range, so no GPU is touched."""
import os
import shutil
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

CHILD = r"""
import ctypes, sys
sys.path.insert(0, sys.argv[1])
from paper_1104_4518_gb300 import build
lib = ctypes.CDLL(build.build())
vp = ctypes.c_void_p
lib.bfs_run.argtypes = [vp, ctypes.c_int32, vp, vp, vp, vp]
lib.bfs_run_batch.argtypes = [vp, vp, ctypes.c_int32, vp, vp, vp, vp]
lib.bfs_graph_create.argtypes = [vp, vp, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, vp]
lib.bfs_graph_info.argtypes = [vp, vp, vp, vp]
assert lib.bfs_run(None, 0, None, None, None, None) == 1
assert lib.bfs_run_batch(None, None, 0, None, None, None, None) == 1
assert lib.bfs_graph_create(None, None, 5, 0, 0, None) == 1
assert lib.bfs_graph_info(None, None, None, None) == 1   # no range: a query, not a call that runs work
"""


def test_public_calls_open_and_close_named_ranges(tmp_path):
    if not shutil.which("gcc"):
        pytest.skip("gcc not available")
    rec = tmp_path / "librecorder.so"
    subprocess.run(["gcc", "-shared", "-fPIC", "-O1", "-o", str(rec), os.path.join(HERE, "nvtx", "nvtx_recorder.c")],
                   check=True)
    out = tmp_path / "ranges.txt"
    env = dict(os.environ, NVTX_INJECTION64_PATH=str(rec), NVTX_RECORD_PATH=str(out))
    subprocess.run([sys.executable, "-c", CHILD, ROOT], env=env, check=True, cwd=ROOT)
    lines = out.read_text().splitlines()
    assert lines == ["push bfs_run", "pop", "push bfs_run_batch", "pop", "push bfs_graph_create", "pop"]
