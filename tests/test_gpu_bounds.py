"""The bounds-checking build (libbfs_gb300_checked.so, -DBFS_BOUNDS_CHECK) on the
GPU, in child processes that load it (BFS_BOUNDS_CHECK=1):

- on well-formed graphs it raises no false alarm and stays bit-identical to the
  oracle for every selector and entry point;
- adjacency ids outside [0, n) in a row that a top-down, pull, batched or
  static traversal reads give BFS_ERR_BOUNDS naming the site, malformed row
  offsets give BFS_ERR_BOUNDS at graph creation (or per static call), and the
  library runs clean graphs correctly afterwards.

The cases themselves are in bounds_child.py; it refuses to run the malformed
inputs unless the library it loaded is the bounds-checking build.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def run_child(case):
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("GPU test run without a CUDA device")
    from paper_1104_4518_gb300 import build as b
    b.build_checked()
    env = dict(os.environ, BFS_BOUNDS_CHECK="1")
    r = subprocess.run([sys.executable, os.path.join(HERE, "bounds_child.py"), case], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=900)
    print(r.stdout)
    assert r.returncode == 0, f"bounds_child {case} failed:\n{r.stdout}\n{r.stderr[-4000:]}"
    assert r.stdout.strip().endswith("done")
    return r.stdout


def test_checked_build_is_bit_identical_on_well_formed_graphs():
    out = run_child("parity")
    for line in ("single-source rmat14: ok", "batched rmat14: ok", "star 5000: ok", "directed rmat13: ok",
                 "ragged union: ok", "static entry: ok"):
        assert line in out


def test_checked_build_reports_bad_indices():
    out = run_child("malformed")
    assert out.count("BFS_ERR_BOUNDS") == 3 + 3 + 1 + 1 + 2 + 2 + 2  # + the tiled variant's tile builder
    assert "clean runs after the errors: ok" in out
