"""The boundary is a C ABI: include/bfs.h compiles as strict C99 (gcc
-std=c99 -pedantic -Wall -Wextra -Werror), a C program links against
libbfs_gb300.so and against its bounds-checking twin, and its calls return
the documented statuses (tests/c_abi/consumer.c; calls that need no GPU)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.mark.parametrize("checked", [False, True])
def test_c_program_compiles_links_and_runs(tmp_path, checked):
    if not shutil.which("gcc"):
        pytest.skip("gcc not available")
    from paper_1104_4518_gb300 import build
    lib = build.build_checked() if checked else build.build()
    libdir, libfile = os.path.split(lib)
    name = libfile[len("lib"):-len(".so")]
    exe = tmp_path / "consumer"
    subprocess.run(["gcc", "-std=c99", "-pedantic", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                    os.path.join(HERE, "c_abi", "consumer.c"), "-o", str(exe), "-L", libdir, f"-l{name}",
                    f"-Wl,-rpath,{libdir}"], check=True)
    r = subprocess.run([str(exe)] + (["--checked"] if checked else []), capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "bounds-checking" in r.stdout if checked else "bounds-checking" not in r.stdout
