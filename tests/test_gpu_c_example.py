"""The C ABI used from C: the example program is built against the in-tree library
and run on the GPU (every call must succeed, the logs be consistent)."""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c_example_runs(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    from paper_1008_5113_gb300.build import LIB, build_library

    build_library()
    libdir = os.path.dirname(LIB)
    exe = tmp_path / "example"
    subprocess.run(["gcc", "-std=c99", "-O2", os.path.join(ROOT, "paper_1008_5113_gb300", "examples",
                                                           "vmc_sweep_example.c"),
                    "-I", os.path.join(ROOT, "include"), libdir + "/libvmc.so", "-Wl,-rpath," + libdir, "-lm",
                    "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "accepted=" in out.stdout
