"""CPU checks of the benchmark script: it compiles, and its argument parser knows the
driver's flags."""
import os
import py_compile
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_compiles():
    py_compile.compile(os.path.join(ROOT, "bench.py"), doraise=True)


def test_bench_help_lists_driver_flags():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--help"], capture_output=True, text=True,
                         check=True).stdout
    for flag in ("--gpus", "--steps", "--warmup", "--impl"):
        assert flag in out
