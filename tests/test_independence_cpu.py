"""Static checks of the separation between the product path and the oracle, and of the
device code's failure handling (CPU only, reads the sources as text).

- The package (CUDA sources, C ABI, binding) never imports, includes or loads the
  oracle, and the oracle never imports or includes the package: they share no code.
- The workload parameter module, which both sides read, holds no arithmetic of the
  method (plain data and seed lists).
- Device code reports failures through status words: no trap, no device assert."""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1008_5113_gb300")
ORC = os.path.join(ROOT, "oracle")


def _files(top, exts):
    for d, _, fs in os.walk(top):
        if "__pycache__" in d:
            continue
        for f in fs:
            if f.endswith(exts):
                yield os.path.join(d, f)


def _py_imports(path):
    tree = ast.parse(open(path, encoding="utf-8").read())
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            for a in node.names:
                yield a.name
        elif isinstance(node, ast.ImportFrom):
            yield (node.module or "") if node.level == 0 else "." * node.level + (node.module or "")


def test_package_does_not_use_the_oracle():
    for path in _files(PKG, (".py",)):
        for mod in _py_imports(path):
            assert not mod.split(".")[0] == "oracle", f"{path} imports {mod}"
    for path in _files(PKG, (".py", ".cu", ".cuh", ".h", ".c")):
        text = open(path, encoding="utf-8").read()
        assert not re.search(r'#\s*include\s*[<"][^>"]*oracle', text), path
        assert "liboracle" not in text and "orc_" not in text, path


def test_oracle_does_not_use_the_package():
    for path in _files(ORC, (".py",)):
        for mod in _py_imports(path):
            assert not mod.startswith("paper_1008_5113_gb300"), f"{path} imports {mod}"
    for path in _files(ORC, (".c", ".h", ".py")):
        text = open(path, encoding="utf-8").read()
        assert "csrc" not in text and "vmc.h" not in text and "libvmc" not in text, path


def test_workload_module_holds_no_method_arithmetic():
    path = os.path.join(PKG, "workloads.py")
    imports = set(_py_imports(path))
    assert imports <= {"__future__", "dataclasses", "math"}, imports
    called = set()
    for node in ast.walk(ast.parse(open(path, encoding="utf-8").read())):
        if isinstance(node, ast.Call):
            f = node.func
            called.add(f.attr if isinstance(f, ast.Attribute) else getattr(f, "id", "?"))
    # parameter sets and seed lists only; sqrt and log derive the paper workload's cutoff
    assert called <= {"Workload", "dataclass", "field", "len", "range", "dict", "sqrt", "log"}, called


def test_device_code_has_no_traps_or_asserts():
    for path in _files(os.path.join(PKG, "csrc"), (".cu", ".cuh", ".h")):
        text = open(path, encoding="utf-8").read()
        assert "__trap" not in text, path
        assert not re.search(r"\bassert\s*\(", text), path
        assert not re.search(r'asm[^;]*"\s*trap', text), path
        assert "brkpt" not in text, path


def test_product_path_fails_loudly_without_its_library(monkeypatch, tmp_path):
    from paper_1008_5113_gb300 import vmc

    monkeypatch.setattr(vmc, "LIB", str(tmp_path / "libvmc.so"))
    monkeypatch.setattr(vmc, "_lib", None)
    try:
        vmc.lib()
    except RuntimeError as e:
        assert "no CPU fallback" in str(e)
    else:
        raise AssertionError("loading a missing library succeeded")
