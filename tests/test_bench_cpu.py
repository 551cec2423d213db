"""CPU checks of the benchmark script: it compiles, its argument parser knows the
contract's flags, the reference arm (the FP64 oracle on the host cores) prints a
consistent JSON line, and the DRAM traffic of a profile summary is used only while
the kernel sources match the ones it was taken from."""
import json
import os
import py_compile
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_bench_compiles():
    py_compile.compile(os.path.join(ROOT, "bench.py"), doraise=True)


def test_bench_help_lists_contract_flags():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--help"], capture_output=True, text=True,
                         check=True).stdout
    for flag in ("--gpus", "--steps", "--warmup", "--impl"):
        assert flag in out


def test_reference_arm_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, check=True, timeout=600).stdout
    lines = [ln for ln in out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 1 and d["higher_is_better"] is True
    assert d["unit"] == "det-ratio evals/s" and d["value"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and "sample" in cb
    # one step = one sweep (1000 moves) of one walker per core: the rate and the step time agree
    assert d["value"] == pytest.approx(cb["cores"] * 1000 / (d["ms_per_step"] / 1000.0), rel=1e-9)
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_profiled_traffic_requires_matching_sources(tmp_path, monkeypatch):
    import bench

    (tmp_path / "profiles").mkdir()
    digest = bench.sources_digest()
    assert len(digest) == 64
    good = tmp_path / "profiles" / "k_good.md"
    good.write_text(f"# summary\n\ntraffic_bytes_per_launch: 1234\nsources_sha256: {digest}\n")
    stale = tmp_path / "profiles" / "k_stale.md"
    stale.write_text("traffic_bytes_per_launch: 1234\nsources_sha256: " + "0" * 64 + "\n")
    monkeypatch.setattr(bench, "ROOT", tmp_path)
    monkeypatch.setattr(bench, "sources_digest", lambda: digest)
    assert bench.profiled_traffic("k_good.md") == 1234.0
    assert bench.profiled_traffic("k_stale.md") is None
    assert bench.profiled_traffic("k_missing.md") is None


def test_source_digest_ignores_comments_only():
    import bench

    code = 'int f(int x) {\n  return x + 1;  // one\n}\nconst char* s = "// kept /* too */";\n'
    commented = '/* header\n   text */\nint f(int x) {\n\n  return x + 1;  // two, longer\n}\n' \
                'const char* s = "// kept /* too */";  /* trailing */\n'
    changed = code.replace("x + 1", "x + 2")
    strip = bench.strip_c_comments
    assert strip(code) == strip(commented)
    assert strip(code) != strip(changed)
    assert '"// kept /* too */"' in strip(code)
    assert strip("char c = '\\''; // q\nint y;") == "char c = '\\'';\nint y;"
