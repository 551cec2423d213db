"""CPU checks of the C ABI library: it loads, exports every entry point that
include/vmc.h declares, and rejects invalid arguments without touching a GPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def vmc():
    from paper_1008_5113_gb300.build import build_library

    build_library()
    from paper_1008_5113_gb300 import vmc as v

    v.lib()
    return v


def _declared():
    src = open(os.path.join(ROOT, "include", "vmc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(vmc_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported_and_bound(vmc):
    names = _declared()
    assert len(names) >= 20
    lib = vmc.lib()
    for name in names:
        assert hasattr(lib, name), name
        assert name in vmc._SIG, f"binding lacks {name}"
    assert set(vmc._SIG) == set(names)


def test_default_params(vmc):
    p = vmc.vmc_default_params()
    assert p.drop_tol == 1e-4 and p.permtol == 0.5 and p.gmres_m == 30
    assert p.N_max == 100.0 and p.slow_factor == 4.0 and p.lfil_extra == -1
    assert p.precision == vmc.PREC_MIXED and p.engine == vmc.ENGINE_PERSISTENT
    assert p.max_updates == -1 and p.refactor_lag == -1 and p.graphs == 1 and p.trisolve == 0
    assert p.trisolve_group == 8 and p.trisolve_row_cap == 0 and p.trisolve_lane_entries == 0


@pytest.mark.parametrize("system,why", [
    ((6, 0, 1.0, 2.0, 3.5), "half the box"),          # r_c >= L/2
    ((6, 0, 1.0, 2.0, 0.8), "covering radius"),       # rows could be empty
    ((1, 0, 1.0, 2.0, 0.9), "K must be"),
    ((6, 2, 1.0, 2.0, 1.5), "lattice"),
    ((6, 0, 1.0, -1.0, 1.5), "kappa"),
    ((40, 0, 1.0, 0.5, 12.0), "256 orbitals"),
])
def test_create_rejects_invalid_systems(vmc, system, why):
    with pytest.raises(vmc.VmcError) as e:
        vmc.vmc_create([system])
    assert e.value.status == 1 and why in str(e.value)


@pytest.mark.parametrize("field,value", [("gmres_m", 0), ("gmres_m", 41), ("max_updates", 129), ("max_updates", -2),
                                         ("block_threads", 100), ("block_threads", 1024), ("precision", 3),
                                         ("engine", 7), ("drop_tol", -1.0), ("trisolve_row_cap", 481),
                                         ("trisolve_row_cap", -1), ("trisolve_lane_entries", 65),
                                         ("trisolve_lane_entries", -1), ("trisolve_group", 65)])
def test_create_rejects_invalid_params(vmc, field, value):
    with pytest.raises(vmc.VmcError) as e:
        vmc.vmc_create([(6, 0, 1.0, 2.0, 1.5)], vmc.params(**{field: value}))
    assert e.value.status == 1


def test_create_rejects_rows_longer_than_a_stream_slot(vmc):
    with pytest.raises(vmc.VmcError) as e:
        vmc.vmc_create([(6, 0, 1.0, 2.0, 1.5)], vmc.params(lfil_extra=1000))
    assert e.value.status == 1 and "stream slot" in str(e.value)


def test_null_arguments(vmc):
    lib = vmc.lib()
    assert lib.vmc_create(None, 1, None, None, None) == 1
    assert lib.vmc_default_params(None) == 1
    assert lib.vmc_destroy(None) == 1
    assert lib.vmc_philox_device(None, None, None, 0) == 1


def test_struct_layouts_match_the_header(vmc, tmp_path):
    """The binding's ctypes structures have the C compiler's sizes and offsets."""
    import shutil
    import subprocess

    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    structs = {"vmc_system": vmc.vmc_system, "vmc_solver_params": vmc.vmc_solver_params,
               "vmc_stats": vmc.vmc_stats, "vmc_tune_trial": vmc.vmc_tune_trial}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "vmc.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name}.{field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                         check=True).stdout.split("\n") if l)
    for name, cls in structs.items():
        assert int(out[name]) == C.sizeof(cls), name
        for field, _ in cls._fields_:
            assert int(out[f"{name}.{field}"]) == getattr(cls, field).offset, f"{name}.{field}"


def test_autotune_rejects_bad_arguments_without_a_gpu(vmc):
    lib = vmc.lib()
    p = vmc.vmc_default_params()
    sysarr = (vmc.vmc_system * 1)(vmc.vmc_system(6, 0, 1.0, 2.0, 1.5))
    seeds = (C.c_uint64 * 1)(1)
    n = C.c_int(-1)
    assert lib.vmc_autotune(None, 1, C.byref(p), seeds, 0.1, 0.2, 64, None, 0, C.byref(n), None) == 1
    assert n.value == 0
    assert lib.vmc_autotune(sysarr, 1, C.byref(p), seeds, 0.1, 0.2, 0, None, 0, None, None) == 1
    p.engine = vmc.ENGINE_DENSE_SM
    assert lib.vmc_autotune(sysarr, 1, C.byref(p), seeds, 0.1, 0.2, 64, None, 0, None, None) == 1


def test_c_example_compiles_against_the_header(tmp_path):
    """The C example of the ABI compiles as plain C against include/vmc.h."""
    import shutil
    import subprocess

    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    src = os.path.join(ROOT, "paper_1008_5113_gb300", "examples", "vmc_sweep_example.c")
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), "-c", src, "-o",
                    str(tmp_path / "example.o")], check=True)
