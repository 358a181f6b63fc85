"""The C-ABI library builds, loads and exports every symbol include/poisson.h
declares; host-only entry points (argument validation, workspace sizing, error
text) work without a GPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "poisson.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2605_03563_gb300 import build as B
    B.build()
    from paper_2605_03563_gb300 import capi
    return capi.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(poisson_\w+|ps_op_\w+|ps_probe_\w+)\s*\(", text)))


def test_every_declared_symbol_is_exported_and_bound(lib):
    from paper_2605_03563_gb300 import capi
    names = declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
        assert n in capi.SIGNATURES, n


def test_struct_layouts_match_the_header(tmp_path):
    """Every field offset and struct size of the ctypes binding equals what a C
    compiler makes of include/poisson.h."""
    import shutil
    import subprocess
    from paper_2605_03563_gb300 import capi
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"ps_grid": capi.PsGrid, "ps_bc": capi.PsBC, "ps_solve_opts": capi.PsSolveOpts,
               "ps_info": capi.PsInfo, "ps_kernel_stat": capi.PsKernelStat,
               "ps_tuning": capi.PsTuning}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "poisson.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    inc = os.path.join(ROOT, "include")
    subprocess.run([cc, "-std=c99", "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    seen = 0
    for line in out:
        if not line.strip():
            continue
        cname, what, val = line.split()
        py = structs[cname]
        got = C.sizeof(py) if what == "size" else getattr(py, what).offset
        assert got == int(val), (cname, what, got, val)
        seen += 1
    assert seen == sum(len(p._fields_) + 1 for p in structs.values())


def test_invalid_arguments_rejected_before_gpu_work(lib):
    from paper_2605_03563_gb300 import capi
    h = C.c_void_p()
    bad = capi.make_grid(32)
    assert lib.poisson_create(C.byref(bad), None, 3, None, 4, C.byref(h)) == capi.PS_ERR_INVALID_ARG
    assert b"stencil_order" in lib.poisson_last_error()
    tiny = capi.make_grid((1, 8, 8))
    assert lib.poisson_create(C.byref(tiny), None, 2, None, 4, C.byref(h)) == capi.PS_ERR_INVALID_ARG
    box = capi.make_grid(16, lo=(0, 0, 0), hi=(1, -1, 1))
    assert lib.poisson_create(C.byref(box), None, 2, None, 4, C.byref(h)) == capi.PS_ERR_INVALID_ARG
    bc = capi.PsBC(capi.PS_BC_MULTIPOLE, capi.PS_INNER_NONE, (C.c_double * 3)(0.5, 0.5, 0.5), 1.0)
    g = capi.make_grid(32)
    assert lib.poisson_create(C.byref(g), None, 2, C.byref(bc), 17, C.byref(h)) == capi.PS_ERR_INVALID_ARG
    sph = capi.make_grid((16, 8, 16), kind=capi.PS_GRID_SPHERICAL)
    assert lib.poisson_create(C.byref(sph), None, 2, None, 4, C.byref(h)) == capi.PS_ERR_INVALID_ARG
    assert not h.value
    assert lib.poisson_solve(None, None, None, 1e-6, None, None) == capi.PS_ERR_INVALID_ARG


def test_workspace_bytes_grows_with_grid_and_shrinks_with_precision(lib):
    from paper_2605_03563_gb300 import capi
    # the hierarchy scales with the volume; the multipole scratch (a few MB) does not
    g128 = capi.make_grid(128)
    g256 = capi.make_grid(256)
    b128 = lib.poisson_workspace_bytes(C.byref(g128), 2, 4, capi.PS_FP64)
    b256 = lib.poisson_workspace_bytes(C.byref(g256), 2, 4, capi.PS_FP64)
    assert 6 < b256 / b128 < 10
    m32 = lib.poisson_workspace_bytes(C.byref(g128), 2, 4, capi.PS_MIXED_FP32)
    mbf = lib.poisson_workspace_bytes(C.byref(g128), 2, 4, capi.PS_MIXED_BF16)
    assert mbf < m32
    # a 256^3 FP64 multigrid hierarchy needs at least the level-0 scaled RHS and delta buffer
    g256 = capi.make_grid(256)
    assert lib.poisson_workspace_bytes(C.byref(g256), 2, 4, capi.PS_FP64) >= 2 * 257 ** 3 * 8
    assert lib.poisson_workspace_bytes(C.byref(g256), 5, 4, capi.PS_FP64) == 0


def test_package_fails_loudly_without_the_library(tmp_path, monkeypatch):
    from paper_2605_03563_gb300 import capi
    monkeypatch.setattr(capi, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(capi, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        capi.lib()
