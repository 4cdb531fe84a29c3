"""The C-ABI library builds for sm_103a, loads, exports every entry point the
header declares, and rejects malformed descriptions on the host (no GPU
needed for these checks)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2506_00263_gb300 import binding as tb
from paper_2506_00263_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return tb.lib()


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tr_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared("tr.h")
    assert "tr_problem_create" in names and "tr_run_power_iteration" in names
    raw = C.CDLL(tb.LIB_PATH)
    missing = [n for n in names if not hasattr(raw, n)]
    assert not missing, missing


def test_version_and_error_strings(lib):
    assert "sm_103a" in tb.version()
    assert isinstance(lib.tr_last_error(), bytes)


def _geom(nx=1, planes=(0.0, 1.0)):
    g = tb.GeometryDesc()
    g.nx = g.ny = g.nz = nx
    arr = np.array(planes, dtype=np.float64)
    g.x_planes = g.y_planes = g.z_planes = arr.ctypes.data_as(C.POINTER(C.c_double))
    cm = np.zeros(max(nx, 1) ** 3, np.int32)
    g.cell_material = cm.ctypes.data_as(C.POINTER(C.c_int32))
    return g, (arr, cm)


@pytest.mark.parametrize("case", ["zero_cells", "descending_planes", "bad_bc", "material_range", "null_out"])
def test_invalid_descriptions_rejected_on_host(lib, case):
    g, keep = _geom()
    x = tb.XsDesc()
    x.kind, x.n_materials, x.n_groups = 0, 1, 1
    s = tb.SourceDesc()
    ctx = tb.DeviceCtx()
    out = C.c_void_p()
    if case == "zero_cells":
        g.nx = 0
    elif case == "descending_planes":
        bad = np.array([1.0, 0.0])
        keep = keep + (bad,)
        g.x_planes = bad.ctypes.data_as(C.POINTER(C.c_double))
    elif case == "bad_bc":
        g.bc[2] = 9
    elif case == "material_range":
        x.n_materials = 0
    st = lib.tr_problem_create(C.byref(g), C.byref(x), C.byref(s), None, 0, C.byref(ctx),
                               None if case == "null_out" else C.byref(out))
    assert st == tb.TR_ERR_INVALID
    assert lib.tr_last_error()
    assert not out.value


def test_destroy_is_null_safe(lib):
    lib.tr_problem_destroy(None)


def test_header_documents_every_entry_point():
    """Every declaration is directly preceded by a comment block."""
    lines = open(os.path.join(ROOT, "include", "tr.h")).read().splitlines()
    for name in _declared("tr.h"):
        decl = [i for i, l in enumerate(lines)
                if re.match(r"^[A-Za-z_].*\b" + name + r"\s*\(", l) and not l.lstrip().startswith("*")]
        assert decl, name
        j = decl[0] - 1
        while j >= 0 and not lines[j].strip():
            j -= 1
        assert lines[j].rstrip().endswith("*/"), name


def test_batched_rejects_null_arguments_on_host(lib):
    opts = tb.RunOpts(n_histories=1, scheme=tb.SCHEME_ASYNC).to_c()
    nh = (C.c_uint64 * 1)(1)
    assert lib.tr_run_batched(None, 1, nh, C.byref(opts), None) == tb.TR_ERR_INVALID
    hs = (C.c_void_p * 1)(None)
    assert lib.tr_run_batched(hs, 0, nh, C.byref(opts), None) == tb.TR_ERR_INVALID
    assert lib.tr_run_batched(hs, 1, nh, C.byref(opts), None) == tb.TR_ERR_INVALID
    assert b"NULL" in lib.tr_last_error()


def test_ctypes_structs_match_the_header(tmp_path):
    """Size and field offsets of every public struct, from the C compiler,
    equal the ctypes mirrors of the binding."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    pairs = {"tr_geometry_desc": tb.GeometryDesc, "tr_xs_desc": tb.XsDesc, "tr_source_desc": tb.SourceDesc,
             "tr_tally_desc": tb.TallyDesc, "tr_device_ctx": tb.DeviceCtx, "tr_run_opts": tb.RunOptsC,
             "tr_run_stats": tb.RunStats, "tr_eig_opts": tb.EigOptsC, "tr_eig_result": tb.EigResultC}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "tr.h"', "int main(void) {"]
    for cname, py in pairs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in py._fields_:
            lines.append(f'printf("{cname} {f[0]} %zu\\n", offsetof({cname}, {f[0]}));')
    lines += ["return 0; }"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line.strip():
            a, b, v = line.split()
            got[(a, b)] = int(v)
    for cname, py in pairs.items():
        assert got[(cname, "size")] == C.sizeof(py), cname
        for f in py._fields_:
            assert got[(cname, f[0])] == getattr(py, f[0]).offset, (cname, f[0])
