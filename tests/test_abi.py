"""The C-ABI library builds, loads and exports every symbol include/cloak.h
declares; argument validation works without a GPU (no compute calls)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2606_18400_gb300 import build
    build.build()
    from paper_2606_18400_gb300 import cloak
    return cloak.load()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "cloak.h")).read()
    return sorted(set(re.findall(r"CLOAK_API\s+[\w\s\*]*?\b(cloak_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ("cloak_create", "cloak_destroy", "cloak_keygen", "cloak_shuffle", "cloak_unshuffle",
              "cloak_linear", "cloak_rekey", "cloak_export_table"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_binding_covers_the_header():
    from paper_2606_18400_gb300 import cloak
    assert sorted(n for n, _, _ in cloak.SIGNATURES) == declared_symbols()
    for n in declared_symbols():
        assert callable(getattr(cloak, n))


def test_version(lib):
    from paper_2606_18400_gb300 import cloak
    assert "sm_103a" in cloak.cloak_version()


def _desc(cloak, **kw):
    t = (cloak.TensorDesc * 1)(cloak.TensorDesc(kw.get("n", 256), kw.get("k", 256), 0, 0,
                                                kw.get("pg", -1), kw.get("axis", 0), kw.get("pg2", -1)))
    g = (cloak.GroupDesc * 1)(cloak.GroupDesc(kw.get("units", 256), 1, -1, 1))
    d = cloak.ModelDesc(1, kw.get("ngroups", 0), t, g, kw.get("dtype", 1), kw.get("tr", 128),
                        kw.get("tc", 128), 0, kw.get("scope", 0), 0, kw.get("page", 2 << 20))
    return d, t, g


@pytest.mark.parametrize("kw,rc", [
    (dict(dtype=7), -1),                      # unknown dtype
    (dict(page=1000), -1),                    # page not a multiple of the tile
    (dict(tr=64, tc=64), -6),                 # BF16 needs 128x128 tiles
    (dict(pg=0, ngroups=1, units=100), -1),   # permuted dim != units * unit
    (dict(pg=3, ngroups=1), -1),              # group out of range
    (dict(pg2=0, ngroups=1, units=100), -1),  # second axis != units * unit
    (dict(pg2=2, ngroups=1), -1),             # second group out of range
    (dict(axis=2), -1),                       # no such axis
    (dict(scope=2), -1),
    (dict(n=0), -1),
])
def test_create_rejects_bad_descriptors(lib, kw, rc):
    from paper_2606_18400_gb300 import cloak
    d, t, g = _desc(cloak, **kw)
    ctx = C.c_void_p()
    assert lib.cloak_create(C.byref(d), 0, C.byref(ctx)) == rc
    assert not ctx.value


def test_null_arguments(lib):
    assert lib.cloak_create(None, 0, None) == -1
    assert lib.cloak_destroy(None) == -1
    assert lib.cloak_linear(None, 0, None, None, 1, 0, 0, None) == -1
    assert lib.cloak_rekey(None, 0, 0, None) == -1


def test_product_path_does_not_touch_the_oracle():
    """The package, the CUDA sources and the benchmark's product leg never
    import or link the oracle."""
    pkg = os.path.join(ROOT, "paper_2606_18400_gb300")
    for dp, _, fs in os.walk(pkg):
        for f in fs:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dp, f)).read()
                assert not re.search(r"(import\s+oracle|from\s+oracle|liboracle|oracle/|cloak_oracle)",
                                     src), f


def test_struct_layouts_match_the_header(tmp_path):
    """Every descriptor struct the binding declares has the header's size and
    field offsets (gcc compiles the header and prints them)."""
    from paper_2606_18400_gb300 import cloak
    structs = {"cloak_tensor_desc": cloak.TensorDesc, "cloak_group_desc": cloak.GroupDesc,
               "cloak_model_desc": cloak.ModelDesc, "cloak_stack_desc": cloak.StackDesc,
               "cloak_serve_desc": cloak.ServeDesc, "cloak_serve_batch": cloak.ServeBatch,
               "cloak_tune_result": cloak.TuneResult, "cloak_moe_desc": cloak.MoeDesc}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "cloak.h"', 'int main(void) {']
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in py._fields_:
            lines.append(f'printf("{cname} {f[0]} %zu\\n", offsetof({cname}, {f[0]}));')
    lines += ['return 0;', '}']
    src, exe = tmp_path / "layout.c", tmp_path / "layout"
    src.write_text("\n".join(lines))
    import subprocess
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = dict()
    for ln in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        a, b, v = ln.split()
        got[(a, b)] = int(v)
    for cname, py in structs.items():
        assert got[(cname, "size")] == C.sizeof(py), cname
        for f in py._fields_:
            assert got[(cname, f[0])] == getattr(py, f[0]).offset, (cname, f[0])
