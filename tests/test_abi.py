"""The C-ABI library builds, loads without a GPU and exports what include/px.h declares."""
import ctypes as C
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2510_12731_gb300 import build as B  # noqa: E402
from paper_2510_12731_gb300 import _lib as L  # noqa: E402


@pytest.fixture(scope="module")
def libpath():
    return B.build()


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(px_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(libpath):
    lib = C.CDLL(libpath)
    for header in os.listdir(os.path.join(ROOT, "include")):
        names = _declared(header)
        assert names, header
        for name in names:
            assert hasattr(lib, name), f"{name} declared in {header} but not exported"


def test_binding_covers_the_header(libpath):
    assert set(_declared("px.h")) | set(_declared("px_serve.h")) == set(L.SIGNATURES)


def test_struct_layouts_match_the_header(tmp_path, libpath):
    """Compile a C program against px.h and compare sizeof/offsetof with the ctypes mirror."""
    structs = {"px_atom_type": L.AtomType, "px_options": L.Options, "px_result": L.Result,
               "px_stats": L.Stats, "px_request": L.Request, "px_server_stats": L.ServerStats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "px.h"', '#include "px_serve.h"',
             "int main(void){"]
    for cname, cls in structs.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = dict(l.split() for l in out if l.strip())
    for cname, cls in structs.items():
        assert int(got[cname]) == C.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert int(got[f"{cname}.{f}"]) == getattr(cls, f).offset, f"{cname}.{f}"


def test_defaults_and_version_without_gpu(libpath):
    lib = L.load(libpath)
    assert lib.px_abi_version() == 2
    o = L.Options()
    assert lib.px_options_default(C.byref(o)) == L.PX_OK
    assert o.restart_m == 0 and o.gs_passes == 1 and o.tol_rel == 1e-7
    assert o.basis == L.PX_BASIS_AUTO and o.gemm_tiles == 0 and o.cycle_graphs == 1
    assert o.solver == L.PX_SOLVER_BATCHED and o.shift_krylov_max == 0
    assert lib.px_options_default(None) == L.PX_EINVAL
    assert lib.px_destroy(None) == L.PX_OK


def test_create_rejects_bad_options(libpath):
    lib = L.load(libpath)
    o = L.Options()
    lib.px_options_default(C.byref(o))
    o.restart_m = -1
    h = C.c_void_p()
    assert lib.px_create(C.byref(h), C.byref(o)) == L.PX_EINVAL
    assert b"restart_m" in lib.px_last_error(None)
    assert lib.px_create(None, C.byref(o)) == L.PX_EINVAL
    lib.px_options_default(C.byref(o))
    o.basis = 4
    assert lib.px_create(C.byref(h), C.byref(o)) == L.PX_EINVAL
    assert b"basis" in lib.px_last_error(None)
    # an FP64 solve keeps an FP64 basis
    o.basis = L.PX_BASIS_FP32
    o.precision = L.PX_FP64
    assert lib.px_create(C.byref(h), C.byref(o)) == L.PX_EINVAL
    assert b"FP64" in lib.px_last_error(None)
    lib.px_options_default(C.byref(o))
    o.gemm_tiles = 3
    assert lib.px_create(C.byref(h), C.byref(o)) == L.PX_EINVAL
    lib.px_options_default(C.byref(o))
    o.cycle_graphs = 2
    assert lib.px_create(C.byref(h), C.byref(o)) == L.PX_EINVAL
    assert b"cycle_graphs" in lib.px_last_error(None)
    lib.px_options_default(C.byref(o))
    o.solver = 2
    assert lib.px_create(C.byref(h), C.byref(o)) == L.PX_EINVAL
    assert b"solver" in lib.px_last_error(None)
    lib.px_options_default(C.byref(o))
    o.shift_krylov_max = -1
    assert lib.px_create(C.byref(h), C.byref(o)) == L.PX_EINVAL
    assert b"shift_krylov_max" in lib.px_last_error(None)


def test_calls_on_null_handle_fail_cleanly(libpath):
    lib = L.load(libpath)
    assert lib.px_set_structure(None, 0, 1, None, None, None, 1) == L.PX_EINVAL
    assert lib.px_solve(None, 1, None, None, 1, None, 1.0, None, None) == L.PX_EINVAL
    st = L.Stats()
    assert lib.px_get_stats(None, C.byref(st)) == L.PX_EINVAL
