"""CPU-side checks of the C-ABI library: it builds, loads, and exports every
symbol that include/fde.h declares.  No compute call is made without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fde.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1305_6653_gb300 import _lib
    if not os.path.exists(_lib.LIB_PATH):
        from paper_1305_6653_gb300 import build
        build.build()
    return ctypes.CDLL(_lib.LIB_PATH)


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:int|void|long long|const char\*|fde_problem\*)\s+\**(\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("fde_problem_create", "bvm_assemble", "strang_precond_factor", "pgmres_solve",
                     "fde_problem_destroy", "fde_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_binding_lists_every_declared_symbol():
    from paper_1305_6653_gb300 import _lib
    assert sorted(_lib.EXPORTED) == _declared_functions()


def test_struct_layouts_match_header(tmp_path):
    """The ctypes structures have the C layout of include/fde.h: every field's offset
    and each struct's size, printed by a C program compiled against the header."""
    import shutil
    import subprocess

    from paper_1305_6653_gb300 import _lib
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"fde_problem_desc": _lib.FdeProblemDesc, "fde_pgmres_opts": _lib.FdePgmresOpts,
               "fde_stats": _lib.FdeStats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "fde.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)


def test_argument_validation_needs_no_gpu(lib):
    """fde_problem_create rejects bad arguments before touching the device."""
    from paper_1305_6653_gb300 import _lib
    L = _lib.load()
    d = _lib.FdeProblemDesc()
    d.m, d.s, d.alpha, d.xL, d.xR, d.t0, d.T, d.family, d.mu = 63, 32, 2.5, 0.0, 1.0, 0.0, 1.0, 1, 3
    h = ctypes.c_void_p()
    assert L.fde_problem_create(ctypes.byref(d), None, ctypes.byref(h)) == _lib.FDE_ERR_ARG
    assert b"alpha" in L.fde_last_error()
    d.alpha = 1.5
    d.s = 30  # not a power of two
    assert L.fde_problem_create(ctypes.byref(d), None, ctypes.byref(h)) == _lib.FDE_ERR_ARG
    d.s, d.family = 32, 9
    assert L.fde_problem_create(ctypes.byref(d), None, ctypes.byref(h)) == _lib.FDE_ERR_ARG
    d.family, d.mu = 3, 4  # ETR needs odd mu
    assert L.fde_problem_create(ctypes.byref(d), None, ctypes.byref(h)) == _lib.FDE_ERR_ARG
    d.family, d.mu = 1, 3
    one = (ctypes.c_double * 1)(1.0)
    d.u0 = d.f = ctypes.cast(one, ctypes.c_void_p)
    d.dplus_t = ctypes.cast(one, ctypes.c_void_p)  # d+(x, t) without d-(x, t)
    assert L.fde_problem_create(ctypes.byref(d), None, ctypes.byref(h)) == _lib.FDE_ERR_ARG
    assert b"dminus_t" in L.fde_last_error()
    d.dplus_t = None
    assert L.bvm_assemble(None) == _lib.FDE_ERR_ARG
    assert L.strang_precond_factor(None, 0) == _lib.FDE_ERR_ARG
    assert L.fde_factor_storage(None, _lib.STORAGES["bf16"]) == _lib.FDE_ERR_ARG


def test_release_of_an_empty_device_cache_needs_no_gpu(lib):
    """With nothing cached, fde_release_cached_memory makes no CUDA call and succeeds."""
    from paper_1305_6653_gb300 import _lib, fde_release_cached_memory
    assert _lib.load().fde_release_cached_memory() == _lib.FDE_OK
    fde_release_cached_memory()


def test_tune_table_is_host_side(tmp_path):
    """fde_tune_set / fde_tune_cache / fde_tune_query need no GPU: argument checks and
    a cache file read back."""
    import ctypes as C

    from paper_1305_6653_gb300 import _lib
    lib = _lib.load()
    assert lib.fde_tune_set(5, 0) == _lib.FDE_ERR_ARG
    assert lib.fde_tune_set(0, 3) == _lib.FDE_ERR_ARG
    f = tmp_path / "t.txt"
    f.write_text("matvec 0 2048 256 0 1\ntrsv 1 2048 129 1 2\ntrsv 1 64 9 1 7\n")
    assert lib.fde_tune_cache(str(f).encode()) == 0
    v = C.c_int()
    assert lib.fde_tune_query(0, 2048, 256, 0, C.byref(v)) == 0 and v.value == 1
    assert lib.fde_tune_query(1, 2048, 129, 1, C.byref(v)) == 0 and v.value == 2
    assert lib.fde_tune_query(1, 64, 9, 1, C.byref(v)) == 0 and v.value == -1  # out-of-range entry dropped
    assert lib.fde_tune_query(1, 128, 9, 1, C.byref(v)) == 0 and v.value == -1
    assert lib.fde_tune_set(1, 0) == 0
    assert lib.fde_tune_query(1, 2048, 129, 1, C.byref(v)) == 0 and v.value == 0  # forced
    assert lib.fde_tune_set(1, -1) == 0
    assert lib.fde_tune_cache(None) == 0


def test_binding_constants_match_header():
    """The binding's enumerations (precisions, factor storages, block solvers, tuner
    kernels) have the values the header defines."""
    from paper_1305_6653_gb300 import PRECISIONS, _lib
    defines = dict((k, int(v)) for k, v in re.findall(r"^#define\s+(FDE_\w+)\s+(-?\d+)", open(HEADER).read(), re.M))
    for name, value in {"fp64": "FDE_FP64", "fp32": "FDE_FP32", "tf32": "FDE_TF32", "bf16": "FDE_BF16",
                        "tf32x3": "FDE_TF32X3"}.items():
        assert PRECISIONS[name] == defines[value], name
    assert _lib.STORAGES == {"fp32": defines["FDE_STORAGE_FP32"], "bf16": defines["FDE_STORAGE_BF16"]}
    assert _lib.BLOCK_SOLVERS == {"auto": defines["FDE_BLOCK_SOLVE_AUTO"],
                                  "cuda_cores": defines["FDE_BLOCK_SOLVE_CUDA_CORES"],
                                  "tensor_cores": defines["FDE_BLOCK_SOLVE_TENSOR_CORES"]}
    assert (_lib.FDE_TUNE_MATVEC, _lib.FDE_TUNE_TRSV, _lib.FDE_TUNE_LU) == (
        defines["FDE_TUNE_MATVEC"], defines["FDE_TUNE_TRSV"], defines["FDE_TUNE_LU"])
