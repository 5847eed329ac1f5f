"""The C-ABI library builds, loads and exports every entry point that
include/qdd.h declares; host-side argument checks answer without a GPU."""

import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qdd.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qdd_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1011_3318_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("qdd_create_lattice", "qdd_load_gauge", "qdd_dslash", "qdd_ras_apply", "qdd_solve"):
        assert required in names


def test_header_is_plain_c(tmp_path, libpath):
    """The boundary is a C ABI: the header compiles as C99 and as C++ with
    no CUDA or torch headers, and a C program linked against the library
    runs its host-side calls."""
    src = tmp_path / "use.c"
    src.write_text('#include "qdd.h"\n'
                   'int main(void) { qdd_solver_params p; qdd_default_params(&p);\n'
                   '  return p.schwarz == QDD_SCHWARZ_RAS && p.outer_mode == 0 ? 0 : 1; }\n')
    inc = os.path.join(ROOT, "include")
    for cc, std in (("gcc", "-std=c99"), ("g++", "-std=c++11")):
        args = [cc, std, "-Wall", "-Wextra", "-Werror", "-fsyntax-only", "-I", inc]
        if cc == "g++":
            args += ["-x", "c++"]
        p = subprocess.run(args + [str(src)], capture_output=True, text=True)
        assert p.returncode == 0, p.stderr
    libdir = os.path.dirname(libpath)
    exe = tmp_path / "use"
    p = subprocess.run(["gcc", "-std=c99", "-I", inc, str(src), "-L", libdir, "-lqdd", "-Wl,-rpath," + libdir,
                        "-o", str(exe)], capture_output=True, text=True)
    assert p.returncode == 0, p.stderr
    assert subprocess.run([str(exe)], timeout=60).returncode == 0


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (qdd_[a-z_0-9]+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(libpath)
    for n in declared_functions():
        getattr(lib, n)


def test_binding_lists_the_abi(libpath):
    from paper_1011_3318_gb300 import qdd
    assert sorted(qdd.ABI) == declared_functions()


def test_host_side_calls_without_gpu(libpath):
    from paper_1011_3318_gb300 import qdd
    assert "sm_103a" in qdd.version()
    p = qdd.default_params()
    assert list(p.block) == [4, 4, 4, 4] and p.n_ras == 3 and p.n_dominv == 4 and p.inner_tol == 1e-3
    assert p.schwarz == qdd.QDD_SCHWARZ_RAS and p.outer_mode == 0 and p.ras_kernel == 0
    lib = qdd.lib()
    h = ctypes.c_void_p()
    bad_dims = (ctypes.c_int * 4)(8, 0, 8, 8)
    bc = (ctypes.c_int * 4)(1, 1, 1, -1)
    assert lib.qdd_create_lattice(ctypes.byref(h), bad_dims, bc, 1, None) == qdd.QDD_ERR_ARG
    assert "extents" in qdd.last_error()
    dims = (ctypes.c_int * 4)(8, 8, 8, 8)
    bad_bc = (ctypes.c_int * 4)(1, 1, 1, 0)
    assert lib.qdd_create_lattice(ctypes.byref(h), dims, bad_bc, 1, None) == qdd.QDD_ERR_ARG
    assert lib.qdd_create_lattice(ctypes.byref(h), dims, bc, 0, None) == qdd.QDD_ERR_ARG
    assert lib.qdd_create_lattice(ctypes.byref(h), dims, bc, 65, None) == qdd.QDD_ERR_ARG
    # 4096 x 4096 x 8 x 1 = 134M sites: above the 32-bit plane-index cap
    big = (ctypes.c_int * 4)(4096, 4096, 8, 1)
    assert lib.qdd_create_lattice(ctypes.byref(h), big, bc, 1, None) == qdd.QDD_ERR_ARG
    assert "119304647" in qdd.last_error()
    assert lib.qdd_destroy_lattice(None) == qdd.QDD_OK
    # the batch work-list switch is process-wide host state: on by default,
    # and each call reports the setting it replaces
    prev = qdd.set_batch_lists(False)
    try:
        assert prev is True
        assert qdd.set_batch_lists(False) is False
        assert qdd.set_batch_lists(True) is False
        assert qdd.set_batch_lists(True) is True
    finally:
        qdd.set_batch_lists(prev)
    assert lib.qdd_set_batch_lists(1, None) == qdd.QDD_OK


def test_oracle_and_library_share_no_code():
    """The oracle and the CUDA path are independent: no file of one includes,
    imports or links the other."""
    pkg = os.path.join(ROOT, "paper_1011_3318_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.sub(r"#.*|//.*", "", text).lower() or f.endswith(".md"), f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c")):
            text = open(os.path.join(ROOT, "oracle", f)).read()
            assert "paper_1011_3318_gb300" not in text and "qdd.h" not in text


def test_binding_structs_mirror_the_header():
    """The ctypes mirrors of qdd_solver_params and qdd_solve_info list the
    header's fields in the header's order."""
    import re
    from paper_1011_3318_gb300 import qdd
    text = open(os.path.join(ROOT, "include", "qdd.h")).read()
    for cname, cls in (("qdd_solver_params", qdd.SolverParams), ("qdd_solve_info", qdd.SolveInfo)):
        end = text.index("} " + cname + ";")
        body = text[text.rindex("typedef struct {", 0, end) + len("typedef struct {"):end]
        body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
        names = []
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            first, *rest = [x.strip() for x in decl.split(",")]
            names.append(re.sub(r"\[.*\]", "", first.split()[-1]))
            names.extend(re.sub(r"\[.*\]", "", x) for x in rest)
        assert names == [f[0] for f in cls._fields_], cname
