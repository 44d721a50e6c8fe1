"""The C-ABI library builds for sm_103a, loads, exports every entry point declared in
include/qed.h, and rejects bad arguments on the host before touching a GPU."""
import ctypes as C
import os
import re

import pytest

import paper_2306_11288_gb300 as q
from paper_2306_11288_gb300 import buildlib as qbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if hdr.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", hdr)).read()
            names += re.findall(r"^\s*(?:qed_status|const char \*)\s*(\w+)\s*\(", txt, flags=re.M)
    return names


@pytest.fixture(scope="module")
def lib():
    qbuild.build()
    return C.CDLL(qbuild.LIB)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 13
    for n in names:
        assert hasattr(lib, n), n
    assert set(q.ABI_FUNCTIONS) == set(names)


def test_header_is_plain_c(tmp_path):
    """include/qed.h compiles as C99 (pedantic) and as C++: the boundary uses no C++ or
    torch types, and a C program can link against the library by its declarations alone."""
    import shutil
    import subprocess
    src = tmp_path / "use.c"
    src.write_text('#include "qed.h"\nint main(void) { qed_ctx *c = 0; (void)c; return (int)QED_OK; }\n')
    for cc, extra in (("gcc", ["-std=c99", "-pedantic", "-Wall", "-Wextra", "-Werror"]),
                      ("g++", ["-std=c++17", "-Wall", "-Werror", "-x", "c++"])):
        exe = shutil.which(cc)
        if exe is None:
            pytest.skip(f"{cc} not available")
        r = subprocess.run([exe, *extra, "-fsyntax-only", "-I", os.path.join(ROOT, "include"), str(src)],
                           capture_output=True, text=True)
        assert r.returncode == 0, (cc, r.stderr)


def test_sm103a_build_flags():
    assert "arch=compute_103a,code=sm_103a" in qbuild.ARCH
    # the build recorded ptxas output for every translation unit, without spills
    for src in qbuild.SOURCES:
        rep = os.path.join(qbuild.OUT_DIR, src.replace(".cu", ".o") + ".ptxas.txt")
        assert os.path.exists(rep)
        assert "bytes spill stores" not in open(rep).read() or " 0 bytes spill stores" in open(rep).read()


def test_host_validation_without_gpu(lib):
    L = q.lib()
    # NULL context / outputs are rejected before any CUDA call
    assert L.qed_step(None, None, None, None, None, 0.0, 1.0, 0, 0, 0, None, None) == q.QED_ERR_NOT_INITIALIZED
    assert L.qed_init_tables(None, None) == q.QED_ERR_INVALID_ARG
    assert "out is NULL" in q.qed_last_error()
    n = C.c_uint64()
    assert L.particles_count(None, C.byref(n), None) == q.QED_ERR_INVALID_ARG
    assert L.particles_destroy(None) == q.QED_ERR_INVALID_ARG
    assert L.qed_destroy(None) == q.QED_ERR_NOT_INITIALIZED
    assert L.qed_read_status(None, None, 0, None) == q.QED_ERR_NOT_INITIALIZED
    assert L.qed_copy_table(None, 0, None, 0, C.byref(n), None) == q.QED_ERR_NOT_INITIALIZED
    assert L.qed_fdtd_advance(None, 0, 1.0, None) == q.QED_ERR_INVALID_ARG
    g = q.qed_grid2d()
    assert L.qed_fdtd_advance(C.byref(g), 0, 1.0, None) == q.QED_ERR_INVALID_ARG
    assert "non-NULL" in q.qed_last_error()
    assert L.qed_philox_blocks(None, 0, None, 0, None) == q.QED_OK          # nothing to do
    assert L.qed_philox_blocks(None, 0, None, 4, None) == q.QED_ERR_INVALID_ARG
    assert "NULL buffer" in q.qed_last_error()
    h = C.c_void_p()
    soa = q.qed_soa()
    assert L.particles_create(None, 0, C.byref(soa), 0, 0, 0, None, C.byref(h)) == q.QED_ERR_NOT_INITIALIZED
    spec = q.diag_spec(q.QED_DIAG_SPECTRUM, 8, 1, 1.0, 10.0)
    assert L.qed_diag(None, None, C.byref(spec), None, None) == q.QED_ERR_NOT_INITIALIZED
    assert "invalid context" in q.qed_last_error()


def test_binding_refuses_missing_library(tmp_path, monkeypatch):
    monkeypatch.setattr(q, "LIB_PATH", str(tmp_path / "absent.so"))
    monkeypatch.setattr(q, "_lib", None)
    with pytest.raises(q.QedError):
        q.lib()
