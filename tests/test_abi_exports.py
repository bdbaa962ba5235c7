"""The C-ABI library builds, loads without a GPU and exports every declared symbol."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "jacobi.h")


def declared_functions(path=HEADER):
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(jac_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libjac():
    from paper_2002_12115_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("jac_create", "jac_upload", "jac_sweep", "jac_residual", "jac_download", "jac_destroy",
                 "jac_sweep_dev", "jac_last_error"):
        assert must in names


def test_every_declared_symbol_is_exported(libjac):
    missing = [n for n in declared_functions() if not hasattr(libjac, n)]
    assert not missing, missing


def test_host_only_calls(libjac):
    libjac.jac_pitch.restype = ctypes.c_int
    libjac.jac_pitch.argtypes = [ctypes.c_int]
    assert [libjac.jac_pitch(n) for n in (3, 8, 9, 129, 513)] == [8, 8, 16, 136, 520]
    libjac.jac_version.restype = ctypes.c_char_p
    assert b"sm_103a" in libjac.jac_version()


def test_binding_loads_and_rejects_bad_arguments_without_gpu():
    import paper_2002_12115_gb300 as pkg
    L = pkg.lib()
    assert pkg.pitch(33) == 40
    # argument checks happen before any CUDA call
    h = ctypes.c_void_p()
    assert L.jac_create(ctypes.byref(h), 2, 5, 5, 1, 0.8, None) == 1        # JAC_EINVAL
    assert b">= 3" in L.jac_last_error(None)
    assert L.jac_create(ctypes.byref(h), 5, 5, 5, 7, 0.8, None) == 1        # unknown precision
    assert L.jac_create(ctypes.byref(h), 5, 5, 5, 1, float("nan"), None) == 1
    g = pkg.jac_grid()
    n = ctypes.c_size_t()
    assert L.jac_sweep_workspace_size(ctypes.byref(g), None, ctypes.byref(n)) == 1


def test_header_is_plain_c(tmp_path):
    """include/jacobi.h is a C header: it compiles as strict C99 (no torch or
    C++ types in the boundary) and its plan constant has the documented value."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use_header.c"
    src.write_text('#include "jacobi.h"\n'
                   "int main(void) { jac_plan p = {8, JAC_KDEPTH_BALANCED, 0, 0};\n"
                   "  jac_fields f; (void)f; return p.kdepth == -1 && JAC_NOALLOC_MAX_CTAS == 2048 ? 0 : 1; }\n")
    exe = tmp_path / "use_header"
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
                        str(src), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    assert subprocess.run([str(exe)]).returncode == 0
