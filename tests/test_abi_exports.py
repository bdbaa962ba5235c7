"""The C-ABI library builds, loads without a GPU and exports every declared symbol."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "jacobi.h")
HEADERS = sorted(os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
                 if f.endswith(".h"))


def declared_functions(paths=HEADERS):
    names = set()
    for path in paths:
        text = open(path).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names.update(re.findall(r"\b((?:jac|jfft)_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def libjac():
    from paper_2002_12115_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("jac_create", "jac_create_borrowed", "jac_workspace_size", "jac_upload", "jac_sweep",
                 "jac_residual", "jac_download", "jac_destroy", "jac_sweep_dev", "jac_last_error",
                 "jac_sweep_adjoint", "jac_batch_sweep", "jfft_plan_create", "jfft_forward", "jfft_inverse",
                 "jfft_evolve"):
        assert must in names, must


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
    src.write_text('#include "jacobi.h"\n#include "jfft.h"\n'
                   "int main(void) { jac_plan p = {8, JAC_KDEPTH_BALANCED, 0, 0};\n"
                   "  jac_fields f; (void)f; return p.kdepth == -1 && JAC_NOALLOC_MAX_CTAS == 2048 ? 0 : 1; }\n")
    exe = tmp_path / "use_header"
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
                        str(src), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    assert subprocess.run([str(exe)]).returncode == 0


def test_borrowed_sizes_without_gpu():
    """jac_field_bytes and jac_workspace_size are host-only: the storage of
    each array is pitch * J * K elements of its type, and a borrowed
    context's workspace is the sweep scratch (256 + 8 * 2048 bytes), one
    FP64 staging array, thirteen more with asynchronous staging, and
    ceil(max/C) + C + 1 state arrays plus 256 bytes for a tape, each part
    rounded up to 256 bytes."""
    import paper_2002_12115_gb300 as pkg

    def r256(n):
        return (n + 255) // 256 * 256

    I, J, K = 129, 33, 17
    pitch = pkg.pitch(I)
    assert pitch == 136
    for prec, p_elem, c_elem in (("f64", 8, 8), ("f32", 4, 4), ("bf16", 4, 2)):
        assert pkg.field_bytes(I, J, K, prec, 0) == pitch * J * K * p_elem
        assert pkg.field_bytes(I, J, K, prec, 11) == pitch * J * K * p_elem          # wrk1
        assert pkg.field_bytes(I, J, K, prec, 4) == pitch * J * K * c_elem           # a3
        n = I * J * K
        base = 256 + 8 * 2048 + r256(8 * n)
        assert pkg.ctx_workspace_size(I, J, K, prec) == base
        assert pkg.ctx_workspace_size(I, J, K, prec, async_upload=True) == base + r256(13 * 8 * n)
        state = r256(pitch * J * K * p_elem)
        assert pkg.ctx_workspace_size(I, J, K, prec, tape=(5, 20)) == base + (4 + 5 + 1) * state + 256
        assert pkg.ctx_workspace_size(I, J, K, prec, tape=(10, 3)) == base + (1 + 3 + 1) * state + 256
    with pytest.raises(pkg.JacError):
        pkg.field_bytes(2, 5, 5, "f32", 0)
    with pytest.raises(pkg.JacError):
        pkg.field_bytes(5, 5, 5, "f32", 13)


def test_fft_sizes_without_gpu():
    """jfft_workspace_size is host-only and rejects extents that are not
    powers of two in [2, 1024]."""
    import paper_2002_12115_gb300 as pkg
    assert pkg.fft_workspace_size(256, 256, 256, "c32") > 256 + 3 * 256 * 8
    assert pkg.fft_workspace_size(64, 32, 16, "c64") >= 256 + (64 + 32 + 16) * 16
    for bad in ((12, 16, 16), (1, 16, 16), (2048, 16, 16)):
        with pytest.raises(pkg.JacError):
            pkg.fft_workspace_size(*bad)
