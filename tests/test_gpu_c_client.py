"""The C ABI from a plain C program: tests/c_client/jac_client.c, built with
gcc against include/jacobi.h and linked to libjac.so, runs the hoisted path
on the GPU, with a context that owns its memory and with a borrowed one
whose storage and workspace the client allocates.  Its state and residual
equal, bitwise, the same calls made through the Python binding, and match
the FP64 CPU oracle."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import jacobi_inputs as ji
from _util import TOL, gpu_run, oracle_ref, rel_g, rel_p

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PRECS = {"f64": 0, "f32": 1, "bf16": 2}


@pytest.fixture(scope="module")
def client(tmp_path_factory):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_2002_12115_gb300 import _build
    lib = _build.build()
    import oracle
    oracle.build()
    d = tmp_path_factory.mktemp("c_client")
    exe = str(d / "jac_client")
    libdir = os.path.dirname(lib)
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    cuda = os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    cudalib = next((os.path.join(cuda, x) for x in ("lib64", "lib", "targets/sbsa-linux/lib",
                                                     "targets/x86_64-linux/lib")
                    if os.path.exists(os.path.join(cuda, x, "libcudart.so"))), os.path.join(cuda, "lib64"))
    r = subprocess.run([cc, "-std=c99", "-O2", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                        "-I", os.path.join(cuda, "include"),
                        os.path.join(ROOT, "tests", "c_client", "jac_client.c"), "-o", exe,
                        "-L", libdir, "-ljac", "-Wl,-rpath," + libdir,
                        "-L", cudalib, "-lcudart", "-Wl,-rpath," + cudalib], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe, d


@pytest.mark.parametrize("borrowed", [False, True])
@pytest.mark.parametrize("prec,dims,n", [("f64", (33, 33, 65), 20), ("f32", (131, 10, 6), 5),
                                         ("bf16", (67, 19, 23), 7)])
def test_c_client_matches_binding_and_oracle(client, prec, dims, n, borrowed):
    exe, d = client
    I, J, K = dims
    f = ji.himeno_fields(I, J, K, seed=400 + I)
    src, dst = d / f"in_{prec}.bin", d / f"out_{prec}_{int(borrowed)}.bin"
    np.concatenate([f[name].ravel() for name in ji.FIELD_NAMES]).astype(np.float64).tofile(src)
    r = subprocess.run([exe, str(I), str(J), str(K), str(PRECS[prec]), str(n), str(src), str(dst)]
                       + (["borrowed"] if borrowed else []), capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = np.fromfile(dst, dtype=np.float64)
    p, g = out[:-1].reshape(K, J, I), float(out[-1])
    want_p, want_g = gpu_run(f, n, prec)
    assert np.array_equal(p, want_p) and g == want_g
    op, og = oracle_ref(f, n, prec)
    assert rel_p(p, op) <= TOL[prec] and rel_g(g, og) <= TOL[prec]
