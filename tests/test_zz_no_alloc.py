"""jac_sweep_dev_noalloc against jac_sweep_dev, through the C ABI.

jac_sweep_dev_noalloc serves callers that may not allocate device memory (a
plugin handed only input and output buffers by a host that owns the GPU's
memory, or a loop that cannot take cudaMalloc's synchronisation): it keeps
its scratch in a fixed array inside the library instead of a caller
workspace.  It launches the same kernel with the same plan as the
workspace entry point, so two calls in a row must give that entry point's
state and residual bit for bit, and both must match the oracle.

The file name sorts last so that pytest collects it last: when a run stops
at the first failure (-x), a failure here comes after every other test has
run.  Nothing in it depends on the tests before it; it also passes alone in
a fresh process.
"""
import ctypes

import numpy as np
import pytest

import jacobi_inputs as ji
from _util import TOL, oracle_ref, rel_g, rel_p

pytestmark = pytest.mark.gpu

FIELDS = ("p", "a0", "a1", "a2", "a3", "b0", "b1", "b2", "c0", "c1", "c2", "wrk1", "bnd")
PRECS = {"f64": 0, "f32": 1, "bf16": 2}


def _elem(prec, name):
    if prec == "f64":
        return 8
    if prec == "f32" or name in ("p", "wrk1"):
        return 4
    return 2


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_12115_gb300 import _build
    _build.build()
    import paper_2002_12115_gb300 as pkg
    return pkg


class Grid:
    """Storage-layout buffers of one grid, owned by torch (the caller)."""

    def __init__(self, pkg, fields, prec, omega=0.8):
        import torch
        K, J, I = fields["p"].shape
        self.pkg, self.I, self.J, self.K, self.prec = pkg, I, J, K, prec
        self.stream = torch.cuda.current_stream()
        self.sh = pkg.stream_handle(self.stream)
        pitch = pkg.pitch(I)
        self.src = {n: torch.from_numpy(np.ascontiguousarray(v)).cuda() for n, v in fields.items()}
        self.buf = {n: torch.zeros(pitch * J * K * _elem(prec, n), dtype=torch.uint8, device="cuda")
                    for n in FIELDS}
        self.p1 = torch.zeros_like(self.buf["p"])
        g = pkg.jac_grid()
        g.I, g.J, g.K, g.prec, g.omega = I, J, K, PRECS[prec], omega
        g.p[0], g.p[1] = self.buf["p"].data_ptr(), self.p1.data_ptr()
        for q, n in enumerate(FIELDS):
            if q:
                g.coef[q] = self.buf[n].data_ptr()
        self.g = g
        self.reset()

    def reset(self):
        lib = self.pkg.lib()
        for q, n in enumerate(FIELDS):
            st = lib.jac_pack_dev(self.I, self.J, self.K, PRECS[self.prec], q, self.src[n].data_ptr(),
                                  self.buf[n].data_ptr(), ctypes.c_void_p(self.sh))
            self.pkg.check(st)
        self.p1.copy_(self.buf["p"])

    def state(self, n):
        import torch
        out = torch.empty((self.K, self.J, self.I), dtype=torch.float64, device="cuda")
        src = self.buf["p"] if n % 2 == 0 else self.p1
        self.pkg.check(self.pkg.lib().jac_unpack_dev(self.I, self.J, self.K, PRECS[self.prec], 0,
                                                     src.data_ptr(), out.data_ptr(), ctypes.c_void_p(self.sh)))
        return out.cpu().numpy()


def _with_workspace(pkg, grid, n, plan):
    import torch
    ws_bytes = pkg.workspace_size(grid.g, *plan)
    ws = torch.zeros(ws_bytes, dtype=torch.uint8, device="cuda")
    res = torch.zeros(1, dtype=torch.float64, device="cuda")
    pkg.sweep_dev(grid.g, n, res.data_ptr(), ws.data_ptr(), ws_bytes, grid.sh, *plan)
    return grid.state(n), float(res.item())


def _no_alloc(pkg, grid, n, plan):
    import torch
    res = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = pkg.lib().jac_sweep_dev_noalloc(ctypes.byref(grid.g), ctypes.byref(pkg.jac_plan(*plan)), n,
                                         ctypes.c_void_p(res.data_ptr()), ctypes.c_void_p(grid.sh))
    pkg.check(st)
    return grid.state(n), float(res.item())


@pytest.mark.parametrize("prec,dims,n,plan", [("f32", (130, 37, 41), 7, (8, 5)),
                                              ("bf16", (67, 29, 33), 4, (4, 3)),
                                              ("f64", (70, 21, 19), 5, (8, 0)),
                                              # two-sweep passes (FP32, fuse = 2): 4 paired sweeps then 1 single
                                              ("f32", (130, 37, 41), 9, (8, 5, 0, 2))])
def test_no_alloc_matches_workspace_entry_point(L, prec, dims, n, plan):
    I, J, K = dims
    fields = ji.himeno_fields(I, J, K, seed=200 + I)
    grid = Grid(L, fields, prec)
    want_p, want_g = _with_workspace(L, grid, n, plan)
    for call in range(2):                      # two calls in a row share the scratch
        grid.reset()
        p, g = _no_alloc(L, grid, n, plan)
        # the same kernel and plan: bit for bit
        assert np.array_equal(p, want_p) and g == want_g, (call, rel_p(p, want_p), rel_g(g, want_g))
    op, og = oracle_ref(fields, n, prec)
    assert rel_p(p, op) <= TOL[prec] and rel_g(g, og) <= TOL[prec], (rel_p(p, op), rel_g(g, og))


def test_no_alloc_scratch_covers_every_launch_of_this_gpu(L):
    """The sweep launches at most one CTA per SM, so the fixed scratch (one
    partial per CTA) must cover the SM count; the workspace the regular entry
    point asks for, minus its 256-byte header, is that partial array."""
    import torch
    import paper_2002_12115_gb300 as pkg
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert sms <= 2048                         # JAC_NOALLOC_MAX_CTAS
    g = pkg.jac_grid()
    g.I, g.J, g.K, g.prec, g.omega = 513, 513, 1025, 1, 0.8
    g.p[0], g.p[1] = 256, 512                  # size query only: never dereferenced
    for q in range(1, 13):
        g.coef[q] = 1024 * q
    ws = pkg.workspace_size(g)
    assert 256 + 8 * sms <= ws <= 256 + 8 * 2048
