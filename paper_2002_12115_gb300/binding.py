"""ctypes binding of libjac (include/jacobi.h): argument marshalling only.

Every step of the sweep runs in the CUDA library; this module converts
numpy arrays / torch tensors to pointers and status codes to exceptions.
If libjac.so has not been built, loading raises: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libjac.so")

# status codes
JAC_OK, JAC_EINVAL, JAC_ENOMEM, JAC_ECUDA, JAC_ESTATE, JAC_ETIMEOUT, JAC_EINTERNAL = range(7)
STATUS_NAMES = {0: "JAC_OK", 1: "JAC_EINVAL", 2: "JAC_ENOMEM", 3: "JAC_ECUDA", 4: "JAC_ESTATE",
                5: "JAC_ETIMEOUT", 6: "JAC_EINTERNAL"}
# precisions
PRECS = {"f64": 0, "f32": 1, "bf16": 2}
# array indices of a field set
FIELDS = ("p", "a0", "a1", "a2", "a3", "b0", "b1", "b2", "c0", "c1", "c2", "wrk1", "bnd")
NFIELDS = len(FIELDS)
# jac_plan.kdepth: balanced ranges of tile-planes instead of a fixed depth
KDEPTH_BALANCED = -1


class JacError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class jac_fields(ctypes.Structure):
    _fields_ = [("f", ctypes.c_void_p * NFIELDS)]


class jac_fields_f32(ctypes.Structure):
    _fields_ = [("f", ctypes.c_void_p * NFIELDS)]


class jac_grid(ctypes.Structure):
    _fields_ = [("I", ctypes.c_int), ("J", ctypes.c_int), ("K", ctypes.c_int), ("prec", ctypes.c_int),
                ("omega", ctypes.c_double), ("p", ctypes.c_void_p * 2),
                ("coef", ctypes.c_void_p * NFIELDS)]


class jac_plan(ctypes.Structure):
    _fields_ = [("tile_j", ctypes.c_int), ("kdepth", ctypes.c_int), ("tile_i", ctypes.c_int),
                ("fuse", ctypes.c_int)]


class jac_ws_spec(ctypes.Structure):
    _fields_ = [("async_upload", ctypes.c_int), ("tape_C", ctypes.c_int), ("tape_max", ctypes.c_int)]


_VP = ctypes.c_void_p
_I = ctypes.c_int
_SIG = {
    "jac_pitch": (_I, [_I]),
    "jac_version": (ctypes.c_char_p, []),
    "jac_sweep_workspace_size": (_I, [ctypes.POINTER(jac_grid), ctypes.POINTER(jac_plan),
                                      ctypes.POINTER(ctypes.c_size_t)]),
    "jac_sweep_dev": (_I, [ctypes.POINTER(jac_grid), ctypes.POINTER(jac_plan), _I, _VP, _VP,
                           ctypes.c_size_t, _VP]),
    "jac_workspace_check": (_I, [_VP, _VP]),
    "jac_resolve_plan": (_I, [ctypes.POINTER(jac_grid), ctypes.POINTER(jac_plan), _I, ctypes.POINTER(jac_plan)]),
    "jac_sweep_dev_noalloc": (_I, [ctypes.POINTER(jac_grid), ctypes.POINTER(jac_plan), _I, _VP, _VP]),
    "jac_pack_dev": (_I, [_I, _I, _I, _I, _I, _VP, _VP, _VP]),
    "jac_unpack_dev": (_I, [_I, _I, _I, _I, _I, _VP, _VP, _VP]),
    "jac_create": (_I, [ctypes.POINTER(_VP), _I, _I, _I, _I, ctypes.c_double, _VP]),
    "jac_field_bytes": (_I, [_I, _I, _I, _I, _I, ctypes.POINTER(ctypes.c_size_t)]),
    "jac_workspace_size": (_I, [_I, _I, _I, _I, ctypes.POINTER(jac_ws_spec), ctypes.POINTER(ctypes.c_size_t)]),
    "jac_create_borrowed": (_I, [ctypes.POINTER(_VP), ctypes.POINTER(jac_grid), _VP, _VP, ctypes.c_size_t,
                                 ctypes.POINTER(jac_ws_spec)]),
    "jac_set_workspace": (_I, [_VP, _VP, ctypes.c_size_t, ctypes.POINTER(jac_ws_spec)]),
    "jac_inject_stall": (_I, [_VP, ctypes.c_ulonglong]),
    "jac_destroy": (_I, [_VP]),
    "jac_last_error": (ctypes.c_char_p, [_VP]),
    "jac_set_plan": (_I, [_VP, ctypes.POINTER(jac_plan)]),
    "jac_upload": (_I, [_VP, ctypes.POINTER(jac_fields)]),
    "jac_upload_dev": (_I, [_VP, ctypes.POINTER(jac_fields)]),
    "jac_upload_async": (_I, [_VP, ctypes.POINTER(jac_fields)]),
    "jac_download_async": (_I, [_VP, _VP, _VP]),
    "jac_upload_f32_async": (_I, [_VP, ctypes.POINTER(jac_fields_f32)]),
    "jac_download_f32_async": (_I, [_VP, _VP, _VP]),
    "jac_sync": (_I, [_VP]),
    "jac_sweep": (_I, [_VP, _I]),
    "jac_residual": (_I, [_VP, ctypes.POINTER(ctypes.c_double)]),
    "jac_download": (_I, [_VP, _VP]),
    "jac_download_dev": (_I, [_VP, _VP]),
    "jac_sweep_count": (_I, [_VP, ctypes.POINTER(ctypes.c_longlong)]),
    "jac_get_grid": (_I, [_VP, ctypes.POINTER(jac_grid)]),
    "jac_sweep_unhoisted": (_I, [_VP, _I, ctypes.POINTER(jac_fields), _VP]),
    "jac_adjoint_step_dev": (_I, [ctypes.POINTER(jac_grid), _VP, _VP, _VP, _VP, _VP, _VP, _I, _VP, ctypes.c_size_t, _VP]),
    "jac_tape_begin": (_I, [_VP, _I, _I]),
    "jac_tape_end": (_I, [_VP]),
    "jac_tape_count": (_I, [_VP, ctypes.POINTER(_I)]),
    "jac_sweep_adjoint": (_I, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "jac_batch_create": (_I, [ctypes.POINTER(_VP), _I, _VP, _I, ctypes.c_double, _VP]),
    "jac_batch_destroy": (_I, [_VP]),
    "jac_batch_last_error": (ctypes.c_char_p, [_VP]),
    "jac_batch_upload": (_I, [_VP, _I, ctypes.POINTER(jac_fields)]),
    "jac_batch_upload_dev": (_I, [_VP, _I, ctypes.POINTER(jac_fields)]),
    "jac_batch_set_plan": (_I, [_VP, _I, _VP, _VP]),
    "jac_batch_grid_plan": (_I, [_VP, _I, ctypes.POINTER(jac_plan)]),
    "jac_batch_sweep": (_I, [_VP, _I, _VP]),
    "jac_batch_sweep_loop": (_I, [_VP, _I, _I, _VP]),
    "jac_batch_download": (_I, [_VP, _I, _VP]),
    "jac_batch_download_dev": (_I, [_VP, _I, _VP]),
    "jac_batch_info": (_I, [_VP, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I),
                            ctypes.POINTER(ctypes.c_longlong)]),
    # 3-D FFT block (include/jfft.h)
    "jfft_workspace_size": (_I, [_I, _I, _I, _I, ctypes.POINTER(ctypes.c_size_t)]),
    "jfft_plan_create": (_I, [ctypes.POINTER(_VP), _I, _I, _I, _I, _VP, _VP, ctypes.c_size_t]),
    "jfft_destroy": (_I, [_VP]),
    "jfft_last_error": (ctypes.c_char_p, [_VP]),
    "jfft_forward": (_I, [_VP, _VP, _VP]),
    "jfft_inverse": (_I, [_VP, _VP, _VP]),
    "jfft_evolve": (_I, [_VP, _VP, ctypes.c_double, ctypes.c_double, _VP, _VP]),
}

_lock = threading.Lock()
_lib = None


def lib() -> ctypes.CDLL:
    """The loaded libjac; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"libjac.so not built ({LIB_PATH}); run __graft_entry__.build() "
                                  "or python -m paper_2002_12115_gb300._build")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIG.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def check(status: int, ctx=None) -> None:
    if status != JAC_OK:
        msg = lib().jac_last_error(ctx)
        raise JacError(status, msg.decode() if msg else "")


def stream_handle(stream=None) -> int:
    """cudaStream_t of a torch stream (default: the current stream)."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def pitch(I: int) -> int:
    return int(lib().jac_pitch(int(I)))


def _host_ptr(a: np.ndarray) -> int:
    if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
        raise ValueError("host fields must be C-contiguous float64 arrays")
    return a.ctypes.data


def field_bytes(I: int, J: int, K: int, prec: str, which: int) -> int:
    """Bytes of storage array `which` (index into FIELDS) of an I x J x K grid."""
    n = ctypes.c_size_t()
    check(lib().jac_field_bytes(int(I), int(J), int(K), PRECS[prec], int(which), ctypes.byref(n)))
    return n.value


def ctx_workspace_size(I: int, J: int, K: int, prec: str, async_upload: bool = False, tape=None) -> int:
    """Bytes of the workspace a borrowed context needs (jac_workspace_size);
    tape = (C, max_sweeps) reserves a checkpoint tape."""
    C, mx = tape if tape else (0, 0)
    n = ctypes.c_size_t()
    check(lib().jac_workspace_size(int(I), int(J), int(K), PRECS[prec],
                                   ctypes.byref(jac_ws_spec(int(bool(async_upload)), int(C), int(mx))),
                                   ctypes.byref(n)))
    return n.value


def _tape_states(C: int, mx: int) -> int:
    if C < 1 or mx < 1:
        return 0
    c = min(C, mx)
    return (mx + c - 1) // c + c + 1


class Jacobi:
    """One grid resident on the GPU (a jac_ctx).

    ``upload`` -> ``sweep(n)`` -> ``residual()`` / ``download()`` is the
    hoisted structure: one copy-in, n sweeps on resident arrays, one copy-out.
    Arrays are (K, J, I) float64, i fastest.

    By default the context is borrowed (jac_create_borrowed): the fourteen
    storage arrays and the workspace are torch tensors held by this object,
    so every device byte comes from torch's allocator and the library
    allocates none.  ``async_upload`` and ``tape=(C, max_sweeps)`` size the
    workspace up front; later calls that need more (upload_async, a longer
    tape) give the context a larger torch workspace.  ``owned=True`` makes
    the library allocate instead (jac_create).
    """

    def __init__(self, I: int, J: int, K: int, prec: str = "f32", omega: float = 0.8, stream=None,
                 owned: bool = False, async_upload: bool = False, tape=None):
        import torch
        if prec not in PRECS:
            raise ValueError(f"prec must be one of {list(PRECS)}")
        self.I, self.J, self.K, self.prec, self.omega = int(I), int(J), int(K), prec, float(omega)
        self._stream_obj = stream if stream is not None else torch.cuda.current_stream()
        self.stream = stream_handle(self._stream_obj)
        self.owned = bool(owned)
        self._pending = []       # host arrays of asynchronous copies, until sync()
        h = _VP()
        if self.owned:
            check(lib().jac_create(ctypes.byref(h), self.I, self.J, self.K, PRECS[prec], self.omega,
                                   _VP(self.stream)))
            self._h = h
            return
        dev = torch.device("cuda", torch.cuda.current_device())
        self.storage = [torch.empty(field_bytes(self.I, self.J, self.K, prec, 0), dtype=torch.uint8, device=dev)
                        for _ in range(2)]
        self.storage += [torch.empty(field_bytes(self.I, self.J, self.K, prec, q), dtype=torch.uint8, device=dev)
                         for q in range(1, NFIELDS)]
        g = jac_grid()
        g.I, g.J, g.K, g.prec, g.omega = self.I, self.J, self.K, PRECS[prec], self.omega
        g.p[0], g.p[1] = self.storage[0].data_ptr(), self.storage[1].data_ptr()
        for q in range(1, NFIELDS):
            g.coef[q] = self.storage[q + 1].data_ptr()
        self._spec = (bool(async_upload), tuple(tape) if tape else (0, 0))
        spec = jac_ws_spec(int(self._spec[0]), *self._spec[1])
        self.workspace = torch.empty(ctx_workspace_size(self.I, self.J, self.K, prec, *self._spec),
                                     dtype=torch.uint8, device=dev)
        check(lib().jac_create_borrowed(ctypes.byref(h), ctypes.byref(g), _VP(self.stream),
                                        _VP(self.workspace.data_ptr()), ctypes.c_size_t(self.workspace.numel()),
                                        ctypes.byref(spec)))
        self._h = h

    def device_bytes(self) -> int:
        """Device bytes this object holds for a borrowed context (storage
        arrays and workspace); 0 for an owned one."""
        if self.owned:
            return 0
        return sum(t.numel() for t in self.storage) + self.workspace.numel()

    def _ensure_workspace(self, async_upload: bool = False, tape=None) -> None:
        """Borrowed contexts: a larger torch workspace if the current one
        lacks the asynchronous staging or the tape asked for."""
        if self.owned:
            return
        import torch
        a0, t0 = self._spec
        want_a = a0 or bool(async_upload)
        want_t = t0
        if tape is not None and _tape_states(*tape) > _tape_states(*t0):
            want_t = tuple(tape)
        if (want_a, want_t) == (a0, t0):
            return
        ws = torch.empty(ctx_workspace_size(self.I, self.J, self.K, self.prec, want_a, want_t),
                         dtype=torch.uint8, device=self.workspace.device)
        self._check(lib().jac_set_workspace(self._h, _VP(ws.data_ptr()), ctypes.c_size_t(ws.numel()),
                                            ctypes.byref(jac_ws_spec(int(want_a), *want_t))))
        self.workspace, self._spec = ws, (want_a, want_t)

    def inject_stall(self, wait_ns: int) -> None:
        """Failure-path test aid (jac_inject_stall): the next sweep launch
        waits on a grid barrier nobody reaches, gives up after wait_ns and
        reports JAC_ETIMEOUT."""
        self._check(lib().jac_inject_stall(self._h, int(wait_ns)))

    # -- lifetime
    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().jac_destroy(self._h)
            self._h = None
        self.storage = []
        self.workspace = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def shape(self):
        return (self.K, self.J, self.I)

    def _check(self, st: int) -> None:
        check(st, self._h)

    def _fields(self, arrays: dict, device: bool) -> jac_fields:
        f = jac_fields()
        for q, name in enumerate(FIELDS):
            a = arrays[name]
            if device:
                if tuple(a.shape) != self.shape or a.dtype.__str__() != "torch.float64" or not a.is_contiguous():
                    raise ValueError(f"{name}: expected a contiguous float64 CUDA tensor of shape {self.shape}")
                f.f[q] = a.data_ptr()
            else:
                if tuple(a.shape) != self.shape:
                    raise ValueError(f"{name}: expected shape {self.shape}")
                f.f[q] = _host_ptr(a)
        return f

    # -- the hoisted path
    def set_plan(self, tile_j: int = 0, kdepth: int = 0, tile_i: int = 0, fuse: int = 0) -> None:
        """Launch plan (0 = default); fuse: 0 library's choice, 1 single sweeps only,
        2 two-sweep passes (FP32 storage)."""
        self._check(lib().jac_set_plan(self._h, ctypes.byref(jac_plan(int(tile_j), int(kdepth), int(tile_i),
                                                                       int(fuse)))))

    def upload(self, fields: dict) -> None:
        """Copy in all thirteen host arrays (float64, shape (K, J, I))."""
        f = self._fields(fields, device=False)
        self._check(lib().jac_upload(self._h, ctypes.byref(f)))

    def upload_tensors(self, fields: dict) -> None:
        """Same, from contiguous float64 CUDA tensors."""
        f = self._fields(fields, device=True)
        self._check(lib().jac_upload_dev(self._h, ctypes.byref(f)))

    def upload_async(self, fields: dict) -> None:
        """Copy in without waiting (pinned host arrays for an asynchronous
        copy).  The arrays are kept referenced until sync()."""
        f = self._fields(fields, device=False)
        self._ensure_workspace(async_upload=True)
        self._check(lib().jac_upload_async(self._h, ctypes.byref(f)))
        self._pending.append(fields)

    def upload_f32_async(self, fields: dict) -> None:
        """Copy in thirteen dense FP32 host arrays (float32, shape (K, J, I))
        without waiting: half the bytes of upload_async, for inputs that are
        FP32 numbers.  The arrays are kept referenced until sync()."""
        f = jac_fields_f32()
        for q, name in enumerate(FIELDS):
            a = fields[name]
            if tuple(a.shape) != self.shape or a.dtype != np.float32 or not a.flags["C_CONTIGUOUS"]:
                raise ValueError(f"{name}: expected a C-contiguous float32 array of shape {self.shape}")
            f.f[q] = a.ctypes.data
        self._ensure_workspace(async_upload=True)
        self._check(lib().jac_upload_f32_async(self._h, ctypes.byref(f)))
        self._pending.append(fields)

    def download_f32_async(self, out: np.ndarray, res_out: np.ndarray | None = None) -> None:
        """Enqueue the copy-out of the state as FP32 to `out` (float32, shape
        (K, J, I)) and, if given, of the residual to res_out[0]; valid after sync()."""
        if tuple(out.shape) != self.shape or out.dtype != np.float32 or not out.flags.c_contiguous:
            raise ValueError(f"out: expected a contiguous float32 array of shape {self.shape}")
        if res_out is not None and (res_out.dtype != np.float64 or res_out.size < 1):
            raise ValueError("res_out: expected a float64 array of at least one element")
        self._check(lib().jac_download_f32_async(self._h, _VP(out.ctypes.data),
                                                 _VP(_host_ptr(res_out)) if res_out is not None else None))
        self._pending.append((out, res_out))

    def download_async(self, out: np.ndarray, res_out: np.ndarray | None = None) -> None:
        """Enqueue the copy-out of the state to `out` (float64, shape (K, J, I))
        and, if given, of the residual to res_out[0] (a float64 array); both
        are valid after sync()."""
        if tuple(out.shape) != self.shape or out.dtype != np.float64 or not out.flags.c_contiguous:
            raise ValueError(f"out: expected a contiguous float64 array of shape {self.shape}")
        if res_out is not None and (res_out.dtype != np.float64 or res_out.size < 1):
            raise ValueError("res_out: expected a float64 array of at least one element")
        self._check(lib().jac_download_async(self._h, _VP(_host_ptr(out)),
                                             _VP(_host_ptr(res_out)) if res_out is not None else None))
        self._pending.append((out, res_out))

    def sync(self) -> None:
        """Wait for this context's stream; raises on a device wait that gave up."""
        st = lib().jac_sync(self._h)
        self._pending.clear()
        self._check(st)

    def sweep(self, n: int) -> None:
        self._check(lib().jac_sweep(self._h, int(n)))

    def residual(self) -> float:
        out = ctypes.c_double()
        self._check(lib().jac_residual(self._h, ctypes.byref(out)))
        return out.value

    def download(self, out: np.ndarray | None = None) -> np.ndarray:
        if out is None:
            out = np.empty(self.shape, dtype=np.float64)
        self._check(lib().jac_download(self._h, _VP(_host_ptr(out))))
        return out

    def download_tensor(self, out=None):
        import torch
        if out is None:
            out = torch.empty(self.shape, dtype=torch.float64, device="cuda")
        self._check(lib().jac_download_dev(self._h, _VP(out.data_ptr())))
        return out

    def count(self) -> int:
        c = ctypes.c_longlong()
        self._check(lib().jac_sweep_count(self._h, ctypes.byref(c)))
        return c.value

    def grid(self) -> jac_grid:
        g = jac_grid()
        self._check(lib().jac_get_grid(self._h, ctypes.byref(g)))
        return g

    # -- reverse mode
    def tape_begin(self, C: int, max_sweeps: int) -> None:
        """Record the next sweeps (at most max_sweeps) with a checkpoint every C."""
        self._ensure_workspace(tape=(int(C), int(max_sweeps)))
        self._check(lib().jac_tape_begin(self._h, int(C), int(max_sweeps)))

    def tape_end(self) -> None:
        self._check(lib().jac_tape_end(self._h))

    def tape_count(self) -> int:
        n = ctypes.c_int()
        self._check(lib().jac_tape_count(self._h, ctypes.byref(n)))
        return n.value

    def sweep_adjoint(self, lam_T, coef_grads: bool = False, want_p0: bool = True) -> dict:
        """Reverse pass over the taped sweeps.  lam_T: float64 CUDA tensor
        (K, J, I) = dL/dp_T.  Returns FP64 tensors g_wrk1, g_a3 and, as
        requested, g_p0 and g_a0..g_c2."""
        import torch
        if tuple(lam_T.shape) != self.shape or lam_T.dtype != torch.float64 or not lam_T.is_cuda:
            raise ValueError(f"lam_T must be a float64 CUDA tensor of shape {self.shape}")
        lam_T = lam_T.contiguous()
        out = {"g_wrk1": torch.empty_like(lam_T), "g_a3": torch.empty_like(lam_T)}
        gc = None
        if coef_grads:
            names = ("a0", "a1", "a2", "b0", "b1", "b2", "c0", "c1", "c2")
            for nm in names:
                out["g_" + nm] = torch.empty_like(lam_T)
            gc = (_VP * 9)(*[out["g_" + nm].data_ptr() for nm in names])
        if want_p0:
            out["g_p0"] = torch.empty_like(lam_T)
        self._check(lib().jac_sweep_adjoint(self._h, _VP(lam_T.data_ptr()), _VP(out["g_wrk1"].data_ptr()),
                                            _VP(out["g_a3"].data_ptr()), gc,
                                            _VP(out["g_p0"].data_ptr()) if want_p0 else None))
        return out

    def sweep_unhoisted(self, n: int, fields: dict, p_host: np.ndarray) -> None:
        """Per-sweep copy-in / copy-out (measurement contrast only)."""
        f = self._fields(fields, device=False)
        self._check(lib().jac_sweep_unhoisted(self._h, int(n), ctypes.byref(f), _VP(_host_ptr(p_host))))


def resolve_plan(I: int, J: int, K: int, prec: str = "f32", sm_count: int = 0, tile_j: int = 0, kdepth: int = 0,
                 tile_i: int = 0, fuse: int = 0) -> dict:
    """The launch plan a sweep of an I x J x K grid runs with on a device of
    sm_count SMs (0: the current device); the zero entries are filled in."""
    g = jac_grid()
    g.I, g.J, g.K, g.prec, g.omega = int(I), int(J), int(K), PRECS[prec], 0.8
    out = jac_plan()
    check(lib().jac_resolve_plan(ctypes.byref(g), ctypes.byref(jac_plan(int(tile_j), int(kdepth), int(tile_i),
                                                                        int(fuse))), int(sm_count),
                                 ctypes.byref(out)))
    return {"tile_j": out.tile_j, "kdepth": out.kdepth, "tile_i": out.tile_i, "fuse": out.fuse}


def workspace_size(grid: jac_grid, tile_j: int = 0, kdepth: int = 0, tile_i: int = 0, fuse: int = 0) -> int:
    n = ctypes.c_size_t()
    check(lib().jac_sweep_workspace_size(ctypes.byref(grid), ctypes.byref(jac_plan(tile_j, kdepth, tile_i, fuse)),
                                         ctypes.byref(n)))
    return n.value


def sweep_dev(grid: jac_grid, n: int, d_residual: int | None, workspace: int, ws_bytes: int,
              stream: int, tile_j: int = 0, kdepth: int = 0, tile_i: int = 0, fuse: int = 0) -> None:
    """The stateless entry point jac_sweep_dev on caller-owned device buffers."""
    check(lib().jac_sweep_dev(ctypes.byref(grid), ctypes.byref(jac_plan(tile_j, kdepth, tile_i, fuse)), int(n),
                              _VP(d_residual) if d_residual else None, _VP(workspace), ctypes.c_size_t(ws_bytes),
                              _VP(stream)))


def workspace_check(workspace: int, stream: int) -> None:
    """Synchronise the stream and raise if a kernel set the workspace error word."""
    check(lib().jac_workspace_check(_VP(workspace), _VP(stream)))


def pack_dev(I: int, J: int, K: int, prec: str, which: int, src: int, dst: int, stream: int) -> None:
    """Dense FP64 device array -> storage layout of array `which` (index into FIELDS)."""
    check(lib().jac_pack_dev(int(I), int(J), int(K), PRECS[prec], int(which), _VP(src), _VP(dst), _VP(stream)))


def unpack_dev(I: int, J: int, K: int, prec: str, which: int, src: int, dst: int, stream: int) -> None:
    """Storage layout of array `which` -> dense FP64 device array."""
    check(lib().jac_unpack_dev(int(I), int(J), int(K), PRECS[prec], int(which), _VP(src), _VP(dst), _VP(stream)))


def adjoint_step_dev(grid: jac_grid, p_t: int, lam_in: int, lam_out: int, g_wrk1: int, g_a3: int,
                     workspace: int, ws_bytes: int, stream: int, g_coef=None, kdepth: int = 0) -> None:
    """The stateless entry point jac_adjoint_step_dev (device pointers)."""
    gc = (_VP * 9)(*g_coef) if g_coef is not None else None
    check(lib().jac_adjoint_step_dev(ctypes.byref(grid), _VP(p_t), _VP(lam_in), _VP(lam_out), _VP(g_wrk1),
                                     _VP(g_a3), gc, int(kdepth), _VP(workspace), ctypes.c_size_t(ws_bytes),
                                     _VP(stream)))


class JacobiBatch:
    """Many independent grids of uneven sizes, swept together in one
    persistent launch replayed from a CUDA graph (a jac_batch)."""

    def __init__(self, dims, prec: str = "f32", omega: float = 0.8, stream=None):
        import torch
        if prec not in PRECS:
            raise ValueError(f"prec must be one of {list(PRECS)}")
        self.dims = [tuple(int(x) for x in d) for d in dims]
        self.n, self.prec, self.omega = len(self.dims), prec, float(omega)
        self._stream_obj = stream if stream is not None else torch.cuda.current_stream()
        self.stream = stream_handle(self._stream_obj)
        flat = (ctypes.c_int * (3 * self.n))(*[x for d in self.dims for x in d])
        h = _VP()
        check(lib().jac_batch_create(ctypes.byref(h), self.n, ctypes.cast(flat, _VP), PRECS[prec], self.omega,
                                     _VP(self.stream)))
        self._h = h

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().jac_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, st: int) -> None:
        if st != JAC_OK:
            msg = lib().jac_batch_last_error(self._h)
            raise JacError(st, msg.decode() if msg else "")

    def shape(self, g: int):
        I, J, K = self.dims[g]
        return (K, J, I)

    def _fields(self, g: int, arrays: dict, device: bool) -> jac_fields:
        f = jac_fields()
        for q, name in enumerate(FIELDS):
            a = arrays[name]
            if tuple(a.shape) != self.shape(g):
                raise ValueError(f"grid {g} {name}: expected shape {self.shape(g)}")
            f.f[q] = a.data_ptr() if device else _host_ptr(a)
        return f

    def upload(self, g: int, fields: dict) -> None:
        f = self._fields(g, fields, device=False)
        self._check(lib().jac_batch_upload(self._h, int(g), ctypes.byref(f)))

    def upload_tensors(self, g: int, fields: dict) -> None:
        f = self._fields(g, fields, device=True)
        self._check(lib().jac_batch_upload_dev(self._h, int(g), ctypes.byref(f)))

    def set_plan(self, warps: int = 0, tile_i=None, kdepth=None) -> None:
        ti = (ctypes.c_int * self.n)(*tile_i) if tile_i is not None else None
        kd = (ctypes.c_int * self.n)(*kdepth) if kdepth is not None else None
        self._check(lib().jac_batch_set_plan(self._h, int(warps), ctypes.cast(ti, _VP) if ti else None,
                                             ctypes.cast(kd, _VP) if kd else None))

    def grid_plan(self, g: int) -> tuple:
        p = jac_plan()
        self._check(lib().jac_batch_grid_plan(self._h, int(g), ctypes.byref(p)))
        return (p.tile_i, p.tile_j, p.kdepth)

    def sweep(self, n: int, residuals: bool = True):
        """n sweeps of every grid in one persistent launch (graph replay)."""
        out = np.empty(self.n) if residuals else None
        self._check(lib().jac_batch_sweep(self._h, int(n), _VP(out.ctypes.data) if residuals else None))
        return out

    def sweep_loop(self, n: int, per_sweep: bool = False, residuals: bool = True):
        """The same sweeps as per-grid launches (comparison)."""
        out = np.empty(self.n) if residuals else None
        self._check(lib().jac_batch_sweep_loop(self._h, int(n), int(bool(per_sweep)),
                                               _VP(out.ctypes.data) if residuals else None))
        return out

    def download(self, g: int, out: np.ndarray | None = None) -> np.ndarray:
        if out is None:
            out = np.empty(self.shape(g), dtype=np.float64)
        self._check(lib().jac_batch_download(self._h, int(g), _VP(_host_ptr(out))))
        return out

    def download_tensor(self, g: int, out=None):
        import torch
        if out is None:
            out = torch.empty(self.shape(g), dtype=torch.float64, device="cuda")
        self._check(lib().jac_batch_download_dev(self._h, int(g), _VP(out.data_ptr())))
        return out

    def info(self) -> dict:
        a, b, c, d = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_longlong()
        self._check(lib().jac_batch_info(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                         ctypes.byref(d)))
        return {"items": a.value, "ctas": b.value, "warps": c.value, "sweeps": d.value}


# ---------------------------------------------------------------- 3-D FFT
FFT_PRECS = {"c64": 0, "c32": 1}


def fft_workspace_size(n1: int, n2: int, n3: int, prec: str = "c32") -> int:
    """Bytes of the workspace an FFT plan of this shape needs (jfft_workspace_size)."""
    n = ctypes.c_size_t()
    check(lib().jfft_workspace_size(int(n1), int(n2), int(n3), FFT_PRECS[prec], ctypes.byref(n)))
    return n.value


class FFT3:
    """3-D complex FFT of an (n3, n2, n1) array (x fastest) on the GPU (a
    jfft_plan).  The workspace is a torch tensor held by this object; data
    arrays are complex64 ("c32") or complex128 ("c64") CUDA tensors."""

    def __init__(self, n1: int, n2: int, n3: int, prec: str = "c32", stream=None):
        import torch
        if prec not in FFT_PRECS:
            raise ValueError(f"prec must be one of {list(FFT_PRECS)}")
        self.n1, self.n2, self.n3, self.prec = int(n1), int(n2), int(n3), prec
        self.dtype = torch.complex64 if prec == "c32" else torch.complex128
        self._stream_obj = stream if stream is not None else torch.cuda.current_stream()
        self.stream = stream_handle(self._stream_obj)
        self.workspace = torch.empty(fft_workspace_size(n1, n2, n3, prec), dtype=torch.uint8, device="cuda")
        h = _VP()
        check(lib().jfft_plan_create(ctypes.byref(h), self.n1, self.n2, self.n3, FFT_PRECS[prec],
                                     _VP(self.stream), _VP(self.workspace.data_ptr()),
                                     ctypes.c_size_t(self.workspace.numel())))
        self._h = h

    @property
    def shape(self):
        return (self.n3, self.n2, self.n1)

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().jfft_destroy(self._h)
            self._h = None
        self.workspace = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, st: int) -> None:
        if st != JAC_OK:
            msg = lib().jfft_last_error(self._h)
            raise JacError(st, msg.decode() if msg else "")

    def _arg(self, x, name):
        if tuple(x.shape) != self.shape or x.dtype != self.dtype or not x.is_cuda or not x.is_contiguous():
            raise ValueError(f"{name}: expected a contiguous {self.dtype} CUDA tensor of shape {self.shape}")
        return _VP(x.data_ptr())

    def forward(self, x, out=None):
        """Unscaled forward transform; out may be x (in place)."""
        import torch
        out = torch.empty_like(x) if out is None else out
        self._check(lib().jfft_forward(self._h, self._arg(x, "x"), self._arg(out, "out")))
        return out

    def inverse(self, X, out=None):
        """Inverse transform scaled by 1/N; out may be X (in place)."""
        import torch
        out = torch.empty_like(X) if out is None else out
        self._check(lib().jfft_inverse(self._h, self._arg(X, "X"), self._arg(out, "out")))
        return out

    def evolve(self, U, alpha: float, t: float, out=None, energy=None):
        """The spectral step inverse(U * exp(-4 pi^2 alpha t |kbar|^2)); energy:
        a float64 CUDA tensor of one element that receives sum |u|^2, or None."""
        import torch
        out = torch.empty_like(U) if out is None else out
        ep = None
        if energy is not None:
            if energy.dtype != torch.float64 or not energy.is_cuda or energy.numel() < 1:
                raise ValueError("energy: expected a float64 CUDA tensor")
            ep = _VP(energy.data_ptr())
        self._check(lib().jfft_evolve(self._h, self._arg(U, "U"), float(alpha), float(t), self._arg(out, "out"),
                                      ep))
        return out
