"""ctypes binding of liblsp.so (the C ABI in include/lsp.h).

Argument marshalling only: every computation of the Strang step runs in the
library's CUDA kernels.  Device buffers are torch CUDA tensors (data_ptr) and
streams are torch CUDA streams; host buffers are numpy arrays.  There is no
CPU fallback: if the library cannot be built or loaded, or a call fails, an
exception is raised.
"""

from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

LSP_OK = 0
C64, C128 = 1, 2
AA_MINL2, AA_EXPLICIT = 0, 1
PHYSICAL, SPECTRAL = 0, 1
PATH_MULTIPASS, PATH_SMALL, PATH_RANK2, PATH_RANK1_4SWEEP, PATH_RANK1_TMA, PATH_MIXED = 0, 1, 2, 3, 4, 5
NUM_PATHS = 6

_lib = None
_lock = threading.Lock()


class LspError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} ({code})")


def library_path() -> str:
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "liblsp.so")


def _declare(lib):
    P, I, I64, D, V = C.c_void_p, C.c_int, C.c_int64, C.c_double, None
    sig = {
        "lsp_plan_create": (I, [C.POINTER(C.c_void_p), I, I, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                C.POINTER(C.c_int32), I64, I, I, D, I]),
        "lsp_plan_destroy": (V, [P]),
        "lsp_set_potential": (I, [P, P, I, P]),
        "lsp_set_state": (I, [P, P, I, I, P]),
        "lsp_strang_steps": (I, [P, D, I64, P]),
        "lsp_get_state": (I, [P, P, I, I, I, P]),
        "lsp_plan_status": (I, [P, P]),
        "lsp_lattice_points": (I, [P, P]),
        "lsp_index_norms": (I, [P, P]),
        "lsp_index_table": (I, [P, P]),
        "lsp_plan_info": (I, [P, P]),
        "lsp_plan_paths": (I, [P, C.POINTER(C.c_int)]),
        "lsp_observables": (I, [P, P, P]),
        "lsp_strang_composed": (I, [P, D, I64, I, P, P]),
        "lsp_plan_set_path": (I, [P, I]),
        "lsp_plan_autotune": (I, [P, D, I64, P, C.POINTER(C.c_int), C.POINTER(C.c_double)]),
        "lsp_batch_create": (I, [C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), I]),
        "lsp_batch_steps": (I, [P, P, I64, P]),
        "lsp_batch_destroy": (V, [P]),
        "lsp_batch_status": (I, [P, P]),
        "lsp_adjoint": (I, [P, D, I64, P, P, P, I64, P]),
        "lsp_strang_steps_noalloc": (I, [I, I64, D, D, I64, P, P, P, P]),
        "lsp_sweep_times": (I, [P, D, I64, P, P]),
        "lsp_cbc_reconstructing": (I, [P, I64, I, I, P, P, I64, P, C.POINTER(C.c_int), I]),
        "lsp_plan_set_wait_limit": (I, [P, I64]),
        "lsp_plan_schedule": (I, [P, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
        "lsp_plan_set_schedule": (I, [P, I]),
        "lsp_autotune_cache": (I, [I, C.POINTER(C.c_int64)]),
        "lsp_fma_rate": (I, [I, I, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
        "lsp_strerror": (C.c_char_p, [I]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


def load_library(build_if_missing: bool = True):
    """Load liblsp.so, compiling it first when it is missing or stale."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = library_path()
        if build_if_missing:
            from . import build as _build
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing; run __graft_entry__.build()")
        _lib = _declare(C.CDLL(path))
        return _lib


def strerror(code: int) -> str:
    lib = load_library()
    return lib.lsp_strerror(int(code)).decode()


def _check(code: int, where: str):
    if code != LSP_OK:
        raise LspError(code, where)


def _prec_code(prec) -> int:
    if prec in (C64, "c64", "complex64"):
        return C64
    if prec in (C128, "c128", "complex128"):
        return C128
    raise ValueError(f"unknown precision {prec!r}")


def _stream_ptr(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


_KEEP = threading.local()


def _buf(x, output: bool = False):
    """(pointer, on_device) for a torch tensor or numpy array.

    Torch views with a lazy conjugate or negative bit do not hold the values
    they represent in memory: inputs are materialised (the copy is kept alive
    until the next call from this thread, and is stream-ordered anyway);
    outputs must be plain tensors."""
    try:
        import torch
        if isinstance(x, torch.Tensor):
            if x.is_complex() and (x.is_conj() or x.is_neg()):
                if output:
                    raise ValueError("output tensor must not be a conjugate or negative view")
                x = x.resolve_conj().resolve_neg()
                _KEEP.t = x
            if not x.is_contiguous():
                raise ValueError("tensor must be contiguous")
            return C.c_void_p(x.data_ptr()), int(x.is_cuda)
    except ImportError:
        pass
    a = np.asarray(x)
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return C.c_void_p(a.ctypes.data), 0


class Plan:
    """One TDSE instance on a rank-r lattice, r <= 4 (lsp_plan_create)."""

    def __init__(self, Z, n, gamma: float, prec="c64", aa: str = "minl2", index_set=None,
                 device: int = 0):
        lib = load_library()
        nn = np.atleast_1d(np.asarray(n, dtype=np.int64))
        r = nn.size
        Zm = np.asarray(Z, dtype=np.int64).reshape(-1, r)
        self.d, self.r = Zm.shape[0], r
        self.n = tuple(int(x) for x in nn)
        self.npoints = int(np.prod(nn))
        self.prec = _prec_code(prec)
        self.gamma = float(gamma)
        self.device = int(device)
        Zc = np.ascontiguousarray(Zm)
        mode = AA_EXPLICIT if aa == "explicit" else AA_MINL2
        if mode == AA_EXPLICIT:
            I = np.ascontiguousarray(np.asarray(index_set, dtype=np.int32))
            iptr, m = I.ctypes.data_as(C.POINTER(C.c_int32)), I.shape[0]
            self._index_set = I
        else:
            iptr, m = None, 0
        h = C.c_void_p()
        _check(lib.lsp_plan_create(C.byref(h), self.d, r, nn.ctypes.data_as(C.POINTER(C.c_int64)),
                                   Zc.ctypes.data_as(C.POINTER(C.c_int64)), iptr, m, mode, self.prec,
                                   self.gamma, self.device), "lsp_plan_create")
        self._h = h
        self._lib = lib

    # -- lifetime ----------------------------------------------------------
    def destroy(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.lsp_plan_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    # -- data --------------------------------------------------------------
    def set_potential(self, v, stream=None):
        ptr, dev = _buf(v)
        _check(self._lib.lsp_set_potential(self._h, ptr, dev, _stream_ptr(stream) if dev else None),
               "lsp_set_potential")

    def set_state(self, u, stream=None):
        ptr, dev = _buf(u)
        prec = C64 if str(getattr(u, "dtype", "")).endswith("complex64") else C128
        _check(self._lib.lsp_set_state(self._h, ptr, prec, dev, _stream_ptr(stream) if dev else None),
               "lsp_set_state")

    def strang_steps(self, dt: float, nsteps: int, stream=None):
        _check(self._lib.lsp_strang_steps(self._h, float(dt), int(nsteps), _stream_ptr(stream)),
               "lsp_strang_steps")

    def strang_composed(self, dt: float, nsteps: int, weights, stream=None):
        """lsp_strang_composed: each step is S(w_s dt) ... S(w_1 dt) (e.g. fourth order with
        weights = yoshida4())."""
        w = np.ascontiguousarray(np.asarray(weights, dtype=np.float64))
        _check(self._lib.lsp_strang_composed(self._h, float(dt), int(nsteps), int(w.size), C.c_void_p(w.ctypes.data),
                                             _stream_ptr(stream)), "lsp_strang_composed")

    def get_state(self, out=None, space: str = "physical", prec=None, stream=None):
        """Copy the state into `out` (torch CUDA tensor or numpy array).  Without `out`
        a new torch tensor on the plan's device is returned."""
        sp = SPECTRAL if space == "spectral" else PHYSICAL
        if out is None:
            import torch
            pc = self.prec if prec is None else _prec_code(prec)
            out = torch.empty(self.npoints, dtype=torch.complex64 if pc == C64 else torch.complex128,
                              device=f"cuda:{self.device}")
        pc = C64 if str(out.dtype).endswith("complex64") else C128
        ptr, dev = _buf(out, output=True)
        _check(self._lib.lsp_get_state(self._h, ptr, pc, sp, dev, _stream_ptr(stream)), "lsp_get_state")
        return out

    def observables(self, stream=None):
        """(norm^2, energy) of the current state (lsp_observables, Sec. 3.3)."""
        out = np.zeros(2, dtype=np.float64)
        _check(self._lib.lsp_observables(self._h, C.c_void_p(out.ctypes.data), _stream_ptr(stream)),
               "lsp_observables")
        return float(out[0]), float(out[1])

    def status(self, stream=None) -> int:
        return int(self._lib.lsp_plan_status(self._h, _stream_ptr(stream)))

    def schedule(self):
        """(path, kernel schedule) of the plan (lsp_plan_schedule)."""
        a, b = C.c_int(), C.c_int()
        _check(self._lib.lsp_plan_schedule(self._h, C.byref(a), C.byref(b)), "lsp_plan_schedule")
        return a.value, b.value

    def set_schedule(self, sched: int):
        _check(self._lib.lsp_plan_set_schedule(self._h, int(sched)), "lsp_plan_set_schedule")

    def set_wait_limit(self, polls: int):
        """lsp_plan_set_wait_limit: polls of a bounded device wait before it gives up (0: default)."""
        _check(self._lib.lsp_plan_set_wait_limit(self._h, int(polls)), "lsp_plan_set_wait_limit")

    # -- queries -----------------------------------------------------------
    def lattice_points(self) -> np.ndarray:
        x = np.empty((self.npoints, self.d), dtype=np.float64)
        _check(self._lib.lsp_lattice_points(self._h, C.c_void_p(x.ctypes.data)), "lsp_lattice_points")
        return x

    def index_norms(self) -> np.ndarray:
        x = np.empty(self.npoints, dtype=np.int64)
        _check(self._lib.lsp_index_norms(self._h, C.c_void_p(x.ctypes.data)), "lsp_index_norms")
        return x

    def index_table(self) -> np.ndarray:
        x = np.empty((self.npoints, self.d), dtype=np.int32)
        _check(self._lib.lsp_index_table(self._h, C.c_void_p(x.ctypes.data)), "lsp_index_table")
        return x

    def paths(self) -> list:
        """Execution paths this plan can run (lsp_plan_paths)."""
        m = C.c_int()
        _check(self._lib.lsp_plan_paths(self._h, C.byref(m)), "lsp_plan_paths")
        return [k for k in range(NUM_PATHS) if m.value >> k & 1]

    def set_path(self, path: int):
        _check(self._lib.lsp_plan_set_path(self._h, int(path)), "lsp_plan_set_path")

    def sweep_times(self, dt: float, nsteps: int, stream=None) -> dict:
        """lsp_sweep_times: mean ms per launch of the P, A / Y, K and A^-1 / Y^-1 sweeps (multi-launch
        paths; the TMA two-sweep path has only the P (column) and K (row) sweeps, the others are -1)."""
        ms = np.zeros(4, dtype=np.float64)
        _check(self._lib.lsp_sweep_times(self.handle, float(dt), int(nsteps), _stream_ptr(stream),
                                         C.c_void_p(ms.ctypes.data)), "lsp_sweep_times")
        return dict(zip(("P", "A", "K", "A_inv"), (float(x) for x in ms)))

    def autotune(self, dt: float, nsteps: int, stream=None):
        """Time nsteps steps on every available path, keep the fastest; returns (path, {path: ms})."""
        chosen = C.c_int()
        ms = (C.c_double * NUM_PATHS)()
        _check(self._lib.lsp_plan_autotune(self._h, float(dt), int(nsteps), _stream_ptr(stream), C.byref(chosen), ms),
               "lsp_plan_autotune")
        return chosen.value, {k: ms[k] for k in range(NUM_PATHS) if ms[k] >= 0}

    def info(self) -> dict:
        x = np.zeros(8, dtype=np.int64)
        _check(self._lib.lsp_plan_info(self._h, C.c_void_p(x.ctypes.data)), "lsp_plan_info")
        keys = ["n", "N1", "N2", "path", "prec", "bytes", "dp_box", "max_norm2"]
        return dict(zip(keys, (int(v) for v in x)))


class Batch:
    """Several plans advanced together (lsp_batch_create / lsp_batch_steps)."""

    def __init__(self, plans):
        lib = load_library()
        self.plans = list(plans)
        arr = (C.c_void_p * len(self.plans))(*[p.handle.value for p in self.plans])
        h = C.c_void_p()
        _check(lib.lsp_batch_create(C.byref(h), arr, len(self.plans)), "lsp_batch_create")
        self._h, self._lib = h, lib

    def steps(self, dts, nsteps: int, stream=None):
        dt = np.ascontiguousarray(np.asarray(dts, dtype=np.float64))
        _check(self._lib.lsp_batch_steps(self._h, C.c_void_p(dt.ctypes.data), int(nsteps), _stream_ptr(stream)),
               "lsp_batch_steps")

    def observables(self, stream=None):
        """(norm^2, energy) of the current state (lsp_observables, Sec. 3.3)."""
        out = np.zeros(2, dtype=np.float64)
        _check(self._lib.lsp_observables(self._h, C.c_void_p(out.ctypes.data), _stream_ptr(stream)),
               "lsp_observables")
        return float(out[0]), float(out[1])

    def status(self, stream=None) -> int:
        return int(self._lib.lsp_batch_status(self._h, _stream_ptr(stream)))

    def destroy(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.lsp_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def autotune_cache(clear: bool = False) -> int:
    """lsp_autotune_cache: number of stored autotune decisions (emptied first when clear)."""
    lib = load_library()
    n = C.c_int64()
    _check(lib.lsp_autotune_cache(int(bool(clear)), C.byref(n)), "lsp_autotune_cache")
    return int(n.value)


def fma_rate(prec="c128", device: int = 0):
    """lsp_fma_rate: measured FMA throughput of the device in TFLOP/s (FP64 for c128, FP32 for c64)."""
    lib = load_library()
    t, ms = C.c_double(), C.c_double()
    _check(lib.lsp_fma_rate(int(device), _prec_code(prec), C.byref(t), C.byref(ms)), "lsp_fma_rate")
    return float(t.value)


def yoshida4():
    """Stage weights (c, 1 - 2c, c), c = 1 / (2 - 2^(1/3)): a fourth-order composition of Strang steps."""
    c = 1.0 / (2.0 - 2.0 ** (1.0 / 3.0))
    return (c, 1.0 - 2.0 * c, c)


def strang_steps_noalloc(u, v, norm2, gamma: float, dt: float, nsteps: int, stream=None):
    """lsp_strang_steps_noalloc: allocation-free Strang steps on device tensors
    (u complex64/complex128 updated in place, v float64, norm2 int32, all with
    u.numel() elements on u's CUDA device).  The kernels take raw pointers, so
    every argument is checked here: a host array, a shorter or differently typed
    buffer or a tensor on another device would be read out of bounds."""
    import torch
    for name, t in (("u", u), ("v", v), ("norm2", norm2)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if t.device != u.device:
            raise ValueError(f"{name} is on {t.device}, u on {u.device}")
    if u.dtype not in (torch.complex64, torch.complex128):
        raise ValueError(f"u must be complex64 or complex128, not {u.dtype}")
    if v.dtype != torch.float64:
        raise ValueError(f"v must be float64, not {v.dtype}")
    if norm2.dtype != torch.int32:
        raise ValueError(f"norm2 must be int32, not {norm2.dtype}")
    n = u.numel()
    if v.numel() != n or norm2.numel() != n:
        raise ValueError(f"v ({v.numel()}) and norm2 ({norm2.numel()}) must hold u.numel() = {n} elements")
    lib = load_library()
    prec = C64 if u.dtype == torch.complex64 else C128
    with torch.cuda.device(u.device):
        up, _ = _buf(u, output=True)
        vp, _ = _buf(v)
        np_, _ = _buf(norm2)
        _check(lib.lsp_strang_steps_noalloc(prec, int(n), float(gamma), float(dt), int(nsteps), vp, np_, up,
                                            _stream_ptr(stream)), "lsp_strang_steps_noalloc")


def adjoint(plan: Plan, dt: float, nsteps: int, lamT, grad_v, grad_u0, ckpt_stride: int = 0, stream=None):
    """lsp_adjoint: gradients of a real objective of u_T w.r.t. v and u_0 (device tensors)."""
    lp, _ = _buf(lamT)
    gv, _ = _buf(grad_v, output=True)
    gu, _ = _buf(grad_u0, output=True)
    _check(plan._lib.lsp_adjoint(plan.handle, float(dt), int(nsteps), lp, gv, gu, int(ckpt_stride),
                                 _stream_ptr(stream)), "lsp_adjoint")


def cbc_reconstructing(index_set, n, candidates, device: int = 0):
    """lsp_cbc_reconstructing: generating vectors built component by component on the GPU.

    index_set (m, d) ints; n an int (rank 1) or (n1, n2); candidates (d - 1, T, r) ints.
    Returns (Z, fixed): Z of shape (d, r) and the number of components fixed (d on
    success; fewer when a component's list held no injective candidate).
    """
    lib = load_library()
    I = np.ascontiguousarray(np.asarray(index_set), dtype=np.int32)
    nt = np.ascontiguousarray(np.atleast_1d(np.asarray(n, dtype=np.int64)))
    r = int(nt.size)
    m, d = I.shape
    cand = np.ascontiguousarray(np.asarray(candidates, dtype=np.int64).reshape(max(d - 1, 0), -1, r))
    Z = np.zeros((d, r), dtype=np.int64)
    fixed = C.c_int(0)
    rc = lib.lsp_cbc_reconstructing(C.c_void_p(I.ctypes.data), int(m), int(d), r, C.c_void_p(nt.ctypes.data),
                                    C.c_void_p(cand.ctypes.data), int(cand.shape[1]) if d > 1 else 0,
                                    C.c_void_p(Z.ctypes.data), C.byref(fixed), int(device))
    if rc != -3:                                   # NOT_INJECTIVE is an answer, not a failure
        _check(rc, "lsp_cbc_reconstructing")
    return Z, int(fixed.value)
