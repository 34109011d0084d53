"""ctypes binding of libigm.so (the C ABI of include/igm.h).

Argument marshalling only: every step of the solver runs in the CUDA
library.  Arrays may be torch CUDA tensors, torch CPU tensors or numpy
arrays; the library itself copies host memory to the device.  There is no
CPU fallback: if libigm.so has not been built the import of the solver
raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

STATUS = {0: "ok", 1: "einval", 2: "ezero_row", 3: "ezero_pivot", 4: "ebreakdown",
          5: "enoconv", 6: "eoom", 7: "etimeout", 8: "ecuda"}
EV_NAMES = ["L5", "L5p", "L7", "L8", "L10", "L11", "L13", "L15", "L16", "L17",
            "vrange", "L2", "r12", "r13", "r14", "r15"]
MAX_M = 128


class IGMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status
        self.name = STATUS.get(status, str(status))


class Params(C.Structure):
    _fields_ = [("df", C.c_int), ("alpha_a", C.c_int), ("m", C.c_int), ("precond", C.c_int),
                ("beta7", C.c_int), ("beta8", C.c_int), ("beta10", C.c_int),
                ("beta11a", C.c_int), ("beta11b", C.c_int), ("beta13", C.c_int),
                ("beta15", C.c_int), ("beta16a", C.c_int), ("beta16b", C.c_int),
                ("tol", C.c_double), ("max_refine", C.c_int), ("inner", C.c_int),
                ("trsv_chunk", C.c_int), ("trsv_cluster", C.c_int), ("s", C.c_int),
                ("order", C.c_int), ("shift_tune", C.c_int), ("mgs_wmax", C.c_int),
                ("wait_us", C.c_int), ("test_stall", C.c_int), ("fuse_steps", C.c_int),
                ("plan_snap", C.c_int), ("reserved", C.c_int * 2)]

    def replace(self, **kw) -> "Params":
        p = Params()
        C.memmove(C.byref(p), C.byref(self), C.sizeof(Params))
        for k, v in kw.items():
            setattr(p, k, v)
        return p


class Report(C.Structure):
    _fields_ = [("ev", C.c_longlong * 16), ("refinements", C.c_int),
                ("inner_steps", C.c_int), ("breakdowns", C.c_int), ("status", C.c_int),
                ("relres", C.c_double), ("relres_unscaled", C.c_double),
                ("gamma_hist", C.c_double * 64), ("relres_hist", C.c_double * 65),
                ("shift_retries", C.c_int), ("beta_final", C.c_int * 5),
                ("fuse_steps", C.c_int), ("plan_snap", C.c_int)]

    def as_dict(self) -> dict:
        k = self.refinements
        return dict(status=STATUS.get(self.status, self.status), refinements=k,
                    inner_steps=self.inner_steps, breakdowns=self.breakdowns,
                    relres=self.relres, relres_unscaled=self.relres_unscaled,
                    ev=np.array(self.ev[:], dtype=np.int64),
                    gamma_hist=np.array(self.gamma_hist[:min(k, 64)]),
                    relres_hist=np.array(self.relres_hist[:min(k + 1, 65)]),
                    shift_retries=self.shift_retries, beta_final=tuple(self.beta_final[:]),
                    fuse_steps=self.fuse_steps, plan_snap=self.plan_snap)


class ServerConfig(C.Structure):
    _fields_ = [("budget_bytes", C.c_longlong), ("max_active", C.c_int), ("m", C.c_int),
                ("inner", C.c_int), ("reserved", C.c_int * 5)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_longlong), ("completed", C.c_longlong),
                ("failed", C.c_longlong), ("rounds", C.c_longlong),
                ("peak_bytes", C.c_longlong), ("busy_s", C.c_double)]


_VP = C.c_void_p
_I = C.c_int


def _declare(lib):
    sig = {
        "igm_params_default": (_I, [C.POINTER(Params), _I, _I]),
        "int_gmres_setup": (_I, [_I, _I, _VP, _VP, _VP, C.POINTER(Params), _VP,
                                 C.POINTER(_VP)]),
        "int_gmres_solve": (_I, [_VP, _VP, _VP, C.POINTER(Report), _VP]),
        "ir_solve": (_I, [_VP, _VP, _VP, C.POINTER(Report), _VP]),
        "ir_solve_batched": (_I, [_I, C.POINTER(_VP), C.POINTER(_VP), C.POINTER(_VP),
                                  C.POINTER(Report), _VP]),
        "int_gmres_get_state": (_I, [_VP, _VP, _VP, _VP, _VP, _VP, C.POINTER(_I),
                                     C.POINTER(C.c_double)]),
        "int_gmres_device_bytes": (C.c_longlong, [_VP]),
        "igm_time_kernels": (_I, [_VP, _I, C.POINTER(C.c_double), _VP]),
        "igm_kernel_launches": (C.c_longlong, []),
        "igm_norm2": (_I, [_VP, _I, _VP, _VP]),
        "igm_norm2_noalloc": (_I, [_VP, _I, _VP, _VP]),
        "int_gmres_destroy": (None, [_VP]),
        "igm_server_create": (_I, [C.POINTER(ServerConfig), C.POINTER(_VP)]),
        "igm_server_submit": (_I, [_VP, _I, _I, _VP, _VP, _VP, _VP, C.POINTER(Params),
                                   C.POINTER(C.c_longlong)]),
        "igm_server_poll": (_I, [_VP, C.c_longlong, _I, _VP, C.POINTER(Report),
                                 C.POINTER(C.c_double), C.POINTER(_I)]),
        "igm_server_get_stats": (_I, [_VP, C.POINTER(ServerStats)]),
        "igm_server_destroy": (None, [_VP]),
        "igm_last_error": (C.c_char_p, []),
        "igm_version": (C.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libigm.so.  Raises if it is missing (no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if build_if_missing:
                path = _build.build()
            if not os.path.exists(path):
                raise ImportError(f"libigm.so not built ({path}); run __graft_entry__.build()")
            lib = C.CDLL(path)
            _declare(lib)
            _lib = lib
    return _lib


def _check(st: int):
    if st != 0:
        raise IGMError(st, load().igm_last_error().decode())


def params_default(precond: int = 0, m: int = 30, **kw) -> Params:
    """The paper's settings (Table 4 without, Table 5 with ILU(0)),
    overridden by keyword arguments."""
    p = Params()
    _check(load().igm_params_default(C.byref(p), int(precond), int(m)))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


class _Buf:
    """A pointer to caller memory: torch tensor (any device) or numpy array.
    Keeps the object alive for the duration of the call."""

    def __init__(self, a, dtype, n=None, writable=False):
        try:
            import torch
        except ImportError:  # pragma: no cover
            torch = None
        if torch is not None and isinstance(a, torch.Tensor):
            tdt = {np.int32: torch.int32, np.float64: torch.float64, np.int64: torch.int64}[dtype]
            if a.dtype != tdt or not a.is_contiguous():
                if writable:
                    raise TypeError(f"output tensor must be contiguous {tdt}")
                a = a.to(tdt).contiguous()
            self.obj = a
            self.ptr = a.data_ptr()
            self.cuda = a.is_cuda
            self.len = a.numel()
        else:
            arr = np.asarray(a)
            if arr.dtype != dtype or not arr.flags.c_contiguous:
                if writable:
                    raise TypeError(f"output array must be contiguous {np.dtype(dtype)}")
                arr = np.ascontiguousarray(arr, dtype=dtype)
            self.obj = arr
            self.ptr = arr.ctypes.data
            self.cuda = False
            self.len = arr.size
        if n is not None and self.len < n:
            raise ValueError(f"array too short: {self.len} < {n}")


def _stream_ptr(stream, *bufs) -> int:
    if stream is not None:
        return int(getattr(stream, "cuda_stream", stream))
    if any(b.cuda for b in bufs):
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    return 0


class Solver:
    """One system Ahat xhat = bhat set up on the GPU (int_gmres_setup)."""

    def __init__(self, rowptr, col, val, params: Params | None = None, stream=None):
        self._h = _VP()
        lib = load()
        rp = _Buf(rowptr, np.int32)
        n = rp.len - 1
        cl = _Buf(col, np.int32)
        vl = _Buf(val, np.float64)
        self.params = params if params is not None else params_default(0, 30)
        self.n, self.nnz = n, cl.len
        sp = _stream_ptr(stream, rp, cl, vl)
        _check(lib.int_gmres_setup(n, cl.len, rp.ptr, cl.ptr, vl.ptr, C.byref(self.params),
                                   sp, C.byref(self._h)))

    @property
    def handle(self):
        return self._h

    def ir_solve(self, bhat, xhat=None, stream=None) -> tuple:
        """Fig. 1 on the original system; returns (xhat, report dict)."""
        b = _Buf(bhat, np.float64, self.n)
        if xhat is None:
            if b.cuda:
                import torch
                xhat = torch.empty(self.n, dtype=torch.float64, device=b.obj.device)
            else:
                xhat = np.empty(self.n)
        x = _Buf(xhat, np.float64, self.n, writable=True)
        rep = Report()
        st = load().ir_solve(self._h, b.ptr, x.ptr, C.byref(rep), _stream_ptr(stream, b, x))
        if st not in (0, 5):
            _check(st)
        return xhat, rep.as_dict()

    def inner_solve(self, bk, xk, stream=None) -> dict:
        """One int-GMRES(m) solve (Fig. 2) of the scaled system; xk is updated."""
        b = _Buf(bk, np.float64, self.n)
        x = _Buf(xk, np.float64, self.n, writable=True)
        rep = Report()
        _check(load().int_gmres_solve(self._h, b.ptr, x.ptr, C.byref(rep),
                                      _stream_ptr(stream, b, x)))
        return rep.as_dict()

    def state(self) -> dict:
        """Integer state of the last inner solve (host numpy arrays)."""
        m, n = self.params.m, self.n
        V = np.zeros((m + 1, n), np.int64)
        H = np.zeros((m, m + 1), np.int64)
        cs = np.zeros(m, np.int64)
        sn = np.zeros(m, np.int64)
        g = np.zeros(m + 1, np.int64)
        jeff = C.c_int(0)
        nu = C.c_double(0)
        _check(load().int_gmres_get_state(self._h, V.ctypes.data, H.ctypes.data,
                                          cs.ctypes.data, sn.ctypes.data, g.ctypes.data,
                                          C.byref(jeff), C.byref(nu)))
        return dict(V=V, H=H.T.copy(), cs=cs, sn=sn, g=g, jeff=jeff.value, nu=nu.value)

    def device_bytes(self) -> int:
        return int(load().int_gmres_device_bytes(self._h))

    def close(self):
        if self._h:
            load().int_gmres_destroy(self._h)
            self._h = _VP()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ir_solve_batched(solvers, bhats, xhats, stream=None) -> list[dict]:
    """Fig. 1 for many independent systems in one launch sequence."""
    k = len(solvers)
    bs = [_Buf(b, np.float64, s.n) for b, s in zip(bhats, solvers)]
    xs = [_Buf(x, np.float64, s.n, writable=True) for x, s in zip(xhats, solvers)]
    hs = (_VP * k)(*[s.handle.value for s in solvers])
    bp = (_VP * k)(*[b.ptr for b in bs])
    xp = (_VP * k)(*[x.ptr for x in xs])
    reps = (Report * k)()
    st = load().ir_solve_batched(k, hs, bp, xp, reps, _stream_ptr(stream, *bs, *xs))
    if st not in (0, 5):
        _check(st)
    return [r.as_dict() for r in reps]


class Server:
    """Continuous-batching solve server (igm_server_*): submit host systems,
    poll for results."""

    def __init__(self, budget_bytes: int, m: int, inner: int = 0, max_active: int = 0):
        self._s = _VP()
        cfg = ServerConfig(int(budget_bytes), int(max_active), int(m), int(inner))
        _check(load().igm_server_create(C.byref(cfg), C.byref(self._s)))
        self.m, self.inner = m, inner
        self._n = {}

    def submit(self, rowptr, col, val, bhat, params: Params) -> int:
        rp, cl = _Buf(rowptr, np.int32), _Buf(col, np.int32)
        vl, b = _Buf(val, np.float64), _Buf(bhat, np.float64)
        if rp.cuda or b.cuda:
            raise TypeError("the server takes host arrays")
        rid = C.c_longlong(0)
        _check(load().igm_server_submit(self._s, rp.len - 1, cl.len, rp.ptr, cl.ptr, vl.ptr,
                                        b.ptr, C.byref(params), C.byref(rid)))
        self._n[rid.value] = rp.len - 1
        return rid.value

    def poll(self, rid: int, wait_ms: int = -1):
        """(done, x, report dict, latency_s); x/report are None while pending."""
        n = self._n[rid]
        x = np.empty(n)
        rep = Report()
        lat = C.c_double(0)
        done = C.c_int(0)
        st = load().igm_server_poll(self._s, rid, int(wait_ms), x.ctypes.data, C.byref(rep),
                                    C.byref(lat), C.byref(done))
        if not done.value:
            return False, None, None, None
        del self._n[rid]
        if st not in (0, 5):
            _check(st)
        return True, x, rep.as_dict(), lat.value

    def stats(self) -> dict:
        st = ServerStats()
        _check(load().igm_server_get_stats(self._s, C.byref(st)))
        return {k: getattr(st, k) for k, _ in ServerStats._fields_}

    def close(self):
        if self._s:
            load().igm_server_destroy(self._s)
            self._s = _VP()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def norm2(x, stream=None) -> float:
    """The reproducible 2-norm of Fig. 1's test (igm_norm2)."""
    b = _Buf(x, np.float64)
    out = C.c_double(0)
    _check(load().igm_norm2(b.ptr if b.len else None, b.len, C.addressof(out),
                            _stream_ptr(stream, b)))
    return out.value


def version() -> str:
    return load().igm_version().decode()
