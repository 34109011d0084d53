"""ctypes marshalling for the C oracle (test infrastructure only).

Every function here is argument marshalling; the arithmetic is in
``igm_oracle.c``.  Section, equation and figure numbers refer to Iwashita,
Suzuki, Fukaya, "An Integer Arithmetic-Based Sparse Linear Solver Using a
GMRES Method and Iterative Refinement" (ScalA'20).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "igm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libigm_oracle.so")
_lock = threading.Lock()
_lib = None

EV_NAMES = ["L5", "L5p", "L7", "L8", "L10", "L11", "L13", "L15", "L16", "L17",
            "vrange", "L2", "r12", "r13", "r14", "r15"]

STATUS = {0: "ok", 1: "einval", 2: "ezero_row", 3: "ezero_pivot",
          4: "ebreakdown", 5: "enoconv", 6: "enomem"}


def build(force: bool = False) -> str:
    """Compile igm_oracle.c into oracle/_build/libigm_oracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(C.Structure):
    _fields_ = [("df", C.c_int), ("alpha_a", C.c_int), ("m", C.c_int),
                ("precond", C.c_int),
                ("beta7", C.c_int), ("beta8", C.c_int), ("beta10", C.c_int),
                ("beta11a", C.c_int), ("beta11b", C.c_int), ("beta13", C.c_int),
                ("beta15", C.c_int), ("beta16a", C.c_int), ("beta16b", C.c_int),
                ("tol", C.c_double), ("max_refine", C.c_int), ("s", C.c_int),
                ("order", C.c_int), ("shift_tune", C.c_int)]


class _Report(C.Structure):
    _fields_ = [("ev", C.c_longlong * 16), ("refinements", C.c_int),
                ("inner_steps", C.c_int), ("breakdowns", C.c_int),
                ("status", C.c_int), ("relres", C.c_double),
                ("relres_unscaled", C.c_double),
                ("gamma_hist", C.c_double * 64), ("relres_hist", C.c_double * 65),
                ("shift_retries", C.c_int), ("beta_final", C.c_int * 5)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            assert lib.or_sizeof_params() == C.sizeof(_Params)
            assert lib.or_sizeof_report() == C.sizeof(_Report)
            _lib = lib
    return _lib


@dataclass
class Params:
    """Parameters of the method (Sec. VII): d_f, alpha_a, m, the
    preconditioner and the operand shifts of Table 4 / Table 5."""
    df: int = 30
    alpha_a: int = 16
    m: int = 30
    precond: int = 0
    beta7: int = 16
    beta8: int = 16
    beta10: int = 16
    beta11a: int = 16
    beta11b: int = 14
    beta13: int = 16
    beta15: int = 16
    beta16a: int = 16
    beta16b: int = 14
    tol: float = 1e-10
    max_refine: int = 60
    s: int = 0               # correction terms of eq. (AA), s(k) = s
    order: int = 0           # 0 natural, 1 multicolour (mc_order)
    shift_tune: int = 0      # cycles the shift auto-tuning may discard (Sec. VII-D)

    @staticmethod
    def table4(m: int = 30, **kw) -> "Params":
        """No preconditioning: alpha_a = 16 and the shifts of Table 4."""
        return Params(m=m, **kw)

    @staticmethod
    def table5(m: int = 30, **kw) -> "Params":
        """ILU(0): alpha_a = 32 and the shifts of Table 5."""
        d = dict(alpha_a=32, m=m, precond=1, beta7=0, beta8=0, beta10=0,
                 beta11a=30, beta11b=0, beta13=0, beta15=0, beta16a=30,
                 beta16b=0)
        d.update(kw)
        return Params(**d)

    def _c(self) -> _Params:
        return _Params(self.df, self.alpha_a, self.m, self.precond, self.beta7,
                       self.beta8, self.beta10, self.beta11a, self.beta11b,
                       self.beta13, self.beta15, self.beta16a, self.beta16b,
                       float(self.tol), self.max_refine, self.s, self.order,
                       self.shift_tune)


@dataclass
class Report:
    status: str
    refinements: int
    inner_steps: int
    breakdowns: int
    relres: float
    relres_unscaled: float
    ev: np.ndarray = field(repr=False)
    gamma_hist: np.ndarray = field(repr=False)
    relres_hist: np.ndarray = field(repr=False)
    shift_retries: int = 0
    beta_final: tuple = ()   # beta7, beta8, beta10, beta13, beta15 at the end


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


_I64 = C.c_longlong
_F64 = C.c_double
_I32 = C.c_int


def _sig(name, res, args):
    f = getattr(_load(), name)
    f.restype = res
    f.argtypes = args
    return f


def shr(x: int, s: int) -> int:
    f = _sig("or_shr", _I64, [_I64, _I32])
    return int(f(x, s))


def isqrt(s: int) -> int:
    """Babylonian integer square root of Sec. V-B."""
    f = _sig("or_isqrt", _I64, [_I64])
    return int(f(s))


def fx_mul(t1: int, t2: int, b1: int, b2: int, df: int = 30):
    """eq. (c1c2).  Returns (value, overflow events)."""
    f = _sig("or_fx_mul", _I64, [_I64, _I64, _I32, _I32, _I32, C.POINTER(_I64)])
    ev = _I64(0)
    r = f(t1, t2, b1, b2, df, C.byref(ev))
    return int(r), int(ev.value)


def fx_div(t1: int, t2: int, b1: int, b2: int, df: int = 30):
    """Fixed-point division of Sec. V-B.  Returns (value, events, zero)."""
    f = _sig("or_fx_div", _I64, [_I64, _I64, _I32, _I32, _I32, C.POINTER(_I64),
                                  C.POINTER(_I32)])
    ev, z = _I64(0), _I32(0)
    r = f(t1, t2, b1, b2, df, C.byref(ev), C.byref(z))
    return int(r), int(ev.value), bool(z.value)


def fx_sqrt(t: int, dfp: int, df: int = 30):
    f = _sig("or_fx_sqrt", _I64, [_I64, _I32, _I32, C.POINTER(_I64)])
    ev = _I64(0)
    r = f(t, dfp, df, C.byref(ev))
    return int(r), int(ev.value)


def norm2(x) -> float:
    """Reproducible FP64 2-norm."""
    x = _f64(x)
    f = _sig("or_norm2", _F64, [_I32, C.POINTER(_F64)])
    return float(f(len(x), _p(x, _F64)))


def scale(rowptr, col, ahat, bhat, alpha_a: int):
    """eq. (1), eq. (3).  Returns (a, b, d) or raises on a zero row."""
    rowptr, col, ahat, bhat = _i32(rowptr), _i32(col), _f64(ahat), _f64(bhat)
    n = len(rowptr) - 1
    a = np.empty_like(ahat)
    b = np.empty(n)
    d = np.empty(n)
    f = _sig("or_scale", _I32, [_I32, C.POINTER(_I32), C.POINTER(_I32),
                                C.POINTER(_F64), C.POINTER(_F64), _I32,
                                C.POINTER(_F64), C.POINTER(_F64), C.POINTER(_F64)])
    st = f(n, _p(rowptr, _I32), _p(col, _I32), _p(ahat, _F64), _p(bhat, _F64),
           alpha_a, _p(a, _F64), _p(b, _F64), _p(d, _F64))
    if st:
        raise ValueError(STATUS[st])
    return a, b, d


def cast(a):
    """Sec. IV-B: Abar_0 = cast(A)."""
    a = _f64(a)
    out = np.empty(len(a), dtype=np.int64)
    f = _sig("or_cast", _I32, [_I32, C.POINTER(_F64), C.POINTER(_I64)])
    st = f(len(a), _p(a, _F64), _p(out, _I64))
    if st:
        raise ValueError(STATUS[st])
    return out


def ilu0(rowptr, col, a):
    """eq. (ilu): FP64 ILU(0).  Returns (f, diagpos)."""
    rowptr, col, a = _i32(rowptr), _i32(col), _f64(a)
    n = len(rowptr) - 1
    fv = np.empty_like(a)
    dp = np.empty(n, dtype=np.int32)
    f = _sig("or_ilu0", _I32, [_I32, C.POINTER(_I32), C.POINTER(_I32),
                               C.POINTER(_F64), C.POINTER(_F64), C.POINTER(_I32)])
    st = f(n, _p(rowptr, _I32), _p(col, _I32), _p(a, _F64), _p(fv, _F64),
           _p(dp, _I32))
    if st:
        raise ValueError(STATUS[st])
    return fv, dp


def mc_order(rowptr, col):
    """Greedy multicolour order.  Returns (perm with perm[new] = old,
    cptr: colour c occupies new indices cptr[c] .. cptr[c+1]-1)."""
    rowptr, col = _i32(rowptr), _i32(col)
    n = len(rowptr) - 1
    perm = np.empty(n, dtype=np.int32)
    cptr = np.empty(n + 1, dtype=np.int32)
    f = _sig("or_mc_order", _I32, [_I32, C.POINTER(_I32), C.POINTER(_I32), C.POINTER(_I32),
                                   C.POINTER(_I32)])
    nc = f(n, _p(rowptr, _I32), _p(col, _I32), _p(perm, _I32), _p(cptr, _I32))
    return perm, cptr[: nc + 1].copy()


def permute_csr(rowptr, col, val, perm):
    """P A P^T for perm[new] = old (columns sorted ascending)."""
    rowptr, col, val, perm = _i32(rowptr), _i32(col), _f64(val), _i32(perm)
    n = len(rowptr) - 1
    rp2 = np.empty(n + 1, dtype=np.int32)
    cl2 = np.empty(max(len(col), 1), dtype=np.int32)
    av2 = np.empty(max(len(col), 1))
    f = _sig("or_permute_csr", None, [_I32, C.POINTER(_I32), C.POINTER(_I32), C.POINTER(_F64),
                                      C.POINTER(_I32), C.POINTER(_I32), C.POINTER(_I32),
                                      C.POINTER(_F64)])
    f(n, _p(rowptr, _I32), _p(col, _I32), _p(val, _F64), _p(perm, _I32), _p(rp2, _I32),
      _p(cl2, _I32), _p(av2, _F64))
    return rp2, cl2[: len(col)].copy(), av2[: len(col)].copy()


def gs_factors(rowptr, col, a):
    """The Gauss-Seidel preconditioner D + L_A in the ILU factor form
    (unit lower a_ij / a_jj, pivots a_ii, no upper part).  Returns
    (f, diagpos)."""
    rowptr, col, a = _i32(rowptr), _i32(col), _f64(a)
    n = len(rowptr) - 1
    f = np.empty_like(a)
    dp = np.empty(n, dtype=np.int32)
    fn = _sig("or_gs_factors", _I32, [_I32, C.POINTER(_I32), C.POINTER(_I32), C.POINTER(_F64),
                                      C.POINTER(_F64), C.POINTER(_I32)])
    st = fn(n, _p(rowptr, _I32), _p(col, _I32), _p(a, _F64), _p(f, _F64), _p(dp, _I32))
    if st:
        raise ValueError(f"gs_factors: status {st}")
    return f, dp


def ilu_int(rowptr, col, fv, diagpos):
    """eq. (dldr)-(ilu2): integer factors.  Returns (fac, ldiag, udiag)."""
    rowptr, col, fv, diagpos = _i32(rowptr), _i32(col), _f64(fv), _i32(diagpos)
    n = len(rowptr) - 1
    fac = np.empty(len(fv), dtype=np.int64)
    ld = np.empty(n, dtype=np.int64)
    ud = np.empty(n, dtype=np.int64)
    f = _sig("or_ilu_int", _I32, [_I32, C.POINTER(_I32), C.POINTER(_I32),
                                  C.POINTER(_F64), C.POINTER(_I32), C.POINTER(_I64),
                                  C.POINTER(_I64), C.POINTER(_I64)])
    st = f(n, _p(rowptr, _I32), _p(col, _I32), _p(fv, _F64), _p(diagpos, _I32),
           _p(fac, _I64), _p(ld, _I64), _p(ud, _I64))
    if st:
        raise ValueError(STATUS[st])
    return fac, ld, ud


def spmv_int(rowptr, col, abar, v):
    """Line 5 of Fig. 2.  Returns (w, events)."""
    rowptr, col, abar, v = _i32(rowptr), _i32(col), _i64(abar), _i64(v)
    n = len(rowptr) - 1
    w = np.empty(n, dtype=np.int64)
    ev = _I64(0)
    f = _sig("or_spmv_int", None, [_I32, C.POINTER(_I32), C.POINTER(_I32),
                                   C.POINTER(_I64), C.POINTER(_I64), C.POINTER(_I64),
                                   C.POINTER(_I64)])
    f(n, _p(rowptr, _I32), _p(col, _I32), _p(abar, _I64), _p(v, _I64),
      _p(w, _I64), C.byref(ev))
    return w, int(ev.value)


def multiterm(a, alpha_a: int, S: int):
    """Eq. (alpha1), (A): Abar_0 ... Abar_s (s <= S, fewer when a remainder
    is zero) and their exponents.  Returns (terms (s+1) x nnz, alphas)."""
    a = _f64(a)
    nnz = len(a)
    terms = np.zeros((S + 1, max(nnz, 1)), dtype=np.int64)
    alphas = np.zeros(S + 1, dtype=np.int32)
    f = _sig("or_multiterm", _I32, [_I32, C.POINTER(_F64), _I32, _I32, C.POINTER(_I64),
                                    C.POINTER(_I32)])
    ns = f(nnz, _p(a, _F64), alpha_a, S, _p(terms, _I64), _p(alphas, _I32))
    return terms[: ns + 1, :nnz].copy(), alphas[: ns + 1].copy()


def spmv_int_s(rowptr, col, terms, alphas, v):
    """Line 5 with eq. (matvec): w = sum_l (Abar_l v) / 2^alpha_l.
    Returns (w, events)."""
    rowptr, col, v = _i32(rowptr), _i32(col), _i64(v)
    terms = np.ascontiguousarray(terms, dtype=np.int64)
    alphas = _i32(alphas)
    n = len(rowptr) - 1
    w = np.empty(n, dtype=np.int64)
    ev = _I64(0)
    f = _sig("or_spmv_int_s", None, [_I32, C.POINTER(_I32), C.POINTER(_I32), _I32,
                                     C.POINTER(_I64), C.POINTER(_I32), C.POINTER(_I64),
                                     C.POINTER(_I64), C.POINTER(_I64)])
    f(n, _p(rowptr, _I32), _p(col, _I32), len(alphas) - 1, _p(terms, _I64), _p(alphas, _I32),
      _p(v, _I64), _p(w, _I64), C.byref(ev))
    return w, int(ev.value)


def _solve_int(name, rowptr, col, fac, diag, z):
    rowptr, col, fac, diag, z = _i32(rowptr), _i32(col), _i64(fac), _i64(diag), _i64(z)
    n = len(rowptr) - 1
    y = np.empty(n, dtype=np.int64)
    ev = _I64(0)
    f = _sig(name, None, [_I32, C.POINTER(_I32), C.POINTER(_I32), C.POINTER(_I64),
                          C.POINTER(_I64), C.POINTER(_I64), C.POINTER(_I64),
                          C.POINTER(_I64)])
    f(n, _p(rowptr, _I32), _p(col, _I32), _p(fac, _I64), _p(diag, _I64),
      _p(z, _I64), _p(y, _I64), C.byref(ev))
    return y, int(ev.value)


def lsolve_int(rowptr, col, fac, ldiag, z):
    """Line 5', forward substitution with Lbar (Sec. VI-A)."""
    return _solve_int("or_lsolve_int", rowptr, col, fac, ldiag, z)


def usolve_int(rowptr, col, fac, udiag, y):
    """Line 5', backward substitution with Ubar (Sec. VI-A)."""
    return _solve_int("or_usolve_int", rowptr, col, fac, udiag, y)


def _solve_fp(name, rowptr, col, fac, diag, z):
    rowptr, col, fac, diag, z = _i32(rowptr), _i32(col), _i64(fac), _i64(diag), _f64(z)
    n = len(rowptr) - 1
    y = np.empty(n)
    f = _sig(name, None, [_I32, C.POINTER(_I32), C.POINTER(_I32), C.POINTER(_I64),
                          C.POINTER(_I64), C.POINTER(_F64), C.POINTER(_F64)])
    f(n, _p(rowptr, _I32), _p(col, _I32), _p(fac, _I64), _p(diag, _I64),
      _p(z, _F64), _p(y, _F64))
    return y


def lsolve_fp(rowptr, col, fac, ldiag, z):
    """Line 1', forward substitution in FP64 on the integer factor."""
    return _solve_fp("or_lsolve_fp", rowptr, col, fac, ldiag, z)


def usolve_fp(rowptr, col, fac, udiag, y):
    """Line 1', backward substitution in FP64 on the integer factor."""
    return _solve_fp("or_usolve_fp", rowptr, col, fac, udiag, y)


def resid_fp(rowptr, col, a, x, b):
    """eq. (b): r = b - A x in FP64, CSR order."""
    rowptr, col, a, x, b = _i32(rowptr), _i32(col), _f64(a), _f64(x), _f64(b)
    n = len(rowptr) - 1
    r = np.empty(n)
    f = _sig("or_resid_fp", None, [_I32, C.POINTER(_I32), C.POINTER(_I32),
                                   C.POINTER(_F64), C.POINTER(_F64), C.POINTER(_F64),
                                   C.POINTER(_F64)])
    f(n, _p(rowptr, _I32), _p(col, _I32), _p(a, _F64), _p(x, _F64), _p(b, _F64),
      _p(r, _F64))
    return r


def setup(rowptr, col, ahat, bhat, params: Params):
    """Setup of Fig. 1: scaling, cast and (precond=1) integer ILU(0).
    Returns a dict with the scaled system and its integer data."""
    perm = None
    if params.order == 1:
        perm, _ = mc_order(rowptr, col)
        rowptr, col, ahat = permute_csr(rowptr, col, ahat, perm)
        bhat = _f64(bhat)[perm]
    a, b, d = scale(rowptr, col, ahat, bhat, params.alpha_a)
    out = dict(rowptr=_i32(rowptr), col=_i32(col), a=a, b=b, d=d, abar=cast(a), perm=perm)
    if params.s > 0:
        terms, alphas = multiterm(a, params.alpha_a, params.s)
        out.update(terms=terms, alphas=alphas)
    n = len(rowptr) - 1
    if params.precond:
        fv, dp = gs_factors(rowptr, col, a) if params.precond == 2 else ilu0(rowptr, col, a)
        fac, ld, ud = ilu_int(rowptr, col, fv, dp)
        out.update(f=fv, diagpos=dp, fac=fac, ldiag=ld, udiag=ud)
    else:
        out.update(fac=np.zeros(max(len(col), 1), np.int64),
                   ldiag=np.ones(n, np.int64), udiag=np.ones(n, np.int64))
    return out


def int_gmres(params: Params, sysd: dict, bk, xk=None):
    """One int-GMRES(m) solve of Fig. 2 (lines 1', 5' when precond=1).
    Returns a dict: x, V, H, Hraw, cs, sn, g, jeff, nu, ev, early."""
    m = params.m
    rowptr, col = sysd["rowptr"], sysd["col"]
    n = len(rowptr) - 1
    bk = _f64(bk)
    x = np.zeros(n) if xk is None else _f64(xk).copy()
    V = np.zeros((m + 1, n), dtype=np.int64)
    H = np.zeros((m, m + 1), dtype=np.int64)     # column-major (m+1) x m
    Hraw = np.zeros((m, m + 1), dtype=np.int64)
    cs = np.zeros(m, dtype=np.int64)
    sn = np.zeros(m, dtype=np.int64)
    g = np.zeros(m + 1, dtype=np.int64)
    ev = np.zeros(16, dtype=np.int64)
    jeff = _I32(0)
    nu = _F64(0)
    pc = params._c()
    abar, fac = _i64(sysd["abar"]), _i64(sysd["fac"])
    ld, ud = _i64(sysd["ldiag"]), _i64(sysd["udiag"])
    tail = [C.POINTER(_I64)] * 3 + [C.POINTER(_F64)] * 2 + [C.POINTER(_I64)] * 6 \
        + [C.POINTER(_I32), C.POINTER(_F64), C.POINTER(_I64)]
    outs = (_p(bk, _F64), _p(x, _F64), _p(V, _I64), _p(H, _I64), _p(Hraw, _I64),
            _p(cs, _I64), _p(sn, _I64), _p(g, _I64), C.byref(jeff), C.byref(nu), _p(ev, _I64))
    if "terms" in sysd and len(sysd["alphas"]) > 1:
        terms = np.ascontiguousarray(sysd["terms"], dtype=np.int64)
        alphas = _i32(sysd["alphas"])
        f = _sig("or_int_gmres_flat_s", _I32,
                 [C.POINTER(_Params), _I32, C.POINTER(_I32), C.POINTER(_I32), _I32,
                  C.POINTER(_I64), C.POINTER(_I32)] + tail)
        early = f(C.byref(pc), n, _p(rowptr, _I32), _p(col, _I32), len(alphas) - 1,
                  _p(terms, _I64), _p(alphas, _I32), _p(fac, _I64), _p(ld, _I64),
                  _p(ud, _I64), *outs)
    else:
        f = _sig("or_int_gmres_flat", _I32,
                 [C.POINTER(_Params), _I32, C.POINTER(_I32), C.POINTER(_I32),
                  C.POINTER(_I64)] + tail)
        early = f(C.byref(pc), n, _p(rowptr, _I32), _p(col, _I32), _p(abar, _I64),
                  _p(fac, _I64), _p(ld, _I64), _p(ud, _I64), *outs)
    return dict(x=x, V=V, H=H.T.copy(), Hraw=Hraw.T.copy(), cs=cs, sn=sn, g=g,
                jeff=int(jeff.value), nu=float(nu.value), ev=ev, early=bool(early))


def ir_solve(rowptr, col, ahat, bhat, params: Params, inner: int = 0):
    """Fig. 1.  inner=0: int-GMRES; inner=1: FP64 GMRES(m) ("Double").
    Returns (x, Report)."""
    rowptr, col, ahat, bhat = _i32(rowptr), _i32(col), _f64(ahat), _f64(bhat)
    n = len(rowptr) - 1
    x = np.zeros(n)
    rep = _Report()
    pc = params._c()
    f = _sig("or_ir_solve", _I32, [C.POINTER(_Params), _I32, _I32, C.POINTER(_I32),
                                   C.POINTER(_I32), C.POINTER(_F64), C.POINTER(_F64),
                                   C.POINTER(_F64), C.POINTER(_Report)])
    st = f(C.byref(pc), inner, n, _p(rowptr, _I32), _p(col, _I32), _p(ahat, _F64),
           _p(bhat, _F64), _p(x, _F64), C.byref(rep))
    r = Report(status=STATUS[st], refinements=rep.refinements,
               inner_steps=rep.inner_steps, breakdowns=rep.breakdowns,
               relres=rep.relres, relres_unscaled=rep.relres_unscaled,
               ev=np.array(rep.ev[:], dtype=np.int64),
               gamma_hist=np.array(rep.gamma_hist[:rep.refinements]),
               relres_hist=np.array(rep.relres_hist[:min(rep.refinements + 1, 65)]),
               shift_retries=rep.shift_retries, beta_final=tuple(rep.beta_final[:]))
    return x, r


def fp_gmres(sysd: dict, params: Params, bk, xk=None):
    """One FP64 GMRES(m) cycle (the comparison solver).  Returns (x, jeff)."""
    rowptr, col, a = sysd["rowptr"], sysd["col"], _f64(sysd["a"])
    n = len(rowptr) - 1
    fv = _f64(sysd.get("f", np.zeros(1)))
    dp = _i32(sysd.get("diagpos", np.zeros(1, np.int32)))
    x = np.zeros(n) if xk is None else _f64(xk).copy()
    bk = _f64(bk)
    jeff = _I32(0)
    f = _sig("or_fp_gmres", _I32, [_I32, C.POINTER(_I32), C.POINTER(_I32),
                                   C.POINTER(_F64), C.POINTER(_F64), C.POINTER(_I32),
                                   _I32, _I32, C.POINTER(_F64), C.POINTER(_F64),
                                   C.POINTER(_I32)])
    f(n, _p(rowptr, _I32), _p(col, _I32), _p(a, _F64), _p(fv, _F64), _p(dp, _I32),
      params.m, params.precond, _p(bk, _F64), _p(x, _F64), C.byref(jeff))
    return x, int(jeff.value)


__all__ = ["build", "Params", "Report", "EV_NAMES", "shr", "isqrt", "fx_mul",
           "fx_div", "fx_sqrt", "norm2", "scale", "cast", "ilu0", "ilu_int",
           "spmv_int", "multiterm", "spmv_int_s", "gs_factors", "mc_order", "permute_csr", "lsolve_int", "usolve_int",
           "lsolve_fp", "usolve_fp",
           "resid_fp", "setup", "int_gmres", "ir_solve", "fp_gmres"]
