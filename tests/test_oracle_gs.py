"""Pins of the integer Gauss-Seidel preconditioner (precond = 2): the
factor form of D + L_A, the substitutions of lines 1'/5' applying
(D + L_A)^-1 up to the truncation of the integer factors, and the
refinement loop with zero operand shifts (Sec. VII-D: like ILU(0), no
overflow without shifts)."""
import numpy as np
import scipy.sparse as sp
from scipy.sparse.linalg import spsolve_triangular

from paper_2009_07495_gb300 import workloads as W


def _csr(s, a):
    return sp.csr_matrix((a, s.col, s.rowptr), shape=(s.n, s.n))


def test_gs_factor_form(orc):
    """Below the diagonal f_ij a_jj = a_ij to one rounding; the pivots are
    a_ii; nothing above the diagonal."""
    s = W.small_cd3d(6, seed=12)
    a, b, d = orc.scale(s.rowptr, s.col, s.val, s.b, 32)
    f, dp = orc.gs_factors(s.rowptr, s.col, a)
    for i in range(s.n):
        for k in range(s.rowptr[i], s.rowptr[i + 1]):
            j = s.col[k]
            if j < i:
                assert abs(f[k] * a[dp[j]] - a[k]) <= 2 * np.spacing(abs(a[k]))
            elif j == i:
                assert f[k] == a[k]
            else:
                assert f[k] == 0.0


def test_gs_substitution_applies_D_plus_L_inverse(orc):
    """Line 1' with the integer Gauss-Seidel factors solves (D + L_A) y = z
    up to the truncation of the factors (relative error far below 1e-3)."""
    s = W.small_cd3d(7, seed=13)
    a, b, d = orc.scale(s.rowptr, s.col, s.val, s.b, 32)
    f, dp = orc.gs_factors(s.rowptr, s.col, a)
    fac, ld, ud = orc.ilu_int(s.rowptr, s.col, f, dp)
    z = np.random.default_rng(2).standard_normal(s.n)
    t = orc.lsolve_fp(s.rowptr, s.col, fac, ld, z)
    y = orc.usolve_fp(s.rowptr, s.col, fac, ud, t)
    M = sp.tril(_csr(s, a)).tocsr()
    y_ref = spsolve_triangular(M, z, lower=True)
    assert np.linalg.norm(y - y_ref) / np.linalg.norm(y_ref) < 1e-3


def test_gs_refinement_converges_without_overflow(orc):
    """Fig. 1 with the Gauss-Seidel preconditioner and the zero shifts of
    Table 5 converges to 1e-10 with no overflow event."""
    for s in (W.config0(), W.small_cd3d(8, seed=14)):
        P = orc.Params.table5(m=30, precond=2)
        x, rep = orc.ir_solve(s.rowptr, s.col, s.val, s.b, P)
        assert rep.status == "ok" and rep.relres < 1e-10
        assert int(np.abs(rep.ev).sum()) == 0, rep.ev
        A = _csr(s, s.val)
        assert np.linalg.norm(A @ x - s.b) / np.linalg.norm(s.b) < 1e-9
