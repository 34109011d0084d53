"""Pins for the oracle's setup (eq. 1, 3; Sec. IV-B; eq. ilu..ilu2) and its
integer kernels (line 5, line 5', line 1'), each checked against a library
routine or an exact property, never against the oracle itself."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from paper_2009_07495_gb300 import workloads as W


def _csr(s):
    return sp.csr_matrix((s.val, s.col, s.rowptr), shape=(s.n, s.n))


def test_scaling_eq3(orc):
    """eq. (3): d_i = max_j |ahat_ij| / 2^alpha_a, A = D^-1 Ahat: every row's
    largest |a_ij| is exactly 2^alpha_a, and a_ij is the IEEE quotient."""
    s = W.small_cd2d(12, seed=3)
    for alpha in (16, 32):
        a, b, d = orc.scale(s.rowptr, s.col, s.val, s.b, alpha)
        rows = np.repeat(np.arange(s.n), np.diff(s.rowptr))
        mx = np.maximum.reduceat(np.abs(a), s.rowptr[:-1])
        assert np.all(mx == 2.0 ** alpha)
        np.testing.assert_array_equal(a, s.val / d[rows])
        np.testing.assert_array_equal(b, s.b / d)
        np.testing.assert_array_equal(d, np.maximum.reduceat(np.abs(s.val), s.rowptr[:-1]) / 2.0 ** alpha)


def test_zero_row_rejected(orc):
    s = W.small_cd2d(4)
    val = s.val.copy()
    val[s.rowptr[3]:s.rowptr[4]] = 0.0
    with pytest.raises(ValueError, match="ezero_row"):
        orc.scale(s.rowptr, s.col, val, s.b, 16)


def test_cast_truncates(orc):
    """Sec. IV-B: Abar_0 = cast(A), truncation toward zero (C cast)."""
    rng = np.random.default_rng(1)
    a = rng.standard_normal(1000) * 2.0 ** 20
    a[:4] = [2.5, -2.5, 0.999, -0.999]
    np.testing.assert_array_equal(orc.cast(a), np.trunc(a).astype(np.int64))


def test_ilu0_tridiagonal_is_exact_lu(orc):
    """On a tridiagonal matrix ILU(0) has no dropped fill, so L D U' = A
    exactly as the textbook LU (scipy.linalg.lu without pivoting agrees)."""
    rng = np.random.default_rng(2)
    n = 40
    A = np.diag(rng.uniform(4, 5, n)) + np.diag(rng.uniform(-1, 1, n - 1), 1) \
        + np.diag(rng.uniform(-1, 1, n - 1), -1)
    s = W.from_dense(A, np.ones(n))
    f, dp = orc.ilu0(s.rowptr, s.col, s.val)
    F = W.System(n, s.rowptr, s.col, f, s.b).dense()
    L = np.tril(F, -1) + np.eye(n)
    U = np.triu(F)
    np.testing.assert_allclose(L @ U, A, rtol=1e-14, atol=1e-14)
    # Doolittle LU without pivoting, written out (unique factorisation)
    Lr, Ur = np.eye(n), A.copy()
    for k in range(n):
        for i in range(k + 1, n):
            Lr[i, k] = Ur[i, k] / Ur[k, k]
            Ur[i, :] -= Lr[i, k] * Ur[k, :]
    np.testing.assert_allclose(L, Lr, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(U, Ur, rtol=1e-13, atol=1e-13)


def test_ilu0_matches_pattern(orc):
    """ILU(0)'s defining property: (L U)_ij = a_ij on the pattern of A
    (Saad, Iterative Methods, Prop. 10.4), for a 2D and a 3D stencil."""
    for s in (W.small_cd2d(9, seed=4), W.small_cd3d(5)):
        a, b, d = orc.scale(s.rowptr, s.col, s.val, s.b, 32)
        f, dp = orc.ilu0(s.rowptr, s.col, a)
        F = W.System(s.n, s.rowptr, s.col, f, b).dense()
        L = np.tril(F, -1) + np.eye(s.n)
        U = np.triu(F)
        LU = L @ U
        Ad = W.System(s.n, s.rowptr, s.col, a, b).dense()
        mask = W.System(s.n, s.rowptr, s.col, np.ones_like(a), b).dense() != 0
        np.testing.assert_allclose(LU[mask], Ad[mask], rtol=1e-12, atol=1e-12 * 2.0 ** 32)


def test_integer_ilu_factors(orc):
    """eq. (dl)-(u1): Ltilde = L D_l, Utilde = D_u U' with
    D_l = |d|^(1/2), D_u = sgn(d)|d|^(1/2); Lbar, Ubar are the truncations:
    |Lbar - Ltilde| < 1 elementwise, and Ltilde Utilde = L D U'."""
    s = W.small_cd3d(5)
    a, b, d = orc.scale(s.rowptr, s.col, s.val, s.b, 32)
    f, dp = orc.ilu0(s.rowptr, s.col, a)
    fac, ld, ud = orc.ilu_int(s.rowptr, s.col, f, dp)
    F = W.System(s.n, s.rowptr, s.col, f, b).dense()
    L = np.tril(F, -1) + np.eye(s.n)
    D = np.diag(F)
    Up = np.triu(F, 1) / D[:, None] + np.eye(s.n)
    Dl = np.sqrt(np.abs(D))
    Du = np.sign(D) * Dl
    Lt, Ut = L * Dl[None, :], Du[:, None] * Up
    Fi = W.System(s.n, s.rowptr, s.col, fac.astype(float), b).dense()
    Lb = np.tril(Fi, -1) + np.diag(ld.astype(float))
    Ub = np.triu(Fi, 1) + np.diag(ud.astype(float))
    mask = W.System(s.n, s.rowptr, s.col, np.ones_like(a), b).dense() != 0
    assert np.all(np.abs(Lb - Lt)[mask | np.eye(s.n, dtype=bool)] < 1.0)
    assert np.all(np.abs(Ub - Ut)[mask | np.eye(s.n, dtype=bool)] < 1.0)
    sl = mask & np.tri(s.n, k=-1, dtype=bool)
    su = mask & np.tri(s.n, k=-1, dtype=bool).T
    np.testing.assert_array_equal(Lb[sl], np.trunc(Lt)[sl])
    np.testing.assert_array_equal(Ub[su], np.trunc(Ut)[su])
    np.testing.assert_array_equal(np.diag(Lb), np.trunc(Dl))
    np.testing.assert_array_equal(np.diag(Ub), np.trunc(Du))
    np.testing.assert_allclose(Lt @ Ut, L @ np.diag(D) @ Up, rtol=1e-12, atol=1e-6)


def test_spmv_int_exact(orc):
    """Line 5 with s = 0 is the exact integer product Abar v (Sec. V-C):
    equal to scipy's int64 sparse product when nothing overflows."""
    s = W.small_cd3d(6)
    a, b, d = orc.scale(s.rowptr, s.col, s.val, s.b, 32)
    abar = orc.cast(a)
    rng = np.random.default_rng(5)
    v = rng.integers(-(1 << 30), 1 << 30, s.n)
    w, ev = orc.spmv_int(s.rowptr, s.col, abar, v)
    M = sp.csr_matrix((abar, s.col, s.rowptr), shape=(s.n, s.n), dtype=np.int64)
    np.testing.assert_array_equal(w, M @ v)
    assert ev == 0


def test_spmv_int_overflow_counts(orc):
    """A product or a row total beyond int64 is counted once and the stored
    value is the exact total modulo 2^64."""
    rowptr = np.array([0, 2, 4], np.int32)
    col = np.array([0, 1, 0, 1], np.int32)
    abar = np.array([1 << 33, 1 << 33, 1 << 40, 1], np.int64)
    v = np.array([1 << 29, 1 << 29], np.int64)
    w, ev = orc.spmv_int(rowptr, col, abar, v)
    # row 0: 2^62 + 2^62 = 2^63 -> total overflow (1 event); wraps to -2^63
    # row 1: 2^69 product overflow (wraps to 0) + 2^29 -> 1 event
    assert ev == 2
    assert w[0] == -(1 << 63)
    assert w[1] == 1 << 29


def _int_tri_system(orc, seed=6):
    s = W.small_cd3d(5, seed=seed)
    a, b, d = orc.scale(s.rowptr, s.col, s.val, s.b, 32)
    f, dp = orc.ilu0(s.rowptr, s.col, a)
    fac, ld, ud = orc.ilu_int(s.rowptr, s.col, f, dp)
    return s, fac, ld, ud


def test_integer_substitution_recovers_exact_solution(orc):
    """Line 5' (Sec. VI-A): with z = Lbar y* for an integer y*, every division
    in the forward substitution is exact, so it must return y* itself; the
    same for the backward substitution with Ubar."""
    s, fac, ld, ud = _int_tri_system(orc)
    rng = np.random.default_rng(7)
    ys = [int(v) for v in rng.integers(-(1 << 28), 1 << 28, s.n)]
    # z = Lbar y* with Python integers (exact)
    z = []
    for i in range(s.n):
        acc = ld[i] * ys[i]
        for k in range(s.rowptr[i], s.rowptr[i + 1]):
            j = s.col[k]
            if j < i:
                acc += int(fac[k]) * ys[j]
        z.append(int(acc))
    y, ev = orc.lsolve_int(s.rowptr, s.col, fac, ld, np.array(z, np.int64))
    assert ev == 0
    np.testing.assert_array_equal(y, np.array(ys))
    z = []
    for i in range(s.n):
        acc = int(ud[i]) * ys[i]
        for k in range(s.rowptr[i], s.rowptr[i + 1]):
            j = s.col[k]
            if j > i:
                acc += int(fac[k]) * ys[j]
        z.append(int(acc))
    w, ev = orc.usolve_int(s.rowptr, s.col, fac, ud, np.array(z, np.int64))
    np.testing.assert_array_equal(w, np.array(ys))


def test_integer_substitution_truncation(orc):
    """For a general right-hand side each y_i is the quotient of its exact
    numerator by Lbar_ii truncated toward zero: |num - y_i Lbar_ii| < |Lbar_ii|
    with the remainder of the numerator's sign; and the integer solution
    tracks the FP64 one (scipy spsolve_triangular) to the truncation error."""
    s, fac, ld, ud = _int_tri_system(orc, 8)
    rng = np.random.default_rng(9)
    z = rng.integers(-(1 << 40), 1 << 40, s.n)
    y, ev = orc.lsolve_int(s.rowptr, s.col, fac, ld, z)
    for i in range(s.n):
        num = int(z[i])
        for k in range(s.rowptr[i], s.rowptr[i + 1]):
            if s.col[k] < i:
                num -= int(fac[k]) * int(y[s.col[k]])
        rem = num - int(y[i]) * int(ld[i])
        assert abs(rem) < abs(int(ld[i]))
        assert rem == 0 or (rem > 0) == (num > 0)
    Lm = sp.csr_matrix((np.where(s.col < np.repeat(np.arange(s.n), np.diff(s.rowptr)), fac, 0).astype(float),
                        s.col, s.rowptr), shape=(s.n, s.n)) + sp.diags(ld.astype(float))
    yf = spla.spsolve_triangular(Lm.tocsr(), z.astype(float), lower=True)
    np.testing.assert_allclose(y, yf, rtol=1e-6, atol=8.0)


def test_fp_substitution_line1p(orc):
    """Line 1': FP64 substitutions on the integer factors match scipy's
    triangular solves to rounding."""
    s, fac, ld, ud = _int_tri_system(orc, 10)
    rows = np.repeat(np.arange(s.n), np.diff(s.rowptr))
    Lm = (sp.csr_matrix((np.where(s.col < rows, fac, 0).astype(float), s.col, s.rowptr),
                        shape=(s.n, s.n)) + sp.diags(ld.astype(float))).tocsr()
    Um = (sp.csr_matrix((np.where(s.col > rows, fac, 0).astype(float), s.col, s.rowptr),
                        shape=(s.n, s.n)) + sp.diags(ud.astype(float))).tocsr()
    rng = np.random.default_rng(11)
    z = rng.uniform(-1, 1, s.n)
    y = orc.lsolve_fp(s.rowptr, s.col, fac, ld, z)
    np.testing.assert_allclose(y, spla.spsolve_triangular(Lm, z, lower=True), rtol=1e-12, atol=1e-300)
    w = orc.usolve_fp(s.rowptr, s.col, fac, ud, y)
    np.testing.assert_allclose(w, spla.spsolve_triangular(Um, y, lower=False), rtol=1e-11, atol=1e-300)


def test_resid_fp(orc):
    """eq. (b): r = b - A x agrees with scipy's product to rounding."""
    s = W.small_cd2d(10, seed=12)
    rng = np.random.default_rng(13)
    x = rng.standard_normal(s.n)
    r = orc.resid_fp(s.rowptr, s.col, s.val, x, s.b)
    np.testing.assert_allclose(r, s.b - _csr(s) @ x, rtol=1e-12, atol=1e-9)
