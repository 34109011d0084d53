"""Pins of the multi-term fixed-point matrix (Sec. IV-C, eq. alpha1, A, AA)
and its SpMV (eq. matvec), against what the definitions fix: the exact
value of A, the exponent order, the word range of every term, the
remainder bound, the floor-division error bound of the product, the s = 0
special case, and the effect on convergence."""
from fractions import Fraction

import numpy as np

from paper_2009_07495_gb300 import workloads as W


def _scaled(orc, sysw, alpha_a):
    a, b, d = orc.scale(sysw.rowptr, sysw.col, sysw.val, sysw.b, alpha_a)
    return a


def test_terms_reconstruct_A_exactly(orc):
    """With enough terms the remainder is zero and sum_l Abar_l 2^-alpha_l
    equals every element of A exactly (eq. A)."""
    s = W.small_cd2d(12, seed=3)
    a = _scaled(orc, s, 16)
    terms, alphas = orc.multiterm(a, 16, 8)
    assert len(alphas) >= 3                      # the fractions need > 1 term
    for k in range(len(a)):
        v = sum(Fraction(int(terms[l, k]), 2 ** int(alphas[l])) for l in range(len(alphas)))
        assert v == Fraction(float(a[k]))


def test_exponents_increase_and_terms_fill_the_word(orc):
    """alpha_1 < alpha_2 < ...; alpha_l = alpha_a - floor(log2 max|A_l|)
    puts the largest |Abar_l| in [2^alpha_a, 2^(alpha_a+1)); term 0 is the
    cast of A (truncation toward zero)."""
    s = W.small_cd3d(6, seed=8)
    for alpha_a in (16, 32):
        a = _scaled(orc, s, alpha_a)
        terms, alphas = orc.multiterm(a, alpha_a, 4)
        np.testing.assert_array_equal(terms[0], np.trunc(a).astype(np.int64))
        assert all(alphas[l] < alphas[l + 1] for l in range(1, len(alphas) - 1))
        assert alphas[1] > alpha_a
        for l in range(1, len(alphas)):
            mx = int(np.abs(terms[l]).max())
            assert 2 ** alpha_a <= mx < 2 ** (alpha_a + 1)


def test_remainder_after_s_terms_is_below_the_last_grid(orc):
    """A - sum_{l<=s} Abar_l 2^-alpha_l is the truncation remainder: the
    same sign as A and smaller than 2^-alpha_s in magnitude."""
    s = W.small_cd2d(10, seed=5)
    a = _scaled(orc, s, 16)
    for S in (1, 2, 3):
        terms, alphas = orc.multiterm(a, 16, S)
        for k in range(len(a)):
            approx = sum(Fraction(int(terms[l, k]), 2 ** int(alphas[l]))
                         for l in range(len(alphas)))
            rem = Fraction(float(a[k])) - approx
            assert abs(rem) < Fraction(1, 2 ** int(alphas[-1]))
            assert rem == 0 or (rem > 0) == (a[k] > 0)


def test_spmv_within_the_floor_error_of_the_exact_product(orc):
    """Each of the s terms is divided by 2^alpha_l with a floor, so w_i lies
    in (exact - s, exact] where exact = sum_l (Abar_l v)_i / 2^alpha_l
    (no overflow at these sizes)."""
    rng = np.random.default_rng(9)
    s = W.small_cd2d(9, seed=6)
    a = _scaled(orc, s, 16)
    terms, alphas = orc.multiterm(a, 16, 3)
    v = rng.integers(-2 ** 30, 2 ** 30, s.n, dtype=np.int64)
    w, ev = orc.spmv_int_s(s.rowptr, s.col, terms, alphas, v)
    assert ev == 0
    ns = len(alphas) - 1
    for i in range(s.n):
        ks = range(s.rowptr[i], s.rowptr[i + 1])
        exact = sum(Fraction(sum(int(terms[l, k]) * int(v[s.col[k]]) for k in ks),
                             2 ** int(alphas[l])) for l in range(ns + 1))
        assert exact - ns < int(w[i]) <= exact


def test_spmv_with_no_correction_terms_is_line_5(orc):
    s = W.small_cd2d(8, seed=7)
    a = _scaled(orc, s, 16)
    terms, alphas = orc.multiterm(a, 16, 0)
    v = np.random.default_rng(1).integers(-2 ** 30, 2 ** 30, s.n, dtype=np.int64)
    w0, e0 = orc.spmv_int(s.rowptr, s.col, orc.cast(a), v)
    w1, e1 = orc.spmv_int_s(s.rowptr, s.col, terms, alphas, v)
    np.testing.assert_array_equal(w0, w1)
    assert e0 == e1


def test_more_terms_fewer_refinements_on_a_coarse_matrix(orc):
    """With a coarse word (alpha_a = 6) Abar_0 is a poor copy of A and the
    refinement loop needs many inner solves; the correction terms of eq. (AA)
    bring A^(k) close to A and the count drops, every run converging."""
    s = W.small_cd2d(16, seed=4)
    counts = []
    for S in (0, 2):
        P = orc.Params.table4(m=30, alpha_a=6, beta7=6, beta8=6, beta10=6, beta11a=6,
                              beta11b=4, beta13=6, beta15=6, beta16a=6, beta16b=4, s=S)
        x, rep = orc.ir_solve(s.rowptr, s.col, s.val, s.b, P)
        assert rep.status == "ok", (S, rep.status, rep.relres)
        counts.append(rep.refinements)
    assert counts[1] < counts[0], counts
