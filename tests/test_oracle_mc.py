"""Pins of the multicolour order (a GPU-motivated reordering, order = 1):
a proper colouring, the closed forms for stencils in natural order
(red-black for 5/7-point grids), the permuted system equal to P A P^T,
colours as independent sets (every strict-lower dependency in an earlier
colour, so a substitution has as many levels as colours), and the
refinement loop on the permuted system solving the original one."""
import numpy as np
import scipy.sparse as sp

from paper_2009_07495_gb300 import workloads as W


def _colors(perm, cptr):
    col = np.empty(len(perm), dtype=np.int64)
    for c in range(len(cptr) - 1):
        col[perm[cptr[c]:cptr[c + 1]]] = c
    return col


def test_proper_colouring_and_order(orc):
    s = W.banded_random(400, np.random.default_rng(7))
    perm, cptr = orc.mc_order(s.rowptr, s.col)
    assert sorted(perm.tolist()) == list(range(s.n))
    color = _colors(perm, cptr)
    for i in range(s.n):
        for k in range(s.rowptr[i], s.rowptr[i + 1]):
            j = s.col[k]
            if j != i:
                assert color[i] != color[j]
    for c in range(len(cptr) - 1):                # ascending within a colour
        blk = perm[cptr[c]:cptr[c + 1]]
        assert np.all(np.diff(blk) > 0)
    # greedy: each row's colour is the smallest not used by an earlier neighbour
    A = sp.csr_matrix((np.ones(len(s.col)), s.col, s.rowptr), shape=(s.n, s.n))
    S = (A + A.T).tocsr()
    for i in range(s.n):
        used = {int(color[j]) for j in S.indices[S.indptr[i]:S.indptr[i + 1]] if j < i}
        assert color[i] == min(c for c in range(len(used) + 1) if c not in used)


def test_red_black_for_5_and_7_point_grids(orc):
    for s, shape in ((W.small_cd2d(9), (9, 9)), (W.small_cd3d(7), (7, 7, 7))):
        perm, cptr = orc.mc_order(s.rowptr, s.col)
        assert len(cptr) - 1 == 2
        color = _colors(perm, cptr)
        idx = np.indices(shape[::-1]).reshape(len(shape), -1)   # natural order: x fastest
        np.testing.assert_array_equal(color, idx.sum(0) % 2)


def test_27_point_grid_colours(orc):
    s = W.small_cd3d(6, points=27)
    perm, cptr = orc.mc_order(s.rowptr, s.col)
    assert len(cptr) - 1 == 8
    color = _colors(perm, cptr)
    z, y, x = np.indices((6, 6, 6)).reshape(3, -1)
    np.testing.assert_array_equal(color, (x % 2) + 2 * (y % 2) + 4 * (z % 2))


def test_permuted_system_and_independent_colours(orc):
    s = W.small_cd3d(5, seed=15, points=27)
    perm, cptr = orc.mc_order(s.rowptr, s.col)
    rp2, cl2, av2 = orc.permute_csr(s.rowptr, s.col, s.val, perm)
    A = sp.csr_matrix((s.val, s.col, s.rowptr), shape=(s.n, s.n)).toarray()
    A2 = sp.csr_matrix((av2, cl2, rp2), shape=(s.n, s.n)).toarray()
    np.testing.assert_array_equal(A2, A[np.ix_(perm, perm)])
    assert all(np.all(np.diff(cl2[rp2[r]:rp2[r + 1]]) > 0) for r in range(s.n))
    newcol = np.repeat(np.arange(len(cptr) - 1), np.diff(cptr))
    for r in range(s.n):
        for k in range(rp2[r], rp2[r + 1]):
            if cl2[k] < r:
                assert newcol[cl2[k]] < newcol[r]


def test_refinement_in_multicolour_order_solves_the_original_system(orc):
    for s, prec in ((W.small_cd3d(8, seed=16), 1), (W.small_cd3d(7, seed=17, points=27), 1),
                    (W.config0(), 2)):
        P = orc.Params.table5(m=30, precond=prec, order=1)
        x, rep = orc.ir_solve(s.rowptr, s.col, s.val, s.b, P)
        assert rep.status == "ok" and rep.relres < 1e-10
        A = sp.csr_matrix((s.val, s.col, s.rowptr), shape=(s.n, s.n))
        assert np.linalg.norm(A @ x - s.b) / np.linalg.norm(s.b) < 1e-9
