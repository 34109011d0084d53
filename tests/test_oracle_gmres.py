"""Pins for the oracle's int-GMRES(m) solve (Fig. 2, Sec. V-D, VI) and its
iterative refinement (Fig. 1, Sec. IV), checked against closed forms worked
out from the paper's formulas, mathematical properties of GMRES (Arnoldi
relation, orthonormal basis, minimal residual over the Krylov space, Givens
QR, residual estimate) computed with numpy, and numpy.linalg.solve."""
import numpy as np
import pytest

from paper_2009_07495_gb300 import workloads as W

Q = 2.0 ** 30


def _sysd(orc, s, P):
    return orc.setup(s.rowptr, s.col, s.val, s.b, P)


def _int_dense(d, n):
    return W.System(n, d["rowptr"], d["col"], d["abar"].astype(float), d["b"]).dense()


def _prec_dense(d, n):
    """M = Lbar Ubar as an FP64 dense matrix."""
    rows = np.repeat(np.arange(n), np.diff(d["rowptr"]))
    F = W.System(n, d["rowptr"], d["col"], d["fac"].astype(float), d["b"]).dense()
    L = np.tril(F, -1) + np.diag(d["ldiag"].astype(float))
    U = np.triu(F, 1) + np.diag(d["udiag"].astype(float))
    del rows
    return L @ U


def test_one_by_one_closed_form(orc):
    """Ahat = [2], bhat = [4] with alpha_a = 16 and Table 4 shifts, worked by
    hand from eq. (3), eq. (c1c2), Sec. V-B and Fig. 2:
    d = 2^-15, A = 2^16, b = 2^17, gamma = 2^17, b^(1) = 1, v1 = 2^30,
    w = 2^46, h11 = (2^30 * 2^30) >> 14 = 2^46, w - h v = 0 (breakdown),
    t = isqrt(2^60) 2^16 = 2^46, c = (2^46 2^16) / (2^46 >> 14) = 2^30, s = 0,
    g1 = 2^30, y = 2^-16, x = 2^17 * 2^-16 = 2 after one refinement."""
    P = orc.Params.table4(m=5)
    rowptr, col = np.array([0, 1], np.int32), np.array([0], np.int32)
    d = orc.setup(rowptr, col, np.array([2.0]), np.array([4.0]), P)
    assert d["abar"][0] == 1 << 16 and d["b"][0] == 2.0 ** 17
    r = orc.int_gmres(P, d, np.array([1.0]))
    assert r["V"][0, 0] == 1 << 30
    assert r["Hraw"][0, 0] == 1 << 46 and r["Hraw"][1, 0] == 0
    assert r["H"][0, 0] == 1 << 46
    assert r["cs"][0] == 1 << 30 and r["sn"][0] == 0
    assert r["g"][0] == 1 << 30 and r["g"][1] == 0
    assert r["jeff"] == 1 and r["early"]
    assert r["x"][0] == 2.0 ** -16
    x, rep = orc.ir_solve(rowptr, col, np.array([2.0]), np.array([4.0]), P)
    assert x[0] == 2.0 and rep.refinements == 1 and rep.status == "ok"
    assert rep.gamma_hist[0] == 2.0 ** 17


def test_degree_two_minimal_polynomial(orc):
    """A = blockdiag([[1, 1/2], [0, 1]]) is unchanged by the row scaling of
    eq. (3) (up to 2^alpha_a) and has minimal polynomial (z - 1)^2, so GMRES
    is exact after 2 steps: the Givens residual estimate |g_3| drops to the
    fixed-point noise floor and x = A^-1 b to the Table 4 precision."""
    n = 16
    A = np.eye(n)
    for i in range(0, n, 2):
        A[i, i + 1] = 0.5
    s = W.from_dense(A, np.linspace(1.0, 2.0, n))
    P = orc.Params.table4(m=4)
    d = _sysd(orc, s, P)
    bk = d["b"] / np.abs(d["b"]).max()
    r = orc.int_gmres(P, d, bk)
    Ai = _int_dense(d, n)
    assert abs(r["g"][2]) < 1 << 8 and abs(r["g"][1]) > 1 << 20
    xe = np.linalg.solve(Ai, bk)
    np.testing.assert_allclose(r["x"], xe, rtol=1e-7, atol=0)


def _krylov_minres(B, r0, j):
    """argmin over x in K_j(B, r0) of ||r0 - B x||, via an orthonormal basis
    from numpy QR (independent of Arnoldi/Givens)."""
    K = np.empty((len(r0), j))
    v = r0 / np.linalg.norm(r0)
    for i in range(j):
        K[:, i] = v
        v = B @ v
        v = v / np.linalg.norm(v)
    Qk, _ = np.linalg.qr(K)
    c, *_ = np.linalg.lstsq(B @ Qk, r0, rcond=None)
    return Qk @ c


CASES = [
    ("none", lambda o: o.Params.table4(m=6), lambda: W.small_cd2d(8, seed=21)),
    ("ilu", lambda o: o.Params.table5(m=6), lambda: W.small_cd3d(4, seed=22)),
]


@pytest.mark.parametrize("name,pf,sf", CASES, ids=[c[0] for c in CASES])
def test_arnoldi_properties(orc, name, pf, sf):
    """Lines 5-11: the integer basis satisfies the Arnoldi relation
    B v_j = sum_i h_ij v_i (B = Abar, or Mbar^-1 Abar with line 5'), is
    orthonormal, and lines 12-19 are a QR of the Hessenberg matrix by
    Givens rotations (c^2 + s^2 = 1, Q^T Hraw = R)."""
    orc_ = orc
    P = pf(orc_)
    s = sf()
    d = _sysd(orc_, s, P)
    n = s.n
    A = _int_dense(d, n)
    B = np.linalg.solve(_prec_dense(d, n), A) if P.precond else A
    bk = d["b"] / np.abs(d["b"]).max()
    r = orc_.int_gmres(P, d, bk)
    j = r["jeff"]
    assert j == P.m and not r["early"]
    V = r["V"].astype(float) / Q
    Hr = r["Hraw"].astype(float) / Q
    for c in range(j):
        lhs = B @ V[c]
        rhs = V[: c + 2].T @ Hr[: c + 2, c]
        assert np.linalg.norm(lhs - rhs) <= 1e-6 * np.linalg.norm(lhs)
    # MGS loses orthogonality like eps / (relative residual) (Greenbaum,
    # Rozloznik, Strakos 1997): check |v_a . v_b| for b <= a against
    # 1e-6 / (|g_a| / 2^30), with eps ~ 2^-30 of the fixed-point words.
    G = V[: j + 1] @ V[: j + 1].T
    res = np.abs(r["g"][: j + 1].astype(float)) / Q
    res = np.maximum.accumulate(res[::-1])[::-1]
    for a in range(j + 1):
        for b in range(a + 1):
            tol = 1e-7 / max(res[a], 1e-12)
            assert abs(G[a, b] - (a == b)) <= max(tol, 1e-7)
    cs, sn = r["cs"][:j] / Q, r["sn"][:j] / Q
    assert np.abs(cs ** 2 + sn ** 2 - 1).max() < 1e-6
    R = Hr[: j + 1, :j].copy()
    for i in range(j):
        G2 = np.array([[cs[i], sn[i]], [-sn[i], cs[i]]])
        R[i: i + 2, :] = G2 @ R[i: i + 2, :]
    Hf = r["H"].astype(float) / Q
    np.testing.assert_allclose(np.triu(R[:j, :j]), Hf[:j, :j], rtol=0, atol=1e-6 * np.abs(Hf).max())
    assert np.abs(R[j, :]).max() < 1e-6 * np.abs(Hf).max()


@pytest.mark.parametrize("name,pf,sf", CASES, ids=[c[0] for c in CASES])
def test_minimal_residual_and_estimate(orc, name, pf, sf):
    """One int-GMRES(m) solve from x = 0 returns (up to fixed-point error) the
    minimiser of ||r0 - B x|| over the Krylov space K_m(B, r0), and
    ||r0|| |g_{m+1}| / 2^30 estimates the true residual of that x."""
    P = pf(orc)
    s = sf()
    d = _sysd(orc, s, P)
    n = s.n
    A = _int_dense(d, n)
    bk = d["b"] / np.abs(d["b"]).max()
    if P.precond:
        M = _prec_dense(d, n)
        B, r0 = np.linalg.solve(M, A), np.linalg.solve(M, bk)
    else:
        B, r0 = A, bk
    r = orc.int_gmres(P, d, bk)
    xs = _krylov_minres(B, r0, P.m)
    assert np.linalg.norm(r["x"] - xs) <= 1e-5 * np.linalg.norm(xs)
    true_res = np.linalg.norm(r0 - B @ r["x"])
    est = r["nu"] * abs(r["g"][r["jeff"]]) / Q
    assert abs(true_res - est) <= 1e-6 * r["nu"]
    assert abs(r["nu"] - np.linalg.norm(r0)) <= 1e-13 * r["nu"]


def test_fp_gmres_is_textbook_gmres(orc):
    """The FP64 comparison solver returns the Krylov minimal-residual iterate."""
    s = W.small_cd2d(8, seed=23)
    P = orc.Params.table5(m=7)
    d = _sysd(orc, s, P)
    Ad = W.System(s.n, d["rowptr"], d["col"], d["a"], d["b"]).dense()
    F = W.System(s.n, d["rowptr"], d["col"], d["f"], d["b"]).dense()
    M = (np.tril(F, -1) + np.eye(s.n)) @ np.triu(F)
    bk = d["b"] / np.abs(d["b"]).max()
    x, j = orc.fp_gmres(d, P, bk)
    B, r0 = np.linalg.solve(M, Ad), np.linalg.solve(M, bk)
    xs = _krylov_minres(B, r0, 7)
    assert j == 7
    np.testing.assert_allclose(x, xs, rtol=1e-9, atol=1e-12 * np.abs(xs).max())


@pytest.mark.parametrize("seed", [31, 32, 33])
def test_ir_solves_tiny_dense(orc, seed):
    """Fig. 1 drives the relative residual below 1e-10 and the answer agrees
    with numpy.linalg.solve (tiny diagonally dominant nonsymmetric systems)."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(5, 40))
    A = rng.standard_normal((n, n)) * (rng.random((n, n)) < 0.4)
    np.fill_diagonal(A, np.abs(A).sum(1) * rng.uniform(1.1, 2.0, n) + 0.5)
    b = rng.standard_normal(n)
    s = W.from_dense(A, b)
    xe = np.linalg.solve(A, b)
    for P in (orc.Params.table4(m=10), orc.Params.table5(m=10)):
        x, rep = orc.ir_solve(s.rowptr, s.col, s.val, s.b, P)
        assert rep.status == "ok" and rep.relres < 1e-10
        assert np.linalg.norm(x - xe) <= 1e-8 * np.linalg.norm(xe)
        assert np.all(rep.ev == 0)


def test_config0_converges_like_fp64(orc):
    """Config 0 (2D 5-point, n = 1024, GMRES(30), no preconditioning): int
    refinement reaches 1e-10 and needs at most one refinement more than
    FP64 GMRES(30) (Sec. VII-B's observation); gamma^(k) decreases
    (Sec. IV-A); no overflow event with the paper's shifts."""
    s = W.config0()
    P = orc.Params.table4(m=30)
    xi, ri = orc.ir_solve(s.rowptr, s.col, s.val, s.b, P, inner=0)
    xf, rf = orc.ir_solve(s.rowptr, s.col, s.val, s.b, P, inner=1)
    assert ri.status == "ok" and ri.relres < 1e-10 and rf.relres < 1e-10
    assert ri.refinements <= rf.refinements + 1
    assert np.all(np.diff(ri.gamma_hist) < 0)
    assert np.all(ri.ev == 0)
    assert np.abs(xi - 1.0).max() < 1e-8


def test_ilu_no_overflow_and_converges(orc):
    """Sec. VII-C: with ILU(0) the shifts can be 0 (Table 5) without
    overflow, and the refinement converges in few cycles."""
    s = W.small_cd3d(10, seed=24)
    P = orc.Params.table5(m=30)
    x, rep = orc.ir_solve(s.rowptr, s.col, s.val, s.b, P, inner=0)
    _, rf = orc.ir_solve(s.rowptr, s.col, s.val, s.b, P, inner=1)
    assert rep.status == "ok" and rep.relres < 1e-10
    assert np.all(rep.ev == 0)
    assert rep.refinements <= rf.refinements + 1


def test_overflow_is_counted(orc):
    """Without operand shifts and with alpha_a = 40 the inner products exceed
    int64: the events are counted per line and the solve still returns."""
    s = W.small_cd2d(6, seed=25)
    P = orc.Params.table5(m=5, precond=0, alpha_a=40, max_refine=2)
    x, rep = orc.ir_solve(s.rowptr, s.col, s.val, s.b, P)
    assert rep.ev[2] > 0 or rep.ev[4] > 0       # lines 7 / 10
    assert rep.status in ("ok", "enoconv")


def test_refinement_stops_when_the_residual_stalls(orc):
    """With a tolerance below what FP64 reaches, the residual of Fig. 1
    falls to rounding level and then stays there; the loop stops
    (ENOCONV) the first time it has not decreased over three refinements,
    instead of running to max_refine."""
    s = W.config0()
    P = orc.Params.table4(m=30, tol=1e-18, max_refine=40)
    x, rep = orc.ir_solve(s.rowptr, s.col, s.val, s.b, P)
    h = rep.relres_hist
    k = rep.refinements
    assert rep.status == "enoconv" and k < 40
    assert h[k] >= h[k - 3]
    assert all(h[q] < h[q - 3] for q in range(3, k))
    assert h[k] < 1e-14
