"""Pins of the shift auto-tuning (Sec. VII-D; params.shift_tune): after an
inner solve that overflowed at line 7, 8, 10, 13 or 15 of Fig. 2, the shift
of each such line is raised by one (up to d_f) and the inner solve is
discarded and run again from the same b^(k).

What fixes it independently of the oracle's own arithmetic:
  - a solve that raises no event is the untuned solve (the rule never fires);
  - discarded inner solves leave no trace: where every retry falls in the
    first refinement, the tuned solve equals, bit for bit, the untuned solve
    run with the final shifts from the start;
  - with shifts too small for the system, the untuned solve stalls while the
    tuned solve reaches the tolerance, and its solution satisfies the
    original system (residual computed here, in numpy);
  - the shifts only grow, stay at or below d_f, and the retry budget bounds
    the retries."""
import numpy as np
import pytest

from paper_2009_07495_gb300 import workloads as W

TUNED = ("beta7", "beta8", "beta10", "beta13", "beta15")


def _small(orc, b, tune, **kw):
    d = {k: b for k in TUNED}
    d.update(kw)
    return orc.Params.table4(m=30, shift_tune=tune, **d)


def _true_relres(s, x):
    r = s.b - s.matvec(x)
    return np.linalg.norm(r) / np.linalg.norm(s.b)


def test_no_events_no_retries(orc):
    """Table 4's shifts raise no event on this system: with tuning on the
    solve is the untuned solve, bit for bit."""
    s = W.config0()
    x0, r0 = orc.ir_solve(s.rowptr, s.col, s.val, s.b, orc.Params.table4(m=30))
    x1, r1 = orc.ir_solve(s.rowptr, s.col, s.val, s.b, orc.Params.table4(m=30, shift_tune=40))
    assert r0.ev.sum() == 0 and r1.shift_retries == 0
    assert r1.beta_final == (16, 16, 16, 16, 16)
    np.testing.assert_array_equal(x0, x1)
    np.testing.assert_array_equal(r0.relres_hist, r1.relres_hist)


def test_ilu_without_shifts_needs_no_tuning(orc):
    """Sec. VII-D: with ILU(0) the shifts can stay at zero (Table 5); the
    tuning finds nothing to raise."""
    s = W.small_cd3d(9, seed=31)
    P0 = orc.Params.table5(m=20)
    P1 = orc.Params.table5(m=20, shift_tune=10)
    x0, r0 = orc.ir_solve(s.rowptr, s.col, s.val, s.b, P0)
    x1, r1 = orc.ir_solve(s.rowptr, s.col, s.val, s.b, P1)
    assert r0.status == "ok" and r1.shift_retries == 0 and r1.beta_final == (0, 0, 0, 0, 0)
    np.testing.assert_array_equal(x0, x1)


@pytest.mark.parametrize("b", [12, 8, 0])
def test_small_shifts_stall_untuned_and_converge_tuned(orc, b):
    """Shifts below what the system needs: the words of lines 7-15 wrap, the
    untuned loop stalls (ENOCONV) far from the solution; the tuned loop
    reaches 1e-10 and x solves Ahat x = bhat."""
    s = W.config0()
    xu, ru = orc.ir_solve(s.rowptr, s.col, s.val, s.b, _small(orc, b, 0))
    xt, rt = orc.ir_solve(s.rowptr, s.col, s.val, s.b, _small(orc, b, 40))
    assert ru.status == "enoconv" and _true_relres(s, xu) > 1e-3
    assert ru.ev[[2, 3, 4, 6, 7]].sum() > 0
    assert rt.status == "ok" and rt.shift_retries > 0
    assert _true_relres(s, xt) < 1e-9
    assert abs(_true_relres(s, xt) - rt.relres_unscaled) <= 1e-3 * rt.relres_unscaled + 1e-15


@pytest.mark.parametrize("sf,b", [(lambda: W.config0(), 12),
                                  (lambda: W.small_cd2d(40, seed=5), 12),
                                  (lambda: W.small_cd2d(40, seed=5), 8),
                                  (lambda: W.small_cd2d(40, seed=5), 0),
                                  (lambda: W.small_cd3d(10), 8),
                                  (lambda: W.small_cd3d(10), 0)])
def test_discarded_solves_leave_no_trace(orc, sf, b):
    """On these systems every retry falls in the first refinement, so the
    tuned solve must equal the untuned solve started at the final shifts:
    the same x, histories and counts (a discarded solve that updated x,
    counted a refinement or entered the residual history would differ)."""
    s = sf()
    xt, rt = orc.ir_solve(s.rowptr, s.col, s.val, s.b, _small(orc, b, 40))
    assert rt.status == "ok" and rt.shift_retries > 0
    Pf = orc.Params.table4(m=30, **dict(zip(TUNED, rt.beta_final)))
    xf, rf = orc.ir_solve(s.rowptr, s.col, s.val, s.b, Pf)
    assert rf.ev[[2, 3, 4, 6, 7]].sum() == 0
    np.testing.assert_array_equal(xt, xf)
    np.testing.assert_array_equal(rt.relres_hist, rf.relres_hist)
    np.testing.assert_array_equal(rt.gamma_hist, rf.gamma_hist)
    assert (rt.refinements, rt.inner_steps, rt.breakdowns) == \
        (rf.refinements, rf.inner_steps, rf.breakdowns)


def test_shift_bounds_and_budget(orc):
    """Shifts only grow, only on the tuned lines, never past d_f; each retry
    raises at least one shift; the budget caps the retries."""
    s = W.config0()
    for tune in (1, 2, 5, 40):
        x, r = orc.ir_solve(s.rowptr, s.col, s.val, s.b, _small(orc, 4, tune))
        assert r.shift_retries == min(tune, 21)   # 21 retries reach convergence
        rise = np.array(r.beta_final) - 4
        assert (rise >= 0).all() and (np.array(r.beta_final) <= 30).all()
        assert rise.sum() >= r.shift_retries
    # a shift already at d_f stays there
    x, r = orc.ir_solve(s.rowptr, s.col, s.val, s.b, _small(orc, 4, 40, beta7=30))
    assert r.beta_final[0] == 30 and r.status == "ok"
