"""GPU parity: the CUDA path, called through the C ABI, against the oracle
on the same seeded inputs.  The integer inner loop (basis V, Hessenberg H,
Givens c, s, g, overflow counts) must be bit-exact; the FP64 steps are
computed in the same order with correctly rounded operations, so they are
compared bit-for-bit too (which is stricter than the 1e-12 relative bound
that the method's FP64 steps need)."""
import numpy as np
import pytest

from paper_2009_07495_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_07495_gb300 import _lib
    from paper_2009_07495_gb300 import build
    build.build()
    return _lib


def _oparams(orc, P):
    return orc.Params(df=P.df, alpha_a=P.alpha_a, m=P.m, precond=P.precond, beta7=P.beta7,
                      beta8=P.beta8, beta10=P.beta10, beta11a=P.beta11a, beta11b=P.beta11b,
                      beta13=P.beta13, beta15=P.beta15, beta16a=P.beta16a, beta16b=P.beta16b,
                      tol=P.tol, max_refine=P.max_refine, s=P.s, order=P.order,
                      shift_tune=P.shift_tune)


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _compare_inner(g, o, n, m):
    """bit-exact comparison of one inner solve's integer state"""
    j = o["jeff"]
    assert g["jeff"] == j
    assert g["nu"] == o["nu"]
    np.testing.assert_array_equal(g["g"][: j + 1], o["g"][: j + 1])
    np.testing.assert_array_equal(g["cs"][:j], o["cs"][:j])
    np.testing.assert_array_equal(g["sn"][:j], o["sn"][:j])
    for c in range(j):
        np.testing.assert_array_equal(g["H"][: c + 2, c], o["H"][: c + 2, c])
    nv = j + 1 if not o["early"] else j
    np.testing.assert_array_equal(g["V"][:nv], o["V"][:nv])


INNER_CASES = [
    ("cfg0_none", lambda: W.config0(), 0, 30),
    ("cd3d_13_ilu_ragged", lambda: W.small_cd3d(13, seed=41), 1, 20),
    ("cd2d_40_none", lambda: W.small_cd2d(40, seed=42), 0, 25),
    ("cd3d_10_27pt_ilu", lambda: W.small_cd3d(10, seed=43, points=27), 1, 15),
]


@pytest.mark.parametrize("name,sf,prec,m", INNER_CASES, ids=[c[0] for c in INNER_CASES])
def test_inner_solve_bit_exact(L, orc, name, sf, prec, m):
    """One int-GMRES(m) solve (Fig. 2, lines 1'/5' with ILU): V, H, c, s, g,
    x and the overflow counts equal the oracle's bit for bit."""
    s = sf()
    P = L.params_default(prec, m)
    d = orc.setup(s.rowptr, s.col, s.val, s.b, _oparams(orc, P))
    bk = d["b"] / np.abs(d["b"]).max()
    rng = np.random.default_rng(5)
    x0 = rng.standard_normal(s.n) * 1e-3
    o = orc.int_gmres(_oparams(orc, P), d, bk, x0)
    solver = L.Solver(_dev(s.rowptr), _dev(s.col), _dev(s.val), P)
    xk = _dev(x0)
    rep = solver.inner_solve(_dev(bk), xk)
    st = solver.state()
    _compare_inner(st, o, s.n, m)
    np.testing.assert_array_equal(xk.cpu().numpy(), o["x"])
    np.testing.assert_array_equal(rep["ev"], o["ev"])
    solver.close()


IR_CASES = [
    ("cfg0", lambda: W.config0(), 0, 30),
    ("cd3d_16_ilu", lambda: W.small_cd3d(16, seed=44), 1, 30),
    ("cd3d_11_ilu_ragged", lambda: W.small_cd3d(11, seed=45), 1, 12),
    ("banded_3000", lambda: W.banded_random(3000, np.random.default_rng(46)), 0, 30),
    ("cd2d_33_none_host", lambda: W.small_cd2d(33, seed=47), 0, 20),
]


@pytest.mark.parametrize("name,sf,prec,m", IR_CASES, ids=[c[0] for c in IR_CASES])
def test_ir_solve_bit_exact(L, orc, name, sf, prec, m):
    """Fig. 1 to 1e-10: same refinement count, gamma and residual histories,
    overflow counts and solution, bit for bit."""
    s = sf()
    P = L.params_default(prec, m)
    xo, ro = orc.ir_solve(s.rowptr, s.col, s.val, s.b, _oparams(orc, P))
    if name.endswith("host"):
        solver = L.Solver(s.rowptr, s.col, s.val, P)   # host (numpy) buffers
        x, rep = solver.ir_solve(s.b)
        xg = x
    else:
        solver = L.Solver(_dev(s.rowptr), _dev(s.col), _dev(s.val), P)
        x, rep = solver.ir_solve(_dev(s.b))
        xg = x.cpu().numpy()
    assert ro.status == "ok" and ro.relres < 1e-10
    assert rep["status"] == "ok" and rep["relres"] < 1e-10
    assert rep["refinements"] == ro.refinements
    np.testing.assert_array_equal(rep["gamma_hist"], ro.gamma_hist)
    np.testing.assert_array_equal(rep["relres_hist"], ro.relres_hist)
    np.testing.assert_array_equal(rep["ev"], ro.ev)
    assert rep["relres_unscaled"] == ro.relres_unscaled
    np.testing.assert_array_equal(xg, xo)
    solver.close()


MT_CASES = [
    ("cd2d_20_s1", lambda: W.small_cd2d(20, seed=48), 0, 20, 1),
    ("cd2d_20_s3", lambda: W.small_cd2d(20, seed=48), 0, 20, 3),
    ("cd3d_10_ilu_s2", lambda: W.small_cd3d(10, seed=49), 1, 15, 2),
]


@pytest.mark.parametrize("name,sf,prec,m,S", MT_CASES, ids=[c[0] for c in MT_CASES])
def test_multiterm_bit_exact(L, orc, name, sf, prec, m, S):
    """Sec. IV-C with s correction terms (eq. AA, matvec): one inner solve
    from a non-zero guess (line 1 with the multi-term matrix) and the whole
    refinement loop equal the oracle's bit for bit."""
    s = sf()
    P = L.params_default(prec, m)
    P.s = S
    d = orc.setup(s.rowptr, s.col, s.val, s.b, _oparams(orc, P))
    assert 2 <= len(d["alphas"]) <= S + 1     # fewer when A is exact sooner
    bk = d["b"] / np.abs(d["b"]).max()
    x0 = np.random.default_rng(6).standard_normal(s.n) * 1e-3
    o = orc.int_gmres(_oparams(orc, P), d, bk, x0)
    solver = L.Solver(_dev(s.rowptr), _dev(s.col), _dev(s.val), P)
    xk = _dev(x0)
    rep = solver.inner_solve(_dev(bk), xk)
    _compare_inner(solver.state(), o, s.n, m)
    np.testing.assert_array_equal(xk.cpu().numpy(), o["x"])
    np.testing.assert_array_equal(rep["ev"], o["ev"])
    xo, ro = orc.ir_solve(s.rowptr, s.col, s.val, s.b, _oparams(orc, P))
    x, rep = solver.ir_solve(_dev(s.b))
    assert rep["status"] == "ok" and rep["refinements"] == ro.refinements
    np.testing.assert_array_equal(rep["relres_hist"], ro.relres_hist)
    np.testing.assert_array_equal(rep["ev"], ro.ev)
    np.testing.assert_array_equal(x.cpu().numpy(), xo)
    solver.close()


def test_multiterm_coarse_word_fewer_refinements(L, orc):
    """A coarse word (alpha_a = 6): s = 0 needs many refinements, s = 2
    far fewer, on the GPU exactly as in the oracle."""
    s = W.small_cd2d(16, seed=4)
    counts = []
    for S in (0, 2):
        P = L.params_default(0, 30)
        P.alpha_a, P.s = 6, S
        P.beta7 = P.beta8 = P.beta10 = P.beta11a = P.beta13 = P.beta15 = P.beta16a = 6
        P.beta11b = P.beta16b = 4
        xo, ro = orc.ir_solve(s.rowptr, s.col, s.val, s.b, _oparams(orc, P))
        solver = L.Solver(_dev(s.rowptr), _dev(s.col), _dev(s.val), P)
        x, rep = solver.ir_solve(_dev(s.b))
        assert rep["status"] == "ok" and rep["refinements"] == ro.refinements
        np.testing.assert_array_equal(x.cpu().numpy(), xo)
        counts.append(rep["refinements"])
        solver.close()
    assert counts[1] < counts[0], counts


GS_CASES = [
    ("cfg0_gs", lambda: W.config0(), 30),
    ("cd3d_12_gs", lambda: W.small_cd3d(12, seed=50), 20),
    ("cd3d_10_27pt_gs", lambda: W.small_cd3d(10, seed=51, points=27), 20),
]


@pytest.mark.parametrize("name,sf,m", GS_CASES, ids=[c[0] for c in GS_CASES])
def test_gauss_seidel_bit_exact(L, orc, name, sf, m):
    """The integer Gauss-Seidel preconditioner (precond = 2): the refinement
    loop equals the oracle's bit for bit and has no overflow event."""
    s = sf()
    P = L.params_default(2, m)
    xo, ro = orc.ir_solve(s.rowptr, s.col, s.val, s.b, _oparams(orc, P))
    solver = L.Solver(_dev(s.rowptr), _dev(s.col), _dev(s.val), P)
    x, rep = solver.ir_solve(_dev(s.b))
    assert ro.status == "ok" and rep["status"] == "ok"
    assert rep["refinements"] == ro.refinements
    np.testing.assert_array_equal(rep["relres_hist"], ro.relres_hist)
    np.testing.assert_array_equal(rep["ev"], ro.ev)
    assert int(np.abs(np.asarray(rep["ev"])).sum()) == 0
    np.testing.assert_array_equal(x.cpu().numpy(), xo)
    solver.close()


MC_CASES = [
    ("cd3d_12_ilu_mc", lambda: W.small_cd3d(12, seed=52), 1),
    ("cd3d_10_27pt_ilu_mc", lambda: W.small_cd3d(10, seed=53, points=27), 1),
    ("cd3d_12_gs_mc", lambda: W.small_cd3d(12, seed=54), 2),
    ("banded_2000_ilu_mc", lambda: W.banded_random(2000, np.random.default_rng(55)), 1),
]


@pytest.mark.parametrize("name,sf,prec", MC_CASES, ids=[c[0] for c in MC_CASES])
def test_multicolour_order_bit_exact(L, orc, name, sf, prec):
    """order = 1: the method on P A P^T (P x) = P b with the multicolour
    permutation; one inner solve (basis and Hessenberg matrix in the new
    order, b and x in the caller's) and the refinement loop equal the
    oracle's bit for bit."""
    s = sf()
    m = 20
    P = L.params_default(prec, m)
    P.order = 1
    d = orc.setup(s.rowptr, s.col, s.val, s.b, _oparams(orc, P))
    perm = d["perm"]
    bk_new = d["b"] / np.abs(d["b"]).max()
    x0 = np.random.default_rng(7).standard_normal(s.n) * 1e-3
    o = orc.int_gmres(_oparams(orc, P), d, bk_new, x0[perm])
    bk = np.empty(s.n)
    bk[perm] = bk_new
    solver = L.Solver(_dev(s.rowptr), _dev(s.col), _dev(s.val), P)
    xk = _dev(x0)
    rep = solver.inner_solve(_dev(bk), xk)
    _compare_inner(solver.state(), o, s.n, m)
    xo_inner = np.empty(s.n)
    xo_inner[perm] = o["x"]
    np.testing.assert_array_equal(xk.cpu().numpy(), xo_inner)
    np.testing.assert_array_equal(rep["ev"], o["ev"])
    xo, ro = orc.ir_solve(s.rowptr, s.col, s.val, s.b, _oparams(orc, P))
    x, rep = solver.ir_solve(_dev(s.b))
    assert ro.status == "ok" and rep["status"] == "ok"
    assert rep["refinements"] == ro.refinements
    np.testing.assert_array_equal(rep["relres_hist"], ro.relres_hist)
    np.testing.assert_array_equal(rep["ev"], ro.ev)
    np.testing.assert_array_equal(x.cpu().numpy(), xo)
    solver.close()


def test_stall_stops_like_the_oracle(L, orc):
    """A tolerance below FP64's reach: the loop stops at the first stall
    (no decrease over three refinements) with ENOCONV, at the same
    refinement as the oracle, with the same residual history."""
    s = W.config0()
    P = L.params_default(0, 30)
    P.tol, P.max_refine = 1e-18, 40
    xo, ro = orc.ir_solve(s.rowptr, s.col, s.val, s.b, _oparams(orc, P))
    solver = L.Solver(_dev(s.rowptr), _dev(s.col), _dev(s.val), P)
    x, rep = solver.ir_solve(_dev(s.b))
    assert ro.status == "enoconv" and rep["status"] == "enoconv"
    assert rep["refinements"] == ro.refinements < 40
    np.testing.assert_array_equal(rep["relres_hist"], ro.relres_hist)
    np.testing.assert_array_equal(x.cpu().numpy(), xo)
    solver.close()


def test_one_by_one(L):
    """n = 1: Ahat = [2], bhat = [4] gives x = 2 exactly in one refinement."""
    P = L.params_default(0, 5)
    solver = L.Solver(np.array([0, 1], np.int32), np.array([0], np.int32), np.array([2.0]), P)
    x, rep = solver.ir_solve(np.array([4.0]))
    assert x[0] == 2.0 and rep["refinements"] == 1 and rep["status"] == "ok"


def test_overflow_events_match(L, orc):
    """Without shifts and alpha_a = 40 the inner products overflow; the event
    counts per line and the wrapped results still match the oracle."""
    s = W.small_cd2d(6, seed=25)
    P = L.params_default(1, 5)
    P.precond = 0
    P.alpha_a = 40
    P.max_refine = 2
    xo, ro = orc.ir_solve(s.rowptr, s.col, s.val, s.b, _oparams(orc, P))
    solver = L.Solver(s.rowptr, s.col, s.val, P)
    x, rep = solver.ir_solve(s.b)
    assert ro.ev[2] > 0 or ro.ev[4] > 0
    np.testing.assert_array_equal(rep["ev"], ro.ev)
    assert rep["refinements"] == ro.refinements
    np.testing.assert_array_equal(x, xo)


def test_errors_are_statuses(L):
    """Malformed input returns a status (never a fault)."""
    s = W.small_cd2d(5)
    val = s.val.copy()
    val[s.rowptr[2]:s.rowptr[3]] = 0.0
    with pytest.raises(L.IGMError) as e:
        L.Solver(s.rowptr, s.col, val, L.params_default(0, 5))
    assert e.value.name == "ezero_row"
    # a row without its diagonal cannot be ILU(0)-factorised
    rp = np.array([0, 1, 2], np.int32)
    with pytest.raises(L.IGMError) as e:
        L.Solver(rp, np.array([1, 0], np.int32), np.array([1.0, 1.0]), L.params_default(1, 5))
    assert e.value.name == "ezero_pivot"
    # unsorted columns
    with pytest.raises(L.IGMError) as e:
        L.Solver(np.array([0, 2, 3], np.int32), np.array([1, 0, 1], np.int32),
                 np.array([1.0, 2.0, 3.0]), L.params_default(0, 5))
    assert e.value.name == "einval"
    # bad parameters
    with pytest.raises(L.IGMError) as e:
        L.Solver(s.rowptr, s.col, s.val, L.params_default(0, 0))
    assert e.value.name == "einval"


def test_batched_equals_solo(L, orc):
    """ir_solve_batched: uneven systems (ragged tiles, one with ILU) solved in
    one launch sequence give exactly their solo results."""
    rng = np.random.default_rng(50)
    systems = [W.banded_random(int(n), rng) for n in (1000, 2500, 4097, 1500)]
    systems.append(W.small_cd3d(12, seed=51))
    params = [L.params_default(0, 30)] * 4 + [L.params_default(1, 30)]
    solos, xs = [], []
    for s, P in zip(systems, params):
        sv = L.Solver(_dev(s.rowptr), _dev(s.col), _dev(s.val), P)
        x, rep = sv.ir_solve(_dev(s.b))
        solos.append((x.cpu().numpy(), rep))
        xs.append(sv)
    bh = [_dev(s.b) for s in systems]
    import torch
    out = [torch.empty(s.n, dtype=torch.float64, device="cuda") for s in systems]
    reps = L.ir_solve_batched(xs, bh, out)
    for k, s in enumerate(systems):
        xo, ro = orc.ir_solve(s.rowptr, s.col, s.val, s.b, _oparams(orc, params[k]))
        np.testing.assert_array_equal(out[k].cpu().numpy(), solos[k][0])
        np.testing.assert_array_equal(out[k].cpu().numpy(), xo)
        assert reps[k]["refinements"] == solos[k][1]["refinements"] == ro.refinements
        np.testing.assert_array_equal(reps[k]["relres_hist"], ro.relres_hist)
    for sv in xs:
        sv.close()


def _variant(L, prec, m, order=0, terms=0):
    P = L.params_default(prec, m)
    P.order, P.s = order, terms
    return P


def test_batched_mixed_variants_equal_solo(L, orc):
    """One batch mixing natural-order ILU(0), multicolour ILU(0) (colour
    launches beside chunk launches), Gauss-Seidel, multi-term and plain
    systems: every result equals its solo solve and the oracle's."""
    import torch
    rng = np.random.default_rng(61)
    systems = [W.small_cd3d(11, seed=62), W.small_cd3d(10, seed=63),
               W.small_cd3d(9, seed=64, points=27), W.small_cd3d(8, seed=65),
               W.banded_random(1800, rng), W.small_cd2d(24, seed=66)]
    params = [_variant(L, 1, 20), _variant(L, 1, 20, order=1), _variant(L, 1, 20, order=1),
              _variant(L, 2, 20), _variant(L, 0, 20, terms=2), _variant(L, 2, 20, order=1)]
    svs, solos = [], []
    for sy, P in zip(systems, params):
        sv = L.Solver(_dev(sy.rowptr), _dev(sy.col), _dev(sy.val), P)
        x, rep = sv.ir_solve(_dev(sy.b))
        solos.append((x.cpu().numpy(), rep))
        svs.append(sv)
    out = [torch.empty(sy.n, dtype=torch.float64, device="cuda") for sy in systems]
    reps = L.ir_solve_batched(svs, [_dev(sy.b) for sy in systems], out)
    for k, sy in enumerate(systems):
        xo, ro = orc.ir_solve(sy.rowptr, sy.col, sy.val, sy.b, _oparams(orc, params[k]))
        assert ro.status == "ok"
        np.testing.assert_array_equal(out[k].cpu().numpy(), solos[k][0])
        np.testing.assert_array_equal(out[k].cpu().numpy(), xo)
        assert reps[k]["refinements"] == solos[k][1]["refinements"] == ro.refinements
        np.testing.assert_array_equal(reps[k]["ev"], ro.ev)
    for sv in svs:
        sv.close()


def test_server_mixed_variants_equal_solo(L, orc):
    """The server with requests of every variant (orders, preconditioners,
    correction terms) returns each request's oracle result."""
    systems = [W.small_cd3d(9, seed=67), W.small_cd3d(10, seed=68),
               W.small_cd3d(8, seed=69, points=27), W.small_cd2d(22, seed=70)]
    params = [_variant(L, 1, 20, order=1), _variant(L, 2, 20), _variant(L, 1, 20, terms=1),
              _variant(L, 0, 20, order=1)]
    srv = L.Server(budget_bytes=1 << 30, m=20)
    ids = [srv.submit(sy.rowptr, sy.col, sy.val, sy.b, P) for sy, P in zip(systems, params)]
    outs = [srv.poll(i, wait_ms=60000) for i in ids]
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(systems) and st["failed"] == 0
    for (done, x, rep, lat), sy, P in zip(outs, systems, params):
        xo, ro = orc.ir_solve(sy.rowptr, sy.col, sy.val, sy.b, _oparams(orc, P))
        assert done and rep["status"] == ro.status == "ok"
        assert rep["refinements"] == ro.refinements
        np.testing.assert_array_equal(x, xo)


def _tuned(L, prec, m, b, tune):
    """shifts of lines 7, 8, 10, 13, 15 set to b, auto-tuning budget tune"""
    P = L.params_default(prec, m)
    for k in ("beta7", "beta8", "beta10", "beta13", "beta15"):
        setattr(P, k, b)
    P.shift_tune = tune
    return P


@pytest.mark.parametrize("b", [12, 8, 4])
def test_shift_tune_bit_exact(L, orc, b):
    """Shift auto-tuning (Sec. VII-D) from shifts too small for the system
    (the retries fall in the first and in later refinements): the discarded
    inner solves, the raised shifts and the whole loop equal the oracle's
    bit for bit; a second solve on the same handle starts again from the
    set-up shifts and repeats the first."""
    s = W.config0()
    P = _tuned(L, 0, 30, b, 40)
    xo, ro = orc.ir_solve(s.rowptr, s.col, s.val, s.b, _oparams(orc, P))
    assert ro.status == "ok" and ro.shift_retries > 0
    solver = L.Solver(_dev(s.rowptr), _dev(s.col), _dev(s.val), P)
    for _ in range(2):
        x, rep = solver.ir_solve(_dev(s.b))
        assert rep["status"] == "ok"
        assert rep["shift_retries"] == ro.shift_retries
        assert rep["beta_final"] == ro.beta_final
        assert (rep["refinements"], rep["inner_steps"], rep["breakdowns"]) == \
            (ro.refinements, ro.inner_steps, ro.breakdowns)
        np.testing.assert_array_equal(rep["relres_hist"], ro.relres_hist)
        np.testing.assert_array_equal(rep["gamma_hist"], ro.gamma_hist)
        np.testing.assert_array_equal(rep["ev"], ro.ev)
        np.testing.assert_array_equal(x.cpu().numpy(), xo)
    # the retry budget binds on the device as in the oracle
    P2 = _tuned(L, 0, 30, b, 2)
    xo2, ro2 = orc.ir_solve(s.rowptr, s.col, s.val, s.b, _oparams(orc, P2))
    solver2 = L.Solver(_dev(s.rowptr), _dev(s.col), _dev(s.val), P2)
    x2, rep2 = solver2.ir_solve(_dev(s.b))
    assert rep2["status"] == ro2.status and rep2["shift_retries"] == ro2.shift_retries == 2
    assert rep2["beta_final"] == ro2.beta_final
    np.testing.assert_array_equal(rep2["relres_hist"], ro2.relres_hist)
    np.testing.assert_array_equal(x2.cpu().numpy(), xo2)
    solver.close()
    solver2.close()


def test_shift_tune_batched_and_served(L, orc):
    """Systems that tune their shifts beside systems that do not, in one
    batch and in the server: each result equals its solo solve and the
    oracle's (retries, final shifts and solution)."""
    import torch
    systems = [W.config0(), W.small_cd2d(40, seed=5), W.small_cd3d(10, seed=71),
               W.small_cd2d(24, seed=72)]
    params = [_tuned(L, 0, 30, 8, 40), _tuned(L, 0, 30, 0, 40), _tuned(L, 1, 30, 0, 10),
              L.params_default(0, 30)]
    svs, solos = [], []
    for sy, P in zip(systems, params):
        sv = L.Solver(_dev(sy.rowptr), _dev(sy.col), _dev(sy.val), P)
        x, rep = sv.ir_solve(_dev(sy.b))
        solos.append((x.cpu().numpy(), rep))
        svs.append(sv)
    out = [torch.empty(sy.n, dtype=torch.float64, device="cuda") for sy in systems]
    reps = L.ir_solve_batched(svs, [_dev(sy.b) for sy in systems], out)
    srv = L.Server(budget_bytes=1 << 30, m=30)
    ids = [srv.submit(sy.rowptr, sy.col, sy.val, sy.b, P) for sy, P in zip(systems, params)]
    served = [srv.poll(i, wait_ms=60000) for i in ids]
    srv.close()
    for k, sy in enumerate(systems):
        xo, ro = orc.ir_solve(sy.rowptr, sy.col, sy.val, sy.b, _oparams(orc, params[k]))
        assert ro.status == "ok"
        for x, rep in ((out[k].cpu().numpy(), reps[k]), solos[k], served[k][1:3]):
            np.testing.assert_array_equal(x, xo)
            assert rep["shift_retries"] == ro.shift_retries
            assert rep["beta_final"] == ro.beta_final
            assert rep["refinements"] == ro.refinements
            np.testing.assert_array_equal(rep["ev"], ro.ev)
    assert solos[0][1]["shift_retries"] > 0 and solos[3][1]["shift_retries"] == 0
    for sv in svs:
        sv.close()


@pytest.mark.parametrize("fuse", [-1, 10])
@pytest.mark.parametrize("count", [64, 80])
def test_batched_many_tiny_systems(L, orc, count, fuse):
    """Tiny systems (n = 9) batched so that every row fits one CTA: 64
    systems run the Arnoldi step's one-CTA mode (its segment cache full),
    80 the cooperative grid mode with one CTA whose segments overflow the
    cache, one step a launch or (fuse = 10) ten steps a fused launch.
    Every result equals the oracle's bit for bit."""
    import torch
    systems = [W.small_cd2d(3, seed=200 + k) for k in range(count)]
    P = L.params_default(0, 10)
    P.fuse_steps = fuse
    svs = [L.Solver(_dev(sy.rowptr), _dev(sy.col), _dev(sy.val), P) for sy in systems]
    out = [torch.empty(sy.n, dtype=torch.float64, device="cuda") for sy in systems]
    reps = L.ir_solve_batched(svs, [_dev(sy.b) for sy in systems], out)
    for k, sy in enumerate(systems):
        xo, ro = orc.ir_solve(sy.rowptr, sy.col, sy.val, sy.b, _oparams(orc, P))
        assert ro.status == "ok" and reps[k]["status"] == "ok"
        assert reps[k]["refinements"] == ro.refinements
        np.testing.assert_array_equal(reps[k]["relres_hist"], ro.relres_hist)
        np.testing.assert_array_equal(out[k].cpu().numpy(), xo)
    for sv in svs:
        sv.close()


@pytest.mark.parametrize("fuse", [-1, 30])
@pytest.mark.parametrize("n", [1024, 1025])
def test_arnoldi_mode_boundary(L, orc, n, fuse):
    """n = 1024 is the largest system of the one-CTA Arnoldi mode, 1025 the
    smallest of the grid mode (two CTAs, one Arnoldi launch a step or a
    whole cycle in one fused launch): all equal the oracle bit for bit."""
    s = W.config0() if n == 1024 else W.banded_random(1025, np.random.default_rng(7))
    P = L.params_default(0, 30)
    P.fuse_steps = fuse
    xo, ro = orc.ir_solve(s.rowptr, s.col, s.val, s.b, _oparams(orc, P))
    solver = L.Solver(_dev(s.rowptr), _dev(s.col), _dev(s.val), P)
    x, rep = solver.ir_solve(_dev(s.b))
    assert ro.status == "ok" and rep["status"] == "ok"
    assert rep["refinements"] == ro.refinements
    np.testing.assert_array_equal(rep["relres_hist"], ro.relres_hist)
    np.testing.assert_array_equal(rep["ev"], ro.ev)
    np.testing.assert_array_equal(x.cpu().numpy(), xo)
    solver.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_fp64_gmres_comparison_solver(L, orc, prec):
    """The FP64 GMRES(m) comparison solver (params.inner = 1) converges like
    the oracle's FP64 GMRES: same refinement count, relres < 1e-10 and the
    same solution to rounding (its sums are ordered differently)."""
    s = W.small_cd3d(12, seed=52) if prec else W.config0()
    P = L.params_default(prec, 30)
    P.inner = 1
    xo, ro = orc.ir_solve(s.rowptr, s.col, s.val, s.b, _oparams(orc, P), inner=1)
    solver = L.Solver(_dev(s.rowptr), _dev(s.col), _dev(s.val), P)
    x, rep = solver.ir_solve(_dev(s.b))
    assert rep["status"] == "ok" and rep["relres"] < 1e-10
    assert abs(rep["refinements"] - ro.refinements) <= 1
    xg = x.cpu().numpy()
    assert np.linalg.norm(xg - xo) <= 1e-8 * np.linalg.norm(xo)
    solver.close()


def test_server_results_equal_solo(L, orc):
    """Continuous batching: requests submitted while others are running are
    admitted into later rounds; every served result is bit-identical to the
    same system solved alone (and to the oracle)."""
    import time
    rng = np.random.default_rng(60)
    systems = [W.small_cd3d(int(N), seed=int(60 + N)) for N in (8, 11, 6, 13, 9)]
    systems += [W.small_cd2d(int(N), seed=int(70 + N)) for N in (20, 35)]
    P_ilu, P_none = L.params_default(1, 20), L.params_default(0, 20)
    params = [P_ilu] * 5 + [P_none] * 2
    srv = L.Server(budget_bytes=1 << 30, m=20)
    ids = []
    for k, (s, P) in enumerate(zip(systems, params)):
        ids.append(srv.submit(s.rowptr, s.col, s.val, s.b, P))
        if k == 2:
            time.sleep(0.05)   # later arrivals join while the first run
    outs = [srv.poll(i, wait_ms=60000) for i in ids]
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(systems) and st["failed"] == 0
    for (done, x, rep, lat), s, P in zip(outs, systems, params):
        assert done and rep["status"] == "ok" and rep["relres"] < 1e-10
        solo = L.Solver(s.rowptr, s.col, s.val, P)
        xs, rs = solo.ir_solve(s.b)
        solo.close()
        np.testing.assert_array_equal(x, xs)
        assert rep["refinements"] == rs["refinements"]
        xo, ro = orc.ir_solve(s.rowptr, s.col, s.val, s.b, _oparams(orc, P))
        np.testing.assert_array_equal(x, xo)


def test_server_budget_admission(L):
    """With a budget that fits about one system at a time, requests are served
    one after another and all complete; a request larger than the whole
    budget is refused at submission."""
    systems = [W.small_cd2d(24, seed=80 + k) for k in range(4)]
    P = L.params_default(0, 10)
    one = 0
    sv = L.Solver(systems[0].rowptr, systems[0].col, systems[0].val, P)
    one = sv.device_bytes()
    sv.close()
    srv = L.Server(budget_bytes=int(one * 1.5), m=10)
    ids = [srv.submit(s.rowptr, s.col, s.val, s.b, P) for s in systems]
    res = [srv.poll(i, wait_ms=60000) for i in ids]
    st = srv.stats()
    assert all(r[0] and r[2]["status"] == "ok" for r in res)
    assert st["peak_bytes"] <= int(one * 1.5)
    big = W.small_cd2d(120, seed=90)
    with pytest.raises(L.IGMError) as e:
        srv.submit(big.rowptr, big.col, big.val, big.b, P)
    assert e.value.name == "eoom"
    srv.close()


@pytest.mark.parametrize("n", [1, 7, 1000, 262144 + 13])
@pytest.mark.parametrize("scale", [1e-150, 1.0, 1e200])
def test_norm2_bit_exact(L, orc, n, scale):
    """igm_norm2 (device and host input) equals the oracle's reproducible
    norm bit for bit, and is independent of the element order."""
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) * scale
    ref = orc.norm2(x)
    assert L.norm2(_dev(x)) == ref
    assert L.norm2(x) == ref
    assert L.norm2(_dev(rng.permutation(x))) == ref
    assert L.norm2(np.zeros(5)) == 0.0


@pytest.mark.parametrize("chunk", [100, 1000, 1024, 1500, 4096, 1 << 20])
def test_chunk_schedule_does_not_change_results(L, orc, chunk):
    """Line 5' runs over chunked level schedules; any chunk size (several
    ragged chunks, one chunk for the whole system) gives the oracle's result
    bit for bit."""
    s = W.small_cd3d(16, seed=44)
    P = L.params_default(1, 30)
    P.trsv_chunk = chunk
    xo, ro = orc.ir_solve(s.rowptr, s.col, s.val, s.b, _oparams(orc, P))
    solver = L.Solver(_dev(s.rowptr), _dev(s.col), _dev(s.val), P)
    x, rep = solver.ir_solve(_dev(s.b))
    np.testing.assert_array_equal(x.cpu().numpy(), xo)
    np.testing.assert_array_equal(rep["relres_hist"], ro.relres_hist)
    solver.close()


@pytest.mark.parametrize("cluster", [1, 2, 4, 8])
def test_substitution_clusters_do_not_change_results(L, orc, cluster):
    """The cluster knob is accepted and ignored: with 16 chunks of the
    substitutions every accepted value (1, 2, 4, 8) gives the oracle's
    result bit for bit."""
    s = W.small_cd3d(16, seed=45)
    P = L.params_default(1, 30)
    P.trsv_chunk = 256
    P.trsv_cluster = cluster
    xo, ro = orc.ir_solve(s.rowptr, s.col, s.val, s.b, _oparams(orc, P))
    solver = L.Solver(_dev(s.rowptr), _dev(s.col), _dev(s.val), P)
    x, rep = solver.ir_solve(_dev(s.b))
    np.testing.assert_array_equal(x.cpu().numpy(), xo)
    np.testing.assert_array_equal(rep["relres_hist"], ro.relres_hist)
    np.testing.assert_array_equal(rep["ev"], ro.ev)
    solver.close()


@pytest.mark.parametrize("N,chunk,cluster", [(12, 0, 0), (12, 300, 1), (12, 300, 4),
                                             (14, 0, 4)])
def test_27_point_ilu_bit_exact(L, orc, N, chunk, cluster):
    """27-point stencil with ILU(0): factor rows have 13 strict entries, more
    than the substitution keeps in registers (the rest come from the packed
    arrays, external values from global memory).  Several chunks, with and
    without clusters: the oracle's result bit for bit."""
    s = W.small_cd3d(N, seed=46, points=27)
    P = L.params_default(1, 30)
    P.trsv_chunk = chunk
    P.trsv_cluster = cluster
    xo, ro = orc.ir_solve(s.rowptr, s.col, s.val, s.b, _oparams(orc, P))
    solver = L.Solver(_dev(s.rowptr), _dev(s.col), _dev(s.val), P)
    x, rep = solver.ir_solve(_dev(s.b))
    np.testing.assert_array_equal(x.cpu().numpy(), xo)
    np.testing.assert_array_equal(rep["relres_hist"], ro.relres_hist)
    np.testing.assert_array_equal(rep["ev"], ro.ev)
    solver.close()


@pytest.fixture(scope="module")
def cfg1():
    return W.config1()


def test_full_size_config1_inner_solve_bit_exact(L, orc, cfg1):
    """Config 1 at full size (128^3, n = 2,097,152, ILU(0), m = 50), in the
    launch configuration of the benchmark: one whole inner solve (Fig. 2) is
    bit-identical to the oracle's -- basis, Hessenberg matrix, rotations, g,
    correction and overflow counts."""
    s = cfg1
    P = L.params_default(1, 50)
    d = orc.setup(s.rowptr, s.col, s.val, s.b, _oparams(orc, P))
    bk = d["b"] / np.abs(d["b"]).max()
    o = orc.int_gmres(_oparams(orc, P), d, bk)
    solver = L.Solver(_dev(s.rowptr), _dev(s.col), _dev(s.val), P)
    xk = _dev(np.zeros(s.n))
    rep = solver.inner_solve(_dev(bk), xk)
    st = solver.state()
    _compare_inner(st, o, s.n, 50)
    np.testing.assert_array_equal(xk.cpu().numpy(), o["x"])
    np.testing.assert_array_equal(rep["ev"], o["ev"])
    solver.close()


def test_full_size_config1_refinement(L, cfg1):
    """The full refinement solve of config 1 reaches 1e-10 in 6 refinements,
    the count of the oracle's own full solve of this system (measured once;
    the two paths agree bit for bit), with no overflow event (Sec. VII-C:
    ILU with zero shifts) and a decreasing gamma (Sec. IV-A)."""
    s = cfg1
    solver = L.Solver(_dev(s.rowptr), _dev(s.col), _dev(s.val), L.params_default(1, 50))
    x, rep = solver.ir_solve(_dev(s.b))
    assert rep["status"] == "ok" and rep["relres"] < 1e-10
    assert rep["refinements"] == 6
    assert np.all(rep["ev"] == 0)
    assert np.all(np.diff(rep["gamma_hist"]) < 0)
    solver.close()
