"""GPU parity on the paths the small cases do not reach: the Arnoldi step
with w in global memory (the path of CTAs with more rows than stay resident
in shared memory, forced here on small systems by params.mgs_wmax; for
preconditioned systems those rows stream through the copy engine's stage
ring), basis entries outside
int32 (d_f > 30: the readers switch from the int32 copy of the basis to
the int64 one), the 27-point
sigma = 2.5 / convection +-100 coefficient regime of the largest
configuration, a batch shaped like the batched configuration (64 systems,
n log-uniform up to 64k), and the bounded waits of the substitutions
(a wait that expires returns IGM_ETIMEOUT and leaves the device usable).
Every comparison with the oracle is bit for bit."""
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


def _compare_inner(g, o):
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


def _check_ir(L, orc, s, P):
    xo, ro = orc.ir_solve(s.rowptr, s.col, s.val, s.b, _oparams(orc, P))
    solver = L.Solver(_dev(s.rowptr), _dev(s.col), _dev(s.val), P)
    x, rep = solver.ir_solve(_dev(s.b))
    assert rep["status"] == ro.status
    assert rep["refinements"] == ro.refinements
    np.testing.assert_array_equal(rep["gamma_hist"], ro.gamma_hist)
    np.testing.assert_array_equal(rep["relres_hist"], ro.relres_hist)
    np.testing.assert_array_equal(rep["ev"], ro.ev)
    np.testing.assert_array_equal(x.cpu().numpy(), xo)
    solver.close()
    return ro


GLOBAL_W = [
    ("cd3d_24_ilu", lambda: W.small_cd3d(24, seed=301), 1, 30),
    ("banded_20000_none", lambda: W.banded_random(20000, np.random.default_rng(302)), 0, 30),
    ("cd2d_120_none", lambda: W.small_cd2d(120), 0, 30),
]


@pytest.mark.parametrize("wmax", [-1, 700])
@pytest.mark.parametrize("name,sf,prec,m", GLOBAL_W, ids=[c[0] for c in GLOBAL_W])
def test_arnoldi_global_w_bit_exact(L, orc, name, sf, prec, m, wmax):
    """Lines 6-19 with w in global memory between the passes (mgs_wmax = -1,
    or a cap below the rows of a CTA): one inner solve (basis, Hessenberg
    matrix, rotations, g, x, overflow counts) and the refinement loop equal
    the oracle's bit for bit."""
    s = sf()
    P = L.params_default(prec, m)
    P.mgs_wmax = wmax
    d = orc.setup(s.rowptr, s.col, s.val, s.b, _oparams(orc, P))
    bk = d["b"] / np.abs(d["b"]).max()
    x0 = np.random.default_rng(9).standard_normal(s.n) * 1e-3
    o = orc.int_gmres(_oparams(orc, P), d, bk, x0)
    solver = L.Solver(_dev(s.rowptr), _dev(s.col), _dev(s.val), P)
    xk = _dev(x0)
    rep = solver.inner_solve(_dev(bk), xk)
    _compare_inner(solver.state(), o)
    np.testing.assert_array_equal(xk.cpu().numpy(), o["x"])
    np.testing.assert_array_equal(rep["ev"], o["ev"])
    solver.close()
    ro = _check_ir(L, orc, s, P)
    assert ro.status == "ok"


# (preconditioned, d_f, shift offset on every tuned line, mgs_wmax, basis
# entries outside int32 at line 11): short solves cut by overflow breakdowns
# and full ones where the basis leaves int32 partway (d_f = 34 with shifts
# raised by 4 gives 2 such entries late in the 30 steps)
WIDE = [(0, 31, 0, 500, False, 0), (0, 32, 2, -1, False, 0), (0, 34, 0, 0, True, -1),
        (0, 34, 0, 0, True, 30), (0, 34, 0, 0, True, 7), (1, 33, 1, -1, True, 0),
        (1, 34, 4, 500, True, 0)]


@pytest.mark.parametrize("prec,df,dd,wmax,wide,fuse", WIDE,
                         ids=[f"p{c[0]}_df{c[1]}_dd{c[2]}_w{c[3]}_f{c[5]}" for c in WIDE])
def test_wide_basis_bit_exact(L, orc, prec, df, dd, wmax, wide, fuse):
    """With d_f > 30 a basis entry (at most 2^d_f in magnitude) can leave
    int32, which the kernels detect (at line 2 or line 11) and answer by
    reading the int64 copy of the basis for the rest of the inner solve
    (one Arnoldi launch a step, or the fused kernel with a whole cycle or 7
    steps a launch, or as the autotuner chooses): the basis,
    Hessenberg matrix, rotations, x and every overflow count equal the
    oracle's bit for bit, line 11's basis entries outside int32 are counted
    alike, and the refinement loop agrees."""
    s = W.small_cd2d(60) if prec else W.banded_random(6000, np.random.default_rng(320))
    P = L.params_default(prec, 30)
    P.fuse_steps = fuse
    P.df = df
    for f in ("beta7", "beta8", "beta10", "beta11a", "beta11b", "beta13", "beta15",
              "beta16a", "beta16b"):
        setattr(P, f, getattr(P, f) + dd)
    P.mgs_wmax = wmax
    d = orc.setup(s.rowptr, s.col, s.val, s.b, _oparams(orc, P))
    bk = d["b"] / np.abs(d["b"]).max()
    x0 = np.zeros(s.n)
    o = orc.int_gmres(_oparams(orc, P), d, bk, x0)
    solver = L.Solver(_dev(s.rowptr), _dev(s.col), _dev(s.val), P)
    xk = _dev(x0)
    rep = solver.inner_solve(_dev(bk), xk)
    _compare_inner(solver.state(), o)
    np.testing.assert_array_equal(xk.cpu().numpy(), o["x"])
    np.testing.assert_array_equal(rep["ev"], o["ev"])
    assert (o["ev"][10] > 0) == wide
    solver.close()
    _check_ir(L, orc, s, P)


FUSED = [
    ("banded_20000", lambda: W.banded_random(20000, np.random.default_rng(330)), 30),
    ("cd2d_120", lambda: W.small_cd2d(120), 30),
    ("banded_3001", lambda: W.banded_random(3001, np.random.default_rng(331)), 20),
]


@pytest.mark.parametrize("fuse,snap,wmax", [(0, 0, 0), (30, -1, 0), (7, 50, 0), (1, 25, 600),
                                            (4, -1, -1), (-1, 0, 0)])
@pytest.mark.parametrize("name,sf,m", FUSED, ids=[c[0] for c in FUSED])
def test_fused_arnoldi_bit_exact(L, orc, name, sf, m, fuse, snap, wmax):
    """Lines 5-19 of several steps in one persistent launch (systems without
    preconditioner): one inner solve and the refinement loop equal the
    oracle bit for bit for every number of steps per launch, every row
    partition and every residency (automatic, none, a cap), and the report
    names the launch configuration that ran (chosen by the autotuner when
    left open)."""
    s = sf()
    P = L.params_default(0, m)
    P.fuse_steps, P.plan_snap, P.mgs_wmax = fuse, snap, wmax
    d = orc.setup(s.rowptr, s.col, s.val, s.b, _oparams(orc, P))
    bk = d["b"] / np.abs(d["b"]).max()
    x0 = np.random.default_rng(9).standard_normal(s.n) * 1e-3
    o = orc.int_gmres(_oparams(orc, P), d, bk, x0)
    solver = L.Solver(_dev(s.rowptr), _dev(s.col), _dev(s.val), P)
    xk = _dev(x0)
    rep = solver.inner_solve(_dev(bk), xk)
    _compare_inner(solver.state(), o)
    np.testing.assert_array_equal(xk.cpu().numpy(), o["x"])
    np.testing.assert_array_equal(rep["ev"], o["ev"])
    solver.close()
    xo, ro = orc.ir_solve(s.rowptr, s.col, s.val, s.b, _oparams(orc, P))
    solver = L.Solver(_dev(s.rowptr), _dev(s.col), _dev(s.val), P)
    x, rep = solver.ir_solve(_dev(s.b))
    assert rep["status"] == ro.status and rep["refinements"] == ro.refinements
    np.testing.assert_array_equal(rep["ev"], ro.ev)
    np.testing.assert_array_equal(x.cpu().numpy(), xo)
    if fuse > 0:
        assert rep["fuse_steps"] == min(fuse, m)
    elif fuse < 0:
        assert rep["fuse_steps"] == 0
    else:
        assert 0 <= rep["fuse_steps"] <= m
    if snap > 0:
        assert rep["plan_snap"] == snap
    elif snap < 0:
        assert rep["plan_snap"] == 0
    else:
        assert rep["plan_snap"] in (0, 25, 50)
    solver.close()


@pytest.mark.parametrize("fuse,snap", [(0, 0), (30, 50), (3, -1), (-1, 25)])
def test_fused_batch_bit_exact(L, orc, fuse, snap):
    """A batch of uneven systems without preconditioner (n log-uniform over
    [1k, 20k], banded random) through the fused Arnoldi kernel, with whole
    systems inside one CTA and systems split over several: every system's
    result equals the oracle's bit for bit."""
    import torch
    rng = np.random.default_rng(340)
    ns = [int(v) for v in np.exp(rng.uniform(np.log(1000), np.log(20000), 24))]
    systems = [W.banded_random(n, rng) for n in ns]
    P = L.params_default(0, 30)
    P.fuse_steps, P.plan_snap = fuse, snap
    svs = [L.Solver(_dev(sy.rowptr), _dev(sy.col), _dev(sy.val), P) for sy in systems]
    out = [torch.empty(sy.n, dtype=torch.float64, device="cuda") for sy in systems]
    reps = L.ir_solve_batched(svs, [_dev(sy.b) for sy in systems], out)
    for k, sy in enumerate(systems):
        xo, ro = orc.ir_solve(sy.rowptr, sy.col, sy.val, sy.b, _oparams(orc, P))
        assert reps[k]["status"] == ro.status and reps[k]["refinements"] == ro.refinements
        np.testing.assert_array_equal(reps[k]["ev"], ro.ev)
        np.testing.assert_array_equal(out[k].cpu().numpy(), xo)
    for sv in svs:
        sv.close()


@pytest.mark.parametrize("wmax", [-1, 500])
def test_arnoldi_ring_tiles_bit_exact(L, orc, wmax):
    """The single-step Arnoldi kernel's ring mode (preconditioned systems
    whose CTAs hold more rows than stay resident): 216,000 rows over 152
    CTAs are 1,421 rows a CTA, streamed through the copy engine's stage ring
    as one full and one partial tile after 0 or 500 resident rows, at every
    alignment of a CTA's first row.  One inner solve (basis, Hessenberg
    matrix, rotations, x, overflow counts) equals the oracle's bit for bit."""
    s = W.small_cd3d(60, seed=303)
    P = L.params_default(1, 12)
    P.mgs_wmax = wmax
    d = orc.setup(s.rowptr, s.col, s.val, s.b, _oparams(orc, P))
    bk = d["b"] / np.abs(d["b"]).max()
    x0 = np.random.default_rng(11).standard_normal(s.n) * 1e-3
    o = orc.int_gmres(_oparams(orc, P), d, bk, x0)
    solver = L.Solver(_dev(s.rowptr), _dev(s.col), _dev(s.val), P)
    xk = _dev(x0)
    rep = solver.inner_solve(_dev(bk), xk)
    _compare_inner(solver.state(), o)
    np.testing.assert_array_equal(xk.cpu().numpy(), o["x"])
    np.testing.assert_array_equal(rep["ev"], o["ev"])
    # a second inner solve on the same handle (the stage ring's barriers go
    # on counting across launches)
    xk = _dev(x0)
    rep = solver.inner_solve(_dev(bk), xk)
    np.testing.assert_array_equal(xk.cpu().numpy(), o["x"])
    solver.close()


def test_arnoldi_global_w_batched_equals_solo(L, orc):
    """A batch whose Arnoldi step keeps w in global memory: each system's
    result equals the oracle's (and so its solo solve)."""
    import torch
    rng = np.random.default_rng(310)
    systems = [W.banded_random(int(n), rng) for n in (5000, 12000, 3001)]
    systems.append(W.small_cd3d(14, seed=311))
    params = [L.params_default(0, 30)] * 3 + [L.params_default(1, 30)]
    params = [P.replace(mgs_wmax=-1) for P in params]
    svs = [L.Solver(_dev(sy.rowptr), _dev(sy.col), _dev(sy.val), P)
           for sy, P in zip(systems, params)]
    out = [torch.empty(sy.n, dtype=torch.float64, device="cuda") for sy in systems]
    reps = L.ir_solve_batched(svs, [_dev(sy.b) for sy in systems], out)
    for k, sy in enumerate(systems):
        xo, ro = orc.ir_solve(sy.rowptr, sy.col, sy.val, sy.b, _oparams(orc, params[k]))
        assert ro.status == "ok" and reps[k]["status"] == "ok"
        assert reps[k]["refinements"] == ro.refinements
        np.testing.assert_array_equal(reps[k]["relres_hist"], ro.relres_hist)
        np.testing.assert_array_equal(reps[k]["ev"], ro.ev)
        np.testing.assert_array_equal(out[k].cpu().numpy(), xo)
    for sv in svs:
        sv.close()


CFG4_REGIME = [(12, 60, 401), (16, 60, 402), (20, 60, 403), (40, 30, 404)]


@pytest.mark.parametrize("N,m,seed", CFG4_REGIME, ids=[f"N{c[0]}_m{c[1]}" for c in CFG4_REGIME])
def test_cfg4_regime_bit_exact(L, orc, N, m, seed):
    """The coefficient regime of the largest configuration (27-point stencil,
    diffusion log-normal with sigma 2.5, convection U[-100, 100], ILU(0),
    Table 5 shifts) on N^3 grids: the refinement loop and the overflow
    counts per line equal the oracle's bit for bit, and reach 1e-10."""
    s = W.config4(N=N, seed=seed)
    P = L.params_default(1, m)
    ro = _check_ir(L, orc, s, P)
    assert ro.status == "ok" and ro.relres < 1e-10
    # one inner solve from a non-zero guess: the whole integer state
    d = orc.setup(s.rowptr, s.col, s.val, s.b, _oparams(orc, P))
    bk = d["b"] / np.abs(d["b"]).max()
    x0 = np.random.default_rng(seed).standard_normal(s.n) * 1e-4
    o = orc.int_gmres(_oparams(orc, P), d, bk, x0)
    solver = L.Solver(_dev(s.rowptr), _dev(s.col), _dev(s.val), P)
    xk = _dev(x0)
    rep = solver.inner_solve(_dev(bk), xk)
    _compare_inner(solver.state(), o)
    np.testing.assert_array_equal(xk.cpu().numpy(), o["x"])
    np.testing.assert_array_equal(rep["ev"], o["ev"])
    solver.close()


def test_cfg2_shaped_batch_bit_exact(L, orc):
    """64 banded random systems with n log-uniform in [1k, 64k] (5-27
    non-zeros per row within +-64, GMRES(30), no preconditioning, Table 4)
    in one batched solve: every system's result equals the oracle's."""
    import torch
    systems = W.config2(count=64, seed=12)
    assert max(sy.n for sy in systems) > 32000
    P = L.params_default(0, 30)
    svs = [L.Solver(_dev(sy.rowptr), _dev(sy.col), _dev(sy.val), P) for sy in systems]
    out = [torch.empty(sy.n, dtype=torch.float64, device="cuda") for sy in systems]
    reps = L.ir_solve_batched(svs, [_dev(sy.b) for sy in systems], out)
    for k, sy in enumerate(systems):
        xo, ro = orc.ir_solve(sy.rowptr, sy.col, sy.val, sy.b, _oparams(orc, P))
        assert ro.status == "ok" and reps[k]["status"] == "ok"
        assert reps[k]["refinements"] == ro.refinements
        np.testing.assert_array_equal(reps[k]["relres_hist"], ro.relres_hist)
        np.testing.assert_array_equal(reps[k]["ev"], ro.ev)
        np.testing.assert_array_equal(out[k].cpu().numpy(), xo)
    for sv in svs:
        sv.close()


@pytest.mark.parametrize("cluster", [1, 4])
def test_bounded_wait_expires(L, orc, cluster):
    """A substitution chunk whose predecessor never signals (params.test_stall,
    wait bound 2 ms): the solve returns IGM_ETIMEOUT instead of hanging, the
    device stays usable, and a fresh handle then solves the same system bit
    for bit like the oracle.  cluster = 1 waits on a progress word in global
    memory, cluster = 4 on a signal in shared memory of the cluster."""
    import time
    s = W.small_cd3d(16, seed=320)
    P = L.params_default(1, 20)
    P.trsv_chunk, P.trsv_cluster = 256, cluster
    stuck = P.replace(test_stall=1, wait_us=2000)
    sv = L.Solver(_dev(s.rowptr), _dev(s.col), _dev(s.val), stuck)
    t0 = time.perf_counter()
    with pytest.raises(L.IGMError) as e:
        sv.ir_solve(_dev(s.b))
    assert e.value.name == "etimeout"
    assert time.perf_counter() - t0 < 30.0
    # the single inner solve reports the same
    with pytest.raises(L.IGMError) as e:
        sv.inner_solve(_dev(s.b / np.abs(s.b).max()), _dev(np.zeros(s.n)))
    assert e.value.name == "etimeout"
    sv.close()
    _check_ir(L, orc, s, P)
