"""The seeded synthetic inputs have the structure their recipes state (no
GPU): sizes and non-zero counts of the stencil systems in closed form, the
M-matrix sign pattern and diagonal dominance that make every system
non-singular with a stored diagonal (ILU(0) needs one), the banded random
systems' band and row lengths, the serving stream's arrival process, and
determinism under a fixed seed."""
import math

import numpy as np
import pytest

from paper_2009_07495_gb300 import workloads as W


def _csr_ok(s):
    assert s.rowptr[0] == 0 and s.rowptr[-1] == s.nnz == s.col.size == s.val.size
    assert np.all(np.diff(s.rowptr) >= 1)
    assert s.col.min() >= 0 and s.col.max() < s.n
    rows = np.repeat(np.arange(s.n), np.diff(s.rowptr))
    # columns sorted within each row, no duplicates
    key = rows.astype(np.int64) * s.n + s.col
    assert np.all(np.diff(key) > 0)
    isd = s.col == rows
    assert np.bincount(rows[isd], minlength=s.n).min() == 1  # one diagonal per row
    d = np.zeros(s.n)
    d[rows[isd]] = s.val[isd]
    off = np.bincount(rows, weights=np.where(isd, 0.0, np.abs(s.val)), minlength=s.n)
    return rows, isd, d, off


def _m_matrix(s):
    """Positive diagonal, non-positive off-diagonals, rows weakly
    diagonally dominant (upwind convection-diffusion)."""
    rows, isd, d, off = _csr_ok(s)
    assert np.all(d > 0)
    assert np.all(s.val[~isd] <= 0)
    assert np.all(off <= d * (1 + 1e-12))


def test_config0_shape_and_rhs():
    s = W.config0()
    assert s.n == 1024 and s.nnz == 5 * 1024 - 4 * 32  # 5-point stencil on 32 x 32
    _m_matrix(s)
    np.testing.assert_allclose(s.b, s.matvec(np.ones(s.n)), rtol=0, atol=0)


@pytest.mark.parametrize("N", [5, 8])
def test_config1_7_point_count_and_sign_pattern(N):
    s = W.config1(N=N)
    assert s.n == N ** 3 and s.nnz == 7 * N ** 3 - 6 * N ** 2
    _m_matrix(s)
    assert 7 * 128 ** 3 - 6 * 128 ** 2 == 14_581_760  # the full-size figure quoted


@pytest.mark.parametrize("N", [4, 7])
def test_config4_27_point_count_and_sign_pattern(N):
    s = W.config4(N=N)
    assert s.n == N ** 3 and s.nnz == (3 * N - 2) ** 3
    lens = np.diff(s.rowptr)
    assert lens.min() == 8 and lens.max() == 27  # corner and interior rows
    _m_matrix(s)
    assert (3 * 200 - 2) ** 3 == 213_847_192  # nnz of the 200^3 system


def test_config2_banded_systems():
    systems = W.config2(count=8, n_lo=1000, n_hi=4000)
    for s in systems:
        assert 1000 <= s.n <= 4000
        rows, isd, d, off = _csr_ok(s)
        assert np.abs(s.col - rows).max() <= 64
        lens = np.diff(s.rowptr)
        assert lens.min() >= 5 and lens.max() <= 27
        # strictly diagonally dominant by at least 5%
        assert np.all(d >= 1.05 * np.maximum(off, 1.0) * (1 - 1e-12))


def test_config2_sizes_log_uniform():
    ns = np.array([s.n for s in W.config2(count=64, n_lo=1000, n_hi=8000)])
    assert ns.min() >= 1000 and ns.max() <= 8000
    # log-uniform: the median near the geometric mean of the range
    assert abs(math.log(np.median(ns)) - 0.5 * math.log(1000 * 8000)) < 0.35


def test_seeded_generators_are_deterministic():
    a, b = W.config2(count=3, n_lo=1000, n_hi=2000), W.config2(count=3, n_lo=1000, n_hi=2000)
    for x, y in zip(a, b):
        for f in ("rowptr", "col", "val", "b"):
            np.testing.assert_array_equal(getattr(x, f), getattr(y, f))
    c, d = W.config4(N=5), W.config4(N=5)
    np.testing.assert_array_equal(c.val, d.val)
    np.testing.assert_array_equal(c.b, d.b)
    assert not np.array_equal(W.config4(N=5, seed=5).val, c.val)


def test_serving_stream_recipe():
    rate = 2000.0
    reqs = W.config3_requests(count=4000, rate=rate)
    t = np.array([r.arrival_s for r in reqs])
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() * rate - 1.0) < 0.05           # Poisson, mean 1/rate
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.08     # exponential gaps
    kinds = {r.kind for r in reqs}
    assert kinds == {"2d5", "3d7", "3d27"}
    sides = np.array([r.side for r in reqs])
    assert sides.min() >= 16 and sides.max() <= 160
    pe = np.array([r.peclet for r in reqs])
    assert pe.min() >= 0.1 and pe.max() <= 100.0
    assert {r.tol for r in reqs} == {1e-8, 1e-10}
    assert len({r.seed for r in reqs}) == len(reqs)


@pytest.mark.parametrize("kind,dims,pts", [("2d5", 2, 5), ("3d7", 3, 7), ("3d27", 3, 27)])
def test_request_systems(kind, dims, pts):
    r = W.Request(0.0, kind, 9, 3.0, 1e-10, 12345)
    s = W.request_system(r)
    assert s.n == 9 ** dims
    N = 9
    if pts == 5:
        assert s.nnz == 5 * N * N - 4 * N
    elif pts == 7:
        assert s.nnz == 7 * N ** 3 - 6 * N ** 2
    else:
        assert s.nnz == (3 * N - 2) ** 3
    _m_matrix(s)
    capped = W.request_system(r, max_side=6)
    assert capped.n == 6 ** dims
