"""Seeded synthetic linear systems shaped like the paper's test problems.

The paper (Sec. VII-A, Table "matInfo") solves ten unsymmetric SuiteSparse
matrices, mostly from CFD and PDE discretisations, with 7-17 non-zeros per
row.  Those matrices are not available here, so these generators build
nonsymmetric convection-diffusion systems and banded random systems of the
same character.  This module holds no arithmetic of the method itself: it
only produces the input matrix in CSR form (ahat, FP64) and a right-hand
side (bhat), for the oracle, the CUDA path and the benchmark alike.

All systems are M-matrices or strictly diagonally dominant, hence
non-singular, and have a stored diagonal in every row (needed by ILU(0)).
Column indices are sorted within each row.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class System:
    """One linear system Ahat xhat = bhat in CSR form (FP64)."""
    n: int
    rowptr: np.ndarray   # int32 [n+1]
    col: np.ndarray      # int32 [nnz]
    val: np.ndarray      # float64 [nnz]
    b: np.ndarray        # float64 [n]
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def dense(self) -> np.ndarray:
        a = np.zeros((self.n, self.n))
        for i in range(self.n):
            s, e = self.rowptr[i], self.rowptr[i + 1]
            a[i, self.col[s:e]] = self.val[s:e]
        return a

    def matvec(self, x: np.ndarray) -> np.ndarray:
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        return np.bincount(rows, weights=self.val * x[self.col], minlength=self.n)


def _assemble(shape, offsets, coef, diag):
    """CSR of a stencil matrix on a grid of `shape` (x fastest).

    offsets: list of integer offset tuples (one per neighbour);
    coef: list of float arrays (one value per grid point, the coefficient to
    the neighbour at that offset; only used where the neighbour exists);
    diag: float array, the diagonal.  Rows are in natural (lexicographic)
    order and columns come out sorted.
    """
    dims = len(shape)
    n = int(np.prod(shape))
    idx = np.arange(n, dtype=np.int64)
    coords = []
    rem = idx.copy()
    for d in range(dims):
        coords.append(rem % shape[d])
        rem //= shape[d]
    strides = [int(np.prod(shape[:d])) for d in range(dims)]
    entries = [(0, (0,) * dims, diag)]
    for off, c in zip(offsets, coef):
        lin = sum(o * s for o, s in zip(off, strides))
        entries.append((lin, tuple(off), c))
    entries.sort(key=lambda e: e[0])
    # one (row, entry) table in entry order (= column order), compacted row
    # by row
    lins = np.array([e[0] for e in entries], dtype=np.int64)
    offs = np.array([e[1] for e in entries], dtype=np.int64)  # (E, dims)
    m2 = np.ones((n, len(entries)), dtype=bool)
    for d in range(dims):
        q = coords[d][:, None] + offs[None, :, d]
        m2 &= (q >= 0) & (q < shape[d])
    counts = m2.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    c2 = (idx[:, None] + lins[None, :]).astype(np.int32)
    v2 = np.stack([e[2] for e in entries], axis=1)
    return rowptr.astype(np.int32), c2[m2], v2[m2]


def _harmonic(k1, k2):
    return 2.0 * k1 * k2 / (k1 + k2)


def convection_diffusion(shape, kappa, conv, points: int = 0):
    """Upwind finite-difference convection-diffusion on the unit square/cube,
    h = 1/(N+1) per axis, zero Dirichlet boundary.

    kappa: per-cell diffusion (array of n); a face uses the harmonic mean of
    its two cells, a boundary face the cell's own value.  conv: per-cell
    convection, shape (dims, n), discretised by first-order upwinding on
    each axis: A_PP += |c_d|/h and A_{P, P - sgn(c_d) e_d} -= |c_d|/h.
    points: 0 for the (2 dims + 1)-point stencil; 27 for the 3D 27-point
    stencil whose 26 neighbours o get kappa_f / (h^2 |o|^2) * {1, 1/2, 1/4}
    for |o|^2 = 1, 2, 3.  The result is a nonsymmetric M-matrix.
    """
    import itertools
    dims = len(shape)
    n = int(np.prod(shape))
    hs = [1.0 / (s + 1) for s in shape]
    idx = np.arange(n, dtype=np.int64)
    coords, rem = [], idx.copy()
    for d in range(dims):
        coords.append(rem % shape[d])
        rem //= shape[d]
    strides = [int(np.prod(shape[:d])) for d in range(dims)]
    kappa = np.asarray(kappa, dtype=np.float64)
    conv = np.asarray(conv, dtype=np.float64).reshape(dims, n)
    if points == 27:
        nbrs = [o for o in itertools.product((-1, 0, 1), repeat=3) if any(o)]
    else:
        nbrs = []
        for d in range(dims):
            for s in (-1, 1):
                o = [0] * dims
                o[d] = s
                nbrs.append(tuple(o))
    diag = np.zeros(n)
    coefs = []
    for o in nbrs:
        inside = np.ones(n, dtype=bool)
        for d in range(dims):
            if o[d]:
                q = coords[d] + o[d]
                inside &= (q >= 0) & (q < shape[d])
        lin = sum(oo * s for oo, s in zip(o, strides))
        kn = np.where(inside, kappa[np.clip(idx + lin, 0, n - 1)], kappa)
        kf = _harmonic(kappa, kn)
        r2 = sum(abs(v) for v in o)
        if points == 27:
            w = kf / (hs[0] ** 2 * r2) * {1: 1.0, 2: 0.5, 3: 0.25}[r2]
        else:
            axis = [d for d in range(dims) if o[d]][0]
            w = kf / hs[axis] ** 2
        diag += w
        c = -w
        if r2 == 1:
            axis = [d for d in range(dims) if o[d]][0]
            a = np.abs(conv[axis]) / hs[axis]
            # the upwind neighbour of P on this axis is P - sgn(c) e_axis
            c = c - np.where(np.sign(conv[axis]) == -o[axis], a, 0.0)
        coefs.append(c)
    for d in range(dims):
        diag += np.abs(conv[d]) / hs[d]
    return _assemble(shape, nbrs, coefs, diag)


def config0() -> System:
    """2D convection-diffusion, 5-point upwind stencil on a 32x32 grid,
    kappa = 1, constant convection (20, -10), b = A * ones."""
    shape = (32, 32)
    n = 32 * 32
    conv = np.stack([np.full(n, 20.0), np.full(n, -10.0)])
    rowptr, col, val = convection_diffusion(shape, np.ones(n), conv)
    s = System(n, rowptr, col, val, np.zeros(n), "cd2d_5pt_32x32")
    s.b = s.matvec(np.ones(n))
    return s


def config1(N: int = 128, seed: int = 1) -> System:
    """3D convection-diffusion, 7-point stencil on an N^3 grid, per-cell
    convection components iid U[-50, 50], log-normal diffusion (sigma 1),
    b ~ U[-1, 1].  N = 128 gives n = 2,097,152 and nnz = 14,581,760."""
    rng = np.random.default_rng(seed)
    n = N ** 3
    kappa = rng.lognormal(0.0, 1.0, n)
    conv = rng.uniform(-50.0, 50.0, (3, n))
    b = rng.uniform(-1.0, 1.0, n)
    rowptr, col, val = convection_diffusion((N, N, N), kappa, conv)
    return System(n, rowptr, col, val, b, f"cd3d_7pt_{N}^3")


def config4(N: int = 200, seed: int = 4) -> System:
    """3D heterogeneous diffusion-convection, 27-point stencil on an N^3 grid,
    log-normal diffusion with sigma 2.5, convection U[-100, 100]."""
    rng = np.random.default_rng(seed)
    n = N ** 3
    kappa = rng.lognormal(0.0, 2.5, n)
    conv = rng.uniform(-100.0, 100.0, (3, n))
    b = rng.uniform(-1.0, 1.0, n)
    rowptr, col, val = convection_diffusion((N, N, N), kappa, conv, points=27)
    return System(n, rowptr, col, val, b, f"cd3d_27pt_{N}^3")


def banded_random(n: int, rng: np.random.Generator, bw: int = 64,
                  nnz_lo: int = 5, nnz_hi: int = 27) -> System:
    """Banded random nonsymmetric system: each row has 5..27 non-zeros
    (diagonal included) at distinct columns within |i - j| <= bw, N(0,1)
    off-diagonals, diagonal = (sum of |off-diagonals|) * U(1.05, 2.0),
    b = A x_true with x_true ~ N(0, 1)."""
    k = rng.integers(nnz_lo, nnz_hi + 1, n)          # non-zeros per row
    cand = np.concatenate([np.arange(-bw, 0), np.arange(1, bw + 1)])
    rows_out, cols_out = [], []
    step = max(1, (1 << 22) // cand.size)             # bound the temporary arrays
    for r0 in range(0, n, step):
        r1 = min(n, r0 + step)
        i = np.arange(r0, r1)
        order = np.argsort(rng.random((r1 - r0, cand.size)), axis=1)
        off = cand[order]
        valid = (i[:, None] + off >= 0) & (i[:, None] + off < n)
        rank = np.cumsum(valid, axis=1) - 1
        keep = valid & (rank < (k[r0:r1] - 1)[:, None])
        rr = np.repeat(i, keep.sum(axis=1))
        rows_out += [rr, i]
        cols_out += [(i[:, None] + off)[keep], i]
    rix = np.concatenate(rows_out)
    col = np.concatenate(cols_out)
    o = np.lexsort((col, rix))
    rix, col = rix[o], col[o].astype(np.int32)
    counts = np.bincount(rix, minlength=n)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    val = rng.standard_normal(col.size)
    isd = col == rix
    offsum = np.bincount(rix, weights=np.where(isd, 0.0, np.abs(val)), minlength=n)
    dscale = rng.uniform(1.05, 2.0, n)
    val[isd] = np.maximum(offsum, 1.0) * dscale
    s = System(n, rowptr.astype(np.int32), col, val, np.zeros(n), f"banded_{n}")
    xt = rng.standard_normal(n)
    s.b = s.matvec(xt)
    return s


def config2(count: int = 512, seed: int = 2, n_lo: int = 1000,
            n_hi: int = 64000) -> list[System]:
    """Batch of independent banded random systems with n log-uniform in
    [n_lo, n_hi] (1k..64k for the full batch of 512)."""
    rng = np.random.default_rng(seed)
    ns = np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), count)).astype(np.int64)
    return [banded_random(int(n), rng) for n in ns]


@dataclass
class Request:
    """One solve request of the serving stream."""
    arrival_s: float
    kind: str          # "2d5", "3d7" or "3d27"
    side: int
    peclet: float
    tol: float
    seed: int


def config3_requests(count: int = 10000, rate: float = 2000.0, seed: int = 3,
                     side_lo: int = 16, side_hi: int = 160) -> list[Request]:
    """Poisson arrivals (mean `rate` per second); each request is a 2D
    5-point or 3D 7/27-point convection-diffusion problem with grid sides
    U[side_lo, side_hi] (3D sides capped so n stays moderate), Peclet number
    log-uniform in [0.1, 100], tolerance 1e-8 or 1e-10."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, count))
    kinds = rng.choice(["2d5", "3d7", "3d27"], count)
    sides = rng.integers(side_lo, side_hi + 1, count)
    pe = np.exp(rng.uniform(math.log(0.1), math.log(100.0), count))
    tols = rng.choice([1e-8, 1e-10], count)
    return [Request(float(t[i]), str(kinds[i]), int(sides[i]), float(pe[i]),
                    float(tols[i]), int(seed * 1000003 + i)) for i in range(count)]


def request_system(r: Request, max_side: int | None = None) -> System:
    """The system of one serving request: kappa = 1 and |c| = 2 Pe / h in a
    random direction (Pe = |c| h / (2 kappa)).  max_side caps the grid side
    (for reduced test streams)."""
    rng = np.random.default_rng(r.seed)
    side = r.side if max_side is None else min(r.side, max_side)
    if r.kind == "2d5":
        shape = (side, side)
        pts = 0
    else:
        shape = (side, side, side)
        pts = 27 if r.kind == "3d27" else 0
    dims = len(shape)
    n = int(np.prod(shape))
    h = 1.0 / (shape[0] + 1)
    d = rng.standard_normal(dims)
    d /= np.linalg.norm(d)
    cmag = 2.0 * r.peclet / h
    conv = np.repeat((d * cmag)[:, None], n, axis=1)
    rowptr, col, val = convection_diffusion(shape, np.ones(n), conv, points=pts)
    b = rng.uniform(-1.0, 1.0, n)
    return System(n, rowptr, col, val, b, f"req_{r.kind}_{shape[0]}")


def small_cd2d(N: int, conv=(20.0, -10.0), seed: int | None = None) -> System:
    """Small 2D 5-point convection-diffusion system (tests)."""
    n = N * N
    if seed is None:
        kappa = np.ones(n)
        c = np.stack([np.full(n, conv[0]), np.full(n, conv[1])])
        b = None
    else:
        rng = np.random.default_rng(seed)
        kappa = rng.lognormal(0.0, 1.0, n)
        c = rng.uniform(-50.0, 50.0, (2, n))
        b = rng.uniform(-1.0, 1.0, n)
    rowptr, col, val = convection_diffusion((N, N), kappa, c)
    s = System(n, rowptr, col, val, np.zeros(n), f"cd2d_{N}")
    s.b = s.matvec(np.ones(n)) if b is None else b
    return s


def small_cd3d(N: int, seed: int = 11, points: int = 0) -> System:
    """Small 3D convection-diffusion system like the large 3D configs."""
    rng = np.random.default_rng(seed)
    n = N ** 3
    kappa = rng.lognormal(0.0, 1.0, n)
    conv = rng.uniform(-50.0, 50.0, (3, n))
    b = rng.uniform(-1.0, 1.0, n)
    rowptr, col, val = convection_diffusion((N, N, N), kappa, conv, points=points)
    return System(n, rowptr, col, val, b, f"cd3d_{N}")


def from_dense(a: np.ndarray, b: np.ndarray, name: str = "dense") -> System:
    """CSR of a small dense matrix (explicit zeros dropped, diagonal kept)."""
    n = a.shape[0]
    rows, cols, vals = [], [], []
    rowptr = [0]
    for i in range(n):
        for j in range(n):
            if a[i, j] != 0.0 or i == j:
                cols.append(j)
                vals.append(a[i, j])
        rowptr.append(len(cols))
    return System(n, np.array(rowptr, np.int32), np.array(cols, np.int32),
                  np.array(vals, np.float64), np.asarray(b, np.float64), name)
