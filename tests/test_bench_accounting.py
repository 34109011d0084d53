"""The benchmark's roofline bookkeeping on the CPU: the algorithmic bytes of
each kernel equal the sizes of the arrays the method must read and write
once (counted here from the data structures of a synthetic system), and a
stored DRAM traffic figure is used only while its kernel source is the one
it was measured on."""
import hashlib
import json

import numpy as np
import pytest

import bench
from paper_2009_07495_gb300 import workloads as W


@pytest.fixture(scope="module")
def sysw():
    return W.small_cd3d(12, seed=3)


def test_spmv_bytes_are_the_arrays_it_touches(sysw):
    n, nnz = sysw.n, sysw.nnz
    i64, i32 = np.dtype(np.int64).itemsize, np.dtype(np.int32).itemsize
    # values (int64, alpha_a = 32) and columns once, the row pointers and
    # the basis vector v_j as 32-bit words (the upper bits of a Q30 basis
    # entry are zero, Sec. V-D); the hot-path scope does not count w out
    want = nnz * i64 + sysw.col.nbytes + sysw.rowptr.nbytes + n * i32
    assert sysw.col.dtype.itemsize == i32
    assert bench.algorithmic_bytes("spmv", n, nnz, 0, 8, 50) == want
    # s correction terms: one more value array per term, same columns
    assert bench.algorithmic_bytes("spmv", n, nnz, 0, 8, 50, terms=2) == want + 2 * nnz * i64


def test_arnoldi_and_substitution_bytes(sysw):
    n, nnz, m = sysw.n, sysw.nnz, 30
    # step j = m - 1: basis vectors v_0 .. v_{m-1} read once and v_m written,
    # 32-bit words each; w stays on chip
    assert bench.algorithmic_bytes("arnoldi", n, nnz, 0, 8, m) == 4 * n * m + 4 * n
    # one triangle: strict entries (int64 factor + int32 column), each row's
    # diagonal (int64) and schedule index (int32), the input and output
    # vectors (the division multipliers are this implementation's, not the
    # method's, and are not counted)
    nnz_l = (nnz - n) // 2
    want = nnz_l * (8 + 4) + n * (8 + 4) + 8 * n + 8 * n
    assert bench.algorithmic_bytes("trsv_l", n, nnz, nnz_l, 8, m) == want


def test_arnoldi_launch_scaling_is_the_mean_step():
    # steps j = 0 .. m-1 make j + 2 passes; the timed step (j = m-1) makes
    # m + 1, so one timed launch stands for sum(j + 2) / (m + 1) launches
    for m in (1, 30, 50):
        mean = sum(j + 2 for j in range(m)) / (m + 1)
        assert bench.launches_per_cycle("arnoldi", m) == pytest.approx(mean)


def test_stored_traffic_only_for_the_measured_source(tmp_path, monkeypatch):
    src = tmp_path / "paper_2009_07495_gb300" / "csrc"
    src.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    (src / "k.cu").write_bytes(b"kernel source as profiled\n")
    sha = hashlib.sha256((src / "k.cu").read_bytes()).hexdigest()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(
        {"cfgX:k_x": {"bytes_per_launch": 123, "source": "k.cu", "sha256": sha}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_for("k_x", "cfgX") == 123
    assert bench.traffic_for("k_y", "cfgX") is None
    (src / "k.cu").write_bytes(b"kernel source changed since\n")
    assert bench.traffic_for("k_x", "cfgX") is None
