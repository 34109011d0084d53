#!/usr/bin/env python3
"""Benchmark of the GB300 int-GMRES + FP64 iterative-refinement solver.

Metric: refined solves per second to a relative residual of 1e-10 (Fig. 1
of Iwashita, Suzuki, Fukaya, ScalA'20 with the int-GMRES(m) inner solve of
Fig. 2).  Default workload, the largest single-GPU one: 3D heterogeneous
diffusion-convection, 27-point stencil on a 200^3 grid (n = 8,000,000,
nnz = 213,847,192), log-normal diffusion (sigma 2.5), convection
U[-100, 100], b ~ U[-1, 1], integer ILU(0) (Sec. VI) and GMRES(60),
synthetic data from a fixed seed.  The same line carries the 128^3 7-point
workload (GMRES(50), ILU(0)) as a secondary measurement.

One step = one ir_solve of the whole system (setup done once, inputs
resident in HBM).  The working set (matrix, factors, basis: ~20 GB, ~2 GB
for the secondary) is far larger than L2, so no flush is needed between
steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

With N > 1 (torchrun, one rank per GPU) every rank solves its own replica
(the systems are independent: weak scaling, no collective on the data
path); value = all solves / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2009_07495_gb300 import workloads as W  # noqa: E402

METRIC = "refined solves/s @1e-10 resid (int vs FP64 GMRES, 1 GB300); SpMV GB/s; p99 ms"
KNAMES = ["spmv", "trsv_l", "trsv_u", "arnoldi", "resid"]
KERNEL_SYMBOL = {"spmv": "k_spmv", "trsv_l": "k_trsv_lv", "trsv_u": "k_trsv_lv",
                 "arnoldi": "k_mgs_step_grid", "resid": "k_resid"}

WORKLOADS = {
    "cfg1": dict(desc="3D convection-diffusion 7-pt 128^3 (n=2,097,152, nnz=14,581,760), "
                      "ILU(0) int-GMRES(50), FP64 refinement to 1e-10",
                 gen=lambda: W.config1(), precond=1, m=50),
    "cfg0": dict(desc="2D convection-diffusion 5-pt 32x32 (n=1024), int-GMRES(30), no "
                      "preconditioning, FP64 refinement to 1e-10",
                 gen=lambda: W.config0(), precond=0, m=30),
    "cfg2": dict(desc="batch of 512 banded random systems, n log-uniform [1k, 64k], 5-27 "
                      "nnz/row within +-64, int-GMRES(30) no preconditioning, refinement "
                      "to 1e-10, one batched launch sequence", precond=0, m=30),
    "cfg4": dict(desc="3D heterogeneous diffusion-convection 27-pt 200^3 (n=8,000,000, "
                      "nnz~216M), log-normal diffusion sigma 2.5, convection U[-100,100], "
                      "ILU(0) int-GMRES(60), FP64 refinement to 1e-10",
                 gen=lambda: W.config4(), precond=1, m=60,
                 # the oracle's bounded sample: the same generator on a 60^3 grid
                 sample=lambda: W.config4(N=60, seed=4), sample_desc="27-pt 60^3"),
    "cfg3": dict(desc="serving stream: Poisson arrivals 2k req/s, 2D 5-pt / 3D 7-pt / 3D "
                      "27-pt convection-diffusion, sides U[16,160], Peclet log-U[0.1,100], "
                      "tol 1e-8 or 1e-10, 150 GB budget, continuous batching", m=30),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cfg4", choices=sorted(WORKLOADS))
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the 128^3 7-point secondary measurement")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--batch", type=int, default=512, help="cfg2: systems in the batch")
    ap.add_argument("--requests", type=int, default=400, help="cfg3: requests served")
    ap.add_argument("--serve-window", type=int, default=128,
                    help="cfg3: requests the client keeps in flight at most")
    ap.add_argument("--precond", type=int, default=None,
                    help="override the workload's preconditioner: 0 none, 1 ILU(0), "
                         "2 Gauss-Seidel")
    ap.add_argument("--order", type=int, default=0,
                    help="0 natural row order (the paper's), 1 multicolour order")
    ap.add_argument("--terms", type=int, default=0,
                    help="correction terms of the multi-term matrix (Sec. IV-C, s)")
    ap.add_argument("--shift-tune", type=int, default=0,
                    help="shift auto-tuning budget (Sec. VII-D): inner solves that may "
                         "be discarded and rerun with raised shifts")
    ap.add_argument("--oracle-sample", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--side", type=int, default=0,
                    help="cfg4 only: grid side of the 27-point workload (0: 200; smaller "
                         "sides are for profiling captures, not bench lines)")
    ap.add_argument("--trsv-chunk", type=int, default=0,
                    help="rows per chunk of the substitutions (0: automatic)")
    ap.add_argument("--shifts", type=int, default=None,
                    help="start the shifts of lines 7, 8, 10, 13, 15 at this value "
                         "(default: Table 4 / Table 5)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
class Clocks:
    """nvidia-smi samples (SM clock, throttle reasons) during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def peak_hbm():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return float(json.load(open(p))["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def job_throughput(local_ms: float, steps: int, dist=None, device="cpu") -> tuple:
    """Whole-job rate of independent replicas: every rank ran `steps` solves
    and the job took as long as its slowest rank (max over ranks).  Returns
    (max_ms, solves/s of all ranks together)."""
    world, ms = 1, float(local_ms)
    if dist is not None and dist.is_initialized():
        import torch
        world = dist.get_world_size()
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * steps / (ms / 1000.0)


def algorithmic_bytes(kind: str, n: int, nnz: int, nnz_l: int, val_bytes: int,
                      m: int, terms: int = 0) -> float:
    """Bytes the method must move per launch, counted as the hot-path scope
    counts them (what the method needs, not what a layout happens to move):
    SpMV nnz ((s+1) b_val + 4) + 4(n+1) + 4n (s correction terms; the basis
    vector v_j read as int32 words: the upper bits of a Q30 basis entry are
    zero, Sec. V-D).  Arnoldi step j = m-1: the m basis vectors read once
    (4n each, w kept on chip) and v_m written (4n).  One triangular solve:
    (nnz_tri + n) 12 + 16n.  FP64 residual: nnz 12 + 4(n+1) + 24n."""
    if kind == "spmv":
        return nnz * ((terms + 1) * val_bytes + 4) + 4 * (n + 1) + 4 * n
    if kind == "arnoldi":
        return 4.0 * n * (m + 1)
    if kind in ("trsv_l", "trsv_u"):
        return (nnz_l + n) * 12 + 16 * n
    if kind == "resid":
        return nnz * 12 + 4 * (n + 1) + 24 * n
    raise KeyError(kind)


def launches_per_cycle(kind: str, m: int) -> float:
    """Launches per inner solve; the Arnoldi kernel is timed at its longest
    step (m+1 passes), so its count is scaled to the average step of
    (j+2) passes, j = 0..m-1."""
    return {"spmv": m, "trsv_l": m, "trsv_u": m, "arnoldi": m * (m + 3) / 2 / (m + 1),
            "resid": 1}[kind]


def traffic_for(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if the kernel
    source has not changed since the capture."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        t = json.load(open(p))[f"{workload}:{kernel}"]
    except Exception:
        return None
    src = os.path.join(ROOT, "paper_2009_07495_gb300", "csrc", t["source"])
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    return t["bytes_per_launch"] if sha == t["sha256"] else None


# ---------------------------------------------------------------------------
def _oracle_sample_solve(name: str):
    """One complete oracle solve of a workload's bounded sample (also the
    worker of the all-core baseline, run in a spawned process)."""
    import oracle
    oracle.build()
    wl = WORKLOADS[name]
    sm = wl["sample"]()
    m = wl["m"]
    P = oracle.Params.table5(m=m) if wl["precond"] else oracle.Params.table4(m=m)
    t0 = time.perf_counter()
    x, ro = oracle.ir_solve(sm.rowptr, sm.col, sm.val, sm.b, P)
    return time.perf_counter() - t0, ro.refinements, sm.n, sm.nnz


def cpu_baseline_scaled(name: str, wl, sysw, refinements: int):
    """The oracle on a bounded sample for a workload too large to set up on
    the host within the budget: complete refined solves of the same
    generator on a smaller grid, scaled to the full system by the work of a
    solve (refinements x m Arnoldi steps of 3 nnz products -- SpMV and the
    two substitutions -- plus (m+3)/2 basis vectors of n rows on average, and
    the set-up's nnz).  One solve on one core, then one independent solve
    per host core at once (each in a process of its own): the host's
    throughput is cores / the slowest of those solves."""
    dt1, refs, n_s, nnz_s = _oracle_sample_solve(name)
    m = wl["m"]

    def work(nnz, n, refs_):
        return refs_ * m * (3.0 * nnz + 0.5 * (m + 3) * n) + nnz

    scale = work(sysw.nnz, sysw.n, refinements) / work(nnz_s, n_s, refs)
    cores = os.cpu_count() or 1
    env = dict(os.environ, OMP_NUM_THREADS="1")
    procs = [subprocess.Popen([sys.executable, os.path.abspath(__file__), "--oracle-sample", name],
                              stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True, env=env)
             for _ in range(cores)]
    dts = []
    for pr in procs:
        out, _ = pr.communicate(timeout=600)
        if pr.returncode == 0 and out.strip():
            dts.append(json.loads(out.strip().splitlines()[-1])["dt"])
    cores = max(len(dts), 1)
    dt_all = max(dts) if dts else dt1
    return {"value": cores / (dt_all * scale), "unit": "solves/s", "cores": cores,
            "kind": "oracle",
            "single_core": {"value": 1.0 / (dt1 * scale), "cores": 1},
            "sample": f"complete oracle solves ({refs} refinements) of the same generator on a "
                      f"{wl['sample_desc']} grid (n={n_s}, nnz={nnz_s}): {cores} at once, one "
                      f"per host core (slowest {dt_all:.1f} s; alone {dt1:.1f} s), scaled "
                      f"x{scale:.0f} by the work of a solve to the full system "
                      f"({refinements} refinements)"}


def cpu_baseline(sysw, precond: int, m: int, refinements: int, budget_s: float = 30.0):
    """The oracle, single-threaded, on a bounded sample: its set-up plus one
    inner solve of the full system (one of the `refinements` the full solve
    needs), extrapolated to solves/s."""
    import oracle
    oracle.build()
    P = oracle.Params.table5(m=m) if precond else oracle.Params.table4(m=m)
    t0 = time.perf_counter()
    d = oracle.setup(sysw.rowptr, sysw.col, sysw.val, sysw.b, P)
    t_setup = time.perf_counter() - t0
    bk = d["b"] / np.abs(d["b"]).max()
    t0 = time.perf_counter()
    r = oracle.resid_fp(d["rowptr"], d["col"], d["a"], np.zeros(sysw.n), d["b"])
    oracle.int_gmres(P, d, bk)
    t_cyc = time.perf_counter() - t0
    per_solve = t_setup + refinements * t_cyc
    del r
    return {"value": 1.0 / per_solve, "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": f"oracle set-up ({t_setup:.2f} s) + 1 of {refinements} refinements "
                      f"(residual + one int-GMRES({m}) solve, {t_cyc:.1f} s) of the full "
                      f"workload, extrapolated x{refinements}"}


def run_reference(args, wl):
    """--impl reference: the oracle on the host cores, same workload/metric."""
    if args.gpus > 1 and int(os.environ.get("RANK", "0")) != 0:
        return
    sysw = wl["gen"]()
    import oracle
    oracle.build()
    P = oracle.Params.table5(m=wl["m"]) if wl["precond"] else oracle.Params.table4(m=wl["m"])
    refinements = wl.get("refinements", 0)
    if "sample" in wl:
        # too large to set up on one core within minutes: complete solves of
        # the same generator on a smaller grid, scaled by the work of a solve
        steps = max(1, min(args.steps, 3))
        vals, dts = [], []
        for _ in range(steps):
            t0 = time.perf_counter()
            cb = cpu_baseline_scaled(args.workload, wl, sysw, refinements)
            dts.append(time.perf_counter() - t0)
            vals.append(cb["value"])
        value = statistics.median(vals)
        dt = sum(dts)
        sample = cb["sample"]
        cores = cb["cores"]
    elif sysw.n <= 50000:
        # small workload: whole refined solves
        steps = args.steps
        t0 = time.perf_counter()
        for _ in range(steps):
            x, rep = oracle.ir_solve(sysw.rowptr, sysw.col, sysw.val, sysw.b, P)
        dt = time.perf_counter() - t0
        value = steps / dt
        sample = f"{steps} full oracle solves"
        cores = 1
    else:
        steps = max(1, min(args.steps, 3))
        t0 = time.perf_counter()
        d = oracle.setup(sysw.rowptr, sysw.col, sysw.val, sysw.b, P)
        t_setup = time.perf_counter() - t0
        bk = d["b"] / np.abs(d["b"]).max()
        ts = []
        for _ in range(steps):
            t0 = time.perf_counter()
            oracle.resid_fp(d["rowptr"], d["col"], d["a"], np.zeros(sysw.n), d["b"])
            oracle.int_gmres(P, d, bk)
            ts.append(time.perf_counter() - t0)
        t_cyc = statistics.median(ts)
        value = 1.0 / (t_setup + refinements * t_cyc)
        dt = sum(ts)
        sample = (f"oracle set-up + {steps} inner solves (one refinement each) of the full "
                  f"workload, extrapolated to the {refinements} refinements of a solve")
        cores = 1
    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": steps, "warmup": 0, "ms_per_step": 1000.0 * dt / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int64", "data": "synthetic", "impl": "reference",
            "config": {"workload": wl["desc"]},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
def run_ours(args, wl):
    import torch
    from paper_2009_07495_gb300 import _lib as L

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    L.load()

    sysw = wl["gen"]()
    n, nnz = sysw.n, sysw.nnz
    precond = wl["precond"] if args.precond is None else args.precond
    P = L.params_default(precond, wl["m"])
    P.s = args.terms
    P.order = args.order
    P.shift_tune = args.shift_tune
    P.trsv_chunk = args.trsv_chunk
    if args.shifts is not None:
        for k in ("beta7", "beta8", "beta10", "beta13", "beta15"):
            setattr(P, k, args.shifts)
    rp = torch.from_numpy(sysw.rowptr).to(dev)
    cl = torch.from_numpy(sysw.col).to(dev)
    vl = torch.from_numpy(sysw.val).to(dev)
    bh = torch.from_numpy(sysw.b).to(dev)
    xh = torch.empty(n, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    solver = L.Solver(rp, cl, vl, P, stream=stream)
    ws_bytes = solver.device_bytes()

    def barrier():
        if dist is not None:
            dist.barrier()

    rep = None
    for _ in range(args.warmup):
        _, rep = solver.ir_solve(bh, xh, stream=stream)
    torch.cuda.synchronize(dev)
    assert rep is None or rep["status"] == "ok", rep

    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    clocks = Clocks(local)
    barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    l0 = L.load().igm_kernel_launches()
    ev[0].record(stream)
    for k in range(args.steps):
        _, rep = solver.ir_solve(bh, xh, stream=stream)
        ev[k + 1].record(stream)
    torch.cuda.synchronize(dev)
    launches = L.load().igm_kernel_launches() - l0
    barrier()
    clk = clocks.stop()
    step_ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    total_ms = ev[0].elapsed_time(ev[-1])
    total_ms, value = job_throughput(total_ms, args.steps, dist, dev)
    assert rep["status"] == "ok" and rep["relres"] < 1e-10, rep
    refinements = rep["refinements"]

    # per-kernel device time (same kernels, same launch configuration)
    import ctypes as C
    buf = (C.c_double * 5)()
    st = L.load().igm_time_kernels(solver.handle, 3, buf, stream.cuda_stream)
    if st != 0:
        raise RuntimeError(L.load().igm_last_error().decode())
    kms = np.array(buf[:])
    nnz_l = (nnz - n) // 2 if wl["precond"] else 0
    val_bytes = 8 if P.alpha_a > 30 else 4
    kern = {}
    for k, name in enumerate(KNAMES):
        if kms[k] < 0:
            continue
        per_cycle = launches_per_cycle(name, wl["m"])
        kern[name] = dict(ms=kms[k], launches_per_solve=per_cycle * refinements,
                          ms_per_solve=kms[k] * per_cycle * refinements,
                          gbs=algorithmic_bytes(name, n, nnz, nnz_l, val_bytes, wl["m"], args.terms)
                          / (kms[k] * 1e6))
    tot_k = sum(v["ms_per_solve"] for v in kern.values())
    dom = max(kern, key=lambda k: kern[k]["ms_per_solve"])
    peak, peak_src = peak_hbm()
    ach = kern[dom]["gbs"]
    roofline = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                "frac": ach / peak, "traffic": traffic_for(KERNEL_SYMBOL[dom], args.workload),
                "kernel": KERNEL_SYMBOL[dom] + (f" ({dom})" if dom.startswith("trsv") else ""),
                "peak_source": peak_src,
                "share_of_solve": kern[dom]["ms_per_solve"] / (total_ms / args.steps)}
    kernels = {k: {"ms_per_launch": round(v["ms"], 5), "algorithmic_GBs": round(v["gbs"], 1),
                   "frac_of_peak": round(v["gbs"] / peak, 4),
                   "share": round(v["ms_per_solve"] / tot_k, 4)} for k, v in kern.items()}

    # the FP64 GMRES(m) comparison solver ("Double" of Sec. VII) on the same
    # GPU, workload and refinement loop
    fp64 = None
    if not args.no_fp64:
        Pf = P.replace(inner=1)
        sf = L.Solver(rp, cl, vl, Pf, stream=stream)
        _, rf = sf.ir_solve(bh, xh, stream=stream)
        kf = max(1, min(args.steps, 3 if n < 4_000_000 else 1))
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(kf):
            _, rf = sf.ir_solve(bh, xh, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / kf
        fp64 = {"value": world * 1000.0 / ms, "unit": "solves/s", "ms_per_solve": ms,
                "refinements": rf["refinements"], "relres": rf["relres"], "steps": kf,
                "status": rf["status"]}
        sf.close()

    # the multicolour order (a GPU-motivated reordering of the preconditioner,
    # not the paper's natural order) on the same workload, for comparison
    variant = None
    if not args.no_fp64 and args.order == 0 and precond != 0 and n < 4_000_000:
        Pm = P.replace(order=1)
        sm_ = L.Solver(rp, cl, vl, Pm, stream=stream)
        _, rm = sm_.ir_solve(bh, xh, stream=stream)
        km = max(1, min(args.steps, 3))
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(km):
            _, rm = sm_.ir_solve(bh, xh, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / km
        variant = {"order": "multicolour", "value": world * 1000.0 / ms, "unit": "solves/s",
                   "ms_per_solve": ms, "refinements": rm["refinements"], "relres": rm["relres"],
                   "steps": km, "status": rm["status"]}
        sm_.close()

    # end to end through the C ABI with host buffers: set-up from pinned host
    # CSR + solve from a pinned host right-hand side + solution back to host
    e2e = None
    if args.e2e_steps > 0:
        hrp = torch.from_numpy(sysw.rowptr).pin_memory()
        hcl = torch.from_numpy(sysw.col).pin_memory()
        hvl = torch.from_numpy(sysw.val).pin_memory()
        hb = torch.from_numpy(sysw.b).pin_memory()
        hx = torch.empty(n, dtype=torch.float64).pin_memory()
        solver.close()
        torch.cuda.synchronize(dev)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            s2 = L.Solver(hrp, hcl, hvl, P, stream=stream)
            _, r2 = s2.ir_solve(hb, hx, stream=stream)
            s2.close()
        torch.cuda.synchronize(dev)
        dt = time.perf_counter() - t0
        assert r2["status"] == "ok"
        e2e = {"value": world * args.e2e_steps / dt, "unit": "solves/s",
               "h2d_bytes_per_step": int(4 * (n + 1) + 4 * nnz + 8 * nnz + 8 * n),
               "d2h_bytes_per_step": int(8 * n + 1192),
               "includes": "int_gmres_setup (scaling, cast, ILU(0)) + ir_solve + destroy"}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int64", "data": "synthetic",
            "config": {"workload": wl["desc"], "n": n, "nnz": nnz, "m": wl["m"],
                       "refinements": refinements, "relres": rep["relres"], "terms_s": args.terms,
                       "precond": ["none", "ILU(0)", "Gauss-Seidel"][precond],
                       "order": ["natural", "multicolour"][args.order],
                       "inner_steps": rep["inner_steps"],
                       "shift_tune": args.shift_tune,
                       "shifts_start": [P.beta7, P.beta8, P.beta10, P.beta13, P.beta15],
                       "shift_retries": rep["shift_retries"],
                       "shifts_final": list(rep["beta_final"]),
                       "arnoldi_launch": {"fuse_steps": rep["fuse_steps"],
                                          "plan_snap": rep["plan_snap"]},
                       "l2": f"working set (~{ws_bytes / 1e9:.0f} GB) > L2 "
                             "(129 MB), no flush",
                       "parallelism": f"replicas x{world}"},
            "p50_ms": float(np.percentile(step_ms, 50)),
            "p99_ms": float(np.percentile(step_ms, 99)),
            "spmv_GBs": kern["spmv"]["gbs"],
            "roofline": roofline, "kernels": kernels,
            "clocks": clk, "gpu_launches": int(launches), "e2e": e2e,
            "fp64_gmres": fp64, "multicolour_variant": variant}
    if not args.no_cpu_baseline and world == 1:
        if "sample" in wl:
            line["cpu_baseline"] = cpu_baseline_scaled(args.workload, wl, sysw, refinements)
        else:
            line["cpu_baseline"] = cpu_baseline(sysw, wl["precond"], wl["m"], refinements)
    if args.workload == "cfg4" and not args.no_secondary:
        line["secondary"] = secondary_cfg1(L, dev, stream, world, args.terms)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def secondary_cfg1(L, dev, stream, world, terms, steps=3, warmup=2):
    """The 128^3 7-point workload (ILU(0), GMRES(50)) measured the same way
    as the headline: refined solves/s over `steps` solves after `warmup`,
    and the per-kernel times with their algorithmic bandwidth."""
    import torch
    import ctypes as C
    wl = WORKLOADS["cfg1"]
    sysw = wl["gen"]()
    n, nnz, m = sysw.n, sysw.nnz, wl["m"]
    P = L.params_default(1, m)
    rp, cl, vl, bh = [torch.from_numpy(a).to(dev) for a in (sysw.rowptr, sysw.col, sysw.val,
                                                              sysw.b)]
    xh = torch.empty(n, dtype=torch.float64, device=dev)
    sv = L.Solver(rp, cl, vl, P, stream=stream)
    for _ in range(warmup):
        _, rep = sv.ir_solve(bh, xh, stream=stream)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        _, rep = sv.ir_solve(bh, xh, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / steps
    assert rep["status"] == "ok" and rep["relres"] < 1e-10, rep
    buf = (C.c_double * 5)()
    if L.load().igm_time_kernels(sv.handle, 3, buf, stream.cuda_stream) != 0:
        raise RuntimeError(L.load().igm_last_error().decode())
    peak, _ = peak_hbm()
    kern = {}
    for k, name in enumerate(KNAMES):
        if buf[k] < 0:
            continue
        gbs = algorithmic_bytes(name, n, nnz, (nnz - n) // 2, 8, m, terms) / (buf[k] * 1e6)
        kern[name] = {"ms_per_launch": round(buf[k], 5), "algorithmic_GBs": round(gbs, 1),
                      "frac_of_peak": round(gbs / peak, 4)}
    sv.close()
    return {"workload": wl["desc"], "value": world * 1000.0 / ms, "unit": "solves/s",
            "ms_per_step": ms, "steps": steps, "warmup": warmup,
            "refinements": rep["refinements"], "relres": rep["relres"], "kernels": kern}


def run_batched(args, wl):
    """cfg2: ir_solve_batched over all systems vs one ir_solve per system
    (same kernels, one system per launch sequence) vs the FP64 solver."""
    import torch
    from paper_2009_07495_gb300 import _lib as L
    dev = torch.device("cuda", 0)
    systems = W.config2(count=args.batch)
    P = L.params_default(0, wl["m"])
    solvers, bs, xs = [], [], []
    for sy in systems:
        solvers.append(L.Solver(torch.from_numpy(sy.rowptr).to(dev), torch.from_numpy(sy.col).to(dev),
                                torch.from_numpy(sy.val).to(dev), P))
        bs.append(torch.from_numpy(sy.b).to(dev))
        xs.append(torch.empty(sy.n, dtype=torch.float64, device=dev))
    reps = L.ir_solve_batched(solvers, bs, xs)          # warm-up (graph capture)
    torch.cuda.synchronize()
    clocks = Clocks(0)
    clocks.start()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        reps = L.ir_solve_batched(solvers, bs, xs)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / args.steps
    clk = clocks.stop()
    assert all(r["status"] == "ok" and r["relres"] < 1e-10 for r in reps)
    # one solve per launch sequence
    for k in range(len(solvers)):
        solvers[k].ir_solve(bs[k], xs[k])
    torch.cuda.synchronize()
    lat = []
    t0 = time.perf_counter()
    for k in range(len(solvers)):
        t1 = time.perf_counter()
        solvers[k].ir_solve(bs[k], xs[k])
        lat.append(time.perf_counter() - t1)
    torch.cuda.synchronize()
    dt_one = time.perf_counter() - t0
    for sv in solvers:
        sv.close()
    # the FP64 comparison solver, batched
    Pf = P.replace(inner=1)
    fsolv = [L.Solver(torch.from_numpy(sy.rowptr).to(dev), torch.from_numpy(sy.col).to(dev),
                      torch.from_numpy(sy.val).to(dev), Pf) for sy in systems]
    L.ir_solve_batched(fsolv, bs, xs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rf = L.ir_solve_batched(fsolv, bs, xs)
    torch.cuda.synchronize()
    dt_f = time.perf_counter() - t0
    for sv in fsolv:
        sv.close()
    nsys = len(systems)
    line = {"metric": METRIC, "value": nsys / dt, "unit": "solves/s", "n_gpus": 1,
            "steps": args.steps, "warmup": 1, "ms_per_step": 1000 * dt, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": wl["desc"], "systems": nsys, "rows": int(sum(x.n for x in systems)),
                       "nnz": int(sum(x.nnz for x in systems)),
                       "refinements_max": max(r["refinements"] for r in reps),
                       "arnoldi_launch": {"fuse_steps": reps[0]["fuse_steps"],
                                          "plan_snap": reps[0]["plan_snap"],
                                          "chosen_by": "autotuner"}},
            "one_solve_per_launch": {"value": nsys / dt_one, "unit": "solves/s",
                                     "p50_ms": 1000 * float(np.percentile(lat, 50)),
                                     "p99_ms": 1000 * float(np.percentile(lat, 99))},
            "fp64_gmres_batched": {"value": nsys / dt_f, "unit": "solves/s",
                                   "ok": all(r["status"] == "ok" for r in rf)},
            "clocks": clk}
    print(json.dumps(line), flush=True)


def run_serve(args, wl):
    """cfg3: the first --requests requests of the serving stream.  Request k
    arrives at its Poisson time and is submitted once it has arrived and
    fewer than --serve-window requests are in flight, so that host memory
    holds only the window's matrices (at 2000 req/s the whole stream
    arrives within seconds, far faster than it can be solved).  Host
    processes build the matrices ahead, in order (at most 64 ready).  A
    request's latency runs from its arrival time to its completion, so the
    wait in the client's window counts as queueing."""
    import concurrent.futures as cf
    import multiprocessing as mp
    from paper_2009_07495_gb300 import _lib as L
    reqs = W.config3_requests()[: args.requests]
    m = wl["m"]
    srv = L.Server(budget_bytes=150 * (1 << 30), m=m)
    # host processes (spawned: this process already uses the GPU) build the
    # matrices
    pool = cf.ProcessPoolExecutor(max(2, (os.cpu_count() or 4) - 2),
                                  mp_context=mp.get_context("spawn"))
    ahead = {}  # request index -> future of its system

    def build_ahead(k0):
        for kk in range(k0, min(len(reqs), k0 + min(args.serve_window, 64))):
            if kk not in ahead:
                ahead[kk] = pool.submit(W.request_system, reqs[kk])

    build_ahead(0)
    t0 = time.perf_counter()
    pending = {}  # id -> (arrival time, submit time)
    lats, oks, rows_total, k = [], 0, 0, 0
    clocks = Clocks(0)
    clocks.start()
    while k < len(reqs) or pending:
        now = time.perf_counter() - t0
        while k < len(reqs) and len(pending) < args.serve_window and reqs[k].arrival_s <= now:
            r = reqs[k]
            sy = ahead.pop(k).result()
            build_ahead(k + 1)
            P = L.params_default(0 if r.kind == "2d5" else 1, m, tol=r.tol)
            ts = time.perf_counter() - t0
            pending[srv.submit(sy.rowptr, sy.col, sy.val, sy.b, P)] = (r.arrival_s, ts)
            rows_total += sy.n
            del sy
            k += 1
            now = time.perf_counter() - t0
        finished = 0
        for i in list(pending):
            done, x, rep, lat = srv.poll(i, wait_ms=0)
            if not done:
                continue
            arr, ts = pending.pop(i)
            lats.append(ts + lat - arr)
            oks += rep["status"] == "ok"
            finished += 1
        if not finished:
            nxt = reqs[k].arrival_s - now if k < len(reqs) and len(pending) < args.serve_window \
                else 0.005
            time.sleep(min(max(nxt, 0.0), 0.005))
    dt = time.perf_counter() - t0
    clk = clocks.stop()
    st = srv.stats()
    srv.close()
    pool.shutdown()
    n = len(reqs)
    line = {"metric": METRIC, "value": n / dt, "unit": "solves/s", "n_gpus": 1,
            "steps": n, "warmup": 0, "ms_per_step": 1000 * dt / n,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic",
            "config": {"workload": wl["desc"], "requests": n, "offered_rate": 2000.0,
                       "client_window": args.serve_window, "rows_total": int(rows_total)},
            "p50_ms": 1000 * float(np.percentile(lats, 50)),
            "p99_ms": 1000 * float(np.percentile(lats, 99)),
            "completed_ok": oks, "wall_s": dt, "server": st, "clocks": clk}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.side and args.workload == "cfg4":
        side = args.side
        WORKLOADS["cfg4"] = dict(WORKLOADS["cfg4"], gen=lambda: W.config4(N=side),
                                 desc=WORKLOADS["cfg4"]["desc"].replace(
                                     "200^3 (n=8,000,000, nnz~216M)", f"{side}^3 (n={side ** 3:,})"))
    if args.oracle_sample:  # one worker of the all-core CPU baseline
        dt, refs, n, nnz = _oracle_sample_solve(args.oracle_sample)
        print(json.dumps({"dt": dt, "refinements": refs}), flush=True)
        return
    wl = dict(WORKLOADS[args.workload])
    if args.impl == "reference":
        wl["refinements"] = REFINEMENTS.get(args.workload, 4)
        run_reference(args, wl)
    elif args.workload == "cfg2":
        run_batched(args, wl)
    elif args.workload == "cfg3":
        run_serve(args, wl)
    else:
        run_ours(args, wl)


# refinements a full solve of each workload takes (identical for the oracle
# and the CUDA path, which agree bit for bit); used only to extrapolate the
# reference arm's bounded sample
REFINEMENTS = {"cfg1": 6, "cfg0": 9, "cfg4": 4}

if __name__ == "__main__":
    main()
