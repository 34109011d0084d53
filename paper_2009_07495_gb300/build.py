"""Builds the CUDA library libigm.so in-tree for sm_103a (GB300).

Each .cu translation unit is compiled by nvcc in parallel and linked into
one shared library with the CUDA runtime linked statically, so the library
has no dependency on the Python process beyond the NVIDIA driver.

Build variants (environment variable IGM_BUILD, or build(variant=...)), each
in its own folder under _build/ with the same exports:
  ""             the product library (_build/libigm.so)
  "checks"       device bounds and alignment checks on the copies and
                 gathers (-DIGM_CHECKS): a failed check skips the access and
                 the solve returns IGM_ECUDA naming the site
  "nvtx"         NVTX ranges around the host-side phases (-DIGM_NVTX)
  "checks+nvtx"  both
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
VARIANTS = {"": [], "checks": ["-DIGM_CHECKS"], "nvtx": ["-DIGM_NVTX"],
            "checks+nvtx": ["-DIGM_CHECKS", "-DIGM_NVTX"]}
VARIANT = os.environ.get("IGM_BUILD", "")
if VARIANT not in VARIANTS:
    raise ValueError(f"IGM_BUILD={VARIANT!r}: expected one of {sorted(VARIANTS)}")


def out_dir(variant: str) -> str:
    return OUT if not variant else os.path.join(OUT, variant.replace("+", "_"))


LIB = os.path.join(out_dir(VARIANT), "libigm.so")
ROOT = os.path.dirname(HERE)
HEADERS = [os.path.join(ROOT, "include", "igm.h")]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-fmad=false", "-Xcompiler", "-fPIC",
         "-Xcompiler", "-O2", "--expt-relaxed-constexpr"]


def _nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libigm")
    return p


def sources() -> list[str]:
    return sorted(os.path.join(SRC, f) for f in os.listdir(SRC) if f.endswith(".cu"))


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, variant: str | None = None) -> str:
    """Compile (if needed) and return the path of libigm.so (of the variant
    named by IGM_BUILD unless one is given)."""
    variant = VARIANT if variant is None else variant
    out = out_dir(variant)
    lib = os.path.join(out, "libigm.so")
    flags = FLAGS + VARIANTS[variant]
    os.makedirs(out, exist_ok=True)
    nvcc = _nvcc()
    hdrs = [os.path.join(SRC, f) for f in os.listdir(SRC) if f.endswith((".h", ".cuh"))]
    hdrs += HEADERS
    objs, jobs = [], []
    for src in sources():
        obj = os.path.join(out, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        if force or _stale(obj, [src] + hdrs):
            cmd = [nvcc, *ARCH, *flags, "-c", src, "-o", obj]
            jobs.append(cmd)

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr)

    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(8, len(jobs))) as ex:
            list(ex.map(run, jobs))
    if force or jobs or _stale(lib, objs):
        tmp = lib + f".{os.getpid()}.tmp"
        run([nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs])
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(verbose=True))
