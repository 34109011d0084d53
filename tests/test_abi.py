"""The C-ABI library loads and exports every entry point of include/igm.h,
and the binding's structs match the header (no GPU needed)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "igm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", src, re.M)
    return sorted({n for n in names if n not in ("if", "while", "for", "return")})


@pytest.fixture(scope="module")
def lib():
    from paper_2009_07495_gb300 import _lib as L
    from paper_2009_07495_gb300 import build
    build.build()
    return L.load()


def test_exports_every_declared_symbol(lib):
    names = _declared_functions()
    assert "int_gmres_setup" in names and "ir_solve" in names and "int_gmres_solve" in names
    for n in names:
        assert hasattr(lib, n), f"libigm.so does not export {n}"


def test_checked_and_nvtx_build_exports(lib):
    """The build variant with device bounds and alignment checks and NVTX
    ranges (build.py IGM_BUILD=checks+nvtx) compiles for sm_103a and its
    library loads and exports every entry point of the header (no GPU)."""
    import ctypes as C
    from paper_2009_07495_gb300 import build
    path = build.build(variant="checks+nvtx")
    assert path != build.LIB and os.path.exists(path)
    var = C.CDLL(path)
    for n in _declared_functions():
        assert hasattr(var, n), f"the checks+nvtx build does not export {n}"


def test_default_params_are_the_papers(lib):
    """igm_params_default follows Table 4 / Table 5 and Sec. VII-B (host-only
    call, no device work)."""
    from paper_2009_07495_gb300 import _lib as L
    p = L.params_default(0, 30)
    assert (p.df, p.alpha_a, p.beta7, p.beta8, p.beta10) == (30, 16, 16, 16, 16)
    assert (p.beta11a, p.beta11b, p.beta13, p.beta15, p.beta16a, p.beta16b) == (16, 14, 16, 16, 16, 14)
    q = L.params_default(1, 50)
    assert (q.alpha_a, q.beta7, q.beta11a, q.beta11b, q.beta16a, q.m) == (32, 0, 30, 0, 30, 50)
    # the paper's method by default: natural order, s = 0, fixed shifts,
    # integer inner solver, tol 1e-10
    for r in (p, q):
        assert (r.order, r.s, r.shift_tune, r.inner, r.tol) == (0, 0, 0, 0, 1e-10)


def test_struct_layouts(tmp_path):
    """ctypes mirrors of igm_params / igm_report have the sizes and field
    offsets that a C compiler gives the header's structs."""
    import ctypes as C
    import subprocess
    from paper_2009_07495_gb300 import _lib as L
    src = tmp_path / "sz.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "igm.h"\n'
        'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n",'
        ' sizeof(igm_params),'
        ' sizeof(igm_report), offsetof(igm_params, tol), offsetof(igm_params, inner),'
        ' offsetof(igm_report, relres), offsetof(igm_report, relres_hist),'
        ' offsetof(igm_params, shift_tune), offsetof(igm_report, shift_retries),'
        ' offsetof(igm_report, beta_final), offsetof(igm_params, mgs_wmax),'
        ' offsetof(igm_params, test_stall), offsetof(igm_params, plan_snap),'
        ' offsetof(igm_report, plan_snap)); return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    assert got == [C.sizeof(L.Params), C.sizeof(L.Report), L.Params.tol.offset,
                   L.Params.inner.offset, L.Report.relres.offset, L.Report.relres_hist.offset,
                   L.Params.shift_tune.offset, L.Report.shift_retries.offset,
                   L.Report.beta_final.offset, L.Params.mgs_wmax.offset,
                   L.Params.test_stall.offset, L.Params.plan_snap.offset,
                   L.Report.plan_snap.offset]


def test_no_oracle_in_product_path():
    """The package never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_2009_07495_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "igm_oracle" not in txt, f
