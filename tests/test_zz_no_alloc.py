"""igm_norm2_noalloc: the reproducible norm for callers that cannot allocate
device memory (its scratch is a static device array).  Called through the C
ABI and compared with igm_norm2, the allocating entry point, on two calls in
a row; the file sorts last so a run that stops at the first failure has run
every other test first, and it also passes alone in a fresh process."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_07495_gb300 import _lib
    from paper_2009_07495_gb300 import build
    build.build()
    return _lib


def _noalloc(L, x_dev, out_dev, n=None):
    import torch
    st = L.load().igm_norm2_noalloc(x_dev.data_ptr() or None, x_dev.numel() if n is None else n,
                                    out_dev.data_ptr(), torch.cuda.current_stream().cuda_stream)
    return st


@pytest.mark.parametrize("n", [0, 1, 4096, 4097, 1_000_003, 8_388_608])
def test_noalloc_matches_allocating_entry_point(lib, n):
    """Two calls in a row equal igm_norm2 bit for bit (the tolerance of the
    norm's tests: it is an exact, order-independent definition)."""
    import torch
    L = lib
    rng = np.random.default_rng(n + 7)
    for call in range(2):
        x = rng.standard_normal(n) * (10.0 ** rng.integers(-5, 5))
        xd = torch.from_numpy(x).cuda()
        out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        assert _noalloc(L, xd, out) == 0, L.load().igm_last_error()
        torch.cuda.synchronize()
        assert out.item() == L.norm2(xd), (call, out.item())


def test_noalloc_rejects_too_large_n(lib):
    import torch
    L = lib
    x = torch.zeros(16, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert _noalloc(L, x, out, n=8_388_609) == 1   # IGM_EINVAL
    assert b"exceeds the static scratch" in L.load().igm_last_error()
    # host memory is refused: nothing is staged
    xh = np.zeros(4)
    st = L.load().igm_norm2_noalloc(xh.ctypes.data, 4, out.data_ptr(), 0)
    assert st == 1


def test_noalloc_grid_sizes_in_sequence(lib):
    """Calls on one stream whose grids shrink and grow (n = 1,000,003, 4097,
    8,388,608 -- every partial-sum slot -- then 1): each call clears its own
    counters, so partial sums an earlier, larger call left behind never
    reach a later result; each equals igm_norm2 bit for bit."""
    import torch
    L = lib
    rng = np.random.default_rng(11)
    for n in (1_000_003, 4097, 8_388_608, 1):
        x = rng.standard_normal(n) * (10.0 ** rng.integers(-3, 3))
        xd = torch.from_numpy(x).cuda()
        out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        assert _noalloc(L, xd, out) == 0, L.load().igm_last_error()
        torch.cuda.synchronize()
        assert out.item() == L.norm2(xd), (n, out.item())
