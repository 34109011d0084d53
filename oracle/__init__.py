"""CPU oracle for the integer-arithmetic GMRES + FP64 iterative refinement
method (Iwashita, Suzuki, Fukaya, ScalA'20).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it to check and time the CUDA library.
The product path never imports it.  The arithmetic lives in plain C
(``igm_oracle.c``, single-threaded, ``__int128`` for exact overflow checks);
this module compiles it with gcc and marshals numpy arrays through ctypes.
"""
from .oracle import *  # noqa: F401,F403
from .oracle import build, Params, Report  # noqa: F401
