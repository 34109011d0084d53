"""Pins for the oracle's fixed-point primitives (Sec. V-B) and its
reproducible FP64 norm, checked against Python integers, the mathematics
of each operation and exact rational arithmetic -- never against the
oracle itself."""
import json
import math
import os
import random
from fractions import Fraction

import numpy as np
import pytest

I64MIN, I64MAX = -(1 << 63), (1 << 63) - 1
GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_params.json")


def test_paper_parameters_match_tables(orc):
    """Params.table4/table5 carry the shifts printed in Tables 4 and 5 and the
    word format / alpha_a of Sec. VII-B."""
    g = json.load(open(GOLD))
    for name, p in (("table4", orc.Params.table4()), ("table5", orc.Params.table5())):
        t = g[name]
        assert (p.beta7, p.beta8, p.beta10) == (t["line7_beta1"], t["line8_beta1"], t["line10_beta1"])
        assert (p.beta11a, p.beta11b) == (t["line11_beta1"], t["line11_beta2"])
        assert p.beta13 == t["line13_beta2"] and p.beta15 == t["line15_beta1"]
        assert (p.beta16a, p.beta16b) == (t["line16_beta1"], t["line16_beta2"])
        assert p.df == g["word"]["df"]
    assert orc.Params.table4().alpha_a == g["alpha_a"]["none"]
    assert orc.Params.table5().alpha_a == g["alpha_a"]["ilu"]


def test_shift_is_floor_division(orc):
    """'right shift by beta' = division by 2^beta (Sec. V-A); on signed
    numbers the arithmetic shift rounds toward -inf, like Python's >>."""
    for x in range(-70000, 70000, 7):
        for s in (0, 1, 2, 5, 14, 16, 30):
            assert orc.shr(x, s) == x >> s
    rnd = random.Random(5)
    for _ in range(3000):
        x = rnd.randint(I64MIN, I64MAX)
        s = rnd.randint(0, 63)
        assert orc.shr(x, s) == x >> s
        assert orc.shr(x, s) == math.floor(Fraction(x, 1 << s))


def test_isqrt_is_floor_sqrt(orc):
    """Babylonian iteration of Sec. V-B reaches floor(sqrt(s)): s >= r^2 and
    s < (r+1)^2, equal to math.isqrt."""
    for s in range(0, 1 << 16):
        assert orc.isqrt(s) == math.isqrt(s)
    rnd = random.Random(7)
    vals = [I64MAX, I64MAX - 1, 1 << 62, (1 << 62) - 1, (3037000499 ** 2),
            3037000499 ** 2 - 1, 3037000500 ** 2 - 1 if 3037000500 ** 2 - 1 <= I64MAX else I64MAX]
    vals += [rnd.randint(0, I64MAX) for _ in range(5000)]
    vals += [k * k + d for k in (rnd.randint(1, 3037000499) for _ in range(2000)) for d in (-1, 0, 1)]
    for s in vals:
        if 0 <= s <= I64MAX:
            r = orc.isqrt(s)
            assert r * r <= s < (r + 1) * (r + 1)


def test_fx_mul_error_bound(orc):
    """eq. (c1c2): the shifted product approximates t1 t2 / 2^df.  Writing
    t = 2^b q + r (0 <= r < 2^b), the operand shifts drop r, so
    |result - t1 t2 / 2^df| <= (|t2| 2^b1 + |t1| 2^b2 + 2^(b1+b2)) / 2^df + 1."""
    rnd = random.Random(11)
    df = 30
    for b1, b2 in ((0, 0), (16, 0), (0, 16), (16, 16), (14, 2)):
        for _ in range(3000):
            t1 = rnd.randint(-(1 << 46), 1 << 46)
            t2 = rnd.randint(-(1 << 46), 1 << 46)
            exact = Fraction(t1 * t2, 1 << df)
            p = (t1 >> b1) * (t2 >> b2)
            if not (I64MIN <= p <= I64MAX):
                continue
            r, ev = orc.fx_mul(t1, t2, b1, b2, df)
            assert ev == 0
            bound = Fraction(abs(t2) * (1 << b1) + abs(t1) * (1 << b2) + (1 << (b1 + b2)), 1 << df) + 1
            assert abs(r - exact) <= bound
            # exact whenever nothing is dropped
            if t1 % (1 << b1) == 0 and t2 % (1 << b2) == 0 and (t1 * t2) % (1 << df) == 0:
                assert r == exact


def test_fx_mul_overflow_events(orc):
    """An int64 product whose exact value leaves [-2^63, 2^63) is counted and
    wrapped modulo 2^64, as the paper's int64 hardware would store it."""
    r, ev = orc.fx_mul(1 << 40, 1 << 40, 0, 0, 30)
    assert ev == 1
    assert r == 0  # 2^80 wraps to 0, then >> 30
    r, ev = orc.fx_mul(1 << 31, 1 << 31, 0, 0, 30)
    assert ev == 0 and r == 1 << 32
    r, ev = orc.fx_mul(-(1 << 32), 1 << 31, 0, 0, 0)
    assert ev == 0 and r == I64MIN
    r, ev = orc.fx_mul(1 << 32, 1 << 31, 0, 0, 0)
    assert ev == 1 and r == I64MIN


def test_fx_div_truncates(orc):
    """Sec. V-B division: for Table 5 shifts (b1 = d_f = 30, b2 = 0) the result
    is the truncated quotient t1 2^30 / t2, |q - t1 2^30/t2| < 1, sign of the
    exact quotient; a zero shifted divisor is reported."""
    rnd = random.Random(13)
    for _ in range(5000):
        t1 = rnd.randint(-(1 << 32), 1 << 32)
        t2 = rnd.choice([1, -1]) * rnd.randint(1, 1 << 40)
        q, ev, z = orc.fx_div(t1, t2, 30, 0, 30)
        assert not z and ev == 0
        ex = Fraction(t1 << 30, t2)
        assert abs(q - ex) < 1
        assert q == 0 or (q > 0) == (ex > 0)
        assert abs(q) <= abs(ex)
    # Table 4 shifts: (t1 2^16) / (t2 >> 14) approximates t1 2^30 / t2
    for _ in range(3000):
        t1 = rnd.randint(-(1 << 40), 1 << 40)
        t2 = rnd.randint(1 << 20, 1 << 44)
        q, ev, z = orc.fx_div(t1, t2, 16, 14, 30)
        ex = Fraction(t1 << 30, t2)
        assert abs(q - ex) <= abs(ex) * Fraction(1 << 15, t2) + 1
    q, ev, z = orc.fx_div(5, (1 << 14) - 1, 16, 14, 30)
    assert z and q == 0


def test_fx_sqrt_formats(orc):
    """Sec. V-B square root: an argument with d_f' fractional bits maps to a
    Q(d_f) result, isqrt(t) 2^(d_f - d_f'/2)."""
    # (0.75)^2 in Q60 -> 0.75 in Q30
    t = (3 << 58)
    t2 = (3 * (1 << 28)) ** 2
    r, ev = orc.fx_sqrt(t2, 60, 30)
    assert r == 3 * (1 << 28) and ev == 0
    # Table 4 norm: argument in Q(2*30-2*16) = Q28, result isqrt * 2^16
    r, ev = orc.fx_sqrt(1 << 28, 28, 30)
    assert r == 1 << 30
    assert t > 0


def _exact_norm(x):
    mx = max(abs(float(v)) for v in x)
    if mx == 0.0:
        return 0.0
    e = math.frexp(mx)[1]
    s = sum((Fraction(float(v)) / Fraction(2) ** e) ** 2 for v in x)
    return math.ldexp(math.sqrt(float(s)), e)


@pytest.mark.parametrize("scale", [1e-200, 1e-8, 1.0, 3.7e5, 1e150])
def test_reproducible_norm(orc, scale):
    """The oracle's 2-norm is within 1 ulp of sqrt(exact sum of squares) and
    does not depend on the order of the elements."""
    rng = np.random.default_rng(3)
    for n in (1, 2, 7, 100, 1000):
        x = rng.standard_normal(n) * scale
        nr = orc.norm2(x)
        ex = _exact_norm(x)
        assert abs(nr - ex) <= 2 * np.spacing(ex)
        for _ in range(3):
            assert orc.norm2(rng.permutation(x)) == nr
    assert orc.norm2(np.zeros(5)) == 0.0
    assert orc.norm2(np.array([3.0, -4.0])) == 5.0
