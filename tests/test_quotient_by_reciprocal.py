"""The quotient w / h from r = 1/h by one fused correction (Markstein's theorem), as the
solve's kernels form v = w / ||w|| and the final normalisation: q0 = RN(w r), the exact
remainder w - q0 h in one fma, q = RN(q0 + rem r).  Each fma is emulated exactly here (the
product and sum in rationals, one rounding), and q must equal Python's correctly rounded
w / h for quotients in the normal range, zeros and their signs included."""
import math
import random
from fractions import Fraction

import pytest


def _fma(a: float, b: float, c: float) -> float:
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def _quotient(w: float, h: float) -> float:
    r = 1.0 / h
    q0 = w * r
    rem = _fma(-q0, h, w)
    return q0 if rem == 0.0 else _fma(rem, r, q0)


def _same(a: float, b: float) -> bool:
    return a == b and math.copysign(1.0, a) == math.copysign(1.0, b)


def _all_ones_tail(x: float, rng: random.Random) -> float:
    m, e = math.frexp(x)
    bits = int(abs(m) * (1 << 53)) | ((1 << rng.randint(40, 52)) - 1)
    return math.copysign(math.ldexp(bits / (1 << 53), e), x)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_quotient_is_correctly_rounded(seed):
    rng = random.Random(seed)
    for k in range(6000):
        w = rng.uniform(-1.0, 1.0) * 2.0 ** rng.randint(-60, 60)
        h = rng.uniform(0.5, 1.0) * 2.0 ** rng.randint(-60, 60)
        if k % 5 == 0:
            h = _all_ones_tail(h, rng)
        if k % 7 == 0:
            w = _all_ones_tail(w, rng)
        assert _same(_quotient(w, h), w / h), (w.hex(), h.hex())


def test_quotient_of_unit_vector_entries():
    # the solve's case: entries of w divided by ||w|| (quotients in [-1, 1])
    rng = random.Random(7)
    w = [rng.gauss(0.0, 1.0) for _ in range(4000)]
    h = math.sqrt(sum(x * x for x in w))
    for x in w:
        assert _same(_quotient(x, h), x / h)


def test_quotient_zeros_keep_their_sign():
    for h in (1.0, 3.0, 0.1, 7.5e10):
        assert _same(_quotient(0.0, h), 0.0)
        assert _same(_quotient(-0.0, h), -0.0)


def test_plain_product_is_not_enough():
    # the correction step matters: w * RN(1/h) alone misses the rounding for some pairs
    rng = random.Random(3)
    misses = 0
    for _ in range(3000):
        w = rng.uniform(-1.0, 1.0)
        h = rng.uniform(0.5, 2.0)
        misses += (w * (1.0 / h)) != (w / h)
    assert misses > 0
