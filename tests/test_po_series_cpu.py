"""The bounds the PO rotation kernel's sinc-product series rests on (Eq. 14's
sinc factors), checked exactly on the CPU.

The kernel writes sinc(k a) sinc(k b) as a power series in t = k^2 through
t^6 and takes it while |k a|, |k b| <= 1.  Its stated tail bound uses the
identity sum_{i+j=n} 1 / ((2i+1)! (2j+1)!) = 2^(2n+1) / (2n+2)!, which is
checked here in exact rationals, together with the tail sum it gives and,
against the exact product at the range's edge, the error of the truncated
series itself.
"""
import math
from fractions import Fraction

import numpy as np
import pytest


def _coef_bound(n):
    return sum(Fraction(1, math.factorial(2 * i + 1) * math.factorial(2 * (n - i) + 1))
               for i in range(n + 1))


@pytest.mark.parametrize("n", range(12))
def test_sum_of_reciprocal_odd_factorial_pairs(n):
    assert _coef_bound(n) == Fraction(2 ** (2 * n + 1), math.factorial(2 * n + 2))


def test_tail_beyond_t6_below_stated_bound():
    tail = sum(Fraction(2 ** (2 * n + 1), math.factorial(2 * n + 2)) for n in range(7, 40))
    assert tail < Fraction(16, 10 ** 10)      # "below 1.6e-9"
    assert tail > Fraction(15, 10 ** 10)      # and the bound is tight


def _series(a, b, t, terms):
    # coefficient of t^n: (-1)^n sum_{i+j=n} a^(2i) b^(2j) / ((2i+1)! (2j+1)!)
    s = 0.0
    for n in range(terms + 1):
        c = sum(a ** (2 * i) * b ** (2 * (n - i)) /
                (math.factorial(2 * i + 1) * math.factorial(2 * (n - i) + 1)) for i in range(n + 1))
        s += (-1) ** n * c * t ** n
    return s


@pytest.mark.parametrize("ka,kb", [(1.0, 1.0), (1.0, 0.0), (0.7, -0.9), (-1.0, 0.3)])
def test_truncated_series_within_tail_bound(ka, kb):
    k = 1.0
    exact = (math.sin(ka) / ka if ka else 1.0) * (math.sin(kb) / kb if kb else 1.0)
    got = _series(ka / k, kb / k, k * k, 6)
    assert abs(got - exact) < 1.6e-9


def test_direct_form_identity():
    # the direct pass: sinc(kA) sinc(kB) = sin(kA) sin(kB) / (k^2 A B)
    rng = np.random.default_rng(4)
    A, B, k = rng.uniform(1e-3, 2e-2, 50), rng.uniform(1e-3, 2e-2, 50), rng.uniform(150, 260, 50)
    lhs = np.sinc(k * A / np.pi) * np.sinc(k * B / np.pi)
    rhs = np.sin(k * A) * np.sin(k * B) / (k * k * A * B)
    assert np.allclose(lhs, rhs, rtol=1e-12, atol=0)
