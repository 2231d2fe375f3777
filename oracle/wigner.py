"""Wigner 3j, 6j and 9j symbols (Racah's sum formulas, exact rational
arithmetic on factorials) for the multipole statistical-equilibrium equations
of the polarized multilevel atom. Test infrastructure only.

Arguments are integers or half-integers given as floats; they are doubled
internally. Pinned against sympy.physics.wigner and the orthogonality
relations (tests/test_oracle_wigner.py).
"""
from fractions import Fraction
from functools import lru_cache
from math import factorial, sqrt


def _two(x):
    t = 2 * x
    r = int(round(t))
    if abs(t - r) > 1e-9:
        raise ValueError("angular momenta must be integers or half-integers")
    return r


@lru_cache(maxsize=None)
def _fact(n):
    return factorial(n)


def _tri2(a, b, c):
    """triangle condition and integer perimeter, doubled arguments"""
    return (a + b >= c and b + c >= a and c + a >= b and (a + b + c) % 2 == 0)


def _delta2(a, b, c):
    """Delta(abc)^2 = (a+b-c)!(a-b+c)!(-a+b+c)!/(a+b+c+1)!, doubled arguments"""
    return Fraction(_fact((a + b - c) // 2) * _fact((a - b + c) // 2) * _fact((-a + b + c) // 2),
                    _fact((a + b + c) // 2 + 1))


@lru_cache(maxsize=None)
def _w3j2(j1, j2, j3, m1, m2, m3):
    if m1 + m2 + m3 != 0 or not _tri2(j1, j2, j3):
        return 0.0
    for j, m in ((j1, m1), (j2, m2), (j3, m3)):
        if abs(m) > j or (j + m) % 2:
            return 0.0
    # Racah: (j1 j2 j3; m1 m2 m3) = (-1)^(j1-j2-m3) sqrt(Delta ...) sum_k ...
    pre = _delta2(j1, j2, j3)
    for j, m in ((j1, m1), (j2, m2), (j3, m3)):
        pre *= _fact((j + m) // 2) * _fact((j - m) // 2)
    kmin = max(0, (j2 - j3 - m1) // 2, (j1 - j3 + m2) // 2)
    kmax = min((j1 + j2 - j3) // 2, (j1 - m1) // 2, (j2 + m2) // 2)
    s = Fraction(0)
    for k in range(kmin, kmax + 1):
        d = (_fact(k) * _fact((j3 - j2 + m1) // 2 + k) * _fact((j3 - j1 - m2) // 2 + k) *
             _fact((j1 + j2 - j3) // 2 - k) * _fact((j1 - m1) // 2 - k) * _fact((j2 + m2) // 2 - k))
        s += Fraction((-1) ** k, d)
    sign = -1 if ((j1 - j2 - m3) // 2) % 2 else 1
    return sign * float(s) * sqrt(float(pre))


def w3j(j1, j2, j3, m1, m2, m3):
    return _w3j2(_two(j1), _two(j2), _two(j3), _two(m1), _two(m2), _two(m3))


@lru_cache(maxsize=None)
def _w6j2(j1, j2, j3, l1, l2, l3):
    for t in ((j1, j2, j3), (j1, l2, l3), (l1, j2, l3), (l1, l2, j3)):
        if not _tri2(*t):
            return 0.0
    pre = _delta2(j1, j2, j3) * _delta2(j1, l2, l3) * _delta2(l1, j2, l3) * _delta2(l1, l2, j3)
    a = [(j1 + j2 + j3) // 2, (j1 + l2 + l3) // 2, (l1 + j2 + l3) // 2, (l1 + l2 + j3) // 2]
    b = [(j1 + j2 + l1 + l2) // 2, (j2 + j3 + l2 + l3) // 2, (j3 + j1 + l3 + l1) // 2]
    s = Fraction(0)
    for k in range(max(a), min(b) + 1):
        d = 1
        for x in a:
            d *= _fact(k - x)
        for y in b:
            d *= _fact(y - k)
        s += Fraction((-1) ** k * _fact(k + 1), d)
    return float(s) * sqrt(float(pre))


def w6j(j1, j2, j3, l1, l2, l3):
    """{j1 j2 j3; l1 l2 l3}"""
    return _w6j2(_two(j1), _two(j2), _two(j3), _two(l1), _two(l2), _two(l3))


@lru_cache(maxsize=None)
def _w9j2(a, b, c, d, e, f, g, h, i):
    # sum over x of (-1)^(2x) (2x+1) {a b c; f i x} {d e f; b x h} {g h i; x a d}
    lo = max(abs(a - i), abs(h - d), abs(b - f))
    hi = min(a + i, h + d, b + f)
    s = 0.0
    for x in range(lo, hi + 1, 2):
        s += ((-1) ** x) * (x + 1) * _w6j2(a, b, c, f, i, x) * _w6j2(d, e, f, b, x, h) * _w6j2(g, h, i, x, a, d)
    return s


def w9j(a, b, c, d, e, f, g, h, i):
    """{a b c; d e f; g h i}"""
    return _w9j2(*(_two(x) for x in (a, b, c, d, e, f, g, h, i)))
