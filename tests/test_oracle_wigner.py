"""Pins of oracle/wigner.py: values against sympy.physics.wigner (exact),
and the orthogonality of the 3j and 6j symbols."""
import itertools

import numpy as np
import pytest

from oracle import wigner as W

sw = pytest.importorskip("sympy.physics.wigner")

HALF = [0, 0.5, 1, 1.5, 2, 2.5, 3, 4]


def test_3j_against_sympy():
    rng = np.random.default_rng(0)
    n = 0
    for j1, j2, j3 in itertools.product([0, 0.5, 1, 1.5, 2, 3], repeat=3):
        for _ in range(3):
            m1 = rng.choice(np.arange(-j1, j1 + 1))
            m2 = rng.choice(np.arange(-j2, j2 + 1))
            m3 = -m1 - m2
            want = _sym(sw.wigner_3j, (j1, j2, j3, m1, m2, m3))
            assert abs(W.w3j(j1, j2, j3, m1, m2, m3) - want) < 1e-13
            n += 1
    assert n > 500


def _R(x):
    import sympy
    return sympy.Rational(str(x))


def _sym(fn, args, **kw):
    """sympy's value, 0 where it rejects a non-integral perimeter (the symbol vanishes)"""
    try:
        return float(fn(*map(_R, args), **kw))
    except ValueError:
        return 0.0


def test_6j_and_9j_against_sympy():
    for args in itertools.product([0, 1, 2], [0.5, 1.5], [1, 2], [0.5, 1.5, 2.5], [1, 2], [0.5, 1.5]):
        want = _sym(sw.wigner_6j, args)
        assert abs(W.w6j(*args) - want) < 1e-13, args
    rng = np.random.default_rng(1)
    for _ in range(300):
        args = [int(x) for x in rng.integers(0, 4, size=9)]
        want = _sym(sw.wigner_9j, args, prec=64)
        assert abs(W.w9j(*args) - want) < 1e-12, args
    # half-integer 9j of the kind used by the rate equations
    for J, Jl, K, Kl, Kr in itertools.product([0.5, 1.5, 2.5], [0.5, 1.5], [0, 1, 2, 3], [0, 1, 2], [0, 1, 2]):
        args = (J, Jl, 1, J, Jl, 1, K, Kl, Kr)
        want = _sym(sw.wigner_9j, args, prec=64)
        assert abs(W.w9j(*args) - want) < 1e-12, args


def test_orthogonality():
    for j1, j2 in [(1, 1), (1.5, 1), (2, 2), (0.5, 1.5)]:
        for j3 in np.arange(abs(j1 - j2), j1 + j2 + 1):
            for m3 in np.arange(-j3, j3 + 1):
                s = sum((2 * j3 + 1) * W.w3j(j1, j2, j3, m1, m2, -m3) ** 2
                        for m1 in np.arange(-j1, j1 + 1) for m2 in np.arange(-j2, j2 + 1))
                assert abs(s - 1) < 1e-12
    # sum_x (2x+1)(2e+1) {a b x; c d e}{a b x; c d e'} = delta_ee'
    a, b, c, d = 1, 2, 1.5, 1.5
    for e in (0.5, 1.5, 2.5):
        for e2 in (0.5, 1.5, 2.5):
            s = sum((2 * x + 1) * (2 * e + 1) * W.w6j(a, b, x, c, d, e) * W.w6j(a, b, x, c, d, e2) for x in range(0, 4))
            assert abs(s - (1.0 if e == e2 else 0.0)) < 1e-12
