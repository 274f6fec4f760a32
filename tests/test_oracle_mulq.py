"""Pins of the oracle's Mul / MatMul quotient (Sec. 4.4.1):
t = (A B - L) / (X^n - 1), A, B the interpolants of a, b over H = <omega_n>
and L that of a o b.

The pins avoid the oracle's DFT and division: interpolants are evaluated
with Lagrange's formula over Python integers, the identity
t(X) (X^n - 1) + L(X) = A(X) B(X) is checked coefficient by coefficient
against an independent interpolation (Python O(n^2) inverse transform), and
the identity at random points zeta is checked through Horner."""
import random

import numpy as np
import pytest

import zkinputs as Z

R = Z.R_MOD


def _omega(n):
    return pow(5, (R - 1) // n, R)


def _interp(v):
    """Coefficients of the interpolant of v over H (plain O(n^2) sum)."""
    n = len(v)
    wi = pow(_omega(n), R - 2, R)
    ninv = pow(n, R - 2, R)
    return [ninv * sum(v[k] * pow(wi, j * k, R) for k in range(n)) % R for j in range(n)]


def _lagrange_eval(v, z):
    n = len(v)
    w = _omega(n)
    zn1 = (pow(z, n, R) - 1) % R
    tot = 0
    for k, a in enumerate(v):
        wk = pow(w, k, R)
        tot += a * wk * zn1 * pow(n * (z - wk) % R, R - 2, R)
    return tot % R


def _horner(c, x):
    y = 0
    for a in reversed(c):
        y = (y * x + a) % R
    return y


def _limbs(v):
    return np.stack([Z.int_to_fr(x % R) for x in v])


def _ints(a):
    return [Z.fr_to_int(x) for x in np.asarray(a).reshape(-1, 4)]


@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 32])
def test_mul_quotient_polynomial_identity(orc, n):
    rng = random.Random(70 + n)
    a = [rng.randrange(R) for _ in range(n)]
    b = [rng.randrange(R) for _ in range(n)]
    t, exact = orc.mul_quotient(_limbs(a), _limbs(b))
    assert exact
    t = _ints(t)
    assert len(t) == n - 1
    A, B = _interp(a), _interp(b)
    L = _interp([x * y % R for x, y in zip(a, b)])
    AB = [0] * (2 * n)
    for i, x in enumerate(A):
        for j, y in enumerate(B):
            AB[i + j] = (AB[i + j] + x * y) % R
    lhs = [0] * (2 * n)
    for i, x in enumerate(t):  # t (X^n - 1)
        lhs[i + n] = (lhs[i + n] + x) % R
        lhs[i] = (lhs[i] - x) % R
    for i, x in enumerate(L):
        lhs[i] = (lhs[i] + x) % R
    assert lhs == AB


def test_mul_quotient_at_random_points(orc):
    rng = random.Random(5)
    n = 64
    a = Z.zkml_scalars(81, n)
    b = Z.fr_uniform(82, n)
    t, exact = orc.mul_quotient(a, b)
    assert exact
    t = _ints(t)
    ai, bi = _ints(a), _ints(b)
    li = [x * y % R for x, y in zip(ai, bi)]
    for _ in range(3):
        z = rng.randrange(R)
        lhs = _horner(t, z) * (pow(z, n, R) - 1) % R
        rhs = (_lagrange_eval(ai, z) * _lagrange_eval(bi, z) - _lagrange_eval(li, z)) % R
        assert lhs == rhs


def test_mul_quotient_special_cases(orc):
    n = 16
    b = Z.fr_uniform(83, n)
    ones = np.tile(Z.int_to_fr(1), (n, 1))
    t, exact = orc.mul_quotient(ones, b)  # A = 1: A B = B has degree < n
    assert exact and not np.asarray(t).any()
    t, exact = orc.mul_quotient(b, np.zeros((n, 4), np.uint64))
    assert exact and not np.asarray(t).any()
    t, exact = orc.mul_quotient(b[:1], b[:1])  # n = 1: no quotient coefficients
    assert exact and len(t) == 0
