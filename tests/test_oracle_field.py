"""Pins of the oracle's F_q / F_r arithmetic.

Each check compares the oracle's schoolbook/long-division C code against a
route that does not share it: Python's own arbitrary-precision integers (a
library routine), Fermat's little theorem, and primality of the moduli.
"""
import random

import pytest
import sympy

import zkinputs as Z

Q, R = Z.Q_MOD, Z.R_MOD


def test_moduli_are_the_bn254_primes():
    # Both moduli are 254-bit primes; r - 1 has 2-adicity 28 (largest NTT 2^28).
    for m in (Q, R):
        assert m.bit_length() == 254
        assert sympy.isprime(m)
    assert ((R - 1) >> 28) & 1 == 1 and (R - 1) % (1 << 28) == 0
    # 5 is a quadratic non-residue mod r, so 5^((r-1)/2^28) has order exactly 2^28.
    assert pow(5, (R - 1) // 2, R) == R - 1


def _edge(m):
    return [0, 1, 2, m - 1, m - 2, (m - 1) // 2, (m + 1) // 2, 1 << 253, (1 << 254) % m,
            (1 << 32) - 1, (1 << 64) - 1, (1 << 128) + 12345, m >> 1]


@pytest.mark.parametrize("f,m", [(0, Q), (1, R)])
def test_add_sub_mul_against_python_integers(orc, f, m):
    rng = random.Random(1234 + f)
    vals = _edge(m) + [rng.randrange(m) for _ in range(300)]
    for i, a in enumerate(vals):
        b = vals[(7 * i + 3) % len(vals)]
        A, B = orc.from_int(a), orc.from_int(b)
        assert orc.to_int(orc.fadd(f, A, B)) == (a + b) % m
        assert orc.to_int(orc.fsub(f, A, B)) == (a - b) % m
        assert orc.to_int(orc.fmul(f, A, B)) == (a * b) % m


@pytest.mark.parametrize("f,m", [(0, Q), (1, R)])
def test_long_division_reduction_of_512_bit_values(orc, f, m):
    rng = random.Random(99 + f)
    vals = [0, 1, m, m * m - 1, (1 << 512) - 1, (m - 1) * (m - 1), (1 << 511), m << 257]
    vals += [rng.getrandbits(512) for _ in range(300)]
    vals += [rng.getrandbits(rng.randrange(1, 512)) for _ in range(200)]
    for x in vals:
        assert orc.to_int(orc.freduce512(f, orc.from_int(x, 8))) == x % m


@pytest.mark.parametrize("f,m", [(0, Q), (1, R)])
def test_inverse_and_power(orc, f, m):
    rng = random.Random(7 + f)
    for a in [1, 2, 3, m - 1, m - 2, (m + 1) // 2] + [rng.randrange(1, m) for _ in range(100)]:
        A = orc.from_int(a)
        inv = orc.finv(f, A)
        assert orc.to_int(orc.fmul(f, A, inv)) == 1
        assert orc.to_int(inv) == pow(a, -1, m)
    assert orc.to_int(orc.finv(f, orc.from_int(0))) == 0  # no inverse: 0 by convention
    for a in [rng.randrange(1, m) for _ in range(10)]:
        # Fermat: a^(m-1) = 1 for the prime m.
        assert orc.to_int(orc.fpow(f, orc.from_int(a), orc.from_int(m - 1))) == 1
        e = rng.getrandbits(256)
        assert orc.to_int(orc.fpow(f, orc.from_int(a), orc.from_int(e))) == pow(a, e, m)
