"""Pins of the oracle's BN254 G1 arithmetic: curve equation, the group order r,
the published doubling of the generator, and the group law's homomorphism."""
import os
import random

import numpy as np

import zkinputs as Z

Q, R = Z.Q_MOD, Z.R_MOD
GOLD = os.path.join(os.path.dirname(__file__), "golden", "bn254_g1_small_multiples.txt")


def _golden():
    out = {}
    for line in open(GOLD):
        if line.strip() and not line.startswith("#"):
            k, x, y = line.split()
            out[int(k)] = (int(x), int(y))
    return out


def test_generator_and_published_doubling(orc):
    G = orc.g1_generator()
    assert orc.point_to_ints(G) == (1, 2)
    assert orc.on_curve(G)
    x, y = _golden()[2]
    assert orc.point_to_ints(orc.g1_dbl(G)) == (x, y)
    assert orc.point_to_ints(orc.g1_add(G, G)) == (x, y)
    assert orc.point_to_ints(orc.g1_mul(G, orc.from_int(2))) == (x, y)
    # The published value itself satisfies y^2 = x^3 + 3 (checked with Python ints).
    assert (y * y - x ** 3 - 3) % Q == 0


def test_group_order_is_r(orc):
    G = orc.g1_generator()
    inf = np.zeros(8, dtype=np.uint64)
    assert (orc.g1_mul(G, orc.from_int(R)) == inf).all()
    assert (orc.g1_mul(G, orc.from_int(R - 1)) == orc.g1_neg(G)).all()
    assert (orc.g1_mul(G, orc.from_int(R + 1)) == G).all()
    P = orc.g1_mul(G, orc.from_int(123456789))
    assert (orc.g1_mul(P, orc.from_int(R)) == inf).all()


def test_special_cases_of_addition(orc):
    G = orc.g1_generator()
    inf = np.zeros(8, dtype=np.uint64)
    P = orc.g1_mul(G, orc.from_int(987654321))
    assert (orc.g1_add(P, orc.g1_neg(P)) == inf).all()          # P + (-P)
    assert (orc.g1_add(P, P) == orc.g1_dbl(P)).all()            # P = Q
    assert (orc.g1_add(P, inf) == P).all() and (orc.g1_add(inf, P) == P).all()
    assert (orc.g1_dbl(inf) == inf).all()
    assert not orc.on_curve(orc.point_from_ints(1, 3))
    assert not orc.on_curve(orc.point_from_ints(Q, 2))            # non-canonical


def test_scalar_multiplication_is_a_homomorphism(orc):
    rng = random.Random(5)
    G = orc.g1_generator()
    for _ in range(6):
        a, b = rng.randrange(R), rng.randrange(R)
        A = orc.g1_mul(G, orc.from_int(a))
        B = orc.g1_mul(G, orc.from_int(b))
        assert orc.on_curve(A) and orc.on_curve(B)
        assert (orc.g1_add(A, B) == orc.g1_mul(G, orc.from_int((a + b) % R))).all()
        assert (orc.g1_mul(A, orc.from_int(b)) == orc.g1_mul(G, orc.from_int(a * b % R))).all()
