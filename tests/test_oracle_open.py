"""Pins of the oracle's KZG opening (Sec. 2.1): y = f(x) and the proof
[q(tau)]_1 with q(X) = (f(X) - y) / (X - x), and the batch opening at one point
with h(X) = sum_i gamma^i (f_i(X) - f_i(x)) / (X - x).

The oracle computes q by synthetic division.  The pins below use nothing of
it: Horner over Python integers for y, polynomial multiplication over Python
integers for q (X - x) + y = f, and the KZG verification equation in the
exponent with the known tau, (tau - x) [q(tau)]_1 = com - y G, whose
commitments come from the oracle's separate closed form [f(tau)]_1."""
import random

import numpy as np
import pytest

import zkinputs as Z

R = Z.R_MOD


def _horner(c, x):
    y = 0
    for a in reversed(c):
        y = (y * x + a) % R
    return y


def _times_x_minus(q, x):
    """Coefficients of q(X) (X - x) over F_r."""
    out = [0] * (len(q) + 1)
    for i, a in enumerate(q):
        out[i + 1] = (out[i + 1] + a) % R
        out[i] = (out[i] - a * x) % R
    return out


def _limbs(v):
    return np.stack([Z.int_to_fr(a % R) for a in v]) if v else np.zeros((0, 4), np.uint64)


def _ints(a):
    return [Z.fr_to_int(v) for v in np.asarray(a).reshape(-1, 4)]


@pytest.mark.parametrize("n", [1, 2, 3, 8, 33])
def test_open_matches_definitions(orc, n):
    rng = random.Random(300 + n)
    c = [rng.randrange(R) for _ in range(n)]
    for x in [0, 1, 2, R - 1, rng.randrange(R), rng.randrange(R)]:
        y, q = orc.open_poly(_limbs(c), Z.int_to_fr(x))
        y, q = Z.fr_to_int(y), _ints(q)
        assert y == _horner(c, x)
        assert len(q) == n - 1
        f = _times_x_minus(q, x)
        f[0] = (f[0] + y) % R
        assert f[:n] == c and all(v == 0 for v in f[n:])


def test_open_at_a_root_gives_zero(orc):
    # f = (X - 5)(X + 7) (X^2 + 3): f(5) = 0, quotient (X + 7)(X^2 + 3).
    q_true = [21, 3, 7, 1]
    c = _times_x_minus(q_true, 5)
    y, q = orc.open_poly(_limbs(c), Z.int_to_fr(5))
    assert Z.fr_to_int(y) == 0 and _ints(q) == q_true


def test_kzg_equation_in_the_exponent(orc):
    tau = Z.tau(0)
    t = Z.fr_to_int(tau)
    G = orc.g1_generator()
    rng = random.Random(7)
    for n in [1, 5, 64]:
        c = _limbs([rng.randrange(R) for _ in range(n)])
        x = rng.randrange(R)
        y, q = orc.open_poly(c, Z.int_to_fr(x))
        com = orc.commit_coeffs_tau(c, tau)
        proof = orc.commit_coeffs_tau(q, tau) if n > 1 else np.zeros(8, np.uint64)
        lhs = orc.g1_mul(proof, Z.int_to_fr((t - x) % R))
        rhs = orc.g1_add(com, orc.g1_neg(orc.g1_mul(G, y)))
        assert np.array_equal(lhs, rhs)


def test_batch_open_matches_definitions(orc):
    tau = Z.tau(0)
    t = Z.fr_to_int(tau)
    G = orc.g1_generator()
    rng = random.Random(11)
    lens = [1, 6, 17, 9, 17]
    polys = [[rng.randrange(R) for _ in range(m)] for m in lens]
    x, gamma = rng.randrange(R), rng.randrange(R)
    ys, h = orc.open_batch([_limbs(p) for p in polys], Z.int_to_fr(x), Z.int_to_fr(gamma))
    ys, h = _ints(ys), _ints(h)
    assert ys == [_horner(p, x) for p in polys]
    # h (X - x) = sum_i gamma^i (f_i - y_i)
    lhs = _times_x_minus(h, x)
    rhs = [0] * max(lens)
    for i, p in enumerate(polys):
        g = pow(gamma, i, R)
        for j, a in enumerate(p):
            rhs[j] = (rhs[j] + g * a) % R
        rhs[0] = (rhs[0] - g * ys[i]) % R
    assert lhs[: len(rhs)] == rhs and all(v == 0 for v in lhs[len(rhs):])
    # (tau - x) [h(tau)] = sum_i gamma^i (com_i - y_i G)
    acc = np.zeros(8, np.uint64)
    for i, p in enumerate(polys):
        term = orc.g1_add(orc.commit_coeffs_tau(_limbs(p), tau), orc.g1_neg(orc.g1_mul(G, Z.int_to_fr(ys[i]))))
        acc = orc.g1_add(acc, orc.g1_mul(term, Z.int_to_fr(pow(gamma, i, R))))
    proof = orc.commit_coeffs_tau(_limbs(h), tau)
    assert np.array_equal(orc.g1_mul(proof, Z.int_to_fr((t - x) % R)), acc)
