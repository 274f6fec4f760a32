"""Pins of the oracle's O(n^2) DFT over F_r: primitive roots, transform pairs of
closed form, the convolution theorem against Python-integer brute force, the
Aurora identity sum_H f = n f(0) (Sec. 4.4, Sum) and polynomial evaluation."""
import numpy as np
import pytest

import zkinputs as Z

R = Z.R_MOD


def _ints(a):
    return [Z.fr_to_int(x) for x in np.asarray(a).reshape(-1, 4)]


def _arr(xs):
    return np.stack([Z.int_to_fr(x % R) for x in xs])


@pytest.mark.parametrize("lg", [1, 2, 5, 10, 16, 28])
def test_root_of_unity_is_primitive(orc, lg):
    n = 1 << lg
    w = Z.fr_to_int(orc.root_of_unity(n))
    assert pow(w, n, R) == 1
    assert pow(w, n // 2, R) == R - 1


@pytest.mark.parametrize("n", [1, 2, 4, 8, 64, 256])
def test_round_trip_and_closed_forms(orc, n):
    x = Z.fr_uniform(2, n)
    assert (orc.intt(orc.ntt(x)) == x).all()
    assert (orc.ntt(orc.intt(x)) == x).all()
    delta = np.zeros((n, 4), dtype=np.uint64)
    delta[0, 0] = 1
    assert _ints(orc.ntt(delta)) == [1] * n               # NTT(e_0) = all ones
    c = Z.fr_uniform(3, 1)[0]
    const = np.tile(c, (n, 1))
    want = [n * Z.fr_to_int(c) % R] + [0] * (n - 1)       # NTT(const c) = n c e_0
    assert _ints(orc.ntt(const)) == want


def test_polynomial_evaluation_at_powers_of_omega(orc):
    n = 32
    c = Z.fr_uniform(4, n)
    cs = _ints(c)
    w = Z.fr_to_int(orc.root_of_unity(n))
    got = _ints(orc.ntt(c))
    for k in range(n):
        x = pow(w, k, R)
        acc = 0
        for cj in reversed(cs):  # Horner with Python integers
            acc = (acc * x + cj) % R
        assert got[k] == acc


def test_convolution_theorem_against_brute_force(orc):
    n = 64
    a, b = Z.fr_uniform(5, n), Z.fr_uniform(6, n)
    ai, bi = _ints(a), _ints(b)
    conv = [sum(ai[j] * bi[(k - j) % n] for j in range(n)) % R for k in range(n)]
    A, B = orc.ntt(a), orc.ntt(b)
    prod = np.stack([orc.fmul(1, A[k], B[k]) for k in range(n)])
    assert _ints(orc.intt(prod)) == conv


def test_aurora_sum_identity(orc):
    n = 128
    v = Z.fr_uniform(7, n)
    f0 = Z.fr_to_int(orc.intt(v)[0])
    assert f0 * n % R == sum(_ints(v)) % R


def test_sampled_rows_match_full_transform(orc):
    n = 256
    x = Z.fr_uniform(8, n)
    rows = np.array([0, 1, 5, 100, 255])
    assert (orc.dft_rows(x, rows, False) == orc.ntt(x)[rows]).all()
    assert (orc.dft_rows(x, rows, True) == orc.intt(x)[rows]).all()
