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


def test_poly_eval_against_python_horner(orc):
    v = Z.fr_uniform(9, 37)
    z = Z.fr_uniform(10, 1)[0]
    zi = Z.fr_to_int(z)
    acc = 0
    for c in reversed(_ints(v)):
        acc = (acc * zi + c) % R
    assert Z.fr_to_int(orc.poly_eval(v, z)) == acc


@pytest.mark.parametrize("n", [1, 2, 4, 16])
def test_fingerprint_against_python_brute_force(orc, n):
    # sum_k z^k sum_j c_j omega^{jk}, every term with Python integers.
    c = Z.fr_uniform(11, n)
    z = Z.fr_uniform(12, 1)[0]
    zi, w = Z.fr_to_int(z), Z.fr_to_int(orc.root_of_unity(n))
    ci = _ints(c)
    want = sum(pow(zi, k, R) * ci[j] * pow(w, j * k, R) for k in range(n) for j in range(n)) % R
    assert Z.fr_to_int(orc.ntt_fingerprint(c, z)) == want


@pytest.mark.parametrize("n", [2, 64, 1024])
def test_fingerprint_matches_evaluated_dft(orc, n):
    c = Z.fr_uniform(13, n)
    z = Z.fr_uniform(14, 1)[0]
    f = orc.ntt(c)
    assert (orc.poly_eval(f, z) == orc.ntt_fingerprint(c, z)).all()
    # the INTT side: NTT(INTT(v)) = v, so the fingerprint of INTT(v) is v(z)
    assert (orc.ntt_fingerprint(orc.intt(c), z) == orc.poly_eval(c, z)).all()
    # a planted error in one output (any position) changes the left side
    for k in (0, n // 2, n - 1):
        bad = f.copy()
        bad[k] = Z.int_to_fr((Z.fr_to_int(bad[k]) + 1) % R)
        assert not (orc.poly_eval(bad, z) == orc.ntt_fingerprint(c, z)).all()


def test_fingerprint_rejects_z_on_the_inverse_subgroup(orc):
    n = 8
    w = Z.fr_to_int(orc.root_of_unity(n))
    z = Z.int_to_fr(pow(w, n - 3, R))  # z omega^3 = 1
    with pytest.raises(ValueError):
        orc.ntt_fingerprint(Z.fr_uniform(15, n), z)
