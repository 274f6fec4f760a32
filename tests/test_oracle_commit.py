"""Pins of the oracle's KZG commitment (Sec. 2.1: com = [f(tau)]_1).

The MSM over the SRS and the closed form (sum c_i tau^i) G take disjoint
routes (affine double-and-add over many points vs one Horner evaluation in F_r
and one scalar multiplication), so their agreement pins both; linearity and the
edge cases below pin the MSM further."""
import numpy as np
import pytest

import zkinputs as Z

R = Z.R_MOD


@pytest.fixture(scope="module")
def tau():
    return Z.tau(0)


@pytest.fixture(scope="module")
def srs(orc, tau):
    return orc.srs_gen(tau, 64)


def test_srs_points_are_powers_of_tau(orc, tau, srs):
    assert orc.count_off_curve(srs) == 0
    G = orc.g1_generator()
    assert (srs[0] == G).all()
    t = Z.fr_to_int(tau)
    for i in [1, 2, 17, 63]:
        assert (srs[i] == orc.g1_mul(G, Z.int_to_fr(pow(t, i, R)))).all()


@pytest.mark.parametrize("n", [1, 2, 7, 64])
def test_msm_equals_tau_closed_form(orc, tau, srs, n):
    c = Z.fr_uniform(11 + n, n)
    assert (orc.msm(srs[:n], c) == orc.commit_coeffs_tau(c, tau)).all()


def test_msm_linearity(orc, srs):
    n = 32
    a, b = Z.fr_uniform(21, n), Z.fr_uniform(22, n)
    ab = np.stack([orc.fadd(1, a[i], b[i]) for i in range(n)])
    assert (orc.g1_add(orc.msm(srs[:n], a), orc.msm(srs[:n], b)) == orc.msm(srs[:n], ab)).all()
    k = Z.fr_uniform(23, 1)[0]
    ka = np.stack([orc.fmul(1, k, a[i]) for i in range(n)])
    assert (orc.g1_mul(orc.msm(srs[:n], a), k) == orc.msm(srs[:n], ka)).all()


def test_msm_edge_cases(orc, srs):
    n = 16
    inf = np.zeros(8, dtype=np.uint64)
    assert (orc.msm(srs[:n], np.zeros((n, 4), dtype=np.uint64)) == inf).all()
    s = np.zeros((n, 4), dtype=np.uint64)
    s[3] = Z.int_to_fr(R - 1)
    assert (orc.msm(srs[:n], s) == orc.g1_neg(srs[3])).all()
    # Repeated points (every base = G): sum s_i G = (sum s_i) G; exercises P = Q.
    G = orc.g1_generator()
    rep = np.tile(G, (n, 1))
    sc = Z.zkml_scalars(24, n)
    total = sum(Z.fr_to_int(x) for x in sc) % R
    assert (orc.msm(rep, sc) == orc.g1_mul(G, Z.int_to_fr(total))).all()
    same = np.tile(Z.int_to_fr(5), (n, 1))
    assert (orc.msm(rep, same) == orc.g1_mul(G, Z.int_to_fr(5 * n))).all()


def test_small_scalar_encoding(orc, srs):
    # x * 2^16 with x < 0 encodes as r - |x| 2^16, i.e. -(|x| 2^16) in F_r.
    q = np.array([-128, -1, 0, 1, 127])
    enc = Z.encode_signed(q, 16)
    for qi, e in zip(q, enc):
        assert Z.fr_to_int(e) == (int(qi) * 65536) % R


def test_evaluation_form_commitment(orc, tau, srs):
    # Commit to the interpolant of v over H: the Lagrange closed form equals
    # the MSM of the O(n^2) INTT coefficients, and the tau form of them.
    for n in (1, 4, 32):
        v = Z.fr_uniform(30 + n, n)
        c = orc.intt(v)
        want = orc.msm(srs[:n], c)
        assert (orc.commit_coeffs_tau(c, tau) == want).all()
        assert (orc.commit_evals_tau(v, tau) == want).all()
    # Lagrange basis sums to 1 (it interpolates the constant 1).
    L = orc.lagrange_at(16, tau)
    assert sum(Z.fr_to_int(x) for x in L) % R == 1
