"""GPU parity of the Mul / MatMul quotient (Sec. 4.4.1):
t = (A B - L)/(X^n - 1) for evaluation vectors a, b over H, L the
interpolant of a o b, and com = [t(tau)]_1.

Small n: every coefficient against the oracle's schoolbook product and long
division, the commitment against the closed form of the oracle's t.  At
2^16 and 2^20 (beyond the oracle's O(n^2)): the identity
t(z) (z^n - 1) = A(z) B(z) - L(z) at random z, with A(z), B(z), L(z) from
the oracle's Lagrange basis values at z, and the commitment against
(A(tau) B(tau) - L(tau)) / (tau^n - 1) G, the Mul verification equation in
the exponent."""
import random

import numpy as np
import pytest

import zkinputs as Z
from _util import pts_equal, to_dev, to_host

pytestmark = pytest.mark.gpu
R = Z.R_MOD


def _mulq(zk, ctx, a, b):
    import torch
    n = a.shape[0]
    t = torch.zeros((max(n - 1, 1), 4), dtype=torch.int64, device="cuda")
    com = torch.zeros(8, dtype=torch.int64, device="cuda")
    zk.zk_mul_quotient(ctx, to_dev(a), to_dev(b), com, t)
    torch.cuda.synchronize()
    return to_host(t)[: n - 1], to_host(com)


def _eval_evals(orc, v, z):
    """Interpolant of v over H evaluated at z (oracle Lagrange values)."""
    Lz = [Z.fr_to_int(x) for x in orc.lagrange_at(v.shape[0], Z.int_to_fr(z))]
    return sum(Z.fr_to_int(a) * l for a, l in zip(v, Lz)) % R


def _horner(t, z):
    y = 0
    for a in reversed([Z.fr_to_int(x) for x in t]):
        y = (y * z + a) % R
    return y


@pytest.mark.parametrize("n", [1, 2, 4, 8, 64, 512, 1024])
def test_mul_quotient_full_oracle(zk, orc, ctx_small, tau, n):
    a = Z.fr_uniform(1100 + n, n)
    b = Z.zkml_scalars(1200 + n, n) if n % 2 else Z.fr_uniform(1200 + n, n)
    t, com = _mulq(zk, ctx_small, a, b)
    ot, exact = orc.mul_quotient(a, b)
    assert exact
    assert np.array_equal(t, ot)
    want = orc.commit_coeffs_tau(ot, tau) if n > 1 else np.zeros(8, np.uint64)
    assert pts_equal(com, want)


@pytest.mark.parametrize("lg", [16, 20])
def test_mul_quotient_at_scale(zk, orc, ctx_big, tau, lg):
    n = 1 << lg
    a = Z.zkml_scalars(1300 + lg, n)
    b = Z.fr_uniform(1400 + lg, n)
    t, com = _mulq(zk, ctx_big, a, b)
    ai = [Z.fr_to_int(x) for x in a]
    bi = [Z.fr_to_int(x) for x in b]
    lv = np.stack([Z.int_to_fr(x * y % R) for x, y in zip(ai, bi)])
    for z in [random.Random(lg).randrange(R), Z.fr_to_int(tau)]:
        A, B, L = _eval_evals(orc, a, z), _eval_evals(orc, b, z), _eval_evals(orc, lv, z)
        lhs = _horner(t, z) * (pow(z, n, R) - 1) % R
        assert lhs == (A * B - L) % R
        if z == Z.fr_to_int(tau):
            tz = (A * B - L) * pow(pow(z, n, R) - 1, R - 2, R) % R
            assert pts_equal(com, orc.g1_mul(orc.g1_generator(), Z.int_to_fr(tz)))


def test_mul_quotient_host_buffers_and_errors(zk, orc, ctx_small, tau):
    import torch
    n = 256
    a = np.ascontiguousarray(Z.fr_uniform(1500, n))
    b = np.ascontiguousarray(Z.fr_uniform(1501, n))
    t = np.zeros((n - 1, 4), np.uint64)
    com = np.zeros(8, np.uint64)
    zk.zk_mul_quotient(ctx_small, a, b, com, t)
    ot, _ = orc.mul_quotient(a, b)
    assert np.array_equal(t, ot) and pts_equal(com, orc.commit_coeffs_tau(ot, tau))
    d = torch.zeros((12, 4), dtype=torch.int64, device="cuda")
    c = torch.zeros(8, dtype=torch.int64, device="cuda")
    with pytest.raises(zk.ZkError) as ei:
        zk.zk_mul_quotient(ctx_small, d, d, c)  # n = 12: not a power of two
    assert ei.value.code == zk.ZK_EINVAL
    big = torch.zeros((1 << 13, 4), dtype=torch.int64, device="cuda")
    with pytest.raises(zk.ZkError) as ei:
        zk.zk_mul_quotient(ctx_small, big, big, c)  # n - 1 > SRS of 2^12
    assert ei.value.code == zk.ZK_ESRS
