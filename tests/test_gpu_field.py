"""GPU parity of the device field arithmetic against the oracle.

Every step of the hot path is built on F_q (curve coordinates) and F_r
(scalars, NTT) Montgomery arithmetic.  zk_field_op runs the device code
(conversion to and from Montgomery form, product, squaring, inverse, sum,
difference) elementwise; each result is compared bit for bit with the
oracle's schoolbook-and-long-division arithmetic.  Inputs: values where
carries and borrows run across all words (0, 1, p - 1, (p +- 1) / 2, 2^k - 1,
2^k, p - 2^k, ...), all pairs of them, and seeded uniform elements."""
import numpy as np
import pytest

import zkinputs as Z
from _util import to_dev, to_host

pytestmark = pytest.mark.gpu


def _edge(M):
    vals = [0, 1, 2, 3, M - 1, M - 2, M - 3, (M - 1) // 2, (M + 1) // 2, (M + 3) // 2]
    for k in (31, 32, 33, 63, 64, 65, 95, 96, 127, 128, 159, 160, 191, 192, 223, 224, 252, 253):
        vals += [(1 << k) - 1, 1 << k, M - (1 << k)]
    return sorted({v % M for v in vals})


def _limbs(xs):
    return np.stack([Z.int_to_fr(x) for x in xs])


def _ints(a):
    return [Z.fr_to_int(v) for v in a]


@pytest.mark.parametrize("field", ["q", "r"])
def test_field_ops_match_oracle(zk, orc, field):
    import torch
    M = Z.Q_MOD if field == "q" else Z.R_MOD
    f_orc = orc.FQ if field == "q" else orc.FR
    f_dev = zk.ZK_FIELD_Q if field == "q" else zk.ZK_FIELD_R
    edge = _edge(M)
    rng = np.random.default_rng(31 if field == "q" else 37)
    uni = [int.from_bytes(rng.bytes(32), "little") % M for _ in range(1500)]
    a = [x for x in edge for _ in edge] + uni + edge
    b = [y for _ in edge for y in edge] + uni[::-1] + edge[::-1]
    A, B = _limbs(a), _limbs(b)
    da, db = to_dev(A), to_dev(B)
    expect = {
        zk.ZK_FOP_MUL: lambda x, y: orc.fmul(f_orc, x, y),
        zk.ZK_FOP_SQR: lambda x, y: orc.fmul(f_orc, x, x),
        # 0 has no inverse; the entry point maps it to 0 (so does the oracle).
        zk.ZK_FOP_INV: lambda x, y: orc.finv(f_orc, x) if x.any() else np.zeros(4, np.uint64),
        zk.ZK_FOP_ADD: lambda x, y: orc.fadd(f_orc, x, y),
        zk.ZK_FOP_SUB: lambda x, y: orc.fsub(f_orc, x, y),
    }
    for op, fn in expect.items():
        out = torch.zeros_like(da)
        zk.zk_field_op(f_dev, op, da, db, out)
        torch.cuda.synchronize()
        got = to_host(out)
        want = np.stack([fn(A[i], B[i]) for i in range(len(a))])
        bad = np.nonzero(~np.all(got == want, axis=1))[0]
        assert bad.size == 0, (op, [(a[i], b[i]) for i in bad[:4]])


@pytest.mark.parametrize("field", ["q", "r"])
def test_field_mul_by_constant_matches_oracle(zk, orc, field):
    """The product by a constant with a precomputed quotient (ZK_FOP_MULC,
    the NTT's butterfly product): every pair of carry-edge values and
    uniform pairs, each first operand fed as all four representatives
    a + m p, m < 4 (elements 4j .. 4j + 3), so the quotient's truncation
    and both corrections are exercised up to the top of [0, 4p); the
    result must be the canonical a b mod p."""
    import torch
    M = Z.Q_MOD if field == "q" else Z.R_MOD
    f_orc = orc.FQ if field == "q" else orc.FR
    f_dev = zk.ZK_FIELD_Q if field == "q" else zk.ZK_FIELD_R
    edge = _edge(M)
    rng = np.random.default_rng(41 if field == "q" else 43)
    uni = [int.from_bytes(rng.bytes(32), "little") % M for _ in range(1000)]
    a = [x for x in edge for _ in edge] + uni
    b = [y for _ in edge for y in edge] + uni[::-1]
    A, B = np.repeat(_limbs(a), 4, axis=0), np.repeat(_limbs(b), 4, axis=0)
    out = torch.zeros((A.shape[0], 4), dtype=torch.int64, device="cuda")
    zk.zk_field_op(f_dev, zk.ZK_FOP_MULC, to_dev(A), to_dev(B), out)
    torch.cuda.synchronize()
    got = to_host(out)
    want = np.repeat(np.stack([orc.fmul(f_orc, _limbs([x])[0], _limbs([y])[0]) for x, y in zip(a, b)]), 4, axis=0)
    bad = np.nonzero(~np.all(got == want, axis=1))[0]
    assert bad.size == 0, [(a[i // 4], b[i // 4], i % 4) for i in bad[:4]]


@pytest.mark.parametrize("field", ["q", "r"])
def test_field_mul_sub_mul_matches_oracle(zk, orc, field):
    """a_i b_i - a_m b_m with m = n - 1 - i (ZK_FOP_MULSUB), the form every
    point addition and doubling takes for Y; F_q reduces the 512-bit
    difference once, lifting it by p 2^256 when negative.  Three layouts:
    every pair of edge values against its mirror pair (both signs, products
    near 0 and near p^2), swapped mirrors (a b - b a = 0 exactly) around
    uniform pairs, and an odd length whose middle element meets itself."""
    import torch
    M = Z.Q_MOD if field == "q" else Z.R_MOD
    f_orc = orc.FQ if field == "q" else orc.FR
    f_dev = zk.ZK_FIELD_Q if field == "q" else zk.ZK_FIELD_R
    edge = _edge(M)
    rng = np.random.default_rng(43 if field == "q" else 47)
    uni = [(int.from_bytes(rng.bytes(32), "little") % M, int.from_bytes(rng.bytes(32), "little") % M)
           for _ in range(1001)]
    grid = [(x, y) for x in edge for y in edge]
    layouts = [grid, grid + uni + [(y, x) for (x, y) in reversed(grid)], uni]
    for pairs in layouts:
        a = [x for x, _ in pairs]
        b = [y for _, y in pairs]
        A, B = _limbs(a), _limbs(b)
        out = torch.zeros((len(a), 4), dtype=torch.int64, device="cuda")
        zk.zk_field_op(f_dev, zk.ZK_FOP_MULSUB, to_dev(A), to_dev(B), out)
        torch.cuda.synchronize()
        got = to_host(out)
        n = len(a)
        want = np.stack([orc.fsub(f_orc, orc.fmul(f_orc, A[i], B[i]), orc.fmul(f_orc, A[n - 1 - i], B[n - 1 - i]))
                         for i in range(n)])
        bad = np.nonzero(~np.all(got == want, axis=1))[0]
        assert bad.size == 0, [(a[i], b[i], a[n - 1 - i], b[n - 1 - i]) for i in bad[:4]]


def test_field_inverse_round_trip(zk, orc):
    """x * x^-1 = 1 for every nonzero input, in both fields (an invariant that
    holds without the oracle)."""
    import torch
    rng = np.random.default_rng(41)
    for M, f in ((Z.Q_MOD, zk.ZK_FIELD_Q), (Z.R_MOD, zk.ZK_FIELD_R)):
        xs = _edge(M)[1:] + [int.from_bytes(rng.bytes(32), "little") % M or 1 for _ in range(4000)]
        d = to_dev(_limbs(xs))
        inv = torch.zeros_like(d)
        zk.zk_field_op(f, zk.ZK_FOP_INV, d, None, inv)
        prod = torch.zeros_like(d)
        zk.zk_field_op(f, zk.ZK_FOP_MUL, d, inv, prod)
        torch.cuda.synchronize()
        assert all(v == 1 for v in _ints(to_host(prod)))


def test_field_op_rejects_bad_arguments(zk):
    import torch
    d = torch.zeros((4, 4), dtype=torch.int64, device="cuda")
    for args in ((7, zk.ZK_FOP_MUL, d, d, d), (zk.ZK_FIELD_Q, 9, d, d, d),
                 (zk.ZK_FIELD_Q, zk.ZK_FOP_MUL, d, None, d)):
        with pytest.raises(zk.ZkError) as ei:
            zk.zk_field_op(*args, n=4)
        assert ei.value.code == zk.ZK_EINVAL
    h = np.zeros((4, 4), np.uint64)
    with pytest.raises(zk.ZkError):
        zk.zk_field_op(zk.ZK_FIELD_R, zk.ZK_FOP_SQR, h, None, h, n=4)
