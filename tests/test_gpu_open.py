"""GPU parity of KZG opening (Sec. 2.1) against the oracle.

zk_open returns y = f(x), the quotient q = (f - y)/(X - x) and the proof
[q(tau)]_1; zk_open_batch returns y_i = f_i(x) and the proof of
sum_i gamma^i (f_i - y_i)/(X - x).  Compared bit for bit with the oracle's
synthetic division (y, every quotient coefficient) and with the closed-form
commitment of the oracle's quotient (the proof); the KZG verification
equation in the exponent, (tau - x) proof = com - y G, is checked with the
GPU's own commitment of f."""
import random

import numpy as np
import pytest

import zkinputs as Z
from _util import pts_equal, to_dev, to_host

pytestmark = pytest.mark.gpu
R = Z.R_MOD


def _open(zk, ctx, c, x, want_q=True):
    import torch
    n = c.shape[0]
    y = torch.zeros(4, dtype=torch.int64, device="cuda")
    proof = torch.zeros(8, dtype=torch.int64, device="cuda")
    q = torch.zeros((max(n - 1, 1), 4), dtype=torch.int64, device="cuda") if want_q else None
    zk.zk_open(ctx, to_dev(c), to_dev(Z.int_to_fr(x)), y, proof, q)
    torch.cuda.synchronize()
    return to_host(y), to_host(proof), (to_host(q)[: n - 1] if want_q else None)


@pytest.mark.parametrize("n", [1, 2, 3, 31, 32, 33, 1000, 4096, 4097])
def test_open_small_full_oracle(zk, orc, ctx_small, tau, n):
    rng = random.Random(n)
    c = Z.fr_uniform(900 + n, n)
    for x in [0, 1, R - 1, rng.randrange(R)]:
        y, proof, q = _open(zk, ctx_small, c, x)
        oy, oq = orc.open_poly(c, Z.int_to_fr(x))
        assert np.array_equal(y, oy), (n, x)
        assert np.array_equal(q, oq), (n, x)
        want = orc.commit_coeffs_tau(oq, tau) if n > 1 else np.zeros(8, np.uint64)
        assert pts_equal(proof, want), (n, x)


def test_open_kzg_equation_with_gpu_commitment(zk, orc, ctx_small, tau):
    import torch
    t = Z.fr_to_int(tau)
    G = orc.g1_generator()
    n = 4000
    c = Z.zkml_scalars(77, n)
    x = 123456789
    y, proof, _ = _open(zk, ctx_small, c, x, want_q=False)
    com = torch.zeros(8, dtype=torch.int64, device="cuda")
    zk.zk_commit(ctx_small, to_dev(c), com)
    torch.cuda.synchronize()
    lhs = orc.g1_mul(proof, Z.int_to_fr((t - x) % R))
    rhs = orc.g1_add(to_host(com), orc.g1_neg(orc.g1_mul(G, y)))
    assert pts_equal(lhs, rhs)


def test_open_at_a_root(zk, orc, ctx_small, tau):
    # f(X) = (X - 5) g(X): y = 0 and the quotient is g.
    g = Z.fr_uniform(31, 300)
    gi = [Z.fr_to_int(v) for v in g]
    f = [0] * 301
    for i, a in enumerate(gi):
        f[i + 1] = (f[i + 1] + a) % R
        f[i] = (f[i] - 5 * a) % R
    y, proof, q = _open(zk, ctx_small, np.stack([Z.int_to_fr(v) for v in f]), 5)
    assert Z.fr_to_int(y) == 0 and np.array_equal(q, g)
    assert pts_equal(proof, orc.commit_coeffs_tau(g, tau))


def test_open_at_scale_2_20(zk, orc, ctx_big, tau):
    n = 1 << 20
    c = Z.fr_uniform(901, n)
    x = 0x1234_5678_9ABC_DEF0_1234
    y, proof, q = _open(zk, ctx_big, c, x)
    oy, oq = orc.open_poly(c, Z.int_to_fr(x))
    assert np.array_equal(y, oy)
    assert np.array_equal(q, oq)
    assert pts_equal(proof, orc.commit_coeffs_tau(oq, tau))


def test_open_host_buffers(zk, orc, ctx_small, tau):
    n = 777
    c = np.ascontiguousarray(Z.fr_uniform(902, n))
    x = np.ascontiguousarray(Z.int_to_fr(42))
    y = np.zeros(4, np.uint64)
    proof = np.zeros(8, np.uint64)
    q = np.zeros((n - 1, 4), np.uint64)
    zk.zk_open(ctx_small, c, x, y, proof, q)
    oy, oq = orc.open_poly(c, x)
    assert np.array_equal(y, oy) and np.array_equal(q, oq)
    assert pts_equal(proof, orc.commit_coeffs_tau(oq, tau))


def test_open_batch_matches_oracle(zk, orc, ctx_small, tau):
    import torch
    lens = [1, 5, 100, 4096, 2000, 33]
    polys = [Z.fr_uniform(950 + i, m) for i, m in enumerate(lens)]
    x, gamma = Z.int_to_fr(987654321), Z.fr_uniform(960, 1)[0]
    ys = torch.zeros((len(lens), 4), dtype=torch.int64, device="cuda")
    proof = torch.zeros(8, dtype=torch.int64, device="cuda")
    zk.zk_open_batch(ctx_small, [to_dev(p) for p in polys], to_dev(x), to_dev(gamma), ys, proof)
    torch.cuda.synchronize()
    oys, oh = orc.open_batch(polys, x, gamma)
    assert np.array_equal(to_host(ys), oys)
    assert pts_equal(to_host(proof), orc.commit_coeffs_tau(oh, tau))
    # host inputs and outputs give the same
    hys = np.zeros((len(lens), 4), np.uint64)
    hproof = np.zeros(8, np.uint64)
    zk.zk_open_batch(ctx_small, [np.ascontiguousarray(p) for p in polys], np.ascontiguousarray(x),
                     np.ascontiguousarray(gamma), hys, hproof)
    assert np.array_equal(hys, oys) and pts_equal(hproof, to_host(proof))


def test_open_rejects_bad_arguments(zk, ctx_small):
    import torch
    c = torch.zeros((8, 4), dtype=torch.int64, device="cuda")
    y = torch.zeros(4, dtype=torch.int64, device="cuda")
    p = torch.zeros(8, dtype=torch.int64, device="cuda")
    with pytest.raises(zk.ZkError) as ei:
        zk.zk_open(ctx_small, c, y, y, p, n=0)
    assert ei.value.code == zk.ZK_EINVAL
    big = torch.zeros(((1 << 12) + 2, 4), dtype=torch.int64, device="cuda")
    with pytest.raises(zk.ZkError) as ei:
        zk.zk_open(ctx_small, big, y, y, p)
    assert ei.value.code == zk.ZK_ESRS
