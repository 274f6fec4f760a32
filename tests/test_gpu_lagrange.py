"""Commitments through the Lagrange basis of H: the basis points derived from
the SRS (an inverse DFT over G1) equal [L_k(tau)]_1 computed by the oracle's
closed form, and every evaluation-form commitment, leaf and fold is the same
point by either route (INTT + SRS, or Lagrange basis)."""
import numpy as np
import pytest

import zkinputs as Z
from _util import pts_equal, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture
def lagrange_route(zk, ctx_small):
    zk.zk_set_commit_route(ctx_small, zk.ZK_ROUTE_LAGRANGE)
    yield
    zk.zk_set_commit_route(ctx_small, zk.ZK_ROUTE_INTT)


def test_lagrange_basis_points_match_closed_form(zk, orc, ctx_small, tau):
    import torch
    n = 1 << 10
    L = orc.lagrange_at(n, tau)
    G = orc.g1_generator()
    ks = [0, 1, 2, 511, n - 1]
    units = []
    for k in ks:
        u = np.zeros((n, 4), np.uint64)
        u[k, 0] = 1
        units.append(to_dev(u))
    out = torch.zeros((len(ks), 8), dtype=torch.int64, device="cuda")
    zk.zk_commit_batch(ctx_small, units, out, flags=zk.ZK_LAGRANGE)
    torch.cuda.synchronize()
    got = to_host(out)
    for i, k in enumerate(ks):
        assert pts_equal(got[i], orc.g1_mul(G, L[k])), k


@pytest.mark.parametrize("dist", ["int8", "uniform"])
def test_lagrange_equals_intt_route(zk, orc, ctx_small, tau, dist):
    import torch
    lens = [1, 2, 3, 64, 100, 1024, 3000, 4096]
    vecs = [Z.zkml_scalars(1500 + i, l) if dist == "int8" else Z.fr_uniform(1500 + i, l)
            for i, l in enumerate(lens)]
    dv = [to_dev(v) for v in vecs]
    a = torch.zeros((len(lens), 8), dtype=torch.int64, device="cuda")
    b = torch.zeros_like(a)
    zk.zk_commit_batch(ctx_small, dv, a, flags=zk.ZK_EVALS)
    zk.zk_commit_batch(ctx_small, dv, b, flags=zk.ZK_LAGRANGE)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    got = to_host(b)
    for k in (3, 6):
        n2 = 1 << (lens[k] - 1).bit_length()
        vp = np.zeros((n2, 4), np.uint64)
        vp[:lens[k]] = vecs[k]
        assert pts_equal(got[k], orc.commit_evals_tau(vp, tau))


def test_lagrange_route_leaf_fold_and_tree(zk, orc, ctx_small, tau, lagrange_route):
    import torch
    from test_gpu_fold import DevAcc, leaf_vectors
    count, n = 8, 512
    devs, orcs = [], []
    for j in range(count):
        m1, m2, m4 = leaf_vectors(j, n)
        d = DevAcc(zk, n)
        d.set_leaf(m1, m2, m4)
        devs.append(d)
        orcs.append(orc.leaf_init(m1, m2, m4, orc.COMMIT_TAU, tau=tau))
    zk.zk_leaf_init(ctx_small, [d.desc for d in devs])
    torch.cuda.synchronize()
    for d, o in zip(devs, orcs):
        assert np.array_equal(to_host(d.x).reshape(44), o.inst)
    gam = np.concatenate([Z.gammas(l, count >> l) for l in range(1, 4)])
    want = orc.fold_tree(orcs, gam, orc.COMMIT_TAU, tau=tau)
    root = DevAcc(zk, n)
    zk.zk_fold_tree(ctx_small, [d.desc for d in devs], np.ascontiguousarray(gam), root.desc)
    torch.cuda.synchronize()
    got = root.oracle(orc)
    assert np.array_equal(got.m, want.m) and np.array_equal(got.e, want.e)
    assert np.array_equal(got.inst, want.inst)


def test_lagrange_route_paper_size_leaves(zk, orc, ctx_big, tau):
    """64 leaves of 2^16: leaf commitments by both routes agree; the quantised
    witness values stay one-window scalars on the Lagrange route."""
    import torch
    from test_gpu_fold import DevAcc, leaf_vectors
    count, n = 64, 1 << 16
    sets = []
    for route in (zk.ZK_ROUTE_INTT, zk.ZK_ROUTE_LAGRANGE):
        zk.zk_set_commit_route(ctx_big, route)
        devs = []
        for j in range(count):
            d = DevAcc(zk, n)
            d.set_leaf(*leaf_vectors(j, n))
            devs.append(d)
        zk.zk_leaf_init(ctx_big, [d.desc for d in devs])
        torch.cuda.synchronize()
        sets.append([d.x.clone() for d in devs])
    zk.zk_set_commit_route(ctx_big, zk.ZK_ROUTE_INTT)
    for a, b in zip(*sets):
        assert torch.equal(a, b)
    x0 = to_host(sets[1][0]).reshape(44)
    m1, _, _ = leaf_vectors(0, n)
    assert pts_equal(x0[:8], orc.commit_evals_tau(m1, tau))
