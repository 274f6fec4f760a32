"""GPU parity of the fold for the degree-3 relation m1 o m2 o m3 - mu^2 m4 = e
(Sec. 4.2 with d = 3: two cross terms E1, E2) against the oracle: leaves,
one fold with its two cross-term commitments, folds of folded accumulators
and a 16-leaf tree, every vector and instance point bit for bit, on both
commitment routes (INTT + SRS, Lagrange basis)."""
import numpy as np
import pytest

import zkinputs as Z
from _util import acc_to_oracle, pts_equal, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx3(zk):
    ctx = zk.zk_init(0)
    zk.zk_srs_generate(ctx, Z.tau(0), 1 << 12)
    zk.zk_set_fold_degree(ctx, 3)
    yield ctx
    zk.zk_destroy(ctx)


@pytest.fixture
def orc3(orc):
    orc.set_degree(3)
    yield orc
    orc.set_degree(2)


class Acc3:
    def __init__(self, zk, n, seed):
        import torch
        self.m = torch.zeros((4, n, 4), dtype=torch.int64, device="cuda")
        self.e = torch.zeros((n, 4), dtype=torch.int64, device="cuda")
        self.x = torch.zeros(44, dtype=torch.int64, device="cuda")
        self.desc = zk.make_acc(self.m, self.e, self.x)
        self.w = [Z.zkml_scalars(seed + i, n) for i in range(3)]
        for i in range(3):
            self.m[i].copy_(to_dev(self.w[i]))

    def oracle(self, orc):
        return acc_to_oracle(orc, self.m, self.e, self.x)


def _same(a, b):
    return np.array_equal(a.m, b.m) and np.array_equal(a.e, b.e) and np.array_equal(a.inst, b.inst)


@pytest.mark.parametrize("route", ["intt", "lagrange"])
def test_degree3_leaf_fold_and_refold(zk, orc3, ctx3, route):
    import torch
    orc = orc3
    tau = Z.tau(0)
    zk.zk_set_commit_route(ctx3, zk.ZK_ROUTE_LAGRANGE if route == "lagrange" else zk.ZK_ROUTE_INTT)
    try:
        n = 1 << 9
        accs = [Acc3(zk, n, 2000 + 10 * i) for i in range(4)]
        zk.zk_leaf_init(ctx3, [a.desc for a in accs])
        torch.cuda.synchronize()
        ol = [orc.leaf_init(*a.w, orc.COMMIT_TAU, tau=tau) for a in accs]
        for a, o in zip(accs, ol):
            assert _same(a.oracle(orc), o)
        g = Z.gammas(1, 2)
        E = torch.zeros(16, dtype=torch.int64, device="cuda")
        zk.zk_fold(ctx3, accs[0].desc, accs[1].desc, to_dev(g[0]), accs[1].desc, E)
        zk.zk_fold(ctx3, accs[2].desc, accs[3].desc, g[1], accs[3].desc)
        torch.cuda.synchronize()
        o1, oE = orc.fold(ol[0], ol[1], g[0], orc.COMMIT_TAU, tau=tau)
        o3, _ = orc.fold(ol[2], ol[3], g[1], orc.COMMIT_TAU, tau=tau)
        assert _same(accs[1].oracle(orc), o1)
        assert pts_equal(to_host(E)[:8], oE[:8]) and pts_equal(to_host(E)[8:], oE[8:])
        assert _same(accs[3].oracle(orc), o3)
        g2 = Z.gammas(2, 1)[0]
        zk.zk_fold(ctx3, accs[1].desc, accs[3].desc, g2, accs[3].desc)
        torch.cuda.synchronize()
        root, _ = orc.fold(o1, o3, g2, orc.COMMIT_TAU, tau=tau)
        got = accs[3].oracle(orc)
        assert _same(got, root)
        assert orc.decide_relation(got) == 0
    finally:
        zk.zk_set_commit_route(ctx3, zk.ZK_ROUTE_INTT)


def test_degree3_tree(zk, orc3, ctx3):
    import torch
    orc = orc3
    tau = Z.tau(0)
    n, count = 1 << 8, 16
    accs = [Acc3(zk, n, 3000 + 10 * i) for i in range(count)]
    zk.zk_leaf_init(ctx3, [a.desc for a in accs])
    ol = [orc.leaf_init(*a.w, orc.COMMIT_TAU, tau=tau) for a in accs]
    gam = np.concatenate([Z.gammas(l, count >> l) for l in range(1, 5)])
    root = Acc3(zk, n, 0)
    zk.zk_fold_tree(ctx3, [a.desc for a in accs], to_dev(gam), root.desc)
    torch.cuda.synchronize()
    want = orc.fold_tree(ol, gam, orc.COMMIT_TAU, tau=tau)
    got = root.oracle(orc)
    assert _same(got, want)
    assert orc.decide_relation(got) == 0


def test_fold_degree_rejects_bad_values(zk, ctx3):
    for d in (0, 1, 4):
        with pytest.raises(zk.ZkError) as ei:
            zk.zk_set_fold_degree(ctx3, d)
        assert ei.value.code == zk.ZK_EINVAL
