"""GPU parity of the generalised-Mira fold and the parallel fold tree
(Sec. 4.2) against the oracle's sequential fold.

Small cases compare every output (witness vectors, error vector, instance
points, mu, E1) bit-exactly.  The 1024-leaf, 2^16 tree (the paper-scale
accumulation workload) compares the whole root witness (m_1..m_4, e, every
position) and mu with the oracle's sequential tree run without commitments,
checks the decider relation on the root, and checks the root commitments
against fresh closed-form commitments of the root witness (homomorphism)."""
import numpy as np
import pytest

import zkinputs as Z
from _util import acc_to_oracle, pts_equal, to_dev, to_host

pytestmark = pytest.mark.gpu
R = Z.R_MOD


def leaf_vectors(j, n):
    """Witness of leaf j of the fold-tree workload: m1, m2, m4 quantised int8
    values times 2^16 (stream 9 * 2^20 + 4 j + i)."""
    base = (9 << 20) + 4 * j
    return Z.zkml_scalars(base, n), Z.zkml_scalars(base + 1, n), Z.zkml_scalars(base + 3, n)


class DevAcc:
    def __init__(self, zk, n):
        import torch
        self.m = torch.zeros((4, n, 4), dtype=torch.int64, device="cuda")
        self.e = torch.zeros((n, 4), dtype=torch.int64, device="cuda")
        self.x = torch.zeros(44, dtype=torch.int64, device="cuda")
        self.desc = zk.make_acc(self.m, self.e, self.x)

    def set_leaf(self, m1, m2, m4):
        import torch
        for i, v in ((0, m1), (1, m2), (3, m4)):
            self.m[i].copy_(to_dev(v))

    def oracle(self, orc):
        return acc_to_oracle(orc, self.m, self.e, self.x)


def _leaves(zk, ctx, orc, tau, count, n, with_oracle=True):
    import torch
    devs, orcs = [], []
    for j in range(count):
        m1, m2, m4 = leaf_vectors(j, n)
        d = DevAcc(zk, n)
        d.set_leaf(m1, m2, m4)
        devs.append(d)
        if with_oracle:
            orcs.append(orc.leaf_init(m1, m2, m4, orc.COMMIT_TAU, tau=tau))
    zk.zk_leaf_init(ctx, [d.desc for d in devs])
    torch.cuda.synchronize()
    return devs, orcs


def _same_acc(a, b):
    return (np.array_equal(a.m, b.m) and np.array_equal(a.e, b.e)
            and np.array_equal(a.inst, b.inst))


def test_leaf_init(zk, orc, ctx_small, tau):
    devs, orcs = _leaves(zk, ctx_small, orc, tau, 3, 256)
    for d, o in zip(devs, orcs):
        assert _same_acc(d.oracle(orc), o)


@pytest.mark.parametrize("alias", [False, True])
def test_single_fold(zk, orc, ctx_small, tau, alias):
    import torch
    n = 512
    (L, R_), (oL, oR) = _leaves(zk, ctx_small, orc, tau, 2, n)
    g = Z.gammas(1, 1)[0]
    want, E1 = orc.fold(oL, oR, g, orc.COMMIT_TAU, tau=tau)
    out = R_ if alias else DevAcc(zk, n)
    E1d = torch.zeros(8, dtype=torch.int64, device="cuda")
    zk.zk_fold(ctx_small, L.desc, R_.desc, np.ascontiguousarray(g), out.desc, E1d)
    torch.cuda.synchronize()
    assert _same_acc(out.oracle(orc), want)
    assert pts_equal(to_host(E1d), E1)
    # Folding two folded accumulators (mu != 1, e != 0, E != infinity).
    (A, B), (oA, oB) = _leaves(zk, ctx_small, orc, tau, 2, n)
    oA2, _ = orc.fold(oA, oB, Z.gammas(1, 2)[1], orc.COMMIT_TAU, tau=tau)
    zk.zk_fold(ctx_small, A.desc, B.desc, to_dev(Z.gammas(1, 2)[1]), B.desc)
    g2 = Z.gammas(2, 1)[0]
    want2, _ = orc.fold(want, oA2, g2, orc.COMMIT_TAU, tau=tau)
    out2 = DevAcc(zk, n)
    zk.zk_fold(ctx_small, out.desc, B.desc, np.ascontiguousarray(g2), out2.desc)
    torch.cuda.synchronize()
    assert _same_acc(out2.oracle(orc), want2)


@pytest.mark.parametrize("count,n", [(2, 64), (8, 256), (16, 1024)])
def test_fold_tree_small(zk, orc, ctx_small, tau, count, n):
    devs, orcs = _leaves(zk, ctx_small, orc, tau, count, n)
    gam = np.concatenate([Z.gammas(l, count >> l) for l in range(1, count.bit_length())])
    want = orc.fold_tree(orcs, gam, orc.COMMIT_TAU, tau=tau)
    root = DevAcc(zk, n)
    zk.zk_fold_tree(ctx_small, [d.desc for d in devs], np.ascontiguousarray(gam), root.desc)
    import torch
    torch.cuda.synchronize()
    assert _same_acc(root.oracle(orc), want)


def test_fold_tree_checkpoint_resume(zk, orc, ctx_small, tau):
    """Checkpoint and resume of the fold tree: 16 leaves of 2^10 folded two
    levels (zk_fold_tree_levels), the four level-2 accumulators copied to
    host memory and the device state dropped; a fresh context with the same
    SRS restores them and folds the remaining levels with the remaining
    challenges.  The root equals the oracle's uninterrupted tree."""
    import torch
    count, n = 16, 1 << 10
    devs, orcs = _leaves(zk, ctx_small, orc, tau, count, n)
    gam = np.ascontiguousarray(np.concatenate([Z.gammas(l, count >> l) for l in range(1, count.bit_length())]))
    want = orc.fold_tree(orcs, gam, orc.COMMIT_TAU, tau=tau)
    for bad in (0, 5):
        with pytest.raises(zk.ZkError) as ei:
            zk.zk_fold_tree_levels(ctx_small, [d.desc for d in devs], gam, bad)
        assert ei.value.code == zk.ZK_EINVAL
    slots = zk.zk_fold_tree_levels(ctx_small, [d.desc for d in devs], gam, 2)
    torch.cuda.synchronize()
    assert slots == [3, 7, 11, 15]
    saved = [(devs[k].m.cpu(), devs[k].e.cpu(), devs[k].x.cpu()) for k in slots]
    del devs
    torch.cuda.empty_cache()
    ctx = zk.zk_init(0)
    try:
        zk.zk_srs_generate(ctx, tau, n)
        restored = []
        for m, e, x in saved:
            d = DevAcc(zk, n)
            d.m.copy_(m)
            d.e.copy_(e)
            d.x.copy_(x)
            restored.append(d)
        root = DevAcc(zk, n)
        used = count - (count >> 2)
        zk.zk_fold_tree(ctx, [d.desc for d in restored], np.ascontiguousarray(gam[used:]), root.desc)
        torch.cuda.synchronize()
        assert _same_acc(root.oracle(orc), want)
    finally:
        zk.zk_destroy(ctx)


def test_fold_tree_paper_scale(zk, orc, ctx_big, tau):
    """1024 leaves of n = 2^16 (about 10 GiB resident), 10 levels, 1023 folds."""
    import torch
    count, n = 1024, 1 << 16
    # Oracle storage, stacked (10 GiB of host memory; the tree runs in place).
    om = np.zeros((count, 4, n, 4), np.uint64)
    oe = np.zeros((count, n, 4), np.uint64)
    oi = np.zeros((count, orc.INST_LIMBS), np.uint64)
    devs = []
    for j in range(count):
        om[j, 0], om[j, 1], om[j, 3] = leaf_vectors(j, n)
        d = DevAcc(zk, n)
        d.set_leaf(om[j, 0], om[j, 1], om[j, 3])
        devs.append(d)
    zk.zk_leaf_init(ctx_big, [d.desc for d in devs])
    gam = np.concatenate([Z.gammas(l, count >> l) for l in range(1, 11)])
    root = DevAcc(zk, n)
    zk.zk_fold_tree(ctx_big, [d.desc for d in devs], np.ascontiguousarray(gam), root.desc)
    torch.cuda.synchronize()
    got = root.oracle(orc)
    del devs
    torch.cuda.empty_cache()
    # The oracle's sequential tree over every position (witness side only).
    for j in range(count):
        orc.leaf_init_into(om[j], oe[j], oi[j], orc.COMMIT_NONE)
    orc.fold_tree_stacked(om, oe, oi, gam, orc.COMMIT_NONE)
    assert np.array_equal(got.m, om[0]) and np.array_equal(got.e, oe[0])
    assert np.array_equal(got.mu, oi[0, 40:44])
    del om, oe, oi
    # Decider on the whole root and homomorphism of its commitments.
    assert orc.decide_relation(got) == 0
    for i in range(4):
        assert pts_equal(got.C[i], orc.commit_evals_tau(got.m[i], tau)), i
    assert pts_equal(got.E, orc.commit_evals_tau(got.e, tau))
