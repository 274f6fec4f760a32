"""CUDA-graph plans: a captured batched commitment and a captured fold tree
give the oracle's results (closed-form commitments of the padded
interpolants; the sequential oracle tree), on the capture's warm-up run and
on every replay, including replays on new inputs."""
import numpy as np
import pytest

import zkinputs as Z
from _util import pts_equal, to_dev, to_host

pytestmark = pytest.mark.gpu


def _padded_commit(orc, v, tau):
    """Oracle commitment of an evaluation vector zero-padded to a power of two
    (the padding zk_commit_batch applies with ZK_EVALS)."""
    n2 = 1 << (len(v) - 1).bit_length()
    vp = np.zeros((n2, 4), np.uint64)
    vp[:len(v)] = v
    return orc.commit_evals_tau(vp, tau)


@pytest.mark.parametrize("flags", ["evals", "lagrange"])
def test_plan_commit_batch_matches_oracle(zk, orc, ctx_small, tau, flags):
    import torch
    fl = zk.ZK_EVALS if flags == "evals" else zk.ZK_LAGRANGE
    lens = [64, 1000, 4096, 7, 2048]
    host = [Z.zkml_scalars(1100 + i, l) for i, l in enumerate(lens)]
    host[1] = Z.fr_uniform(1150, lens[1])  # one full-width vector in the batch
    vecs = [to_dev(v) for v in host]
    want = [_padded_commit(orc, v, tau) for v in host]
    ref = torch.zeros((len(lens), 8), dtype=torch.int64, device="cuda")
    zk.zk_commit_batch(ctx_small, vecs, ref, flags=fl)
    out = torch.zeros_like(ref)
    plan = zk.zk_plan_commit_batch(ctx_small, vecs, out, flags=fl)
    try:
        assert zk.zk_plan_nodes(plan) > 10
        torch.cuda.synchronize()
        got = to_host(out)  # the capture's warm-up run
        for k in range(len(lens)):
            assert pts_equal(got[k], want[k]), k
        assert torch.equal(out, ref)
        for rep in range(2):  # replays, on new inputs the second time
            out.zero_()
            if rep == 1:
                host[2] = Z.zkml_scalars(1200, lens[2])
                host[0] = Z.fr_uniform(1201, lens[0])
                for k in (0, 2):
                    vecs[k].copy_(to_dev(host[k]))
                    want[k] = _padded_commit(orc, host[k], tau)
            zk.zk_plan_launch(plan)
            torch.cuda.synchronize()
            got = to_host(out)
            for k in range(len(lens)):
                assert pts_equal(got[k], want[k]), (rep, k)
    finally:
        zk.zk_plan_destroy(plan)


def test_plan_rejects_host_buffers(zk, ctx_small):
    vec = np.ascontiguousarray(Z.fr_uniform(1300, 16))
    out = np.zeros(8, dtype=np.uint64)
    with pytest.raises(zk.ZkError) as ei:
        zk.zk_plan_commit_batch(ctx_small, [vec], out)
    assert ei.value.code == zk.ZK_EINVAL


def test_plan_fold_tree(zk, orc, ctx_small, tau):
    import torch
    from test_gpu_fold import DevAcc, leaf_vectors
    count, n = 8, 256
    devs, orcs = [], []
    for j in range(count):
        d = DevAcc(zk, n)
        vs = leaf_vectors(j, n)
        d.set_leaf(*vs)
        devs.append(d)
        orcs.append(orc.leaf_init(*vs, orc.COMMIT_TAU, tau=tau))
    zk.zk_leaf_init(ctx_small, [d.desc for d in devs])
    torch.cuda.synchronize()
    saved = [(d.m.clone(), d.e.clone(), d.x.clone()) for d in devs]
    gam_h = np.concatenate([Z.gammas(l, count >> l) for l in range(1, 4)])
    gam = to_dev(gam_h)
    want = orc.fold_tree(orcs, gam_h, orc.COMMIT_TAU, tau=tau)
    ref = DevAcc(zk, n)
    zk.zk_fold_tree(ctx_small, [d.desc for d in devs], gam, ref.desc)
    root = DevAcc(zk, n)

    def restore():
        for d, (m, e, x) in zip(devs, saved):
            d.m.copy_(m)
            d.e.copy_(e)
            d.x.copy_(x)

    restore()
    plan = zk.zk_plan_fold_tree(ctx_small, [d.desc for d in devs], gam, root.desc)
    try:
        for _ in range(2):
            restore()
            root.m.zero_()
            zk.zk_plan_launch(plan)
            torch.cuda.synchronize()
            got = root.oracle(orc)
            assert np.array_equal(got.m, want.m) and np.array_equal(got.e, want.e)
            assert np.array_equal(got.inst, want.inst)
            assert torch.equal(root.x, ref.x)
    finally:
        zk.zk_plan_destroy(plan)
