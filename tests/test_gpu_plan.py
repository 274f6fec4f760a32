"""CUDA-graph plans: a captured batched commitment and a captured fold tree
replay to exactly the results of the direct calls."""
import numpy as np
import pytest

import zkinputs as Z
from _util import pts_equal, to_dev, to_host

pytestmark = pytest.mark.gpu


def test_plan_commit_batch_replays_direct_result(zk, ctx_small):
    import torch
    lens = [64, 1000, 4096, 7, 2048]
    vecs = [to_dev(Z.zkml_scalars(1100 + i, l)) for i, l in enumerate(lens)]
    ref = torch.zeros((len(lens), 8), dtype=torch.int64, device="cuda")
    zk.zk_commit_batch(ctx_small, vecs, ref, flags=zk.ZK_EVALS)
    out = torch.zeros_like(ref)
    plan = zk.zk_plan_commit_batch(ctx_small, vecs, out, flags=zk.ZK_EVALS)
    try:
        assert zk.zk_plan_nodes(plan) > 10
        torch.cuda.synchronize()
        assert torch.equal(out, ref)  # the capture's warm-up run
        for k in range(2):           # replays, on new inputs the second time
            out.zero_()
            if k == 1:
                vecs[2].copy_(to_dev(Z.zkml_scalars(1200, lens[2])))
                zk.zk_commit_batch(ctx_small, vecs, ref, flags=zk.ZK_EVALS)
            zk.zk_plan_launch(plan)
            torch.cuda.synchronize()
            assert torch.equal(out, ref), k
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
    devs = []
    for j in range(count):
        d = DevAcc(zk, n)
        d.set_leaf(*leaf_vectors(j, n))
        devs.append(d)
    zk.zk_leaf_init(ctx_small, [d.desc for d in devs])
    torch.cuda.synchronize()
    saved = [(d.m.clone(), d.e.clone(), d.x.clone()) for d in devs]
    gam = to_dev(np.concatenate([Z.gammas(l, count >> l) for l in range(1, 4)]))
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
            assert torch.equal(root.m, ref.m) and torch.equal(root.e, ref.e)
            assert torch.equal(root.x, ref.x)
    finally:
        zk.zk_plan_destroy(plan)
