"""Serving loop: jobs of different sizes give the same results alone and in
the mix (bit-exact), admission respects the HBM budget, and waits are
bounded."""
import numpy as np
import pytest

import zkinputs as Z
from _util import to_dev

pytestmark = pytest.mark.gpu


class Slot:
    """Device buffers of one job: witness inputs, leaf and fold output."""

    def __init__(self, zk, n, seed):
        import torch
        self.n = n
        self.w = [to_dev(Z.zkml_scalars(seed + i, n)) for i in range(3)]

        def acc():
            m = torch.zeros((4, n, 4), dtype=torch.int64, device="cuda")
            e = torch.zeros((n, 4), dtype=torch.int64, device="cuda")
            x = torch.zeros(44, dtype=torch.int64, device="cuda")
            return (m, e, x), zk.make_acc(m, e, x)

        self.leaf_t, self.leaf = acc()
        self.out_t, self.out = acc()

    def result(self):
        import torch
        return [t.clone() for t in self.leaf_t + self.out_t]


def _resident(zk, ctx, n, seed):
    s = Slot(zk, n, seed)
    for i, k in ((0, 0), (1, 1), (3, 2)):
        s.leaf_t[0][i].copy_(s.w[k])
    zk.zk_leaf_init(ctx, [s.leaf])
    return s


def test_serving_alone_equals_mix(zk, ctx_small):
    import torch
    sizes = [1 << 12, 1 << 10, 1 << 11, 1 << 12, 1 << 9, 1 << 10, 1 << 12, 1 << 8]
    gam = to_dev(Z.gammas(1, len(sizes)))
    res = {n: _resident(zk, ctx_small, n, 5000 + n) for n in set(sizes)}
    slots = [Slot(zk, n, 6000 + 10 * i) for i, n in enumerate(sizes)]
    jobs = [zk.make_job(s.n, s.w, s.leaf, res[s.n].leaf, s.out, gam[i]) for i, s in enumerate(slots)]
    torch.cuda.synchronize()
    srv = zk.zk_server_create(ctx_small, lanes=4)
    try:
        alone = []
        for j, s in zip(jobs, slots):                # one at a time
            info = zk.zk_wait(srv, zk.zk_submit(srv, j), 60000)
            assert info.status == zk.ZK_JOB_DONE and info.error == 0
            alone.append(s.result())
        for s in slots:
            for t in s.leaf_t + s.out_t:
                t.zero_()
        torch.cuda.synchronize()
        tickets = [zk.zk_submit(srv, j) for j in jobs]  # all at once
        lanes = set()
        for t in tickets:
            info = zk.zk_wait(srv, t, 60000)
            assert info.status == zk.ZK_JOB_DONE and info.error == 0
            assert info.end_ms >= info.start_ms >= info.submit_ms
            lanes.add(info.lane)
        assert len(lanes) > 1
        for s, a in zip(slots, alone):
            for u, v in zip(s.result(), a):
                assert torch.equal(u, v)
        st = zk.zk_server_stats(srv)
        assert st.completed == 2 * len(jobs) and st.queued == 0 and st.reserved_bytes == 0
    finally:
        zk.zk_server_destroy(srv)


def test_serving_budget_admission_and_bounded_waits(zk, ctx_small):
    import torch
    n = 1 << 12
    res = _resident(zk, ctx_small, n, 7000)
    slots = [Slot(zk, n, 7100 + 10 * i) for i in range(4)]
    gam = to_dev(Z.gammas(2, 4))
    jobs = [zk.make_job(n, s.w, s.leaf, res.leaf, s.out, gam[i]) for i, s in enumerate(slots)]
    torch.cuda.synchronize()
    # The workspace estimate of one job is the peak reservation of a server
    # that ran just that job; a budget of 1.5 estimates admits one at a time.
    probe = zk.zk_server_create(ctx_small, lanes=1)
    try:
        zk.zk_wait(probe, zk.zk_submit(probe, jobs[0]), 60000)
        est = zk.zk_server_stats(probe).peak_reserved_bytes
    finally:
        zk.zk_server_destroy(probe)
    budget = est * 3 // 2
    srv = zk.zk_server_create(ctx_small, lanes=4, hbm_budget_bytes=budget)
    try:
        tickets = [zk.zk_submit(srv, j) for j in jobs]
        infos = [zk.zk_wait(srv, t, 60000) for t in tickets]
        assert all(i.status == zk.ZK_JOB_DONE for i in infos)
        st = zk.zk_server_stats(srv)
        assert st.peak_reserved_bytes == est <= budget
        spans = sorted((i.start_ms, i.end_ms) for i in infos)
        for (s0, e0), (s1, e1) in zip(spans, spans[1:]):
            assert s1 >= e0 - 1e-6  # never two at once
        with pytest.raises(zk.ZkError) as ei:
            zk.zk_wait(srv, 10 ** 9, 10)  # unknown ticket
        assert ei.value.code == zk.ZK_EINVAL
    finally:
        zk.zk_server_destroy(srv)
    small = zk.zk_server_create(ctx_small, lanes=1, hbm_budget_bytes=1 << 20)
    try:
        with pytest.raises(zk.ZkError) as ei:
            zk.zk_submit(small, jobs[0])
        assert ei.value.code == zk.ZK_ENOMEM
    finally:
        zk.zk_server_destroy(small)
