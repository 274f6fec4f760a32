"""Serving loop: every job's leaf accumulator and fold output equal the
oracle's (leaf_init, then fold into the resident accumulator of its size,
with closed-form commitments), alone and in a mix of sizes that reaches the
full-width MSM path (2^16); the degree-3 relation is served the same way;
admission respects the HBM budget; and waits are bounded."""
import numpy as np
import pytest

import zkinputs as Z
from _util import acc_to_oracle, to_dev

pytestmark = pytest.mark.gpu


class Slot:
    """Device buffers of one job: witness inputs, leaf and fold output."""

    def __init__(self, zk, n, seed):
        import torch
        self.n = n
        self.h = [Z.zkml_scalars(seed + i, n) for i in range(3)]
        self.w = [to_dev(v) for v in self.h]

        def acc():
            m = torch.zeros((4, n, 4), dtype=torch.int64, device="cuda")
            e = torch.zeros((n, 4), dtype=torch.int64, device="cuda")
            x = torch.zeros(44, dtype=torch.int64, device="cuda")
            return (m, e, x), zk.make_acc(m, e, x)

        self.leaf_t, self.leaf = acc()
        self.out_t, self.out = acc()

    def result(self):
        return [t.clone() for t in self.leaf_t + self.out_t]

    def oracle_leaf(self, orc, tau):
        return orc.leaf_init(*self.h, orc.COMMIT_TAU, tau=tau)


def _resident(zk, ctx, n, seed, degree=2):
    s = Slot(zk, n, seed)
    third = 2 if degree == 3 else 3
    for i, k in ((0, 0), (1, 1), (third, 2)):
        s.leaf_t[0][i].copy_(s.w[k])
    zk.zk_leaf_init(ctx, [s.leaf])
    return s


def _same(a, b):
    return np.array_equal(a.m, b.m) and np.array_equal(a.e, b.e) and np.array_equal(a.inst, b.inst)


def _check_against_oracle(orc, tau, slots, res, gam_h):
    """Each job: leaf = leaf_init(w), out = fold(resident, leaf, gamma)."""
    res_orc = {n: r.oracle_leaf(orc, tau) for n, r in res.items()}
    for i, s in enumerate(slots):
        leaf = s.oracle_leaf(orc, tau)
        assert _same(acc_to_oracle(orc, *s.leaf_t), leaf), (i, s.n)
        want, _ = orc.fold(res_orc[s.n], leaf, gam_h[i], orc.COMMIT_TAU, tau=tau)
        assert _same(acc_to_oracle(orc, *s.out_t), want), (i, s.n)


def _run_alone_and_mixed(zk, srv, jobs, slots):
    import torch
    alone = []
    for j, s in zip(jobs, slots):                # one at a time
        info = zk.zk_wait(srv, zk.zk_submit(srv, j), 120000)
        assert info.status == zk.ZK_JOB_DONE and info.error == 0
        alone.append(s.result())
    for s in slots:
        for t in s.leaf_t + s.out_t:
            t.zero_()
    torch.cuda.synchronize()
    tickets = [zk.zk_submit(srv, j) for j in jobs]  # all at once
    lanes = set()
    for t in tickets:
        info = zk.zk_wait(srv, t, 120000)
        assert info.status == zk.ZK_JOB_DONE and info.error == 0
        assert info.end_ms >= info.start_ms >= info.submit_ms
        lanes.add(info.lane)
    for s, a in zip(slots, alone):
        for u, v in zip(s.result(), a):
            assert torch.equal(u, v)
    return lanes


def test_serving_mix_matches_oracle(zk, orc, ctx_big, tau):
    import torch
    sizes = [1 << 12, 1 << 10, 1 << 16, 1 << 11, 1 << 12, 1 << 9, 1 << 16, 1 << 8]
    gam_h = Z.gammas(1, len(sizes))
    gam = to_dev(gam_h)
    res = {n: _resident(zk, ctx_big, n, 5000 + n) for n in set(sizes)}
    slots = [Slot(zk, n, 6000 + 10 * i) for i, n in enumerate(sizes)]
    jobs = [zk.make_job(s.n, s.w, s.leaf, res[s.n].leaf, s.out, gam[i]) for i, s in enumerate(slots)]
    torch.cuda.synchronize()
    srv = zk.zk_server_create(ctx_big, lanes=4)
    try:
        lanes = _run_alone_and_mixed(zk, srv, jobs, slots)
        assert len(lanes) > 1
        st = zk.zk_server_stats(srv)
        assert st.completed == 2 * len(jobs) and st.queued == 0 and st.reserved_bytes == 0
    finally:
        zk.zk_server_destroy(srv)
    _check_against_oracle(orc, tau, slots, res, gam_h)


def test_serving_degree3_matches_oracle(zk, orc, ctx_small, tau):
    import torch
    sizes = [1 << 10, 1 << 12, 1 << 8, 1 << 10]
    gam_h = Z.gammas(3, len(sizes))
    gam = to_dev(gam_h)
    zk.zk_set_fold_degree(ctx_small, 3)
    orc.set_degree(3)
    try:
        res = {n: _resident(zk, ctx_small, n, 8000 + n, degree=3) for n in set(sizes)}
        slots = [Slot(zk, n, 8500 + 10 * i) for i, n in enumerate(sizes)]
        jobs = [zk.make_job(s.n, s.w, s.leaf, res[s.n].leaf, s.out, gam[i]) for i, s in enumerate(slots)]
        torch.cuda.synchronize()
        srv = zk.zk_server_create(ctx_small, lanes=3)
        try:
            _run_alone_and_mixed(zk, srv, jobs, slots)
        finally:
            zk.zk_server_destroy(srv)
        _check_against_oracle(orc, tau, slots, res, gam_h)
        for s in slots:  # the degree-3 leaf keeps m3 and derives m4
            m = acc_to_oracle(orc, *s.leaf_t).m
            assert np.array_equal(m[2], s.h[2])
    finally:
        zk.zk_set_fold_degree(ctx_small, 2)
        orc.set_degree(2)


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


def test_wait_times_out_on_a_queued_job(zk, ctx_big):
    """A job queued behind others on a one-lane server is not done after 1 ms:
    zk_wait returns ZK_ETIMEOUT (a host-side bounded wait), the ticket is
    still pending, and it completes later."""
    import torch
    n = 1 << 18
    res = _resident(zk, ctx_big, n, 9000)
    slots = [Slot(zk, n, 9100 + 10 * i) for i in range(3)]
    gam = to_dev(Z.gammas(4, 3))
    jobs = [zk.make_job(n, s.w, s.leaf, res.leaf, s.out, gam[i]) for i, s in enumerate(slots)]
    torch.cuda.synchronize()
    srv = zk.zk_server_create(ctx_big, lanes=1)
    try:
        tickets = [zk.zk_submit(srv, j) for j in jobs]
        with pytest.raises(zk.ZkError) as ei:
            zk.zk_wait(srv, tickets[-1], 1)
        assert ei.value.code == zk.ZK_ETIMEOUT
        assert zk.zk_poll(srv, tickets[-1]).status in (zk.ZK_JOB_QUEUED, zk.ZK_JOB_RUNNING)
        for t in tickets:
            assert zk.zk_wait(srv, t, 120000).status == zk.ZK_JOB_DONE
    finally:
        zk.zk_server_destroy(srv)


def test_cancel_a_queued_job(zk, ctx_big):
    """A job still waiting in the queue can be cancelled: it never runs (its
    output buffer stays untouched), waiters return at once; running or
    finished jobs cannot be cancelled."""
    import torch
    n = 1 << 18
    res = _resident(zk, ctx_big, n, 9500)
    slots = [Slot(zk, n, 9600 + 10 * i) for i in range(3)]
    gam = to_dev(Z.gammas(5, 3))
    jobs = [zk.make_job(n, s.w, s.leaf, res.leaf, s.out, gam[i]) for i, s in enumerate(slots)]
    slots[2].out_t[0].fill_(7)
    torch.cuda.synchronize()
    srv = zk.zk_server_create(ctx_big, lanes=1)
    try:
        tickets = [zk.zk_submit(srv, j) for j in jobs]
        zk.zk_cancel(srv, tickets[2])
        info = zk.zk_wait(srv, tickets[2], 1000)
        assert info.status == zk.ZK_JOB_CANCELLED
        with pytest.raises(zk.ZkError) as ei:
            zk.zk_cancel(srv, tickets[2])  # no longer queued
        assert ei.value.code == zk.ZK_EBUSY
        with pytest.raises(zk.ZkError) as ei:
            zk.zk_cancel(srv, 10 ** 9)
        assert ei.value.code == zk.ZK_EINVAL
        for t in tickets[:2]:
            assert zk.zk_wait(srv, t, 120000).status == zk.ZK_JOB_DONE
        with pytest.raises(zk.ZkError) as ei:
            zk.zk_cancel(srv, tickets[0])  # finished
        assert ei.value.code == zk.ZK_EBUSY
        st = zk.zk_server_stats(srv)
        assert st.cancelled == 1 and st.completed == 2 and st.queued == 0
        torch.cuda.synchronize()
        assert bool((slots[2].out_t[0] == 7).all())  # never written
    finally:
        zk.zk_server_destroy(srv)
