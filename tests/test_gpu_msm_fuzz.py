"""Seeded random batches across the MSM's switching points, each job against
the commitment's closed form [f(tau)]_1: job counts that do and do not give
the batch-only paths (shared-memory histogram sort, thread-level reduction
level, the batch window rule), lengths from 1 to 2^17 (several window widths
per call), and scalar distributions that move buckets between the piece
classes (uniform, quantised int8 x 2^16, all zero, one repeated value,
values from a tiny set, short values)."""
import numpy as np
import pytest

import zkinputs as Z
from _util import pts_equal, to_dev, to_host

pytestmark = pytest.mark.gpu
R = Z.R_MOD


def _vector(rng, seed, n):
    kind = rng.integers(0, 6)
    if kind == 0:
        return Z.fr_uniform(seed, n)
    if kind == 1:
        return Z.zkml_scalars(seed, n)
    if kind == 2:
        return np.zeros((n, 4), dtype=np.uint64)
    if kind == 3:
        return np.tile(Z.fr_uniform(seed, 1)[0], (n, 1))
    if kind == 4:  # a handful of distinct values: a few heavy buckets
        vals = Z.fr_uniform(seed, 5)
        return np.ascontiguousarray(vals[rng.integers(0, 5, n)])
    small = rng.integers(-(1 << 20), 1 << 20, n)  # short values, both signs
    return np.stack([Z.int_to_fr(int(v) % R) for v in small]) if n <= 4096 else Z.zkml_scalars(seed, n)


@pytest.mark.parametrize("case", range(4))
def test_random_batches(zk, orc, ctx_big, tau, case):
    import torch
    rng = np.random.default_rng(900 + case)
    count = int([3, 80, 300, 700][case])
    logs = rng.integers(0, 18, count) if case < 2 else rng.integers(8, 17, count)
    lens = [max(1, int(1 << l) - int(rng.integers(0, 3))) for l in logs]
    vecs = [_vector(rng, 90_000 + 1000 * case + i, n) for i, n in enumerate(lens)]
    out = torch.zeros((count, 8), dtype=torch.int64, device="cuda")
    zk.zk_commit_batch(ctx_big, [to_dev(v) for v in vecs], out)
    torch.cuda.synchronize()
    got = to_host(out)
    for k, v in enumerate(vecs):
        assert pts_equal(got[k], orc.commit_coeffs_tau(v, tau)), (case, k, lens[k])
