"""GPU parity of the hiding commitment [f(tau)]_1 + s H (Sec. 4.2) against
the oracle (MSM over the SRS plus s H by affine double-and-add), for digit
patterns that exercise every window sign: s = 0, 1, r - 1, (r - 1)/2,
(r + 1)/2, 2^k, values with 0x80 / 0x81 bytes, and uniform s."""
import numpy as np
import pytest

import zkinputs as Z
from _util import pts_equal, to_dev, to_host

pytestmark = pytest.mark.gpu
R = Z.R_MOD


def test_hiding_commitment_matches_oracle(zk, orc, ctx_small, srs_small):
    import torch
    G = orc.g1_generator()
    H = orc.g1_mul(G, Z.int_to_fr(0x5EED_1234_5678))
    zk.zk_set_hiding_base(ctx_small, np.ascontiguousarray(H))
    n = 1000
    c = Z.fr_uniform(1600, n)
    specials = [0, 1, R - 1, (R - 1) // 2, (R + 1) // 2, 1 << 128, (1 << 253) - 1,
                int("80" * 31, 16), int("81" * 31, 16), int("7f" * 31, 16)]
    specials += [Z.fr_to_int(v) for v in Z.fr_uniform(1601, 4)]
    out = torch.zeros(8, dtype=torch.int64, device="cuda")
    for sv in specials:
        s = Z.int_to_fr(sv % R)
        zk.zk_commit_hiding(ctx_small, to_dev(c), to_dev(s), out)
        torch.cuda.synchronize()
        assert pts_equal(to_host(out), orc.commit_hiding(srs_small, c, H, s)), hex(sv)
    # host buffers
    hout = np.zeros(8, np.uint64)
    s = Z.fr_uniform(1602, 1)[0]
    zk.zk_commit_hiding(ctx_small, np.ascontiguousarray(c), np.ascontiguousarray(s), hout)
    assert pts_equal(hout, orc.commit_hiding(srs_small, c, H, s))


def test_hiding_base_validation(zk, orc):
    ctx = zk.zk_init(0)
    try:
        zk.zk_srs_generate(ctx, Z.tau(0), 64)
        c = Z.fr_uniform(1603, 8)
        out = np.zeros(8, np.uint64)
        with pytest.raises(zk.ZkError) as ei:  # no base yet
            zk.zk_commit_hiding(ctx, np.ascontiguousarray(c), np.ascontiguousarray(Z.int_to_fr(3)), out)
        assert ei.value.code == zk.ZK_EINVAL
        bad = orc.g1_generator().copy()
        bad[4] ^= np.uint64(1)  # off the curve
        for H in (bad, np.zeros(8, np.uint64)):
            with pytest.raises(zk.ZkError) as ei:
                zk.zk_set_hiding_base(ctx, np.ascontiguousarray(H))
            assert ei.value.code == zk.ZK_EINVAL
    finally:
        zk.zk_destroy(ctx)
