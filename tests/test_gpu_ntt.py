"""GPU parity of the F_r NTT / INTT against the oracle's O(n^2) DFT.

Full comparison up to 2^12 (every radix split of one and two passes).  At
2^20, 2^21 (three passes) and 2^22 every output is checked by the O(n)
geometric fingerprint sum_k z^k NTT(c)_k = sum_j c_j (z^n - 1)/(z omega^j - 1)
at a seeded z (a wrong output at any position changes the left side), next
to sampled DFT rows, exact round trips and the Aurora identity."""
import numpy as np
import pytest

import zkinputs as Z
from _util import to_dev, to_host

pytestmark = pytest.mark.gpu
R = Z.R_MOD


def _run(zk, ctx, x, inverse):
    import torch
    t = to_dev(x)
    (zk.zk_intt if inverse else zk.zk_ntt)(ctx, t)
    torch.cuda.synchronize()
    return to_host(t)


@pytest.mark.parametrize("lg", list(range(0, 13)))
def test_ntt_intt_full_oracle(zk, orc, ctx_small, lg):
    n = 1 << lg
    x = Z.fr_uniform(500 + lg, n)
    assert np.array_equal(_run(zk, ctx_small, x, False), orc.ntt(x))
    assert np.array_equal(_run(zk, ctx_small, x, True), orc.intt(x))


@pytest.mark.parametrize("lg", [20, 21, 22])
def test_ntt_at_scale_sampled(zk, orc, ctx_small, lg):
    n = 1 << lg
    x = Z.fr_uniform(600 + lg, n)
    rng = np.random.default_rng(lg)
    rows = np.unique(np.concatenate([[0, 1, n // 2, n - 1], rng.integers(0, n, 12)]))
    f = _run(zk, ctx_small, x, False)
    assert np.array_equal(f[rows], orc.dft_rows(x, rows, False))
    b = _run(zk, ctx_small, x, True)
    assert np.array_equal(b[rows], orc.dft_rows(x, rows, True))
    # exact round trips and sum_H f = n f(0) (Aurora)
    assert np.array_equal(_run(zk, ctx_small, f, True), x)
    assert np.array_equal(_run(zk, ctx_small, b, False), x)
    total = sum(Z.fr_to_int(v) for v in x[:: 1]) % R
    assert Z.fr_to_int(b[0]) * n % R == total


@pytest.mark.parametrize("lg", [20, 21, 22])
def test_ntt_at_scale_fingerprint(zk, orc, ctx_small, lg):
    n = 1 << lg
    x = Z.fr_uniform(650 + lg, n)
    z = Z.fr_uniform(660 + lg, 1)[0]
    # NTT: the transform's output evaluated at z equals the closed form of x.
    f = _run(zk, ctx_small, x, False)
    assert np.array_equal(orc.poly_eval(f, z), orc.ntt_fingerprint(x, z))
    # INTT: NTT(INTT(x)) = x, so the closed form of the output is x(z).
    b = _run(zk, ctx_small, x, True)
    assert np.array_equal(orc.ntt_fingerprint(b, z), orc.poly_eval(x, z))


def test_ntt_batch_and_host_buffers(zk, orc, ctx_small):
    import torch
    lens = [2, 8, 8, 1024, 4096, 1, 64]
    xs = [Z.fr_uniform(700 + i, l) for i, l in enumerate(lens)]
    ts = [to_dev(x) for x in xs]
    zk.zk_ntt_batch(ctx_small, ts, inverse=False)
    torch.cuda.synchronize()
    for x, t in zip(xs, ts):
        assert np.array_equal(to_host(t), orc.ntt(x))
    h = np.ascontiguousarray(xs[4].copy())
    zk.zk_intt(ctx_small, h)
    assert np.array_equal(h, orc.intt(xs[4]))


def test_ntt_rejects_bad_sizes(zk, ctx_small):
    import torch
    t = torch.zeros((3, 4), dtype=torch.int64, device="cuda")
    with pytest.raises(zk.ZkError) as ei:
        zk.zk_ntt(ctx_small, t)
    assert ei.value.code == zk.ZK_EINVAL
    with pytest.raises(zk.ZkError):
        zk.zk_ntt(ctx_small, t, n=1 << 29)


@pytest.fixture(scope="module")
def ntt_case_2_11(orc):
    x = Z.fr_uniform(801, 1 << 11)
    return x, orc.ntt(x), orc.intt(x)


@pytest.mark.parametrize("radix", list(range(1, 12)))
def test_ntt_every_pass_radix(zk, ctx_small, ntt_case_2_11, radix):
    x, f, b = ntt_case_2_11
    try:
        zk.zk_tune_set(ctx_small, zk.ZK_TUNE_NTT_RADIX, 11, radix)
        assert np.array_equal(_run(zk, ctx_small, x, False), f)
        assert np.array_equal(_run(zk, ctx_small, x, True), b)
    finally:
        zk.zk_tune_set(ctx_small, zk.ZK_TUNE_NTT_RADIX, 11, 0)


def test_ntt_two_pass_radix_2_11_at_2_22(zk, orc, ctx_small):
    n = 1 << 22
    x = Z.fr_uniform(802, n)
    rows = np.array([0, 1, 12345, n - 1])
    try:
        zk.zk_tune_set(ctx_small, zk.ZK_TUNE_NTT_RADIX, 22, 11)
        f = _run(zk, ctx_small, x, False)
        assert np.array_equal(f[rows], orc.dft_rows(x, rows, False))
        z = Z.fr_uniform(803, 1)[0]
        assert np.array_equal(orc.poly_eval(f, z), orc.ntt_fingerprint(x, z))
        assert np.array_equal(_run(zk, ctx_small, f, True), x)
    finally:
        zk.zk_tune_set(ctx_small, zk.ZK_TUNE_NTT_RADIX, 22, 0)
