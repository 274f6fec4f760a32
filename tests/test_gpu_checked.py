"""The bounds-checked build (-DZK_CHECK): the hot path runs through it with
every in-kernel check passing and results equal to the oracle's; a
non-canonical scalar (a violated precondition) raises its flag instead of
trapping; the normal build reports itself unchecked."""
import ctypes

import numpy as np
import pytest

import zkinputs as Z
from _util import pts_equal, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def checked(zk):
    import importlib.util
    import os
    spec = importlib.util.spec_from_file_location(
        "zk_b300_build", os.path.join(os.path.dirname(zk.__file__), "build.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    b.build(checked=True)
    L = zk.load_checked()
    h = ctypes.c_void_p()
    assert L.zk_init(ctypes.byref(h), 0, 0) == 0
    tau = np.ascontiguousarray(Z.tau(0))
    assert L.zk_srs_generate(h, tau.ctypes.data, 1 << 18) == 0
    yield L, h.value
    L.zk_destroy(h.value)


def _status(L, ctx):
    f, c = ctypes.c_uint(), ctypes.c_int()
    assert L.zk_check_status(ctx, ctypes.byref(f), ctypes.byref(c)) == 0
    return f.value, c.value


def test_hot_path_passes_every_check(zk, orc, checked, tau):
    import torch
    L, ctx = checked
    assert _status(L, ctx) == (0, 1)
    stream = torch.cuda.current_stream().cuda_stream
    n = 1 << 18
    for c in (Z.fr_uniform(71, n), Z.zkml_scalars(72, n), Z.fr_uniform(73, 1000),
              np.zeros((4096, 4), np.uint64)):
        out = torch.zeros(8, dtype=torch.int64, device="cuda")
        assert L.zk_commit(ctx, to_dev(c).data_ptr(), c.shape[0], out.data_ptr(), stream) == 0
        torch.cuda.synchronize()
        assert pts_equal(to_host(out), orc.commit_coeffs_tau(c, tau))
    # NTT on both pass kernels: radix 2^9 (register-tiled) and 2^6.
    x = Z.fr_uniform(74, n)
    z = Z.fr_uniform(75, 1)[0]
    for radix in (9, 6):
        assert L.zk_tune_set(ctx, zk.ZK_TUNE_NTT_RADIX, 18, radix) == 0
        t = to_dev(x)
        assert L.zk_ntt(ctx, t.data_ptr(), n, stream) == 0
        torch.cuda.synchronize()
        assert np.array_equal(orc.poly_eval(to_host(t), z), orc.ntt_fingerprint(x, z)), radix
    assert L.zk_tune_set(ctx, zk.ZK_TUNE_NTT_RADIX, 18, 0) == 0
    assert _status(L, ctx) == (0, 1)


def test_batch_paths_pass_every_check(zk, orc, checked, tau):
    """A batch on the batch-only paths (shared-memory histogram sort, the
    thread-level first reduction level, the team tail of quantised jobs)
    through the checked build: every check passes, results equal the
    oracle's."""
    import torch
    L, ctx = checked
    stream = torch.cuda.current_stream().cuda_stream
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    n = 1 << 16
    count = (2 * sms + 7) // 8 + 2  # chunks of 8192 scalars: two per SM
    vecs = [Z.zkml_scalars(80 + i, n) if i % 4 == 3 else Z.fr_uniform(80 + i, n) for i in range(count)]
    devs = [to_dev(v) for v in vecs]
    ptrs = (ctypes.c_void_p * count)(*[d.data_ptr() for d in devs])
    lens = (ctypes.c_size_t * count)(*[n] * count)
    out = torch.zeros((count, 8), dtype=torch.int64, device="cuda")
    assert L.zk_commit_batch(ctx, ctypes.addressof(ptrs), ctypes.addressof(lens), count, 0, out.data_ptr(),
                             stream) == 0
    torch.cuda.synchronize()
    got = to_host(out)
    for k, v in enumerate(vecs):
        assert pts_equal(got[k], orc.commit_coeffs_tau(v, tau)), k
    assert _status(L, ctx) == (0, 1)


def test_non_canonical_scalar_raises_its_flag(zk, checked):
    import torch
    L, ctx = checked
    stream = torch.cuda.current_stream().cuda_stream
    c = Z.fr_uniform(76, 5000)
    c[17] = np.array([~np.uint64(0)] * 3 + [np.uint64(0x7FFFFFFFFFFFFFFF)], dtype=np.uint64)  # >= r
    out = torch.zeros(8, dtype=torch.int64, device="cuda")
    assert L.zk_commit(ctx, to_dev(c).data_ptr(), c.shape[0], out.data_ptr(), stream) == 0
    flags, is_checked = _status(L, ctx)
    assert is_checked == 1 and flags & zk.ZK_CHECK_SCALAR
    assert _status(L, ctx) == (0, 1)  # read clears


def test_normal_build_is_unchecked(zk, ctx_small):
    assert zk.zk_check_status(ctx_small) == (0, False)
