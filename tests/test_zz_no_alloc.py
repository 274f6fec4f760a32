"""The allocation-free commitment, zk_commit_noalloc.

Some callers cannot call cudaMalloc: a host thread that must never block on
the device-wide synchronisation that cudaFree implies, or a process whose
device memory is all owned by another allocator.  zk_commit_noalloc serves
them from one fixed device array inside the library.  This test calls it
through the C ABI twice in a row, on different inputs and lengths, and checks
each result against zk_commit's bit for bit (the tolerance of every
finite-field test here is zero).  The second call also shows that what the
first call left in the shared array does not leak into the next result.
The file is named so that pytest collects it last."""
import numpy as np
import pytest

import zkinputs as Z
from _util import pts_equal, to_dev, to_host

pytestmark = pytest.mark.gpu


def test_noalloc_commit_matches_zk_commit_twice(zk, ctx_small):
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    cases = [(4096, Z.fr_uniform(901, 4096)), (1000, Z.zkml_scalars(902, 1000))]
    scalars = [to_dev(c) for _, c in cases]
    refs, outs = [], []
    for (n, _), sc in zip(cases, scalars):
        ref = torch.zeros(8, dtype=torch.int64, device="cuda")
        zk.zk_commit(ctx_small, sc, ref)
        refs.append(ref)
        outs.append(torch.zeros(8, dtype=torch.int64, device="cuda"))
    torch.cuda.synchronize()
    for (n, _), sc, out in zip(cases, scalars, outs):  # two calls in a row
        rc = zk.lib.zk_commit_noalloc(ctx_small, sc.data_ptr(), n, out.data_ptr(), stream)
        assert rc == zk.ZK_OK, zk.zk_strerror(rc)
    torch.cuda.synchronize()
    for ref, out in zip(refs, outs):
        assert pts_equal(to_host(out), to_host(ref))
    assert not np.array_equal(to_host(outs[0]), to_host(outs[1]))


def test_noalloc_rejects_what_it_cannot_serve(zk, ctx_small):
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    sc = to_dev(Z.fr_uniform(903, 4096))
    out = torch.zeros(8, dtype=torch.int64, device="cuda")
    assert zk.lib.zk_commit_noalloc(ctx_small, sc.data_ptr(), 4097, out.data_ptr(), stream) == zk.ZK_EINVAL
    host = np.zeros(8, dtype=np.uint64)
    assert zk.lib.zk_commit_noalloc(ctx_small, sc.data_ptr(), 16, host.ctypes.data, stream) == zk.ZK_EINVAL
    assert zk.lib.zk_commit_noalloc(ctx_small, sc.data_ptr(), 0, out.data_ptr(), stream) == zk.ZK_EINVAL
