"""Shared helpers of the GPU parity tests (conversion between torch device
tensors and the uint64 limb arrays the oracle takes)."""
import numpy as np

import zkinputs as Z


def to_dev(a):
    import torch
    a = np.ascontiguousarray(np.asarray(a, dtype=np.uint64))
    return torch.from_numpy(a.view(np.int64)).cuda()


def to_host(t):
    return np.ascontiguousarray(t.detach().cpu().numpy()).view(np.uint64)


def pts_equal(a, b):
    return np.array_equal(np.asarray(a, dtype=np.uint64).reshape(-1, 8),
                          np.asarray(b, dtype=np.uint64).reshape(-1, 8))


def acc_to_oracle(orc, m, e, x):
    """Device accumulator tensors -> oracle Acc (bit patterns unchanged)."""
    return orc.Acc(to_host(m).reshape(4, -1, 4), to_host(e), to_host(x).reshape(44))


def zkml_vec(seed, n):
    return Z.zkml_scalars(seed, n)
