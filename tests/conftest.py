import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running oracle case")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.lib()
    return oracle


TAU_SEED = 0
SMALL_SRS = 1 << 12
BIG_SRS = 1 << 22


@pytest.fixture(scope="session")
def zk():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2507_07031_b300 as z
    return z


@pytest.fixture(scope="session")
def tau():
    import zkinputs
    return zkinputs.tau(TAU_SEED)


@pytest.fixture(scope="session")
def ctx_small(zk, tau):
    ctx = zk.zk_init(0)
    zk.zk_srs_generate(ctx, tau, SMALL_SRS)
    yield ctx
    zk.zk_destroy(ctx)


@pytest.fixture(scope="session")
def ctx_big(zk, tau):
    ctx = zk.zk_init(0)
    zk.zk_srs_generate(ctx, tau, BIG_SRS)
    yield ctx
    zk.zk_destroy(ctx)


@pytest.fixture(scope="session")
def srs_small(orc, tau):
    return orc.srs_gen(tau, SMALL_SRS)
