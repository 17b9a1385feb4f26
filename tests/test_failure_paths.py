"""Failure detection without a GPU fault: a bounded device wait that runs out sets the
device error word and the host reads LC_ERR_TIMEOUT; the context stays usable."""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1405_7470_gb300 import lc as lcmod
    lcmod.load()
    return lcmod


def test_wait_timeout_is_reported_and_context_survives(lc):
    import torch
    assert lc.device_error(clear=True) == 0
    lc.check(lc.load().lc_selftest_wait_timeout(2_000_000, None), "lc_selftest_wait_timeout")  # 2 ms
    torch.cuda.synchronize()
    assert lc.device_error(clear=False) == 8      # LC_ERR_TIMEOUT, still set
    assert lc.device_error(clear=True) == 8       # read and clear
    assert lc.device_error(clear=True) == 0
    # the context still works: a normal contraction afterwards is correct
    D, u = synth.operands(500, 20, 2, np.float32, seed=1)
    kernel = lc.Kernel()
    v = lc.variant_default(kernel, 500, 20, 2, "elem", "fp32")
    out = lc.contract(kernel, v, torch.from_numpy(D).cuda(), torch.from_numpy(u).cuda())
    torch.cuda.synchronize()
    assert oracle.rel_fro_error(out.cpu().numpy(), oracle.contract(D, u)) < 1e-6
    assert lc.device_error() == 0
