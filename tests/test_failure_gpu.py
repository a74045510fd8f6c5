"""Failure detection on the GPU without a GPU fault: a bounded wait inside the
tensor-core kernel is made to expire (it waits on a barrier nothing ever
completes); the kernel must record CORR_E_TIMEOUT, release its resources and
return, leaving the context and the device usable."""
import numpy as np
import pytest
import torch

import oracle
from paper_1501_05992_gb300 import corr

from _gpu import path_available

pytestmark = pytest.mark.gpu


def test_injected_stall_times_out_and_context_recovers():
    if not path_available("tc_fp8", 128):
        pytest.skip("tc_fp8 unsupported")
    N, F, T = 128, 8, 256
    volt = np.random.default_rng(61).integers(0, 256, (T, F, N), dtype=np.uint8)
    v = torch.from_numpy(volt).cuda()
    c = corr.Correlator(N, F, T, path="tc_fp8")
    c.set_wait_limit(20_000_000)              # about 10 ms of SM clock
    c.inject_stall()
    c.accumulate(v)
    with pytest.raises(corr.CorrError) as e:
        c.sync()
    assert e.value.status == corr.CORR_E_TIMEOUT
    c.sync()                                   # the error was reported once
    c.dump()                                   # discard the partial integration
    c.set_wait_limit(0)
    c.accumulate(v)
    got = c.dump().cpu().numpy()
    c.sync()
    assert np.array_equal(got, oracle.to_int32(oracle.xmac(volt)))
    # the device is still healthy for other work
    x = torch.arange(1 << 20, device="cuda", dtype=torch.float32)
    assert float(x.sum()) == float((1 << 20) * ((1 << 20) - 1) / 2)
    c.close()


def test_batch_stall_reported_by_batch_sync():
    if not path_available("tc_fp8", 128):
        pytest.skip("tc_fp8 unsupported")
    b = corr.Batch([{"n_inputs": 128, "n_chan": 4, "n_time_per_int": 64, "path": "tc_fp8"},
                    {"n_inputs": 256, "n_chan": 2, "n_time_per_int": 64, "path": "tc_fp8"}])
    lib = corr.load()
    lead = b._ctx(0)
    assert lib.corr_set_wait_limit(lead, 20_000_000) == 0
    assert lib.corr_debug_inject(lead, 1) == 0
    vs = [torch.zeros((64, 4, 128), dtype=torch.uint8, device="cuda"),
          torch.zeros((64, 2, 256), dtype=torch.uint8, device="cuda")]
    b.accumulate(vs)
    with pytest.raises(corr.CorrError) as e:
        b.sync()
    assert e.value.status == corr.CORR_E_TIMEOUT
    b.dump()
    b.accumulate(vs)
    outs = b.dump()
    b.sync()
    assert not outs[0].any() and not outs[1].any()

