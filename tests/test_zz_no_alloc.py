"""corr_xmac_noalloc, the entry point for callers that may not allocate device
memory (hosts that own all device memory through their own pool, real-time
loops that may not allocate once data flows).

It is called here directly through the C ABI (ctypes), with device buffers
that the test allocates up front, and its output is compared with the regular
corr_accumulate + corr_dump path on the same input and with the CPU oracle:
bit for bit, the tolerance of every parity test in this suite.  Two calls in a row with different inputs
show that the shared static scratch carries nothing over between calls.
This file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1501_05992_gb300 import corr

pytestmark = pytest.mark.gpu


def _noalloc(lib, volt: torch.Tensor, out: torch.Tensor, flags: int = 0) -> int:
    T, F, N = volt.shape
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.corr_xmac_noalloc(ctypes.c_void_p(volt.data_ptr()), T, F, N,
                                 ctypes.c_void_p(out.data_ptr()), flags, stream)


def _regular(volt: torch.Tensor, zero_invalid: bool = False) -> np.ndarray:
    T, F, N = volt.shape
    c = corr.Correlator(N, F, max(T, 1), path="cudacore", zero_invalid=zero_invalid)
    c.accumulate(volt)
    out = c.dump().cpu().numpy()
    c.sync()
    c.close()
    return out


def test_noalloc_matches_regular_path_twice_in_a_row():
    lib = corr.load()
    torch.cuda.init()
    rng = np.random.default_rng(2024)
    shapes = [(700, 8, 64), (333, 5, 40)]
    vols = [torch.from_numpy(rng.integers(0, 256, s, dtype=np.uint8)).cuda() for s in shapes]
    outs = [torch.full((s[1], s[2] * (s[2] + 1) // 2, 2), -12345, dtype=torch.int32,
                       device="cuda") for s in shapes]
    for volt, out in zip(vols, outs):
        assert _noalloc(lib, volt, out) == corr.CORR_OK, corr.strerror(lib.corr_last_error())
    torch.cuda.synchronize()
    for volt, out in zip(vols, outs):
        got = out.cpu().numpy()
        assert np.array_equal(got, _regular(volt))
        assert np.array_equal(got, oracle.to_int32(oracle.xmac(volt.cpu().numpy())))


def test_noalloc_zero_invalid_and_empty_block():
    lib = corr.load()
    rng = np.random.default_rng(7)
    volt = torch.from_numpy(rng.integers(0, 256, (129, 3, 17), dtype=np.uint8)).cuda()
    out = torch.empty((3, 17 * 18 // 2, 2), dtype=torch.int32, device="cuda")
    assert _noalloc(lib, volt, out, flags=corr.ZERO_INVALID) == corr.CORR_OK
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), _regular(volt, zero_invalid=True))
    assert np.array_equal(out.cpu().numpy(),
                          oracle.to_int32(oracle.xmac(volt.cpu().numpy(), zero_invalid=True)))
    empty = torch.empty((0, 3, 17), dtype=torch.uint8, device="cuda")
    out.fill_(99)
    assert _noalloc(lib, empty, out) == corr.CORR_OK
    torch.cuda.synchronize()
    assert not out.cpu().numpy().any()


def test_noalloc_rejects_requests_larger_than_its_scratch():
    lib = corr.load()
    # 256 inputs x 5000 samples need 5.2 MB per channel: 13 channels exceed 64 MiB
    volt = torch.zeros((5000, 13, 256), dtype=torch.uint8, device="cuda")
    out = torch.zeros((13, 256 * 257 // 2, 2), dtype=torch.int32, device="cuda")
    assert _noalloc(lib, volt, out) == corr.CORR_E_BUDGET
    assert lib.corr_last_error() == corr.CORR_E_BUDGET
    assert _noalloc(lib, volt[:, :12].contiguous(), out[:12]) == corr.CORR_OK
    assert lib.corr_xmac_noalloc(None, 10, 1, 4, None, 0, None) == corr.CORR_E_ARG
    torch.cuda.synchronize()
