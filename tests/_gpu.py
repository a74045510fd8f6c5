"""Helpers for the GPU parity tests: run the library through its binding on
numpy inputs and return numpy outputs."""
from __future__ import annotations

import numpy as np
import torch

from paper_1501_05992_gb300 import corr

ALL_PATHS = ["cudacore", "mma_i8", "tc_fp8"]


def path_available(path: str, n_inputs: int = 256, n_chan: int = 1, t: int = 64) -> bool:
    try:
        c = corr.Correlator(n_inputs, n_chan, t, path=path)
    except corr.CorrError as e:
        if e.status == corr.CORR_E_UNSUPPORTED:
            return False
        raise
    c.close()
    return True


def correlate(volt: np.ndarray, path: str, chunks=None, zero_invalid: bool = False,
              t_max: int | None = None, host: bool = False) -> np.ndarray:
    """Packed triangle int32 [F][P][2] of one integration over `volt` [T][F][N]."""
    T, F, N = volt.shape
    c = corr.Correlator(N, F, t_max or max(T, 1), path=path, zero_invalid=zero_invalid)
    try:
        if chunks is None:
            chunks = [(0, T)]
        if host:
            vt = torch.from_numpy(np.ascontiguousarray(volt)).pin_memory()
            for a, b in chunks:
                c.accumulate_host(vt[a:b])
            out = c.dump_host()
        else:
            vt = torch.from_numpy(np.ascontiguousarray(volt)).cuda()
            for a, b in chunks:
                c.accumulate(vt[a:b])
            out = c.dump()
        c.sync()
        torch.cuda.synchronize()
        return out.cpu().numpy()
    finally:
        c.close()
