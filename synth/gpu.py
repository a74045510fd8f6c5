"""Device-side generation of the voltgen.py recipes (same bytes), for inputs
too large to create on the host.  Builds ``synth/_build/libvoltgen.so`` from
``voltgen.cu`` with nvcc on first use."""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess
import threading

import numpy as np
import torch

from . import voltgen as vg

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "voltgen.cu")
_LIB = os.path.join(_HERE, "_build", "libvoltgen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                    "-Xcompiler", "-fPIC", "-shared", "-o", tmp, _SRC], check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            vp, ci, cll, u64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong, ctypes.c_uint64
            lib.vg_gauss3.argtypes = [vp, ci, ci, ci, cll, ci, ci, u64, u64, u64, u64, vp, ci, ci, vp]
            lib.vg_gauss3.restype = ci
            lib.vg_uniform_tone.argtypes = [vp, ci, ci, ci, cll, ci, ci, u64, vp, vp]
            lib.vg_uniform_tone.restype = ci
            _lib = lib
        return _lib


class DeviceGenerator:
    """Generates slices of one array's voltages into device memory."""

    def __init__(self, params, device="cuda"):
        self.params = params
        self.device = torch.device(device)
        if isinstance(params, vg.Gauss3Params):
            self._gains = torch.from_numpy(np.ascontiguousarray(params.gains)).to(self.device)

    def fill(self, out: torch.Tensor, t0: int, f0: int = 0, stream=None) -> torch.Tensor:
        """Write samples [t0, t0 + out.shape[0]) x channels [f0, f0 + out.shape[1])."""
        p = self.params
        if out.dtype != torch.uint8 or out.dim() != 3 or not out.is_contiguous():
            raise ValueError("out must be a contiguous uint8 [T][F][N] device tensor")
        nt, nf, n = out.shape
        if n != p.n_inputs:
            raise ValueError("input count mismatch")
        s = ctypes.c_void_p((stream or torch.cuda.current_stream()).cuda_stream)
        lib = _load()
        if isinstance(p, vg.Gauss3Params):
            rc = lib.vg_gauss3(ctypes.c_void_p(out.data_ptr()), nt, p.n_chan, n, t0, f0, nf,
                               p.key_noise, p.key_src(0), p.key_src(1), p.key_src(2),
                               ctypes.c_void_p(self._gains.data_ptr()), vg.K_NOISE, vg.K_SOURCE, s)
        else:
            tone = torch.from_numpy(vg.tone_table(p, t0, nt)).to(self.device)
            rc = lib.vg_uniform_tone(ctypes.c_void_p(out.data_ptr()), nt, p.n_chan, n, t0, f0, nf,
                                     p.key, ctypes.c_void_p(tone.data_ptr()), s)
            # keep the table alive until the kernel has read it
            (stream or torch.cuda.current_stream()).synchronize()
        if rc != 0:
            raise RuntimeError(f"voltage generator failed ({rc})")
        return out

    def make(self, t0: int, n_time: int, f0: int = 0, n_f: int | None = None) -> torch.Tensor:
        n_f = self.params.n_chan - f0 if n_f is None else n_f
        out = torch.empty((n_time, n_f, self.params.n_inputs), dtype=torch.uint8, device=self.device)
        return self.fill(out, t0, f0)
