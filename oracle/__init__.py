"""CPU oracle for the X-engine (test infrastructure only).

The correlation itself is the plain int64 triple loop in ``xmac_oracle.c``
(Eq. 3 of Section 2 integrated over time as in Section 3.4.2, emitted as the
packed lower triangle of Appendix C); the same file holds the plain fp64
statements of the fine polyphase filterbank (Section 3.2.1), the incoherent
beam, the output remap and the packet ingest.  This module only builds that
file with gcc and marshals numpy arrays to it.

Only the test-suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline may import this package.  It shares no code with the CUDA library in
``paper_1501_05992_gb300`` and imports nothing from it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "xmac_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lock = threading.Lock()
_default = None


def build(force: bool = False, src: str = _SRC, out: str = _LIB_PATH) -> str:
    """Compile ``xmac_oracle.c`` (or another source) into a shared library."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= os.path.getmtime(src)):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
           "-Wall", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def n_pairs(n_inputs: int) -> int:
    """Packed lower triangle size including autos: N(N+1)/2."""
    return n_inputs * (n_inputs + 1) // 2


def _u8(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def _i64(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _check_volt(volt: np.ndarray) -> np.ndarray:
    volt = np.ascontiguousarray(volt)
    if volt.dtype != np.uint8 or volt.ndim != 3:
        raise ValueError("volt must be a uint8 array shaped [T][F][N]")
    return volt


class OracleLib:
    """ctypes view of one build of the oracle source."""

    def __init__(self, path: str):
        lib = ctypes.CDLL(path)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        i64p = ctypes.POINTER(ctypes.c_int64)
        i32p = ctypes.POINTER(ctypes.c_int32)
        c_int = ctypes.c_int
        lib.oracle_xmac_tri.argtypes = [u8p, c_int, c_int, c_int, c_int, i64p]
        lib.oracle_xmac_tri.restype = c_int
        lib.oracle_xmac_full.argtypes = [u8p, c_int, c_int, c_int, c_int, i64p]
        lib.oracle_xmac_full.restype = c_int
        lib.oracle_xmac_pair.argtypes = [u8p, c_int, c_int, c_int, c_int,
                                         c_int, c_int, c_int, i64p]
        lib.oracle_xmac_pair.restype = c_int
        lib.oracle_decode.argtypes = [u8p, ctypes.c_int64, c_int, i32p, i32p]
        lib.oracle_decode.restype = None
        lib.oracle_beam.argtypes = [u8p, c_int, c_int, c_int, c_int, c_int, i64p]
        lib.oracle_beam.restype = c_int
        lib.oracle_remap.argtypes = [i64p, c_int, c_int, c_int, c_int, i32p, i64p]
        lib.oracle_remap.restype = c_int
        lib.oracle_ingest.argtypes = [u8p, ctypes.c_int64, c_int, u8p, i64p]
        lib.oracle_ingest.restype = c_int
        lib.oracle_fine_pfb.argtypes = [ctypes.POINTER(ctypes.c_int8), c_int, c_int, ctypes.c_int64,
                                        ctypes.POINTER(ctypes.c_double), c_int, ctypes.c_double,
                                        ctypes.POINTER(ctypes.c_double), u8p]
        lib.oracle_fine_pfb.restype = c_int
        lib.oracle_set_threads.argtypes = [c_int]
        lib.oracle_set_threads.restype = c_int
        lib.oracle_threads.argtypes = []
        lib.oracle_threads.restype = c_int
        self.lib = lib
        self.path = path

    def decode(self, volt: np.ndarray, zero_invalid: bool = False):
        """Decode packed 4+4-bit samples (Appendix A) into int32 (re, im) arrays."""
        v = np.ascontiguousarray(volt, dtype=np.uint8)
        re = np.empty(v.shape, np.int32)
        im = np.empty(v.shape, np.int32)
        i32p = ctypes.POINTER(ctypes.c_int32)
        self.lib.oracle_decode(_u8(v), v.size, int(zero_invalid),
                               re.ctypes.data_as(i32p), im.ctypes.data_as(i32p))
        return re, im

    def xmac(self, volt: np.ndarray, zero_invalid: bool = False,
             vis: np.ndarray | None = None) -> np.ndarray:
        """Packed lower-triangle visibilities, int64 [F][N(N+1)/2][2] (re, im).

        If ``vis`` is given the products are added into it (one more
        accumulate call of the same integration) and it is returned.
        """
        volt = _check_volt(volt)
        T, F, N = volt.shape
        if vis is None:
            vis = np.zeros((F, n_pairs(N), 2), np.int64)
        elif (vis.dtype != np.int64 or vis.shape != (F, n_pairs(N), 2)
              or not vis.flags.c_contiguous):
            raise ValueError("vis must be a contiguous int64 [F][P][2] array")
        if self.lib.oracle_xmac_tri(_u8(volt), N, F, T, int(zero_invalid), _i64(vis)) != 0:
            raise RuntimeError("oracle_xmac_tri failed")
        return vis

    def xmac_full(self, volt: np.ndarray, zero_invalid: bool = False) -> np.ndarray:
        """Full matrix int64 [F][N][N][2]; element [f][i][j] is V_ij(f)."""
        volt = _check_volt(volt)
        T, F, N = volt.shape
        out = np.zeros((F, N, N, 2), np.int64)
        if self.lib.oracle_xmac_full(_u8(volt), N, F, T, int(zero_invalid), _i64(out)) != 0:
            raise RuntimeError("oracle_xmac_full failed")
        return out

    def xmac_pair(self, volt: np.ndarray, f: int, i: int, j: int,
                  zero_invalid: bool = False) -> tuple[int, int]:
        """One visibility V_ij(f) as (re, im) Python ints."""
        volt = _check_volt(volt)
        T, F, N = volt.shape
        out = np.zeros(2, np.int64)
        if self.lib.oracle_xmac_pair(_u8(volt), N, F, T, int(zero_invalid), f, i, j,
                                     _i64(out)) != 0:
            raise ValueError("oracle_xmac_pair: index out of range")
        return int(out[0]), int(out[1])

    def beam(self, volt: np.ndarray, n_avg: int = 1, zero_invalid: bool = False) -> np.ndarray:
        """Incoherent beam int64 [T / n_avg][F]: total power of all inputs per channel."""
        volt = _check_volt(volt)
        T, F, N = volt.shape
        out = np.zeros((T // max(n_avg, 1), F), np.int64)
        if self.lib.oracle_beam(_u8(volt), N, F, T, int(n_avg), int(zero_invalid), _i64(out)) != 0:
            raise ValueError("oracle_beam: bad arguments")
        return out

    def remap(self, tri: np.ndarray, nat_of_pfb, f_avg: int = 1) -> np.ndarray:
        """Station x polarisation products in natural order, int64
        [F / f_avg][S(S+1)/2][2][2][2], from PFB-order triangles int64
        [n_dumps][F][P][2] (or one [F][P][2]), summed over the dumps."""
        t = np.ascontiguousarray(tri, dtype=np.int64)
        if t.ndim == 3:
            t = t[None]
        D, F, P, _ = t.shape
        N = int(round((np.sqrt(8 * P + 1) - 1) / 2))
        perm = np.ascontiguousarray(nat_of_pfb, dtype=np.int32)
        if N * (N + 1) // 2 != P or perm.shape != (N,):
            raise ValueError("triangle size and permutation length disagree")
        S = N // 2
        out = np.zeros((F // max(f_avg, 1), S * (S + 1) // 2, 2, 2, 2), np.int64)
        i32p = ctypes.POINTER(ctypes.c_int32)
        if self.lib.oracle_remap(_i64(t), N, F, D, int(f_avg), perm.ctypes.data_as(i32p), _i64(out)) != 0:
            raise ValueError("oracle_remap: bad arguments")
        return out

    def ingest(self, packets: np.ndarray, bank: int):
        """One bank of 264-byte PFB packets (uint8 [n][264]) -> the voltage block
        uint8 [500][3072][256] and the counters (good, bad header, bad checksum,
        bad field, duplicate, missing slots)."""
        pk = np.ascontiguousarray(packets, dtype=np.uint8).reshape(-1, 264)
        volt = np.zeros((500, 3072, 256), np.uint8)
        counters = np.zeros(6, np.int64)
        if self.lib.oracle_ingest(_u8(pk), pk.shape[0], int(bank), _u8(volt), _i64(counters)) != 0:
            raise ValueError("oracle_ingest: bad arguments")
        return volt, counters

    def fine_pfb(self, x: np.ndarray, window: np.ndarray, scale: float = 1.0):
        """Fine polyphase filterbank (Section 3.2.1) of int8 coarse-channel
        samples x [Q][N][S][2] with the window h [n_taps * 128]; returns the
        spectra complex128 [M][Q * 128][N] and their 4+4-bit codes uint8
        [M][Q * 128][N] (M = S / 128 - n_taps + 1, channel q * 128 + c with
        c = (k + 64) mod 128 for DFT bin k)."""
        xx = np.ascontiguousarray(x, dtype=np.int8)
        h = np.ascontiguousarray(window, dtype=np.float64).ravel()
        if xx.ndim != 4 or xx.shape[3] != 2 or h.size % 128 != 0:
            raise ValueError("x must be int8 [Q][N][S][2] and the window n_taps * 128 long")
        Q, N, S, _ = xx.shape
        taps = h.size // 128
        if S % 128 != 0 or S < 128 * taps:
            raise ValueError("S must be a multiple of 128 and at least 128 * n_taps")
        M = S // 128 - taps + 1
        spec = np.zeros((M, Q * 128, N, 2), np.float64)
        volt = np.zeros((M, Q * 128, N), np.uint8)
        dp = ctypes.POINTER(ctypes.c_double)
        if self.lib.oracle_fine_pfb(xx.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)), Q, N, S,
                                    h.ctypes.data_as(dp), taps, float(scale),
                                    spec.ctypes.data_as(dp), _u8(volt)) != 0:
            raise ValueError("oracle_fine_pfb: bad arguments")
        return spec[..., 0] + 1j * spec[..., 1], volt

    def set_threads(self, n: int) -> int:
        """Set the OpenMP threads of the triangle routine; returns the count in effect."""
        return int(self.lib.oracle_set_threads(int(n)))

    def threads(self) -> int:
        """OpenMP threads the triangle routine uses."""
        return int(self.lib.oracle_threads())


def default() -> OracleLib:
    global _default
    with _lock:
        if _default is None:
            _default = OracleLib(build())
        return _default


def decode(volt, zero_invalid=False):
    return default().decode(volt, zero_invalid)


def xmac(volt, zero_invalid=False, vis=None):
    return default().xmac(volt, zero_invalid, vis)


def xmac_full(volt, zero_invalid=False):
    return default().xmac_full(volt, zero_invalid)


def xmac_pair(volt, f, i, j, zero_invalid=False):
    return default().xmac_pair(volt, f, i, j, zero_invalid)


def beam(volt, n_avg=1, zero_invalid=False):
    return default().beam(volt, n_avg, zero_invalid)


def remap(tri, nat_of_pfb, f_avg=1):
    return default().remap(tri, nat_of_pfb, f_avg)


def ingest(packets, bank):
    return default().ingest(packets, bank)


def fine_pfb(x, window, scale=1.0):
    return default().fine_pfb(x, window, scale)


def pfb_order(n_inputs: int) -> np.ndarray:
    """nat_of_pfb for the PFB input order of Appendix A: within each PFB's 64
    inputs, position k carries input (k mod 4) * 16 + k div 4 (0, 16, 32, 48,
    1, 17, ...), and the PFBs' blocks of 64 follow each other (Appendix B)."""
    if n_inputs % 64 != 0:
        raise ValueError("the PFB order is defined for whole PFBs of 64 inputs")
    k = np.arange(n_inputs)
    return ((k // 64) * 64 + (k % 64 % 4) * 16 + (k % 64) // 4).astype(np.int32)


def set_threads(n: int) -> int:
    return default().set_threads(n)


def threads() -> int:
    return default().threads()


def to_int32(vis: np.ndarray) -> np.ndarray:
    """Narrow int64 visibilities to the int32 output format, checking they fit."""
    lo, hi = np.iinfo(np.int32).min, np.iinfo(np.int32).max
    if vis.size and (vis.min() < lo or vis.max() > hi):
        raise OverflowError("visibility does not fit in int32")
    return vis.astype(np.int32)


SOURCE = _SRC
