"""Python binding of libcorr.so (include/corr.h): argument marshalling only.

Every step of the X-engine runs in the library's CUDA kernels; this module
turns torch tensors into device pointers, torch streams into cudaStream_t
handles, and status codes into exceptions.  PyTorch supplies device memory
(the workspace and output tensors) and streams, nothing else.  If the library
is not built, or its calls fail, these functions raise: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import build as _build

CORR_OK = 0
CORR_E_ARG = -1
CORR_E_STATE = -2
CORR_E_OVERFLOW = -3
CORR_E_NOMEM = -4
CORR_E_BUDGET = -5
CORR_E_CUDA = -6
CORR_E_TIMEOUT = -7
CORR_E_UNSUPPORTED = -8

PATH_AUTO = 0
PATH_CUDACORE = 1
PATH_MMA_I8 = 2
PATH_TC_FP8 = 3
PATHS = {"auto": PATH_AUTO, "cudacore": PATH_CUDACORE, "mma_i8": PATH_MMA_I8,
         "tc_fp8": PATH_TC_FP8}
PATH_NAMES = {v: k for k, v in PATHS.items()}

ZERO_INVALID = 1


K_UNPACK, K_XENGINE, K_DUMP, K_OTHER = 0, 1, 2, 3
KIND_NAMES = ["unpack", "xengine", "dump", "other"]


class Profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_longlong * 4), ("timed", ctypes.c_longlong * 4),
                ("ms", ctypes.c_double * 4)]

    def as_dict(self) -> dict:
        return {KIND_NAMES[k]: {"launches": int(self.launches[k]), "timed": int(self.timed[k]),
                                "ms": float(self.ms[k])} for k in range(4)}


class ArrayDesc(ctypes.Structure):
    _fields_ = [("n_inputs", ctypes.c_int), ("n_chan", ctypes.c_int),
                ("n_time_per_int", ctypes.c_int), ("path", ctypes.c_int), ("flags", ctypes.c_uint),
                ("tile", ctypes.c_int)]


BATCH_MAX = 16


class CorrError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {strerror(status)} ({status})")


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB_PATH


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libcorr.so (building it first if it is missing and allowed)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB_PATH
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"{path} is not built; run paper_1501_05992_gb300.build.build()")
            _build.build()
        lib = ctypes.CDLL(path)
        vp, c_int, c_size = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
        sig = {
            "corr_create": ([c_int, c_int, c_int], vp),
            "corr_destroy": ([vp], c_int),
            "corr_set_path": ([vp, c_int], c_int),
            "corr_get_path": ([vp], c_int),
            "corr_set_tile": ([vp, c_int], c_int),
            "corr_set_wait_limit": ([vp, ctypes.c_longlong], c_int),
            "corr_debug_inject": ([vp, ctypes.c_uint], c_int),
            "corr_set_flags": ([vp, ctypes.c_uint], c_int),
            "corr_workspace_bytes": ([vp], c_size),
            "corr_workspace_bytes_for": ([c_int, c_int, c_int], c_size),
            "corr_bind_workspace": ([vp, vp, c_size], c_int),
            "corr_accumulate": ([vp, vp, c_int, vp], c_int),
            "corr_dump": ([vp, vp, vp], c_int),
            "corr_samples": ([vp], ctypes.c_longlong),
            "corr_integrate": ([vp, vp, c_int, vp, vp], c_int),
            "corr_integrate_beam": ([vp, vp, c_int, vp, vp, c_int, vp], c_int),
            "corr_accumulate_host": ([vp, vp, c_int, vp], c_int),
            "corr_dump_host": ([vp, vp, vp], c_int),
            "corr_sync": ([vp, vp], c_int),
            "corr_state_bytes": ([vp], c_size),
            "corr_get_state": ([vp, vp, c_size, vp], c_int),
            "corr_set_state": ([vp, vp, c_size, vp], c_int),
            "corr_unpack": ([vp, c_int, c_int, c_int, vp, ctypes.c_uint, vp], c_int),
            "corr_xmac_noalloc": ([vp, c_int, c_int, c_int, vp, ctypes.c_uint, vp], c_int),
            "corr_incoherent_beam": ([vp, c_int, c_int, c_int, c_int, ctypes.c_uint, vp, vp], c_int),
            "corr_ingest_packets": ([vp, ctypes.c_longlong, c_int, vp, vp, vp, vp], c_int),
            "corr_remap": ([ctypes.POINTER(vp), c_int, c_int, c_int, c_int, vp, vp, vp], c_int),
            "corr_fine_pfb": ([vp, c_int, c_int, ctypes.c_longlong, vp, c_int, ctypes.c_float, vp, vp, vp],
                              c_int),
            "corr_batch_create": ([c_int, ctypes.POINTER(ArrayDesc)], vp),
            "corr_batch_destroy": ([vp], c_int),
            "corr_batch_workspace_bytes": ([vp], c_size),
            "corr_batch_bind_workspace": ([vp, vp, c_size], c_int),
            "corr_batch_path": ([vp, c_int], c_int),
            "corr_batch_samples": ([vp, c_int], ctypes.c_longlong),
            "corr_batch_array": ([vp, c_int], vp),
            "corr_batch_accumulate": ([vp, ctypes.POINTER(vp), ctypes.POINTER(c_int), vp], c_int),
            "corr_batch_dump": ([vp, ctypes.POINTER(vp), vp], c_int),
            "corr_batch_integrate": ([vp, ctypes.POINTER(vp), ctypes.POINTER(c_int), ctypes.POINTER(vp), vp],
                                     c_int),
            "corr_batch_sync": ([vp, vp], c_int),
            "corr_batch_graph_capture": ([vp, ctypes.POINTER(vp), ctypes.POINTER(c_int),
                                          ctypes.POINTER(vp), vp, ctypes.POINTER(vp)], c_int),
            "corr_graph_launch": ([vp, vp], c_int),
            "corr_graph_destroy": ([vp], c_int),
            "corr_profile_enable": ([vp, c_int], c_int),
            "corr_profile_read": ([vp, ctypes.POINTER(Profile), c_int], c_int),
            "corr_last_error": ([], c_int),
            "corr_strerror": ([c_int], ctypes.c_char_p),
            "corr_version": ([], c_int),
            "corr_probe_rate": ([c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), vp],
                                c_int),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def strerror(status: int) -> str:
    try:
        return load().corr_strerror(int(status)).decode()
    except Exception:  # library not loadable: still give a message
        return f"status {status}"


def _check(status: int, what: str) -> None:
    if status != CORR_OK:
        raise CorrError(status, what)


def _stream_handle(stream) -> int | None:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def n_pairs(n_inputs: int) -> int:
    return n_inputs * (n_inputs + 1) // 2


def workspace_bytes(n_inputs: int, n_chan: int, n_time_per_int: int) -> int:
    """Device workspace a context of this shape needs (no device required)."""
    nb = load().corr_workspace_bytes_for(n_inputs, n_chan, n_time_per_int)
    if nb == 0:
        raise CorrError(load().corr_last_error(), "corr_workspace_bytes_for")
    return int(nb)


class Correlator:
    """One X-engine context: accumulators for n_chan x N(N+1)/2 visibilities.

    accumulate(volt) adds a block of uint8 [T][F][N] voltages to the running
    integration; dump() returns (or writes) the int32 [F][P][2] packed lower
    triangle and starts a new integration.
    """

    def __init__(self, n_inputs: int, n_chan: int, n_time_per_int: int,
                 path: str | int = "auto", zero_invalid: bool = False,
                 device: torch.device | int | None = None):
        self._lib = load()
        self.n_inputs, self.n_chan, self.n_time_per_int = n_inputs, n_chan, n_time_per_int
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   (device if isinstance(device, int) else device.index or 0))
        with torch.cuda.device(self.device):
            ctx = self._lib.corr_create(n_inputs, n_chan, n_time_per_int)
            if not ctx:
                raise CorrError(self._lib.corr_last_error(), "corr_create")
            self._ctx = ctypes.c_void_p(ctx)
            try:
                if zero_invalid:
                    _check(self._lib.corr_set_flags(self._ctx, ZERO_INVALID), "corr_set_flags")
                self.set_path(path)
                nbytes = self._lib.corr_workspace_bytes(self._ctx)
                self._ws = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=self.device)
                _check(self._lib.corr_bind_workspace(self._ctx, ctypes.c_void_p(self._ws.data_ptr()),
                                                     nbytes), "corr_bind_workspace")
            except Exception:
                self._lib.corr_destroy(self._ctx)
                self._ctx = None
                raise

    # -- properties -------------------------------------------------------
    @property
    def n_pairs(self) -> int:
        return n_pairs(self.n_inputs)

    @property
    def workspace_bytes(self) -> int:
        return int(self._ws.numel())

    @property
    def samples(self) -> int:
        return int(self._lib.corr_samples(self._ctx))

    @property
    def path(self) -> str:
        return PATH_NAMES[self._lib.corr_get_path(self._ctx)]

    def set_tile(self, tile: int) -> None:
        """Tile shape (corr_set_tile): 32 or 64 for the CUDA-core path, 128
        (single tile-pair items) or 256 (pair items) for the tcgen05 path,
        0 to choose by shape."""
        _check(self._lib.corr_set_tile(self._ctx, int(tile)), f"corr_set_tile({tile})")

    def set_wait_limit(self, cycles: int) -> None:
        """Bounded-wait limit of the tensor-core kernel (SM cycles; 0 = default)."""
        _check(self._lib.corr_set_wait_limit(self._ctx, int(cycles)), "corr_set_wait_limit")

    def inject_stall(self) -> None:
        """Test hook: the next tensor-core launch times out on purpose."""
        _check(self._lib.corr_debug_inject(self._ctx, 1), "corr_debug_inject")

    def set_path(self, path: str | int) -> None:
        code = PATHS[path] if isinstance(path, str) else int(path)
        _check(self._lib.corr_set_path(self._ctx, code), f"corr_set_path({path})")

    # -- integration -------------------------------------------------------
    def _check_volt(self, volt: torch.Tensor, device: bool) -> int:
        if volt.dtype != torch.uint8 or volt.dim() != 3 or not volt.is_contiguous():
            raise ValueError("volt must be a contiguous uint8 tensor [T][F][N]")
        if volt.shape[1] != self.n_chan or volt.shape[2] != self.n_inputs:
            raise ValueError(f"volt shape {tuple(volt.shape)} does not match "
                             f"[T][{self.n_chan}][{self.n_inputs}]")
        if device and volt.device != self.device:
            raise ValueError(f"volt must be on {self.device}")
        if not device and volt.device.type != "cpu":
            raise ValueError("volt must be a host tensor")
        return int(volt.shape[0])

    def accumulate(self, volt: torch.Tensor, stream=None) -> None:
        nt = self._check_volt(volt, device=True)
        _check(self._lib.corr_accumulate(self._ctx, ctypes.c_void_p(volt.data_ptr()), nt,
                                         _stream_handle(stream)), "corr_accumulate")

    def dump(self, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        if out is None:
            out = torch.empty((self.n_chan, self.n_pairs, 2), dtype=torch.int32, device=self.device)
        elif (out.dtype != torch.int32 or out.shape != (self.n_chan, self.n_pairs, 2)
              or not out.is_contiguous() or out.device != self.device):
            raise ValueError("out must be a contiguous int32 [F][P][2] tensor on the device")
        _check(self._lib.corr_dump(self._ctx, ctypes.c_void_p(out.data_ptr()),
                                   _stream_handle(stream)), "corr_dump")
        return out

    def integrate(self, volt: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """One whole integration of `volt` written straight to `out` (see corr_integrate);
        the running integration is not touched."""
        nt = self._check_volt(volt, device=True)
        if out is None:
            out = torch.empty((self.n_chan, self.n_pairs, 2), dtype=torch.int32, device=self.device)
        elif (out.dtype != torch.int32 or out.shape != (self.n_chan, self.n_pairs, 2)
              or not out.is_contiguous() or out.device != self.device):
            raise ValueError("out must be a contiguous int32 [F][P][2] tensor on the device")
        vptr = ctypes.c_void_p(volt.data_ptr()) if nt > 0 else ctypes.c_void_p(0)
        _check(self._lib.corr_integrate(self._ctx, vptr, nt, ctypes.c_void_p(out.data_ptr()),
                                        _stream_handle(stream)), "corr_integrate")
        return out

    def integrate_beam(self, volt: torch.Tensor, n_avg: int = 1, out: torch.Tensor | None = None,
                       beam: torch.Tensor | None = None, stream=None):
        """integrate() plus the incoherent beam of the same samples, int32
        [T / n_avg][F] (corr_integrate_beam): returns (triangle, beam)."""
        nt = self._check_volt(volt, device=True)
        if out is None:
            out = torch.empty((self.n_chan, self.n_pairs, 2), dtype=torch.int32, device=self.device)
        elif (out.dtype != torch.int32 or out.shape != (self.n_chan, self.n_pairs, 2)
              or not out.is_contiguous() or out.device != self.device):
            raise ValueError("out must be a contiguous int32 [F][P][2] tensor on the device")
        shape = (nt // max(n_avg, 1), self.n_chan)
        if beam is None:
            beam = torch.empty(shape, dtype=torch.int32, device=self.device)
        elif (beam.dtype != torch.int32 or tuple(beam.shape) != shape or not beam.is_contiguous()
              or beam.device != self.device):
            raise ValueError(f"beam must be a contiguous int32 {list(shape)} tensor on the device")
        vptr = ctypes.c_void_p(volt.data_ptr()) if nt > 0 else ctypes.c_void_p(0)
        _check(self._lib.corr_integrate_beam(self._ctx, vptr, nt, ctypes.c_void_p(out.data_ptr()),
                                             ctypes.c_void_p(beam.data_ptr()), int(n_avg),
                                             _stream_handle(stream)), "corr_integrate_beam")
        return out, beam

    def accumulate_host(self, volt: torch.Tensor, stream=None) -> None:
        nt = self._check_volt(volt, device=False)
        _check(self._lib.corr_accumulate_host(self._ctx, ctypes.c_void_p(volt.data_ptr()), nt,
                                              _stream_handle(stream)), "corr_accumulate_host")

    def dump_host(self, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        if out is None:
            out = torch.empty((self.n_chan, self.n_pairs, 2), dtype=torch.int32, pin_memory=True)
        elif (out.dtype != torch.int32 or out.shape != (self.n_chan, self.n_pairs, 2)
              or not out.is_contiguous() or out.device.type != "cpu"):
            raise ValueError("out must be a contiguous int32 [F][P][2] host tensor")
        _check(self._lib.corr_dump_host(self._ctx, ctypes.c_void_p(out.data_ptr()),
                                        _stream_handle(stream)), "corr_dump_host")
        return out

    def sync(self, stream=None) -> None:
        _check(self._lib.corr_sync(self._ctx, _stream_handle(stream)), "corr_sync")

    # -- profiling ---------------------------------------------------------
    def profile_enable(self, on: bool = True) -> None:
        _check(self._lib.corr_profile_enable(self._ctx, int(on)), "corr_profile_enable")

    def profile_read(self, reset: bool = True) -> dict:
        prof = Profile()
        _check(self._lib.corr_profile_read(self._ctx, ctypes.byref(prof), int(reset)),
               "corr_profile_read")
        return prof.as_dict()

    # -- checkpoint / resume ---------------------------------------------
    def get_state(self, stream=None) -> bytes:
        nb = self._lib.corr_state_bytes(self._ctx)
        buf = ctypes.create_string_buffer(nb)
        _check(self._lib.corr_get_state(self._ctx, buf, nb, _stream_handle(stream)),
               "corr_get_state")
        return buf.raw

    def set_state(self, state: bytes, stream=None) -> None:
        buf = ctypes.create_string_buffer(bytes(state), len(state))
        _check(self._lib.corr_set_state(self._ctx, buf, len(state), _stream_handle(stream)),
               "corr_set_state")

    # -- lifetime -----------------------------------------------------------
    def close(self) -> None:
        if getattr(self, "_ctx", None):
            self._lib.corr_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Graph:
    """An executable CUDA graph holding one whole integration of a Batch."""

    def __init__(self, lib, handle, keep):
        self._lib, self._h, self._keep = lib, handle, keep

    def launch(self, stream=None) -> None:
        _check(self._lib.corr_graph_launch(self._h, _stream_handle(stream)), "corr_graph_launch")

    def close(self) -> None:
        if self._h:
            self._lib.corr_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Several arrays correlated together; tensor-core arrays share one
    persistent launch.  ``arrays`` holds (n_inputs, n_chan, n_time_per_int)
    tuples or dicts with those keys plus optional ``path`` / ``zero_invalid``."""

    def __init__(self, arrays, device: torch.device | int | None = None):
        self._lib = load()
        specs = []
        for a in arrays:
            if isinstance(a, dict):
                specs.append((a["n_inputs"], a["n_chan"], a["n_time_per_int"],
                              a.get("path", "auto"), bool(a.get("zero_invalid", False)),
                              int(a.get("tile", 0))))
            else:
                specs.append((a[0], a[1], a[2], "auto", False, 0))
        self.specs = specs
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   (device if isinstance(device, int) else device.index or 0))
        descs = (ArrayDesc * len(specs))()
        for k, (n, f, t, path, zi, tile) in enumerate(specs):
            descs[k] = ArrayDesc(n, f, t, PATHS[path] if isinstance(path, str) else int(path),
                                 ZERO_INVALID if zi else 0, tile)
        with torch.cuda.device(self.device):
            h = self._lib.corr_batch_create(len(specs), descs)
            if not h:
                raise CorrError(self._lib.corr_last_error(), "corr_batch_create")
            self._h = ctypes.c_void_p(h)
            nbytes = self._lib.corr_batch_workspace_bytes(self._h)
            self._ws = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=self.device)
            _check(self._lib.corr_batch_bind_workspace(self._h, ctypes.c_void_p(self._ws.data_ptr()),
                                                       nbytes), "corr_batch_bind_workspace")

    def __len__(self):
        return len(self.specs)

    @property
    def paths(self) -> list[str]:
        return [PATH_NAMES[self._lib.corr_batch_path(self._h, a)] for a in range(len(self))]

    def samples(self, a: int) -> int:
        return int(self._lib.corr_batch_samples(self._h, a))

    def _ctx(self, a: int):
        h = self._lib.corr_batch_array(self._h, a)
        if not h:
            raise CorrError(self._lib.corr_last_error(), "corr_batch_array")
        return ctypes.c_void_p(h)

    def profile_enable(self, on: bool = True) -> None:
        for a in range(len(self)):
            _check(self._lib.corr_profile_enable(self._ctx(a), int(on)), "corr_profile_enable")

    def profile_read(self, reset: bool = True) -> list[dict]:
        out = []
        for a in range(len(self)):
            prof = Profile()
            _check(self._lib.corr_profile_read(self._ctx(a), ctypes.byref(prof), int(reset)),
                   "corr_profile_read")
            out.append(prof.as_dict())
        return out

    def _ptrs(self, tensors, what):
        arr = (ctypes.c_void_p * len(self))()
        for a, t in enumerate(tensors):
            arr[a] = ctypes.c_void_p(t.data_ptr()) if t is not None else None
        return arr

    def _volts(self, volts):
        if len(volts) != len(self):
            raise ValueError("one voltage tensor (or None) per array")
        nt = (ctypes.c_int * len(self))()
        for a, v in enumerate(volts):
            if v is None:
                continue
            n, f = self.specs[a][0], self.specs[a][1]
            if (v.dtype != torch.uint8 or v.dim() != 3 or not v.is_contiguous() or
                    v.shape[1] != f or v.shape[2] != n or v.device != self.device):
                raise ValueError(f"array {a}: voltages must be a contiguous uint8 [T][{f}][{n}] "
                                 f"tensor on {self.device}")
            nt[a] = int(v.shape[0])
        return self._ptrs(volts, "volt"), nt

    def _outs(self, outs):
        if outs is None:
            outs = [torch.empty((f, n * (n + 1) // 2, 2), dtype=torch.int32, device=self.device)
                    for (n, f, *_rest) in self.specs]
        if len(outs) != len(self):
            raise ValueError("one output tensor (or None) per array")
        for a, o in enumerate(outs):
            n, f = self.specs[a][0], self.specs[a][1]
            if o is not None and (o.dtype != torch.int32 or o.shape != (f, n * (n + 1) // 2, 2)
                                  or not o.is_contiguous() or o.device != self.device):
                raise ValueError(f"array {a}: output must be a contiguous int32 [{f}][P][2] tensor")
        return outs

    def accumulate(self, volts, stream=None) -> None:
        ptrs, nt = self._volts(volts)
        _check(self._lib.corr_batch_accumulate(self._h, ptrs, nt, _stream_handle(stream)),
               "corr_batch_accumulate")

    def dump(self, outs=None, stream=None):
        outs = self._outs(outs)
        _check(self._lib.corr_batch_dump(self._h, self._ptrs(outs, "vis"), _stream_handle(stream)),
               "corr_batch_dump")
        return outs

    def dump_host(self, a: int, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """corr_dump_host on array `a` of the batch: its packed triangle into a host tensor."""
        n, f = self.specs[a][0], self.specs[a][1]
        if out is None:
            out = torch.empty((f, n * (n + 1) // 2, 2), dtype=torch.int32, pin_memory=True)
        elif (out.dtype != torch.int32 or out.shape != (f, n * (n + 1) // 2, 2)
              or not out.is_contiguous() or out.device.type != "cpu"):
            raise ValueError("out must be a contiguous int32 [F][P][2] host tensor")
        _check(self._lib.corr_dump_host(self._ctx(a), ctypes.c_void_p(out.data_ptr()),
                                        _stream_handle(stream)), "corr_dump_host")
        return out

    def integrate(self, volts, outs=None, stream=None):
        """Whole integrations of every array straight into `outs` (see corr_batch_integrate)."""
        ptrs, nt = self._volts(volts)
        outs = self._outs(outs)
        _check(self._lib.corr_batch_integrate(self._h, ptrs, nt, self._ptrs(outs, "vis"),
                                              _stream_handle(stream)), "corr_batch_integrate")
        return outs

    def sync(self, stream=None) -> None:
        _check(self._lib.corr_batch_sync(self._h, _stream_handle(stream)), "corr_batch_sync")

    def capture(self, volts, outs=None, stream=None) -> tuple[Graph, list]:
        """Capture integrate(volts, outs) as one replayable graph."""
        if stream is None:
            stream = torch.cuda.Stream(self.device)
        ptrs, nt = self._volts(volts)
        outs = self._outs(outs)
        h = ctypes.c_void_p()
        _check(self._lib.corr_batch_graph_capture(self._h, ptrs, nt, self._ptrs(outs, "vis"),
                                                  _stream_handle(stream), ctypes.byref(h)),
               "corr_batch_graph_capture")
        return Graph(self._lib, h, (list(volts), outs)), outs

    def close(self) -> None:
        if getattr(self, "_h", None):
            self._lib.corr_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def incoherent_beam(volt: torch.Tensor, n_avg: int = 1, zero_invalid: bool = False,
                    out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Total power of all inputs per channel: int32 [T / n_avg][F] (corr_incoherent_beam)."""
    if volt.dtype != torch.uint8 or volt.dim() != 3 or not volt.is_contiguous() or not volt.is_cuda:
        raise ValueError("volt must be a contiguous uint8 CUDA tensor [T][F][N]")
    T, F, N = volt.shape
    if n_avg < 1 or T % n_avg:
        raise ValueError("n_time must be a multiple of n_avg")
    shape = (T // n_avg, F)
    if out is None:
        out = torch.empty(shape, dtype=torch.int32, device=volt.device)
    elif out.dtype != torch.int32 or tuple(out.shape) != shape or not out.is_contiguous():
        raise ValueError(f"out must be a contiguous int32 {shape} tensor")
    _check(load().corr_incoherent_beam(ctypes.c_void_p(volt.data_ptr()), T, F, N, n_avg,
                                       ZERO_INVALID if zero_invalid else 0,
                                       ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)),
           "corr_incoherent_beam")
    return out


PKT_BYTES, PKT_FRAMES, PKT_CHANNELS, PKT_INPUTS = 264, 500, 3072, 256
PKT_SLOTS = PKT_FRAMES * (PKT_CHANNELS // 4) * 4
PKT_COUNTER_NAMES = ("good", "bad_header", "bad_checksum", "bad_field", "duplicate", "missing")
PKT_COUNTERS = len(PKT_COUNTER_NAMES)


def ingest_packets(packets: torch.Tensor, bank: int, out: torch.Tensor | None = None,
                   seen: torch.Tensor | None = None, counters: torch.Tensor | None = None,
                   stream=None):
    """One bank of PFB packets (uint8 CUDA tensor [n][264]) -> the voltage block
    uint8 [500][3072][256] and int32 counters [6] (corr_ingest_packets)."""
    if (packets.dtype != torch.uint8 or packets.dim() != 2 or packets.shape[1] != PKT_BYTES
            or not packets.is_contiguous() or not packets.is_cuda):
        raise ValueError("packets must be a contiguous uint8 CUDA tensor [n][264]")
    dev = packets.device
    if out is None:
        out = torch.empty((PKT_FRAMES, PKT_CHANNELS, PKT_INPUTS), dtype=torch.uint8, device=dev)
    if seen is None:
        seen = torch.empty(PKT_SLOTS, dtype=torch.uint8, device=dev)
    if counters is None:
        counters = torch.empty(PKT_COUNTERS, dtype=torch.int32, device=dev)
    if tuple(out.shape) != (PKT_FRAMES, PKT_CHANNELS, PKT_INPUTS) or out.dtype != torch.uint8:
        raise ValueError("out must be uint8 [500][3072][256]")
    if (seen.numel() * seen.element_size() < PKT_SLOTS or counters.numel() < PKT_COUNTERS
            or counters.dtype != torch.int32):
        raise ValueError(f"seen must hold one byte per slot and counters {PKT_COUNTERS} int32")
    _check(load().corr_ingest_packets(ctypes.c_void_p(packets.data_ptr()), packets.shape[0], bank,
                                      ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(seen.data_ptr()),
                                      ctypes.c_void_p(counters.data_ptr()), _stream_handle(stream)),
           "corr_ingest_packets")
    return out, counters


def remap(tris, nat_of_pfb: torch.Tensor | None = None, f_avg: int = 1,
          out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Station-pair products in natural input order, summed over the dumps in
    `tris` (one [F][P][2] int32 tensor or a list of them) and f_avg channels:
    int32 [F / f_avg][S(S+1)/2][2][2][2] (corr_remap).  nat_of_pfb: int32
    tensor [N] on the device, or None for the Appendix A PFB order."""
    if isinstance(tris, torch.Tensor):
        tris = [tris]
    if not tris or len(tris) > 8:
        raise ValueError("between 1 and 8 triangles")
    F, P, two = tris[0].shape
    N = int(round(((8 * P + 1) ** 0.5 - 1) / 2))
    for t in tris:
        if (t.dtype != torch.int32 or tuple(t.shape) != (F, P, 2) or not t.is_contiguous()
                or not t.is_cuda or N * (N + 1) // 2 != P):
            raise ValueError("triangles must be contiguous int32 CUDA tensors [F][N(N+1)/2][2]")
    S = N // 2
    shape = (F // max(f_avg, 1), S * (S + 1) // 2, 2, 2, 2)
    if out is None:
        out = torch.empty(shape, dtype=torch.int32, device=tris[0].device)
    elif out.dtype != torch.int32 or tuple(out.shape) != shape or not out.is_contiguous():
        raise ValueError(f"out must be a contiguous int32 {shape} tensor")
    perm_ptr = ctypes.c_void_p(0)
    if nat_of_pfb is not None:
        if (nat_of_pfb.dtype != torch.int32 or tuple(nat_of_pfb.shape) != (N,) or not nat_of_pfb.is_cuda
                or not nat_of_pfb.is_contiguous()):
            raise ValueError(f"nat_of_pfb must be a contiguous int32 CUDA tensor [{N}]")
        perm_ptr = ctypes.c_void_p(nat_of_pfb.data_ptr())
    ptrs = (ctypes.c_void_p * len(tris))(*[t.data_ptr() for t in tris])
    _check(load().corr_remap(ptrs, len(tris), N, F, f_avg, perm_ptr, ctypes.c_void_p(out.data_ptr()),
                             _stream_handle(stream)), "corr_remap")
    return out


PFB_POINTS = 128


def fine_pfb(x: torch.Tensor, window: torch.Tensor, scale: float = 1.0, volt: bool | torch.Tensor = True,
             spec: bool | torch.Tensor = False, stream=None):
    """Fine polyphase filterbank (corr_fine_pfb, Section 3.2.1) of int8 coarse-
    channel samples x [Q][N][S][2] with the window float32 [n_taps * 128]
    (n_taps 1 or 12).  Returns (volt, spec): the 4+4-bit codes uint8
    [M][Q * 128][N] (the X-engine's input layout) and the spectra float32
    [M][Q * 128][N][2], M = S / 128 - n_taps + 1; pass True for a new tensor,
    a tensor to write into, or False to skip that output (None returned)."""
    if x.dtype != torch.int8 or x.dim() != 4 or x.shape[3] != 2 or not x.is_contiguous() or not x.is_cuda:
        raise ValueError("x must be a contiguous int8 CUDA tensor [Q][N][S][2]")
    if (window.dtype != torch.float32 or window.dim() != 1 or window.numel() % PFB_POINTS
            or not window.is_contiguous() or not window.is_cuda):
        raise ValueError("window must be a contiguous float32 CUDA tensor [n_taps * 128]")
    Q, N, S, _ = x.shape
    taps = window.numel() // PFB_POINTS
    if S % PFB_POINTS or S < PFB_POINTS * taps:
        raise ValueError("S must be a multiple of 128 and at least 128 * n_taps")
    M = S // PFB_POINTS - taps + 1

    def _out(arg, shape, dtype):
        if arg is False or arg is None:
            return None
        if arg is True:
            return torch.empty(shape, dtype=dtype, device=x.device)
        if arg.dtype != dtype or tuple(arg.shape) != shape or not arg.is_contiguous():
            raise ValueError(f"output must be a contiguous {dtype} {shape} tensor")
        return arg
    v = _out(volt, (M, Q * PFB_POINTS, N), torch.uint8)
    sp = _out(spec, (M, Q * PFB_POINTS, N, 2), torch.float32)
    if v is None and sp is None:
        raise ValueError("ask for at least one of volt and spec")
    _check(load().corr_fine_pfb(ctypes.c_void_p(x.data_ptr()), Q, N, S, ctypes.c_void_p(window.data_ptr()), taps,
                                float(scale), ctypes.c_void_p(0 if v is None else v.data_ptr()),
                                ctypes.c_void_p(0 if sp is None else sp.data_ptr()), _stream_handle(stream)),
           "corr_fine_pfb")
    return v, sp


def unpack(volt: torch.Tensor, zero_invalid: bool = False, stream=None) -> torch.Tensor:
    """K1 on its own: uint8 [T][F][N] -> int8 [F][N][T][2] (real, imaginary)."""
    if volt.dtype != torch.uint8 or volt.dim() != 3 or not volt.is_contiguous() or not volt.is_cuda:
        raise ValueError("volt must be a contiguous uint8 CUDA tensor [T][F][N]")
    T, F, N = volt.shape
    out = torch.empty((F, N, T, 2), dtype=torch.int8, device=volt.device)
    _check(load().corr_unpack(ctypes.c_void_p(volt.data_ptr()), T, F, N,
                              ctypes.c_void_p(out.data_ptr()), ZERO_INVALID if zero_invalid else 0,
                              _stream_handle(stream)), "corr_unpack")
    return out


PROBES = {"tc_fp8": 0, "mma_s8": 1, "dp4a": 2, "ffma": 3}


def probe_rate(kind: str, stream=None) -> tuple[float, float]:
    """Measured peak rate of one instruction form on the current device
    (corr_probe_rate): (ops per second, ms of the timed launch)."""
    rate, ms = ctypes.c_double(), ctypes.c_double()
    _check(load().corr_probe_rate(PROBES[kind], ctypes.byref(rate), ctypes.byref(ms), _stream_handle(stream)),
           f"corr_probe_rate({kind})")
    return rate.value, ms.value
