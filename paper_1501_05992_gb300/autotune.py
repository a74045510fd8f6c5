"""Measured choice of X-engine form and tile shape per array shape.

For an array of N inputs x F channels x T samples per integration, every
candidate (path, tile) the device supports is timed on a probe block of the
same N and T (random bytes: the kernels' speed does not depend on the values)
with a bounded number of channels, and the fastest is kept in a JSON cache
keyed by device name and shape.  The candidates are the library's tile shapes
(Section 3.4.2: the tile sets the arithmetic intensity): tcgen05 FP8 with
every work item one 128 x 128 tile pair (tile 128; each item's epilogue
overlaps the next item's MMAs) or with pair items, a diagonal tile and the
tile left of it as one 256-row column sharing one conversion (tile 256);
int8 mma.sync on 64 x 64; and the dp4a CUDA-core kernel on 64 x 64 or
32 x 32 tiles.
"""
from __future__ import annotations

import json
import os
import threading

import torch

from . import corr

CANDIDATES = [("tc_fp8", 256), ("tc_fp8", 128), ("mma_i8", 0), ("cudacore", 64), ("cudacore", 32)]
_lock = threading.Lock()


def _key(device: torch.device, n_inputs: int, n_chan: int, n_time: int) -> str:
    return f"{torch.cuda.get_device_name(device)}|{n_inputs}x{n_chan}x{n_time}"


def _load(path: str | None) -> dict:
    if path and os.path.exists(path):
        try:
            with open(path) as f:
                return json.load(f)
        except (OSError, ValueError):
            return {}
    return {}


def _save(path: str | None, cache: dict) -> None:
    if not path:
        return
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune(n_inputs: int, n_chan: int, n_time: int, cache_path: str | None = None,
         reps: int = 3, probe_bytes: int = 1 << 30, device=None,
         candidates=CANDIDATES) -> dict:
    """Fastest (path, tile) for the shape: {"path", "tile", "ms": {...}}."""
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else
                       (device if isinstance(device, int) else device.index or 0))
    key = _key(dev, n_inputs, n_chan, n_time)
    with _lock:
        cache = _load(cache_path)
        if key in cache:
            return cache[key]
    f_probe = max(1, min(n_chan, probe_bytes // max(1, n_time * n_inputs)))
    volt = torch.randint(0, 256, (n_time, f_probe, n_inputs), dtype=torch.uint8, device=dev)
    times = {}
    for path, tile in candidates:
        try:
            c = corr.Correlator(n_inputs, f_probe, n_time, path=path, device=dev)
        except corr.CorrError as e:
            if e.status == corr.CORR_E_UNSUPPORTED:
                continue
            raise
        try:
            if tile:
                c.set_tile(tile)
            out = c.dump()
            c.accumulate(volt)
            c.dump(out)
            torch.cuda.synchronize(dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                c.accumulate(volt)
                c.dump(out)
            e1.record()
            torch.cuda.synchronize(dev)
            c.sync()
            # scale the probe to the full channel count
            times[f"{path}/{tile}"] = e0.elapsed_time(e1) / reps * (n_chan / f_probe)
        finally:
            c.close()
    if not times:
        raise RuntimeError(f"no X-engine path supports {n_inputs} inputs on {dev}")
    best = min(times, key=times.get)
    path, tile = best.split("/")
    result = {"path": path, "tile": int(tile), "ms": times, "probe_channels": f_probe}
    with _lock:
        cache = _load(cache_path)
        cache[key] = result
        _save(cache_path, cache)
    return result


def plan(arrays, cache_path: str | None = None, **kw) -> list[dict]:
    """Batch array descriptors with the measured best path and tile."""
    out = []
    for a in arrays:
        n, f, t = (a["n_inputs"], a["n_chan"], a["n_time_per_int"]) if isinstance(a, dict) else a[:3]
        best = tune(n, f, t, cache_path=cache_path, **kw)
        d = dict(a) if isinstance(a, dict) else {"n_inputs": n, "n_chan": f, "n_time_per_int": t}
        d.update(path=best["path"], tile=best["tile"])
        out.append(d)
    return out
