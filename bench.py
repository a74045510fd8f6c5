#!/usr/bin/env python3
"""Benchmark of the X-engine hot path: complex MAC/s and x real time.

Workload (default "full_band"): 256 inputs x 3072 fine channels, 16
consecutive integrations of 5000 samples (0.5 s at 10 kHz), 4+4-bit voltages
from the seeded gauss3 recipe, generated in device memory before timing.  One
step = 16 whole integrations, each unpacked, correlated and written out as its
packed triangle: the whole hot path over 8 s of data (62.9 GB of voltages,
larger than L2, so no flush is needed between steps).  Graph mode (default)
replays one captured corr_batch_integrate per integration (the X-engine
epilogue stores the triangle straight into the output); direct mode issues
corr_batch_accumulate + corr_batch_dump per integration.

Prints one JSON line (rank 0).  `value` is device-resident throughput, `e2e`
the same metric through the host-buffer C-ABI calls (host->device copies of
every step's voltages and device->host copies of every dump inside the timed
region).  After the timed region, rank 0 adds `extras`: the incoherent beam,
packet ingest, output remap and fine filterbank with their rooflines; the
dp4a CUDA-core, int8 mma.sync and tcgen05 FP8 X-engines on the same
integration (times, fractions of their rooflines, identical triangles, oracle
check); the uneven three-array batch in one persistent launch with
autotuned paths; and the streaming service of three arrays, paced and
unpaced, with every dump checked against the oracle on sampled channels.
`--impl reference` times the CPU oracle on a bounded sample instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Correlator CMAC/s and ×real-time, 256 inputs×3072 ch; TC vs CUDA-core, bit-exact"
UNIT = "CMAC/s"
SAMPLE_RATE_HZ = 1.0e4            # 10 kHz fine channels: one sample per channel per 100 us

WORKLOADS = {
    # name: arrays [(n_inputs, n_chan, samples per integration)], integrations per step, seed
    "full_band": ([(256, 3072, 5000)], 16, 1503),
    "coarse_channel": ([(256, 128, 5000)], 1, 1502),
    # one integration of the full band (3.9 GB of voltages): a small case for traffic captures
    "integration": ([(256, 3072, 5000)], 1, 1503),
    # a quarter of the band, one integration (1 GB of voltages, 1536 items: about ten per CTA, so
    # the steady state rather than the tail): a small case for full profiles
    "quarter_band": ([(256, 768, 5000)], 1, 1507),
    "uneven_batch": ([(128, 1536, 2000), (256, 3072, 5000), (1024, 512, 10000)], 1, 1504),
    # one 50 ms bank of the full band (the packet ingest's unit): a small case for profiles
    "bank": ([(256, 3072, 500)], 1, 1506),
}


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=16)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--path", default="auto", choices=["auto", "cudacore", "mma_i8", "tc_fp8"])
    ap.add_argument("--workload", default="full_band", choices=sorted(WORKLOADS))
    ap.add_argument("--mode", default="graph", choices=["graph", "direct"],
                    help="graph: one captured CUDA graph per integration; direct: C-ABI calls")
    ap.add_argument("--autotune", action="store_true",
                    help="pick path and tile per array by measurement (cached)")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target CPU time of the oracle baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the incoherent-beam and output-remap measurements")
    return ap.parse_args()


# ---------------------------------------------------------------- clocks ---
class ClockSampler:
    """nvidia-smi clock / throttle sampling around the timed region: started
    before the warm-up (nvidia-smi takes a while to produce its first line),
    one reading every 50 ms, and only the readings that arrive between
    mark_start() and mark_stop() (plus one interval) are reported."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    INTERVAL_MS = 50

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None
        self.lines: list[tuple[float, str]] = []
        self.t_start = self.t_stop = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", str(self.INTERVAL_MS)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        t0 = time.perf_counter()
        while not self.lines and time.perf_counter() - t0 < 3.0 and self.proc.poll() is None:
            time.sleep(0.01)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def mark_start(self):
        self.t_start = time.perf_counter()

    def mark_stop(self):
        self.t_stop = time.perf_counter()

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        if self.t_stop is None:
            self.mark_stop()
        time.sleep(self.INTERVAL_MS * 1.5e-3)          # the reading that covers the end
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self._t.join(timeout=2)
        lo = self.t_start if self.t_start is not None else 0.0
        hi = self.t_stop + self.INTERVAL_MS * 1.5e-3
        window = [line for t, line in self.lines if lo <= t <= hi]
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in window:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ distributed ---
def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        import torch
        if args.impl == "ours":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    """The slowest rank's time: the job is done when every rank is."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_array_index(a: int, rank: int) -> int:
    """Generator stream of array a on this rank: every rank correlates its own
    data (weak scaling; channels shard across GPUs with no exchange)."""
    return a + 8 * rank


def job_units(step_cmac: int, steps: int, world: int) -> int:
    """Complex MACs done by the whole job: each rank does the full workload."""
    return step_cmac * steps * world


# ----------------------------------------------------------- CPU baseline ---
def oracle_sample(volt_host_slab, seconds_budget: float):
    """Time the oracle on channels of one integration: returns (CMAC/s, cores, sample str)."""
    import numpy as np
    import oracle
    T, F, N = volt_host_slab.shape
    P = N * (N + 1) // 2
    probe = np.ascontiguousarray(volt_host_slab[:, :2, :])
    t0 = time.perf_counter()
    oracle.xmac(probe)
    per_chan = (time.perf_counter() - t0) / 2
    k = int(max(2, min(F, seconds_budget / max(per_chan, 1e-6))))
    sample = np.ascontiguousarray(volt_host_slab[:, :k, :])
    t0 = time.perf_counter()
    oracle.xmac(sample)
    dt = time.perf_counter() - t0
    cmac = P * k * T
    desc = f"{k} channels x {T} samples x {N} inputs of integration 0 ({cmac:.3e} CMAC, {dt:.1f} s)"
    return cmac / dt, oracle.threads(), desc


def oracle_single_core(volt_host_slab):
    """The oracle on one core, over one channel of the same slab: (CMAC/s, sample str)."""
    import numpy as np
    import oracle
    T, F, N = volt_host_slab.shape
    P = N * (N + 1) // 2
    before = oracle.threads()
    oracle.set_threads(1)
    try:
        one = np.ascontiguousarray(volt_host_slab[:, :1, :])
        t0 = time.perf_counter()
        oracle.xmac(one)
        dt = time.perf_counter() - t0
    finally:
        oracle.set_threads(before)
    return P * T / dt, f"1 channel x {T} samples x {N} inputs on one core ({dt:.1f} s)"


def host_sample_slab(n_inputs, n_chan, n_time, seed, channels):
    from synth import voltgen as vg
    p = vg.gauss3_params(seed, n_inputs, n_chan)
    return vg.gauss3(p, 0, n_time, 0, channels)


def run_reference(args, world, rank):
    if rank != 0:
        return
    arrays, n_int, seed = WORKLOADS[args.workload]
    import oracle
    oracle.build()
    n_inputs, n_chan, t_int = arrays[0]
    P = n_inputs * (n_inputs + 1) // 2
    slab = host_sample_slab(n_inputs, n_chan, t_int, seed, channels=min(n_chan, 64))
    budget = max(1.0, 150.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        oracle_sample(slab[:, :2], 0.5)
    rates, descs, cores = [], [], 1
    for _ in range(args.steps):
        r, cores, d = oracle_sample(slab, min(budget, args.cpu_seconds))
        rates.append(r)
        descs.append(d)
    value = statistics.median(rates)
    step_cmac = sum(n * (n + 1) // 2 * f * t for n, f, t in arrays) * n_int
    rt_rate = sum(n * (n + 1) // 2 * f for n, f, t in arrays) * SAMPLE_RATE_HZ
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": step_cmac / value * 1e3, "higher_is_better": True,
        "ms_per_step_note": ("extrapolated: each timed step runs the oracle on a bounded channel "
                             "sample of the workload, and ms_per_step is the whole step's "
                             "CMAC divided by the median sampled rate"),
        "sampled": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "x_real_time": value / rt_rate,
        "config": workload_config(args, ["oracle (CPU, int64 triple loop)"]),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": descs[-1]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def workload_config(args, paths):
    arrays, n_int, seed = WORKLOADS[args.workload]
    desc = " + ".join(f"{n} inputs x {f} ch x {t} samples" for n, f, t in arrays)
    gb = sum(n * f * t for n, f, t in arrays) * n_int / 1e9
    return {"workload": f"{args.workload}: {desc}, {n_int} integration(s) per step "
                        f"(4+4-bit, gauss3 recipe, seed {seed})",
            "arrays": [{"n_inputs": n, "n_chan": f, "samples_per_integration": t, "path": p}
                       for (n, f, t), p in zip(arrays, paths)],
            "integrations_per_step": n_int, "mode": args.mode,
            "l2": "no flush: each step reads %.1f GB of voltages (> 129 MB L2)" % gb,
            "parallelism": "replicas (channels shard with no exchange)"}


# ------------------------------------------------------------------ ours ---
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")


def load_peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


def measured_traffic(kernel_src: str, profile_md: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, but only while the
    kernel source still matches the one the counters were taken from."""
    import hashlib
    import re
    try:
        text = open(profile_md).read()
        sha = hashlib.sha256(open(kernel_src, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    m = re.search(r"sha256 prefix `([0-9a-f]{16})`", text)
    t = re.search(r"traffic_bytes_per_full_band_launch: ([0-9.e+]+)", text)
    if not m or not t or m.group(1) != sha or workload != "full_band":
        return None
    return float(t.group(1))


_PROBES: dict = {}


def measured_probes(dev) -> dict:
    """Peak rates of the instruction forms the kernels use, measured on this
    device by the library's probes (corr_probe_rate), in Tops/s, with the SM
    clock sampled while they ran.  Taken once per process."""
    if _PROBES:
        return _PROBES
    from paper_1501_05992_gb300 import corr
    clk = ClockSampler(dev.index or 0)
    clk.start()
    clk.mark_start()
    for kind in ("tc_fp8", "mma_s8", "dp4a", "ffma"):
        try:
            rate, ms = corr.probe_rate(kind)
            _PROBES[kind] = {"tops": rate / 1e12, "ms": ms}
        except corr.CorrError as e:
            _PROBES[kind] = {"tops": None, "error": str(e)}
    clk.mark_stop()
    c = clk.stop()
    _PROBES["clocks"] = c
    return _PROBES


def roofline_for(path, ops_per_launch, avg_ms, peaks, src, sm_count, probes=None):
    achieved = ops_per_launch / (avg_ms * 1e-3) / 1e12          # Tops/s
    probes = probes or {}
    if path == "tc_fp8":
        # fp8 dense = 2 x bf16 (the nominal ratio) x the measured bf16 burst
        # rate: the X-engine launch lasts about 2 ms, far shorter than the
        # seconds-long loop the sustained figure comes from
        peak = peaks["bf16_tflops"] * 2.0
        out = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
               "frac": achieved / peak,
               "peak_note": f"fp8 dense = 2 x bf16 burst ({src}); ops = 8 per useful CMAC"}
        pr = (probes.get("tc_fp8") or {}).get("tops")
        if pr:
            out["probe_peak"] = pr
            out["frac_of_probe"] = achieved / pr
            out["probe_note"] = ("tcgen05.mma kind::f8f6f4 M128 N256 K32 back to back from shared memory, "
                                 "one issuing thread per SM (corr_probe_rate), sampled SM clock %s MHz"
                                 % ((probes.get("clocks") or {}).get("sm_mhz")))
        return out
    if path == "mma_i8":
        # int8 tensor rates on this part are far below 2 x bf16; the peak is
        # the measured rate of back-to-back mma.sync m16n8k32 s8 in registers
        peak = (probes.get("mma_s8") or {}).get("tops")
        return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TOPS",
                "frac": achieved / peak if peak else None,
                "peak_note": "mma.sync m16n8k32 s8 on registers, measured in this run (corr_probe_rate); "
                             "ops = 8 per useful CMAC"}
    # dp4a: the measured rate of register-resident dp4a (8 ops each)
    peak = (probes.get("dp4a") or {}).get("tops")
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TOPS",
            "frac": achieved / peak if peak else None,
            "peak_note": "dp4a on registers, measured in this run (corr_probe_rate); 8 ops per dp4a"}


def _time_ms(fn, stream, reps=5):
    """Median CUDA-event time of fn() on `stream` after one warm-up call."""
    import torch
    with torch.cuda.stream(stream):
        fn()
    stream.synchronize()
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        with torch.cuda.stream(stream):
            fn()
        e1.record(stream)
        stream.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def measure_extras(arrays, volts, outs, stream_, dev, peaks, src, full=True):
    """The stages around the X-engine on the first array's first integration,
    against the HBM roofline: the incoherent beam (reads every voltage byte
    once, writes one int32 per channel and sample), the packet ingest of one
    50 ms bank (reads the packets, writes the voltage block) and the output
    remap with 2 x 2 averaging (reads two dumps' triangles, writes the
    station-order products of channel pairs).  Then the three X-engine forms
    on the same integration; with `full`, the uneven batch and the streaming
    service too.  Not part of the timed step."""
    import torch
    from paper_1501_05992_gb300 import corr
    n, f, t = arrays[0]
    hbm = peaks.get("hbm_gbs")
    res = {}
    volt = volts[0][:t]
    beam = torch.empty((t, f), dtype=torch.int32, device=dev)
    ms = _time_ms(lambda: corr.incoherent_beam(volt, 1, out=beam, stream=stream_), stream_)
    nbytes = n * f * t + 4 * f * t
    res["incoherent_beam"] = {"ms": ms, "bytes": nbytes, "gbs": nbytes / ms / 1e6,
                              "frac": (nbytes / ms / 1e6) / hbm if hbm else None,
                              "peak_gbs": hbm, "bound": "hbm"}
    if (n, f) == (256, 3072) and t >= 500:
        # packet ingest of one 50 ms bank: the bank's packets built on the host
        # by the synthetic packetiser from the first 500 samples, in the order a
        # receiver collects them (2000-packet blocks of the 32 lanes in turn,
        # Sections 3.3.3 and 3.4.1); the same packets lane after lane (each
        # lane's whole bank in turn) are timed too, the order with the least
        # write locality
        from synth import packets as pkts
        host = volts[0][:500].cpu().numpy()
        blk = torch.empty((500, f, n), dtype=torch.uint8, device=dev)
        seen = torch.empty(corr.PKT_SLOTS, dtype=torch.uint8, device=dev)
        cnt = torch.empty(corr.PKT_COUNTERS, dtype=torch.int32, device=dev)
        for key, order in (("packet_ingest", pkts.arrival_order), ("packet_ingest_lane_order", pkts.packetise)):
            stream = torch.from_numpy(order(host, 0)).to(dev)
            blk.zero_()
            torch.cuda.synchronize(dev)
            ms = _time_ms(lambda: corr.ingest_packets(stream, 0, blk, seen, cnt, stream=stream_), stream_)
            ok = bool(torch.equal(blk, volts[0][:500])) and cnt.tolist() == [stream.shape[0], 0, 0, 0, 0, 0]
            nbytes = stream.numel() + blk.numel()
            res[key] = {"ms": ms, "bytes": nbytes, "gbs": nbytes / ms / 1e6,
                        "frac": (nbytes / ms / 1e6) / hbm if hbm else None,
                        "peak_gbs": hbm, "bound": "hbm", "packets": int(stream.shape[0]),
                        "order": ("2000-packet blocks of the 32 lanes in turn" if order is pkts.arrival_order
                                  else "each lane's whole bank in turn"),
                        "round_trip_exact": ok}
            del stream
        del blk, seen
    if n % 64 == 0 and f % 2 == 0:
        tris = [outs[0][0], outs[1][0]]
        S = n // 2
        rm = torch.empty((f // 2, S * (S + 1) // 2, 2, 2, 2), dtype=torch.int32, device=dev)
        ms = _time_ms(lambda: corr.remap(tris, None, 2, out=rm, stream=stream_), stream_)
        nbytes = 2 * f * n * (n + 1) // 2 * 8 + rm.numel() * 4
        res["remap_2x2"] = {"ms": ms, "bytes": nbytes, "gbs": nbytes / ms / 1e6,
                            "frac": (nbytes / ms / 1e6) / hbm if hbm else None,
                            "peak_gbs": hbm, "bound": "hbm"}
    if n % 8 == 0 and f % 128 == 0:
        res["fine_pfb"] = measure_fine_pfb(n, f // 128, t, stream_, dev)
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    res["paths_one_integration"] = measure_paths(n, f, t, volt, stream_, dev, peaks, sm_count)
    res["beam_fused"] = measure_beam_fused(n, f, t, volt, stream_, dev)
    torch.cuda.empty_cache()
    if full:
        res["uneven_batch"] = measure_uneven_batch(stream_, dev, peaks, sm_count)
        torch.cuda.empty_cache()
        res["service"] = measure_service(dev)
        torch.cuda.empty_cache()
    return res


def _oracle_channels(volt_dev, chans):
    """Oracle triangles (int32) of whole channels of a device voltage block."""
    import oracle
    sub = volt_dev[:, chans].cpu().numpy()
    return oracle.to_int32(oracle.xmac(sub))


def measure_paths(n, f, t, volt, stream_, dev, peaks, sm_count):
    """The same integration through the three X-engine forms, each as a
    whole-integration call: the dp4a CUDA-core kernel, the int8 mma.sync
    kernel and the tcgen05 FP8 kernel.  Time per integration, CMAC/s, the
    fraction of each form's own roofline, whether the three triangles are
    identical, and whether they equal the oracle on four whole channels."""
    import torch
    from paper_1501_05992_gb300 import corr
    out = {}
    tri = {}
    cmac = n * (n + 1) // 2 * f * t
    for path in ("cudacore", "mma_i8", "tc_fp8"):
        try:
            c = corr.Correlator(n, f, t, path=path, device=dev)
        except corr.CorrError:
            out[path] = None
            continue
        dst = torch.empty((f, n * (n + 1) // 2, 2), dtype=torch.int32, device=dev)
        ms = _time_ms(lambda: c.integrate(volt, dst, stream=stream_), stream_, reps=3)
        c.sync(stream_)
        c.close()
        tri[path] = dst
        roof = roofline_for(path, 8.0 * cmac, ms, peaks, "measured", sm_count, measured_probes(dev))
        out[path] = {"ms_per_integration": ms, "value": cmac / (ms * 1e-3), "unit": "CMAC/s",
                     "x_real_time": t / SAMPLE_RATE_HZ / (ms * 1e-3),
                     "achieved": roof["achieved"], "peak": roof["peak"], "frac": roof["frac"],
                     "peak_unit": roof["unit"], "peak_note": roof["peak_note"]}
    have = [p for p in ("cudacore", "mma_i8", "tc_fp8") if out.get(p)]
    if out.get("cudacore") and out.get("tc_fp8"):
        out["tc_speedup"] = out["cudacore"]["ms_per_integration"] / out["tc_fp8"]["ms_per_integration"]
    if out.get("mma_i8") and out.get("tc_fp8"):
        out["fp8_vs_int8_speedup"] = out["mma_i8"]["ms_per_integration"] / out["tc_fp8"]["ms_per_integration"]
    out["identical"] = all(bool(torch.equal(tri[have[0]], tri[p])) for p in have[1:])
    chans = sorted({0, 1, f // 2, f - 1})
    want = _oracle_channels(volt, chans)
    out["exact"] = bool(out["identical"]) and all(
        bool((tri[p][chans].cpu().numpy() == want).all()) for p in have)
    out["exact_note"] = (f"the {len(have)} triangles are compared element by element over all "
                         f"{f} channels, and against the oracle on whole channels {chans}")
    del tri
    return out


def measure_beam_fused(n, f, t, volt, stream_, dev):
    """One integration with its incoherent beam: the X-engine alone, the
    X-engine forming the beam from its own unpack (corr_integrate_beam), and
    the X-engine followed by the stand-alone beam pass; the fused beam must
    equal the stand-alone one and the oracle's on sampled channels."""
    import torch
    import oracle
    from paper_1501_05992_gb300 import corr
    c = corr.Correlator(n, f, t, device=dev)
    tri = torch.empty((f, n * (n + 1) // 2, 2), dtype=torch.int32, device=dev)
    fused = torch.empty((t, f), dtype=torch.int32, device=dev)
    alone = torch.empty((t, f), dtype=torch.int32, device=dev)
    ms_x = _time_ms(lambda: c.integrate(volt, tri, stream=stream_), stream_, reps=5)
    ms_f = _time_ms(lambda: c.integrate_beam(volt, 1, tri, fused, stream=stream_), stream_, reps=5)
    ms_s = _time_ms(lambda: (c.integrate(volt, tri, stream=stream_),
                             corr.incoherent_beam(volt, 1, out=alone, stream=stream_)), stream_, reps=5)
    c.sync(stream_)
    c.close()
    chans = [0, f // 2, f - 1]
    want = oracle.beam(volt[:, chans].cpu().numpy())
    exact = bool(torch.equal(fused, alone)) and bool((fused[:, chans].cpu().numpy() == want).all())
    return {"xengine_ms": ms_x, "fused_ms": ms_f, "separate_ms": ms_s, "fused_added_ms": ms_f - ms_x,
            "separate_added_ms": ms_s - ms_x, "exact": exact,
            "exact_note": f"fused beam equal to the stand-alone kernel's on all {f} channels and to the "
                          f"oracle's on channels {chans}"}


def measure_uneven_batch(stream_, dev, peaks, sm_count):
    """The uneven batch (three arrays of 128, 256 and 1024 inputs) correlated
    in one persistent launch, each array's path chosen by the autotuner:
    whole-batch and per-array throughput, and whole triangles of two channels
    of every array against the oracle (the 1024-input array at its full
    10000 samples)."""
    import tempfile

    import torch
    from paper_1501_05992_gb300 import autotune, corr
    from synth import voltgen as vg
    from synth.gpu import DeviceGenerator
    arrays, _, seed = WORKLOADS["uneven_batch"]
    volts = [DeviceGenerator(vg.gauss3_params(seed, n, f, array=a), dev).make(0, t)
             for a, (n, f, t) in enumerate(arrays)]
    cache = os.path.join(tempfile.gettempdir(), "corr_autotune_bench.json")
    specs = autotune.plan([{"n_inputs": n, "n_chan": f, "n_time_per_int": t} for n, f, t in arrays],
                          cache_path=cache)
    tuned = [autotune.tune(n, f, t, cache_path=cache) for n, f, t in arrays]
    batch = corr.Batch(specs, device=dev)
    outs = batch._outs(None)
    ms_all = _time_ms(lambda: batch.integrate(volts, outs, stream=stream_), stream_, reps=5)
    batch.sync(stream_)
    res = {"arrays": [], "paths": batch.paths, "autotune_cache": cache}
    cmac_all = 0
    for a, ((n, f, t), spec) in enumerate(zip(arrays, specs)):
        cmac = n * (n + 1) // 2 * f * t
        cmac_all += cmac
        one = corr.Batch([spec], device=dev)
        o1 = one._outs(None)
        ms = _time_ms(lambda: one.integrate([volts[a]], o1, stream=stream_), stream_, reps=3)
        one.sync(stream_)
        same = bool(torch.equal(o1[0], outs[a]))
        one.close()
        del o1
        chans = [0, f - 1]
        exact = bool((outs[a][chans].cpu().numpy() == _oracle_channels(volts[a], chans)).all())
        roof = roofline_for(spec["path"], 8.0 * cmac, ms, peaks, "measured", sm_count, measured_probes(dev))
        res["arrays"].append({
            "n_inputs": n, "n_chan": f, "samples": t, "path": spec["path"], "tile": spec["tile"],
            "autotune_ms": tuned[a]["ms"], "ms_alone": ms, "value_alone": cmac / (ms * 1e-3),
            "frac_alone": roof["frac"], "same_as_in_batch": same, "exact": exact,
            "exact_channels": chans})
    roof = roofline_for("tc_fp8" if all(p == "tc_fp8" for p in batch.paths) else batch.paths[0],
                        8.0 * cmac_all, ms_all, peaks, "measured", sm_count, measured_probes(dev))
    res.update({"ms_batch": ms_all, "value": cmac_all / (ms_all * 1e-3), "unit": "CMAC/s",
                "achieved": roof["achieved"], "peak": roof["peak"], "frac": roof["frac"],
                "exact": all(x["exact"] and x["same_as_in_batch"] for x in res["arrays"]),
                "launch": "one corr_batch_integrate: the tensor-core arrays share one persistent launch"})
    batch.close()
    del volts, outs
    return res


def measure_service(dev, seconds: float = 10.0):
    """The streaming service of three arrays (256, 128 and 512 inputs x 3072
    channels, 50 ms blocks of 500 samples, 0.5 s dumps): one run paced to
    real time for `seconds` and one run of the same data delivered as fast as
    the service accepts it.  Every dump is checked against the oracle on
    sampled channels, its blocks regenerated from the seeded generator."""
    import numpy as np
    import oracle
    from paper_1501_05992_gb300.service import GpuBackend, Service, StreamSpec
    from synth import voltgen as vg
    specs = [StreamSpec("mwa256", 256, 3072, array=0), StreamSpec("aux128", 128, 3072, array=1),
             StreamSpec("aux512", 512, 3072, array=2)]
    n_blocks = int(round(seconds / specs[0].period_s))
    expected = {}

    def want(spec, pool_blocks, f, seqs):
        key = (spec.name, f, tuple(q % pool_blocks for q in seqs))
        if key not in expected:
            params = vg.gauss3_params(spec.seed, spec.n_inputs, spec.n_chan, array=spec.array)
            block = np.concatenate([vg.gauss3(params, (q % pool_blocks) * spec.block_samples,
                                              spec.block_samples, f, 1) for q in seqs])
            expected[key] = oracle.to_int32(oracle.xmac(block))[0]
        return expected[key]

    out = {}
    for label, paced in (("paced", True), ("unpaced", False)):
        import torch
        free, _ = torch.cuda.mem_get_info(dev)
        be = GpuBackend(device=dev.index or 0, pool_blocks=2, verify_channels=2)
        svc = Service(specs, int(free * 0.9), be, paced=paced, mode="block")
        rep = svc.run(n_blocks)
        checked = bad = 0
        for a, d, rows in be.kept:
            spec = specs[a]
            seqs = list(range(d * spec.blocks_per_dump, (d + 1) * spec.blocks_per_dump))
            for f, got in rows.items():
                checked += 1
                bad += int(not np.array_equal(got.numpy(), want(spec, be.pool_blocks, f, seqs)))
        rep["dumps_checked"] = checked
        rep["dumps_checked_channels"] = {s.name: be.kept_channels[a] for a, s in enumerate(specs)}
        rep["exact"] = checked > 0 and bad == 0
        out[label] = rep
        del svc, be
    out["exact"] = all(out[k]["exact"] for k in ("paced", "unpaced"))
    out["gaps"] = sum(a["gaps"] for k in ("paced", "unpaced") for a in out[k]["arrays"])
    return out


FP32_LANES_PER_SM = 128          # fp32 FMA lanes per SM (4 sub-partitions x 32)


def measure_fine_pfb(n, n_coarse, frames, stream_, dev):
    """The F stage's fine filterbank (12 taps, 128 points) producing one
    integration's voltages for every coarse channel: n_coarse x n inputs x
    `frames` output samples from seeded int8 coarse-channel noise, the codes
    written in the X-engine's input layout.  The kernel is bound by fp32
    arithmetic: 12 x 128 complex-by-real multiply-adds (4 flops each) and a
    128-point FFT (5 N log2 N = 4480 flops) per frame and input, against the
    fp32 peak of 128 FMA lanes x 2 flops per SM and clock at the maximum SM
    clock (2070 MHz)."""
    import numpy as np
    import torch
    from paper_1501_05992_gb300 import corr
    from synth import coarse
    taps = 12
    S = 128 * (frames + taps - 1)
    g = torch.Generator(device=dev)
    g.manual_seed(1505)
    x = torch.empty((n_coarse, n, S, 2), dtype=torch.int8, device=dev)
    for q in range(n_coarse):       # N(0, 8^2) per component, rounded and clipped
        x[q] = torch.randn((n, S, 2), device=dev, generator=g).mul_(8.0).round_().clamp_(-127, 127).to(torch.int8)
    h_np = coarse.kaiser_sinc_window(taps)
    h = torch.from_numpy(h_np.astype(np.float32)).to(dev)
    scale = coarse.output_scale(h_np, 8.0)
    volt = torch.empty((frames, n_coarse * 128, n), dtype=torch.uint8, device=dev)
    torch.cuda.synchronize(dev)
    ms = _time_ms(lambda: corr.fine_pfb(x, h, scale, volt=volt, stream=stream_), stream_)
    units = n_coarse * n * frames
    flops = units * (taps * 128 * 4 + 5 * 128 * 7)
    sm = torch.cuda.get_device_properties(dev).multi_processor_count
    derived = sm * FP32_LANES_PER_SM * 2 * 2.070e9 / 1e12
    probe = (measured_probes(dev).get("ffma") or {}).get("tops")
    peak = probe or derived
    tflops = flops / ms / 1e9
    out = {"ms": ms, "frames": frames, "coarse_channels": n_coarse, "inputs": n,
           "x_real_time": frames / SAMPLE_RATE_HZ / (ms * 1e-3), "tflops": tflops, "peak_tflops": peak,
           "frac": tflops / peak, "bound": "alu",
           "peak_note": ("fp32 FMA on registers measured in this run (corr_probe_rate)" if probe else
                         f"{sm} SMs x {FP32_LANES_PER_SM} fp32 lanes x 2 flops x 2.07 GHz"),
           "derived_peak_tflops": derived, "frac_of_derived": tflops / derived,
           "bytes": x.numel() + volt.numel()}
    del x, volt
    return out


def run_ours(args, world, rank, local):
    import torch
    from paper_1501_05992_gb300 import autotune, corr
    from synth import voltgen as vg
    from synth.gpu import DeviceGenerator

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    arrays, n_int, seed = WORKLOADS[args.workload]
    # every rank correlates its own arrays (weak scaling, no exchange)
    volts = []
    for a, (n, f, t) in enumerate(arrays):
        gen = DeviceGenerator(vg.gauss3_params(seed, n, f, array=rank_array_index(a, rank)), dev)
        v = torch.empty((t * n_int, f, n), dtype=torch.uint8, device=dev)
        for k in range(n_int):
            gen.fill(v[k * t:(k + 1) * t], t0=k * t)
        volts.append(v)
    specs = [{"n_inputs": n, "n_chan": f, "n_time_per_int": t, "path": args.path}
             for n, f, t in arrays]
    tuned = None
    if args.autotune:
        cache = os.environ.get("CORR_AUTOTUNE_CACHE") or None
        specs = autotune.plan(specs, cache_path=cache)
        tuned = [{k: s[k] for k in ("path", "tile")} for s in specs]
    batch = corr.Batch(specs, device=dev)
    paths = batch.paths
    stream = torch.cuda.Stream(dev)
    outs = [batch._outs(None) for _ in range(2)]
    step_cmac = sum(n * (n + 1) // 2 * f * t for n, f, t in arrays) * n_int
    rt_rate = sum(n * (n + 1) // 2 * f for n, f, t in arrays) * SAMPLE_RATE_HZ

    def integration(k):
        return [v[k * t:(k + 1) * t] for v, (n, f, t) in zip(volts, arrays)]

    # kernel timing: the library profiler brackets every X-engine and dump
    # launch with CUDA events on the launch stream (direct mode: accumulate +
    # dump per integration); in graph mode each integration is one captured
    # corr_batch_integrate (the X-engine epilogue writes the triangle straight
    # into the output, no dump pass), and the bench brackets every graph launch
    # with its own events on the same stream
    graphs = []
    if args.mode == "graph":
        for k in range(n_int):
            g, _ = batch.capture(integration(k), outs[k & 1], stream=stream)
            graphs.append(g)
        # one event pair per graph launch of every timed step
        gev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                for _ in range(n_int)] for _ in range(args.steps)]
        timed_step = [0]

        def step(timed=False):
            evs = gev[timed_step[0]] if timed else None
            for k, g in enumerate(graphs):
                if timed:
                    evs[k][0].record(stream)
                g.launch(stream)
                if timed:
                    evs[k][1].record(stream)
            if timed:
                timed_step[0] += 1
    else:
        def step(timed=False):
            for k in range(n_int):
                batch.accumulate(integration(k), stream=stream)
                batch.dump(outs[k & 1], stream=stream)

    clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if clocks:
        clocks.start()           # before the warm-up: nvidia-smi is slow to produce its first reading
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    stream.synchronize()
    batch.profile_read(reset=True)
    if args.mode == "direct":
        batch.profile_enable(True)
    barrier(world)
    torch.cuda.synchronize(dev)
    if clocks:
        clocks.mark_start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for st in range(args.steps):
        step(timed=(args.mode == "graph"))
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    if clocks:
        clocks.mark_stop()
    barrier(world)
    clk = clocks.stop() if clocks else None
    batch.sync(stream)
    elapsed_ms = max_over_ranks(ev0.elapsed_time(ev1), world)
    value = job_units(step_cmac, args.steps, world) / (elapsed_ms * 1e-3)

    if args.mode == "direct":
        prof = batch.profile_read(reset=True)
        batch.profile_enable(False)
        launches_per_step = sum(p[k]["launches"] for p in prof for k in p) // max(1, args.steps)
        xe_ms = sum(p["xengine"]["ms"] for p in prof)
        xe_timed = sum(p["xengine"]["timed"] for p in prof)
        kernel_ms = {k: sum(p[k]["ms"] for p in prof) / args.steps for k in prof[0]}
        timing_note = "library CUDA events around every X-engine launch in the timed region"
    else:
        # launch counts and the X-engine's share of a graph (other kernels, such
        # as the CUDA-core path's unpack, run inside it too) from one profiled
        # direct integration after the timed region
        batch.profile_enable(True)
        with torch.cuda.stream(stream):
            batch.integrate(integration(0), outs[0], stream=stream)
        stream.synchronize()
        prof = batch.profile_read(reset=True)
        batch.profile_enable(False)
        per_int_launches = sum(p[k]["launches"] for p in prof for k in p)
        launches_per_step = per_int_launches * n_int
        all_ms = sum(p[k]["ms"] for p in prof for k in p)
        xe_share = sum(p["xengine"]["ms"] for p in prof) / all_ms if all_ms > 0 else 1.0
        g_ms = [a.elapsed_time(b) for evs in gev for a, b in evs]
        xe_ms = sum(g_ms) * xe_share
        xe_timed = len(g_ms) * max(1, sum(p["xengine"]["launches"] for p in prof))
        kernel_ms = {"graph_per_integration": sum(g_ms) / len(g_ms),
                     "graph_per_integration_min": min(g_ms), "graph_per_integration_max": max(g_ms),
                     "xengine_per_integration": xe_ms / len(g_ms), "xengine_share": xe_share,
                     "xengine_ms_per_step": xe_ms / args.steps}
        timing_note = ("CUDA events around every graph launch (one integration each) of every "
                       "timed step, times the X-engine's share of a profiled direct integration")
    xe_per_step = xe_timed // max(1, args.steps)
    peaks, src = load_peaks()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    ops_per_launch = 8.0 * step_cmac / max(1, xe_per_step)
    avg_ms = xe_ms / max(1, xe_timed)
    main_path = paths[max(range(len(arrays)), key=lambda a: arrays[a][0] ** 2 * arrays[a][1] * arrays[a][2])]
    roof = roofline_for(main_path, ops_per_launch, avg_ms, peaks, src, sm_count, measured_probes(dev))
    roof["traffic"] = (measured_traffic(os.path.join(ROOT, "paper_1501_05992_gb300", "csrc", "xeng_tc.cu"),
                                        os.path.join(ROOT, "profiles", "xeng_tc_full_band_traffic.md"),
                                        args.workload) if main_path == "tc_fp8" else None)
    roof["kernel"] = {"cudacore": "xeng_dp4a_kernel", "mma_i8": "xeng_mma8_kernel",
                      "tc_fp8": "xeng_tc_kernel"}[main_path]
    roof["launches_per_step"] = xe_per_step
    roof["avg_launch_ms"] = avg_ms
    roof["timing"] = timing_note

    # ---- end to end through the host-buffer C-ABI calls -------------------
    e2e = None
    if args.e2e_steps > 0:
        ctxs = [corr.Correlator(n, f, t, path=p, device=dev) for (n, f, t), p in zip(arrays, paths)]
        h_volts = [v[:t].cpu().pin_memory() for v, (n, f, t) in zip(volts, arrays)]
        h_outs = [[torch.empty((f, n * (n + 1) // 2, 2), dtype=torch.int32).pin_memory()
                   for _ in range(2)] for n, f, t in arrays]

        def step_host():
            for k in range(n_int):
                for a, c in enumerate(ctxs):
                    c.accumulate_host(h_volts[a], stream=stream)
                    c.dump_host(h_outs[a][k & 1], stream=stream)

        # as many untimed steps as the device-resident loop's warm-up: the first
        # passes over a freshly pinned buffer run slower and less evenly
        for _ in range(max(1, args.warmup)):
            step_host()
        stream.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.e2e_steps):
            step_host()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        wall = time.perf_counter() - t0
        for c in ctxs:
            c.sync(stream)
            c.close()
        e_ms = max_over_ranks(max(e0.elapsed_time(e1), wall * 1e3), world)
        e2e = {"value": step_cmac * args.e2e_steps * world / (e_ms * 1e-3), "unit": UNIT,
               "h2d_bytes_per_step": n_int * sum(n * f * t for n, f, t in arrays),
               "d2h_bytes_per_step": n_int * sum(f * n * (n + 1) // 2 * 8 for n, f, t in arrays),
               "note": "corr_accumulate_host / corr_dump_host from pinned memory; one pinned "
                       "integration per array, re-sent for each integration of the step"}
        del h_volts, h_outs

    extras = None
    if not args.no_extras and rank == 0:
        extras = measure_extras(arrays, volts, outs, stream, dev, peaks, src,
                                full=args.workload == "full_band")

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        n, f, t = arrays[0]
        slab = volts[0][:t, :min(f, 256)].cpu().numpy()
        rate, cores, desc = oracle_sample(slab, args.cpu_seconds)
        one_rate, one_desc = oracle_single_core(slab)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc,
               "single_core": {"value": one_rate, "unit": UNIT, "sample": one_desc}}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"cudacore": "int8", "mma_i8": "int8", "tc_fp8": "e4m3"}[main_path],
            "data": "synthetic", "x_real_time": value / (rt_rate * world),
            "config": workload_config(args, paths),
            "gpu_launches": launches_per_step * args.steps, "clocks": clk, "roofline": roof,
            "cpu_baseline": cpu, "e2e": e2e, "kernel_ms": kernel_ms,
        }
        if extras:
            line["extras"] = extras
        if tuned:
            line["autotune"] = tuned
        print(json.dumps(line), flush=True)
    for g in graphs:
        g.close()
    batch.close()


def main():
    args = parse_args()
    world, rank, local = dist_setup(args)
    try:
        if args.impl == "reference":
            run_reference(args, world, rank)
        else:
            run_ours(args, world, rank, local)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
