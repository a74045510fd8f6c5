"""Streaming X-engine service: voltage blocks of several arrays arriving in
real time, correlated on one GPU with device-resident accumulators.

This is the GB300 counterpart of the XMAC host's input management (Section
3.4.1): there, receiver threads fill a one-second buffer, a management thread
releases it to the GPU and frees the threads for the next buffer, and products
are integrated on the GPU for an operator-chosen time before being copied out
(Section 3.4.3).  Here:

* one arrival thread per array delivers 50 ms blocks (500 samples of every
  channel and input) from pinned host memory, paced to real time or, for
  capacity measurement, as fast as the GPU accepts them;
* arrays are admitted by an HBM budget: each needs its library workspace, a
  ring of device block slots and two dump buffers, and arrays that do not fit
  are rejected with ``CORR_E_BUDGET``;
* a dispatcher gathers the blocks that have arrived (at most one per array per
  tick), copies them into the arrays' device rings on a copy stream and
  correlates them with one batched call (tensor-core arrays share one
  persistent launch); every ``blocks_per_dump`` blocks an array's integration
  is dumped and copied to pinned host memory;
* sequence numbers are checked: a missing block is counted and the
  integration it belonged to is flagged (no unsynchronised data are merged
  silently, the rule the paper's capture system applies at its input, Section
  3.3.1); an arrival thread that delivers nothing for ``stall_s`` is reported
  as stalled; an arrival thread that raises is reported and its array stops;
* block latency is measured from a block's arrival to the completion of the
  GPU work that correlated it; the report gives p50/p99 latency and the
  x-real-time margin (tick period / GPU time per tick).

Two ways to correlate (``mode``):

* ``"block"`` (default): every block is added to the array's running
  integration as it arrives, so its latency is one block's copy and
  correlation;
* ``"dump"``: the blocks of an integration wait in a device ring of
  ``blocks_per_dump`` slots and are correlated together, as one whole
  integration written straight into the dump buffer, when the last one has
  arrived -- the paper's own arrangement (one GPU launch per input block of a
  second, Section 3.4.1).  A block then waits up to one integration, but the
  GPU does a single fresh pass per integration instead of adding every block
  into the accumulators.

The GPU side lives behind a small backend interface so that the control logic
can be exercised without a GPU (tests/test_service.py uses a fake backend).
"""
from __future__ import annotations

import json
import queue
import statistics
import threading
import time
from dataclasses import dataclass, field

SAMPLE_RATE_HZ = 1.0e4


@dataclass
class StreamSpec:
    """One array of the service."""
    name: str
    n_inputs: int
    n_chan: int
    block_samples: int = 500            # 50 ms at 10 kHz
    blocks_per_dump: int = 10           # 0.5 s integrations
    seed: int = 1505
    array: int = 0

    @property
    def block_bytes(self) -> int:
        return self.block_samples * self.n_chan * self.n_inputs

    @property
    def vis_bytes(self) -> int:
        return self.n_chan * self.n_inputs * (self.n_inputs + 1) // 2 * 8

    @property
    def period_s(self) -> float:
        return self.block_samples / SAMPLE_RATE_HZ

    @property
    def n_time_per_int(self) -> int:
        return self.block_samples * self.blocks_per_dump


def footprint(spec: StreamSpec, ring_blocks: int, workspace_bytes) -> int:
    """Device bytes an admitted array holds: workspace + block ring + 2 dumps."""
    return (workspace_bytes(spec.n_inputs, spec.n_chan, spec.n_time_per_int)
            + ring_blocks * spec.block_bytes + 2 * spec.vis_bytes)


def admit(specs, hbm_budget: int, ring_blocks: int, workspace_bytes):
    """Admit arrays in order while their summed footprint fits the budget."""
    admitted, rejected, used = [], [], 0
    for s in specs:
        need = footprint(s, ring_blocks, workspace_bytes)
        if used + need <= hbm_budget:
            admitted.append(s)
            used += need
        else:
            rejected.append((s, f"CORR_E_BUDGET: needs {need} bytes, {hbm_budget - used} left"))
    return admitted, rejected, used


@dataclass
class Block:
    array: int
    seq: int
    arrival: float
    data: object            # backend-specific host buffer


@dataclass
class ArrayStats:
    blocks: int = 0
    dumps: int = 0
    gaps: int = 0
    lost_blocks: int = 0
    tainted_dumps: int = 0
    stalls: int = 0
    failed: str | None = None
    latencies_ms: list = field(default_factory=list)


class Source(threading.Thread):
    """Arrival thread of one array: block k becomes available at t0 + k * period
    (paced) or as soon as the dispatcher has room for it (unpaced)."""

    def __init__(self, index, spec, n_blocks, make_block, out: queue.Queue, paced: bool,
                 t0: float, room: threading.Semaphore, faults=None):
        super().__init__(daemon=True)
        self.index, self.spec, self.n_blocks = index, spec, n_blocks
        self.make_block, self.out, self.paced, self.t0 = make_block, out, paced, t0
        self.room = room
        self.faults = faults or {}
        self.error = None
        self.done = threading.Event()

    def run(self):
        try:
            for k in range(self.n_blocks):
                if k in self.faults.get("skip", ()):
                    continue                              # block lost upstream
                if k in self.faults.get("stall", {}):
                    time.sleep(self.faults["stall"][k])
                if k in self.faults.get("raise", ()):
                    raise RuntimeError(f"source {self.spec.name} failed at block {k}")
                if self.paced:
                    # block k exists at its real-time instant, whether or not
                    # the service has room for it yet
                    arrival = self.t0 + k * self.spec.period_s
                    delay = arrival - time.perf_counter()
                    if delay > 0:
                        time.sleep(delay)
                    self.room.acquire()
                else:
                    self.room.acquire()
                    arrival = time.perf_counter()
                self.out.put(Block(self.index, k, arrival, self.make_block(k)))
        except Exception as e:  # reported, never raised into the service
            self.error = repr(e)
        finally:
            self.done.set()


class Service:
    def __init__(self, specs, hbm_budget: int, backend, ring_blocks: int = 3,
                 paced: bool = True, stall_s: float = 1.0, max_queue: int = 8, mode: str = "block"):
        if mode not in ("block", "dump"):
            raise ValueError("mode is 'block' or 'dump'")
        self.mode = mode
        if mode == "dump":
            # a ring slot per block of an integration
            ring_blocks = max([ring_blocks] + [s.blocks_per_dump for s in specs])
        backend.per_dump = mode == "dump"
        self.backend = backend
        self.ring_blocks = ring_blocks
        self.paced = paced
        self.stall_s = stall_s
        self.max_queue = max_queue
        self.admitted, self.rejected, self.hbm_used = admit(
            specs, hbm_budget, ring_blocks, backend.workspace_bytes)
        self.stats = [ArrayStats() for _ in self.admitted]
        self.dumps = []                  # (array, dump index, seqs, tainted, backend handle)
        self.tick_gpu_ms = []

    def run(self, n_blocks: int, faults=None) -> dict:
        faults = faults or {}
        specs = self.admitted
        if not specs:
            return self.report(0.0)
        self.backend.open(specs, self.ring_blocks)
        qs = [queue.Queue() for _ in specs]
        rooms = [threading.Semaphore(self.max_queue) for _ in specs]
        t0 = time.perf_counter() + 0.05
        sources = [Source(a, s, n_blocks, (lambda k, a=a: self.backend.host_block(a, k)), qs[a],
                          self.paced, t0, rooms[a], faults.get(s.name)) for a, s in enumerate(specs)]
        for src in sources:
            src.start()
        expected = [0] * len(specs)
        in_dump = [[] for _ in specs]
        in_dump_arrivals = [[] for _ in specs]
        per_dump = self.mode == "dump"
        tainted = [False] * len(specs)
        last_arrival = [t0] * len(specs)
        stalled = [False] * len(specs)
        completer_q: queue.Queue = queue.Queue()

        def completer():
            while True:
                item = completer_q.get()
                if item is None:
                    return
                handle, arrivals = item
                gpu_ms = self.backend.wait(handle)
                done = time.perf_counter()
                if gpu_ms is not None:
                    self.tick_gpu_ms.append(gpu_ms)
                for a, arr in arrivals:
                    self.stats[a].latencies_ms.append((done - arr) * 1e3)

        cthread = threading.Thread(target=completer, daemon=True)
        cthread.start()
        while True:
            got = {}
            for a, q in enumerate(qs):
                try:
                    got[a] = q.get_nowait()
                except queue.Empty:
                    pass
            now = time.perf_counter()
            if not got:
                if all(s.done.is_set() for s in sources) and all(q.empty() for q in qs):
                    break
                for a, s in enumerate(sources):
                    if (not s.done.is_set() and not stalled[a] and now > t0
                            and now - last_arrival[a] > self.stall_s):
                        stalled[a] = True
                        self.stats[a].stalls += 1
                time.sleep(0.0005)
                continue
            for a, blk in got.items():
                last_arrival[a] = blk.arrival
                stalled[a] = False
                if blk.seq != expected[a]:
                    # blocks lost upstream: the integration they belong to is tainted
                    self.stats[a].gaps += 1
                    self.stats[a].lost_blocks += blk.seq - expected[a]
                    tainted[a] = True
                expected[a] = blk.seq + 1
                rooms[a].release()
            handle = self.backend.submit({a: blk for a, blk in got.items()})
            if not per_dump:
                completer_q.put((handle, [(a, blk.arrival) for a, blk in got.items()]))
            due = []
            for a, blk in got.items():
                self.stats[a].blocks += 1
                in_dump[a].append(blk.seq)
                in_dump_arrivals[a].append(blk.arrival)
                if len(in_dump[a]) == specs[a].blocks_per_dump:
                    due.append(a)
            if due:
                h = self.backend.dump(due)
                if per_dump:
                    # the blocks of these integrations are correlated by this dump
                    completer_q.put((h, [(a, arr) for a in due for arr in in_dump_arrivals[a]]))
                for a in due:
                    in_dump_arrivals[a] = []
                for a in due:
                    self.dumps.append((a, self.stats[a].dumps, list(in_dump[a]), tainted[a], h))
                    self.stats[a].dumps += 1
                    if tainted[a]:
                        self.stats[a].tainted_dumps += 1
                    in_dump[a] = []
                    tainted[a] = False
        completer_q.put(None)
        cthread.join()                   # every tick's GPU work has completed
        wall = time.perf_counter() - t0
        for a, s in enumerate(sources):
            s.join(timeout=5)
            if s.error:
                self.stats[a].failed = s.error
        self.backend.finish()
        return self.report(wall)

    def report(self, wall_s: float) -> dict:
        arrays = []
        all_lat = []
        for spec, st in zip(self.admitted, self.stats):
            lat = sorted(st.latencies_ms)
            all_lat += lat
            arrays.append({
                "name": spec.name, "n_inputs": spec.n_inputs, "n_chan": spec.n_chan,
                "blocks": st.blocks, "dumps": st.dumps, "gaps": st.gaps,
                "lost_blocks": st.lost_blocks, "tainted_dumps": st.tainted_dumps,
                "stalls": st.stalls, "failed": st.failed,
                "p50_ms": _pct(lat, 50), "p99_ms": _pct(lat, 99)})
        all_lat.sort()
        # the GPU work is timed per tick (block mode) or per integration (dump mode)
        period = min(((s.period_s * (s.blocks_per_dump if self.mode == "dump" else 1))
                      for s in self.admitted), default=0.0)
        gpu = statistics.median(self.tick_gpu_ms) if self.tick_gpu_ms else None
        data_s = max((st.blocks * s.period_s for s, st in zip(self.admitted, self.stats)), default=0.0)
        return {
            "arrays": arrays,
            "rejected": [{"name": s.name, "reason": r} for s, r in self.rejected],
            "hbm_budget_used": self.hbm_used,
            "p50_ms": _pct(all_lat, 50), "p99_ms": _pct(all_lat, 99),
            "gpu_ms_per_tick_median": gpu,
            "x_real_time_margin": (period * 1e3 / gpu) if gpu else None,
            "margin_note": ("tick period / median GPU correlation time per tick" if self.mode == "block" else
                            "integration period / median GPU correlation time per integration") +
                           " (copies excluded); x_real_time_wall = data seconds / wall seconds (copies included)",
            "mode": self.mode,
            "x_real_time_wall": (data_s / wall_s) if wall_s > 0 else None,
            "wall_s": wall_s, "paced": self.paced,
        }


def _pct(sorted_vals, p):
    if not sorted_vals:
        return None
    k = min(len(sorted_vals) - 1, max(0, int(round(p / 100.0 * (len(sorted_vals) - 1)))))
    return sorted_vals[k]


class GpuBackend:
    """The GPU side: device rings, one batched correlator, dump buffers."""

    per_dump = False      # set by Service: correlate whole integrations at dump time

    def __init__(self, device=None, pool_blocks: int = 2, path: str = "auto",
                 verify_channels: int = 2):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.pool_blocks = pool_blocks
        self.path = path
        self.verify_channels = verify_channels

    @staticmethod
    def workspace_bytes(n_inputs, n_chan, n_time_per_int):
        from . import corr
        return corr.workspace_bytes(n_inputs, n_chan, n_time_per_int)

    def open(self, specs, ring_blocks):
        torch = self.torch
        from . import corr
        from synth import voltgen as vg
        from synth.gpu import DeviceGenerator
        self.specs = specs
        self.ring_blocks = ring_blocks
        self.batch = corr.Batch([{"n_inputs": s.n_inputs, "n_chan": s.n_chan,
                                  "n_time_per_int": s.n_time_per_int, "path": self.path}
                                 for s in specs], device=self.device)
        self.rings = [torch.empty((ring_blocks, s.block_samples, s.n_chan, s.n_inputs),
                                  dtype=torch.uint8, device=self.device) for s in specs]
        self.slot_free = [[None] * ring_blocks for _ in specs]
        self.vis = [[torch.empty((s.n_chan, s.n_inputs * (s.n_inputs + 1) // 2, 2), dtype=torch.int32,
                                 device=self.device) for _ in range(2)] for s in specs]
        self.dump_count = [0] * len(specs)
        # the full dump goes to a two-slot pinned ring per array (the service's
        # output); a few channel rows are kept for verification
        self.host_ring = [[torch.empty(v.shape, dtype=torch.int32, pin_memory=True) for v in vis]
                          for vis in self.vis]
        self.d2h_done = [[None, None] for _ in specs]
        self.kept_channels = [sorted({0, s.n_chan // 2, s.n_chan - 1})[:max(1, self.verify_channels)]
                              for s in specs]
        self.kept = []                  # (array, dump index, {channel: int32 [P][2]})
        # host block pool: distinct blocks generated once, cycled by sequence number
        self.params = [vg.gauss3_params(s.seed, s.n_inputs, s.n_chan, array=s.array) for s in specs]
        self.pool = []
        for s, p in zip(specs, self.params):
            gen = DeviceGenerator(p, self.device)
            blocks = []
            for k in range(self.pool_blocks):
                d = gen.make(k * s.block_samples, s.block_samples)
                blocks.append(d.cpu().pin_memory())
            self.pool.append(blocks)
        self.copied = None                                    # last block copies (dump mode)
        self.copy_stream = torch.cuda.Stream(self.device)     # host -> device blocks
        self.d2h_stream = torch.cuda.Stream(self.device)      # dumps -> host, so that block
        self.compute = torch.cuda.Stream(self.device)         # uploads never queue behind them
        self._warm_up()

    def _warm_up(self):
        """One correlation, dump and copy of each kind before the clock starts,
        so that the first blocks do not pay for loading kernels or for first
        use of the copy paths.  The dump resets the integration."""
        torch = self.torch
        for a in range(len(self.specs)):
            self.rings[a][0].copy_(self.pool[a][0])
        torch.cuda.synchronize(self.device)
        self.batch.accumulate([r[0] for r in self.rings], stream=self.compute)
        self.batch.dump([v[0] for v in self.vis], stream=self.compute)
        if self.per_dump:
            self.batch.integrate([r[:sp.blocks_per_dump].view(-1, sp.n_chan, sp.n_inputs)
                                  for r, sp in zip(self.rings, self.specs)],
                                 [v[0] for v in self.vis], stream=self.compute)
        self.compute.synchronize()
        for a in range(len(self.specs)):
            with torch.cuda.stream(self.d2h_stream):
                self.host_ring[a][0][:1].copy_(self.vis[a][0][:1], non_blocking=True)
        self.d2h_stream.synchronize()

    def host_block(self, a, k):
        return self.pool[a][k % self.pool_blocks]

    def _slot(self, a, seq):
        # in dump mode the slots of one integration hold its blocks in order
        return seq % (self.specs[a].blocks_per_dump if self.per_dump else self.ring_blocks)

    def submit(self, blocks: dict):
        torch = self.torch
        ptrs = [None] * len(self.specs)
        start = torch.cuda.Event(enable_timing=True)
        end = torch.cuda.Event(enable_timing=True)
        copied = torch.cuda.Event()
        for a, blk in blocks.items():
            slot = self._slot(a, blk.seq)
            free = self.slot_free[a][slot]
            if free is not None:
                self.copy_stream.wait_event(free)
            with torch.cuda.stream(self.copy_stream):
                self.rings[a][slot].copy_(blk.data, non_blocking=True)
            ptrs[a] = self.rings[a][slot]
        copied.record(self.copy_stream)
        if self.per_dump:
            self.copied = copied           # the dump waits for the last copies
            return None
        self.compute.wait_event(copied)
        start.record(self.compute)
        self.batch.accumulate(ptrs, stream=self.compute)
        end.record(self.compute)
        for a, blk in blocks.items():
            self.slot_free[a][self._slot(a, blk.seq)] = end
        return (start, end)

    def dump(self, arrays):
        torch = self.torch
        outs = [None] * len(self.specs)
        for a in arrays:
            slot = self.dump_count[a] & 1
            if self.d2h_done[a][slot] is not None:   # the copy out of this buffer has finished
                self.compute.wait_event(self.d2h_done[a][slot])
            outs[a] = self.vis[a][slot]
        handle = None
        if self.per_dump:
            # the whole integration from the ring, written straight into the dump buffer
            volts = [None] * len(self.specs)
            for a in arrays:
                sp = self.specs[a]
                volts[a] = self.rings[a][:sp.blocks_per_dump].view(-1, sp.n_chan, sp.n_inputs)
            if self.copied is not None:
                self.compute.wait_event(self.copied)
            start = torch.cuda.Event(enable_timing=True)
            end = torch.cuda.Event(enable_timing=True)
            start.record(self.compute)
            self.batch.integrate(volts, outs, stream=self.compute)
            end.record(self.compute)
            for a in arrays:
                self.slot_free[a] = [end] * self.ring_blocks
            handle = (start, end)
        else:
            self.batch.dump(outs, stream=self.compute)
        done = torch.cuda.Event()
        done.record(self.compute)
        self.d2h_stream.wait_event(done)
        for a in arrays:
            slot = self.dump_count[a] & 1
            host = self.host_ring[a][slot]
            rows = {}
            with torch.cuda.stream(self.d2h_stream):
                host.copy_(outs[a], non_blocking=True)
                for f in self.kept_channels[a]:
                    rows[f] = torch.empty(outs[a][f].shape, dtype=torch.int32, pin_memory=True)
                    rows[f].copy_(outs[a][f], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(self.d2h_stream)
            self.d2h_done[a][slot] = ev
            self.kept.append((a, self.dump_count[a], rows))
            self.dump_count[a] += 1
        return handle if self.per_dump else done

    def wait(self, handle):
        start, end = handle
        end.synchronize()
        return start.elapsed_time(end)

    def finish(self):
        self.torch.cuda.synchronize(self.device)
        self.batch.sync(self.compute)


def main(argv=None):
    import argparse
    ap = argparse.ArgumentParser(description="run the streaming X-engine service")
    ap.add_argument("--seconds", type=float, default=10.0)
    ap.add_argument("--unpaced", action="store_true", help="deliver blocks as fast as accepted")
    ap.add_argument("--hbm-budget-gb", type=float, default=64.0)
    ap.add_argument("--channels", type=int, default=3072)
    ap.add_argument("--mode", choices=("block", "dump"), default="block",
                    help="block: add every block as it arrives; dump: correlate each integration "
                         "as one launch when its last block has arrived")
    args = ap.parse_args(argv)
    specs = [StreamSpec("mwa256", 256, args.channels, array=0),
             StreamSpec("aux128", 128, args.channels, array=1),
             StreamSpec("aux512", 512, args.channels, array=2)]
    svc = Service(specs, int(args.hbm_budget_gb * 1e9), GpuBackend(), paced=not args.unpaced, mode=args.mode)
    n_blocks = int(round(args.seconds / specs[0].period_s))
    print(json.dumps(svc.run(n_blocks)))


if __name__ == "__main__":
    main()
