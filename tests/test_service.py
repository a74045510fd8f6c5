"""Control logic of the streaming service on the CPU (fake GPU backend):
HBM-budget admission, sequence gaps, stalled and failing arrival threads,
latency accounting.  Every failure here is made on the host."""
import time

import pytest

from paper_1501_05992_gb300.service import Service, StreamSpec, admit, footprint


class FakeBackend:
    """Completes every submitted tick after a fixed delay; records calls."""

    def __init__(self, gpu_ms=0.2):
        self.gpu_ms = gpu_ms
        self.submits, self.dumps = [], []

    @staticmethod
    def workspace_bytes(n, f, t):
        return n * (n + 1) // 2 * f * 8 + 4096

    def open(self, specs, ring_blocks):
        self.specs = specs

    def host_block(self, a, k):
        return (a, k)

    def submit(self, blocks):
        self.submits.append({a: b.seq for a, b in blocks.items()})
        return time.perf_counter()

    def dump(self, arrays):
        self.dumps.append(list(arrays))
        return None

    def wait(self, handle):
        time.sleep(self.gpu_ms / 1e3)
        return self.gpu_ms

    def finish(self):
        pass


SPECS = [StreamSpec("a256", 256, 8, block_samples=50, blocks_per_dump=4),
         StreamSpec("a128", 128, 8, block_samples=50, blocks_per_dump=4, array=1),
         StreamSpec("a512", 512, 8, block_samples=50, blocks_per_dump=4, array=2)]


def test_admission_by_hbm_budget():
    ws = FakeBackend.workspace_bytes
    need = [footprint(s, 3, ws) for s in SPECS]
    admitted, rejected, used = admit(SPECS, need[0] + need[1] + 10, 3, ws)
    assert [s.name for s in admitted] == ["a256", "a128"]
    assert [s.name for s, _ in rejected] == ["a512"] and "CORR_E_BUDGET" in rejected[0][1]
    assert used == need[0] + need[1]
    svc = Service(SPECS, need[0] + need[1] + 10, FakeBackend(), paced=False)
    rep = svc.run(8)
    assert [a["name"] for a in rep["arrays"]] == ["a256", "a128"]
    assert rep["rejected"][0]["name"] == "a512"


def test_every_block_correlated_and_dumped():
    be = FakeBackend()
    svc = Service(SPECS, 1 << 40, be, paced=False)
    rep = svc.run(12)
    for a in rep["arrays"]:
        assert a["blocks"] == 12 and a["dumps"] == 3 and a["gaps"] == 0
        assert a["p50_ms"] is not None and a["p99_ms"] >= a["p50_ms"]
    seen = {}
    for tick in be.submits:
        for arr, seq in tick.items():
            seen.setdefault(arr, []).append(seq)
    assert all(v == list(range(12)) for v in seen.values())
    assert rep["x_real_time_margin"] == pytest.approx(5.0 / 0.2)     # 5 ms period / 0.2 ms per tick


def test_lost_blocks_taint_their_integration():
    svc = Service(SPECS[:1], 1 << 40, FakeBackend(), paced=False)
    rep = svc.run(12, faults={"a256": {"skip": {5}}})
    a = rep["arrays"][0]
    assert a["gaps"] == 1 and a["lost_blocks"] == 1 and a["blocks"] == 11
    assert a["tainted_dumps"] == 1
    tainted = [d for d in svc.dumps if d[3]]
    assert len(tainted) == 1 and 6 in tainted[0][2]


def test_stalled_and_failing_sources_are_reported():
    svc = Service(SPECS[:2], 1 << 40, FakeBackend(), paced=True, stall_s=0.05)
    rep = svc.run(8, faults={"a256": {"stall": {3: 0.25}}, "a128": {"raise": {5}}})
    a256, a128 = rep["arrays"]
    assert a256["stalls"] >= 1 and a256["blocks"] == 8 and a256["failed"] is None
    assert a128["failed"] and "block 5" in a128["failed"] and a128["blocks"] == 5


def test_paced_latency_is_measured_from_real_time_arrival():
    svc = Service(SPECS[:1], 1 << 40, FakeBackend(gpu_ms=1.0), paced=True)
    rep = svc.run(6)
    a = rep["arrays"][0]
    assert a["blocks"] == 6
    assert 0.5 < a["p50_ms"] < 200


class FakeDumpBackend(FakeBackend):
    """As FakeBackend; records which blocks each dump correlates."""

    def dump(self, arrays):
        self.dumps.append(list(arrays))
        return ("dump", tuple(arrays))


def test_dump_mode_times_whole_integrations():
    be = FakeDumpBackend(gpu_ms=1.0)
    svc = Service(SPECS, 1 << 40, be, paced=False, mode="dump")
    assert be.per_dump and svc.ring_blocks == 4
    rep = svc.run(8)
    assert rep["mode"] == "dump"
    for a in rep["arrays"]:
        assert a["blocks"] == 8 and a["dumps"] == 2 and a["gaps"] == 0
    # latencies are recorded when the dump that correlates a block completes:
    # one per block, timed once per dump call (the arrays' dumps fall in the
    # same call when their blocks arrive together, else in separate ones)
    assert 2 <= len(svc.tick_gpu_ms) <= 6
    assert sum(len(st.latencies_ms) for st in svc.stats) == 3 * 8
    assert abs(rep["x_real_time_margin"] - 4 * SPECS[0].period_s * 1e3 / 1.0) < 1e-9
    with pytest.raises(ValueError):
        Service(SPECS, 1 << 40, FakeBackend(), mode="tick")
