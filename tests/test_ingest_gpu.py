"""Packet ingest on the GPU against the oracle: the hand-written packet of
the golden fixture, streams built by the packetiser (in and out of order,
partial), rejected and repeated packets, and a whole bank feeding the
X-engine."""
import numpy as np
import pytest
import torch

import oracle
import _pins
from paper_1501_05992_gb300 import corr
from synth import packets as pkts

pytestmark = pytest.mark.gpu


def _ingest(packets_np, bank):
    p = torch.from_numpy(np.ascontiguousarray(packets_np).reshape(-1, 264)).cuda()
    volt, cnt = corr.ingest_packets(p, bank)
    torch.cuda.synchronize()
    return volt.cpu().numpy(), cnt.cpu().numpy().astype(np.int64)


def test_golden_packet():
    pk, bank, samples = _pins._golden_packet()
    volt, cnt = _ingest(pk[None], bank)
    want_v, want_c = oracle.ingest(pk[None], bank)
    assert np.array_equal(cnt, want_c)
    assert np.array_equal(volt, want_v)
    for t, f, n, v in samples:
        assert volt[t, f, n] == v


def test_partial_stream_any_order_and_rejections():
    block = np.random.default_rng(5).integers(0, 256, (500, 3072, 256), dtype=np.uint8)
    stream = np.concatenate([pkts.lane_packets(block, p, m, 2) for p, m in [(0, 1), (2, 6), (3, 0)]])
    rng = np.random.default_rng(6)
    stream = stream[rng.permutation(len(stream))]
    bad = stream[:40].copy()
    bad[0:10, 1] = 0x01                          # header
    bad[10:20, 50] ^= 0x40                       # checksum
    bad[20:30, 2] |= 0x08                        # mgt_bank 6 instead of 2
    stream = np.concatenate([stream, bad, stream[100:130]])        # 30 repeated packets
    volt, cnt = _ingest(stream, 2)
    want_v, want_c = oracle.ingest(stream, 2)
    assert np.array_equal(cnt, want_c)
    assert cnt[corr.PKT_COUNTER_NAMES.index("duplicate")] == 40       # 30 repeats + 10 unmodified copies in `bad`
    assert np.array_equal(volt, want_v)


def test_whole_bank_round_trip_into_xengine():
    block = np.random.default_rng(7).integers(0, 256, (500, 3072, 256), dtype=np.uint8)
    stream = pkts.packetise(block, 0)[::-1].copy()
    volt_t, cnt = corr.ingest_packets(torch.from_numpy(stream).cuda(), 0)
    torch.cuda.synchronize()
    assert cnt.cpu().tolist() == [len(stream), 0, 0, 0, 0, 0]
    assert torch.equal(volt_t.cpu(), torch.from_numpy(block))
    # the ingested block is the X-engine's input as it stands
    c = corr.Correlator(256, 3072, 500)
    tri = c.integrate(volt_t)
    got = tri[[0, 2047]].cpu().numpy()
    c.sync()
    c.close()
    assert np.array_equal(got, oracle.to_int32(oracle.xmac(block[:, [0, 2047]])))


def test_whole_bank_in_arrival_order():
    """The order a receiver collects the lanes' 2000-packet blocks in (the
    benchmark's order) gives the same block and no rejections."""
    block = np.random.default_rng(8).integers(0, 256, (500, 3072, 256), dtype=np.uint8)
    stream = pkts.arrival_order(block, 3)
    volt_t, cnt = corr.ingest_packets(torch.from_numpy(stream).cuda(), 3)
    torch.cuda.synchronize()
    assert cnt.cpu().tolist() == [len(stream), 0, 0, 0, 0, 0]
    assert torch.equal(volt_t.cpu(), torch.from_numpy(block))


def test_missing_packets_are_invalid_samples():
    """A lane that sent nothing leaves invalid samples, which the zero-invalid
    reading turns into zeros: the correlation equals that of the zeroed block."""
    block = np.random.default_rng(8).integers(0, 256, (500, 3072, 256), dtype=np.uint8)
    block[block == 0x88] = 0x77
    stream = np.concatenate([pkts.lane_packets(block, p, m, 1) for p in range(4) for m in range(8)
                             if (p, m) != (1, 4)])
    volt_t, cnt = corr.ingest_packets(torch.from_numpy(stream).cuda(), 1)
    c = corr.Correlator(256, 3072, 500, zero_invalid=True)
    chans = [16 * 4 + 3, 128 * 7 + 64 + 9, 5]                # two channels of the silent lane, one other
    tri = c.integrate(volt_t)[chans].cpu().numpy()
    c.sync()
    c.close()
    assert cnt.cpu().tolist()[corr.PKT_COUNTER_NAMES.index("missing")] == 48000
    zeroed = block[:, chans].copy()
    for k, f in enumerate(chans):
        if (f % 128) // 16 == 4:
            zeroed[:, k, 64:128] = 0x88
    assert np.array_equal(tri, oracle.to_int32(oracle.xmac(zeroed, zero_invalid=True)))


def test_arguments():
    with pytest.raises(ValueError):
        corr.ingest_packets(torch.zeros((3, 263), dtype=torch.uint8, device="cuda"), 0)
    with pytest.raises(corr.CorrError):
        corr.ingest_packets(torch.zeros((3, 264), dtype=torch.uint8, device="cuda"), 40)


@pytest.mark.parametrize("offset,count", [(0, 6407), (4, 6400), (0, 31), (8, 96)])
def test_shuffled_corrupted_repeated_and_offset_streams(offset, count):
    """Streams of shuffled packets with corrupted checksums and headers and
    repeated packets mixed in, starting 0, 4 or 8 bytes past a 16-byte
    boundary: the block and every counter equal the oracle's (the repeats are
    counted as good packets beyond the distinct slots they filled)."""
    rng = np.random.default_rng(offset * 1000 + count)
    block = rng.integers(0, 256, (500, 3072, 256), dtype=np.uint8)
    full = pkts.packetise(block, 1)
    idx = rng.choice(len(full), count, replace=False)
    sel = full[idx].copy()
    sel[::97, 100] ^= 0x40                       # bad checksums
    sel[::131, 0] = 0x09                         # bad headers
    sel = np.concatenate([sel, sel[:5]])         # repeats
    raw = torch.zeros(sel.size + offset, dtype=torch.uint8, device="cuda")
    raw[offset:] = torch.from_numpy(sel.reshape(-1)).cuda()
    p = raw[offset:].view(-1, 264)
    assert (p.data_ptr() - raw.data_ptr()) == offset
    volt, cnt = corr.ingest_packets(p, 1)
    torch.cuda.synchronize()
    want_v, want_c = oracle.ingest(sel, 1)
    got = cnt.cpu().numpy().astype(np.int64)
    assert np.array_equal(got, want_c)
    assert np.array_equal(volt.cpu().numpy(), want_v)
