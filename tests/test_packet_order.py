"""The synthetic packet streams (an input generator, no correlator
arithmetic): the receiver's arrival order holds the same packets as the
lane-by-lane stream, in 2000-packet blocks of one lane and one coarse
channel (Sections 3.3.3 and 3.4.1), the lanes taking turns."""
import numpy as np

from synth import packets as pkts


def _fields(stream):
    w2 = stream[:, 2].astype(np.int64) << 8 | stream[:, 3]
    w3 = stream[:, 4].astype(np.int64) << 8 | stream[:, 5]
    return (w2 >> 4) & 3, (w2 >> 6) & 7, w3 >> 11, (w3 >> 9) & 3, w3 & 511


def test_arrival_order_is_the_lane_stream_in_blocks():
    block = np.zeros((pkts.FRAMES, pkts.CHANNELS, pkts.INPUTS), np.uint8)
    block[:, :, 0] = np.arange(pkts.CHANNELS, dtype=np.int64)[None, :] % 251
    lane = pkts.packetise(block, 5)
    arr = pkts.arrival_order(block, 5)
    assert arr.shape == lane.shape == (32 * 48000, pkts.PKT_BYTES)
    # the same packets: headers unique and equal as sets, payloads follow them
    key = lambda s: (s[:, 2:6].astype(np.int64) * np.array([1 << 24, 1 << 16, 1 << 8, 1])).sum(1)
    kl, ka = key(lane), key(arr)
    assert len(np.unique(ka)) == len(ka)
    il, ia = np.argsort(kl), np.argsort(ka)
    assert np.array_equal(lane[il], arr[ia])
    # block b: lane b mod 32 (pfb_id slowest, then mgt_id), coarse channel b / 32,
    # four groups x 500 frames with the frame fastest
    pfb, mgt, chan, grp, frame = _fields(arr)
    b = np.arange(len(arr)) // 2000
    assert np.array_equal(pfb, (b % 32) // 8)
    assert np.array_equal(mgt, b % 8)
    assert np.array_equal(chan, b // 32)
    k = np.arange(len(arr)) % 2000
    assert np.array_equal(grp, k // 500)
    assert np.array_equal(frame, k % 500)
