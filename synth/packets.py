"""PFB packet streams (Appendix A) built from a voltage block, for feeding the
packet ingest with synthetic data.

This is an input generator: it formats bytes and holds none of the
correlator's arithmetic.  The packet format is the one Appendix A describes
(264 bytes: header word 0x0800, two words of second tick and counters, 256
bytes of samples for four fine channels x 64 PFB inputs, a 16-bit XOR
checksum of the 128 data words), with the readings documented where the
appendix is silent (see ``FIELD_LAYOUT``):

* 16-bit words are sent most significant byte first;
* word two: bit 0 sec_tick, bits 1-3 unused, bits 4-5 pfb_id, bits 6-8
  mgt_id, bits 9-13 mgt_bank, bits 14-15 unused;
* word three: bits 11-15 mgt_channel, bits 9-10 mgt_group, bits 0-8
  mgt_frame (the appendix gives mgt_frame 5 bits but values 0-499, so it is
  read as 9 bits);
* data byte f2 * 64 + k holds fine channel f2 of the packet's group of four
  and PFB position k; PFB p's positions are inputs 64 p + k of the assembled
  block (Appendix B keeps each packet's order and concatenates the PFBs);
* fine channel of (mgt_channel c, mgt_id m, mgt_group g, f2) is
  128 c + 16 m + 4 g + f2 (Appendix A: lane n carries channel groups
  0, 4, 8, 12, 128, ... + 16 n).

A voltage block is uint8 [500][3072][256] (one 50 ms bank, every fine channel,
the four PFBs' inputs in PFB order).
"""
from __future__ import annotations

import numpy as np

PKT_BYTES = 264
FRAMES = 500            # samples per 50 ms bank
COARSE = 24             # coarse channels per lane
LANES_PER_PFB = 8       # mgt_id 0..7
PFBS = 4
GROUPS = 4              # 40 kHz groups of 4 fine channels per 160 kHz
FINE_PER_COARSE = 128
CHANNELS = COARSE * FINE_PER_COARSE     # 3072
INPUTS_PER_PFB = 64
INPUTS = PFBS * INPUTS_PER_PFB          # 256
HEADER = 0x0800

FIELD_LAYOUT = {
    "word2": {"sec_tick": (0, 1), "pfb_id": (4, 2), "mgt_id": (6, 3), "mgt_bank": (9, 5)},
    "word3": {"mgt_frame": (0, 9), "mgt_group": (9, 2), "mgt_channel": (11, 5)},
}


def fine_channel(c, m, g, f2):
    return 128 * c + 16 * m + 4 * g + f2


def lane_packets(block: np.ndarray, pfb: int, mgt: int, bank: int) -> np.ndarray:
    """The 48000 packets of one lane for one bank, in stream order
    (channel, group, frame): uint8 [96 * 500][264]."""
    T, F, N = block.shape
    assert (T, F, N) == (FRAMES, CHANNELS, INPUTS)
    # data[c][g][frame][f2][k]
    chans = (np.arange(COARSE)[:, None, None] * 128 + 16 * mgt + 4 * np.arange(GROUPS)[None, :, None]
             + np.arange(4)[None, None, :])                                   # [c][g][f2]
    sub = block[:, chans.reshape(-1), pfb * 64:(pfb + 1) * 64]                # [frame][c*g*f2][k]
    sub = sub.reshape(FRAMES, COARSE, GROUPS, 4, 64).transpose(1, 2, 0, 3, 4)  # [c][g][frame][f2][k]
    n_pk = COARSE * GROUPS * FRAMES
    pk = np.zeros((n_pk, PKT_BYTES), np.uint8)
    pk[:, 6:262] = sub.reshape(n_pk, 256)
    c = np.repeat(np.arange(COARSE), GROUPS * FRAMES)
    g = np.tile(np.repeat(np.arange(GROUPS), FRAMES), COARSE)
    fr = np.tile(np.arange(FRAMES), COARSE * GROUPS)
    tick = ((bank == 0) & (c == 0) & (g == 0) & (fr == 0)).astype(np.uint32)
    w2 = tick | (pfb << 4) | (mgt << 6) | (bank << 9)
    w3 = fr | (g << 9) | (c << 11)
    for off, w in ((0, np.full(n_pk, HEADER, np.uint32)), (2, w2), (4, w3)):
        pk[:, off] = (w >> 8) & 0xFF
        pk[:, off + 1] = w & 0xFF
    pk[:, 262] = np.bitwise_xor.reduce(pk[:, 6:262:2], axis=1)
    pk[:, 263] = np.bitwise_xor.reduce(pk[:, 7:262:2], axis=1)
    return pk


def packetise(block: np.ndarray, bank: int = 0) -> np.ndarray:
    """Every lane's packets for one bank: uint8 [32 * 48000][264], lanes in
    order pfb_id 0..3, mgt_id 0..7."""
    return np.concatenate([lane_packets(block, p, m, bank) for p in range(PFBS)
                           for m in range(LANES_PER_PFB)])


def arrival_order(block: np.ndarray, bank: int = 0) -> np.ndarray:
    """The same packets in the order a receiver collects them (Sections 3.3.3
    and 3.4.1: each lane's packets travel in time-contiguous blocks of 2000,
    one coarse channel's four groups x 500 frames, one connection per lane,
    and each block is placed as it arrives): the 32 lanes' blocks of coarse
    channel 0, then of coarse channel 1, and so on, lanes in order pfb_id
    0..3, mgt_id 0..7.  uint8 [32 * 48000][264]."""
    per_block = GROUPS * FRAMES
    lanes = [lane_packets(block, p, m, bank) for p in range(PFBS) for m in range(LANES_PER_PFB)]
    return np.concatenate([lane[c * per_block:(c + 1) * per_block] for c in range(COARSE) for lane in lanes])
