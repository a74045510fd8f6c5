"""Pins of the CPU oracle to facts outside itself.

Each pin takes an ``oracle.OracleLib`` and raises AssertionError if the oracle
disagrees with something the paper or mathematics fixes:

* the sample code table of Appendix A (golden file);
* a library routine on a different formulation: numpy's complex matrix
  product X @ X^H (V_ij = sum_t x_i conj(x_j) is exactly that product);
* invariants: Hermitian symmetry, real non-negative autos equal to sum |x|^2,
  rank one at T = 1, additivity over time, permutation equivariance;
* closed forms: constant inputs give T c_i conj(c_j); an injected tone of known
  per-input phase gives arg V_ij = phi_i - phi_j within the rounding bound;
* the invalid-sample reading (code 8) and the output sizes printed in
  Section 3.4.3.

The same pins run against deliberately broken copies of the oracle source
(tests/test_oracle_pins.py::test_pins_catch_planted_mistakes) to show that each
plausible mistake is caught by at least one of them.
"""
from __future__ import annotations

import math
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_table(name: str) -> list[list[str]]:
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append(line.split())
    return rows


def code_values() -> np.ndarray:
    vals = np.zeros(16, np.int64)
    for code, value in read_table("nibble_codes.txt"):
        vals[int(code)] = int(value)
    return vals


def numpy_decode(volt: np.ndarray, zero_invalid: bool = False) -> np.ndarray:
    """Complex128 samples from the golden code table (independent of the oracle)."""
    vals = code_values()
    hi = (volt >> 4) & 0xF
    lo = volt & 0xF
    x = vals[hi].astype(np.float64) + 1j * vals[lo].astype(np.float64)
    if zero_invalid:
        x[(hi == 8) | (lo == 8)] = 0
    return x


def tri_index(i: int, j: int) -> int:
    return i * (i + 1) // 2 + j


def tri_to_full(tri: np.ndarray, n: int) -> np.ndarray:
    """[F][P][2] packed lower triangle -> complex [F][N][N] using V_ji = conj(V_ij)."""
    F = tri.shape[0]
    out = np.zeros((F, n, n), np.complex128)
    ii, jj = np.tril_indices(n)
    p = ii * (ii + 1) // 2 + jj
    v = tri[:, p, 0].astype(np.float64) + 1j * tri[:, p, 1].astype(np.float64)
    out[:, ii, jj] = v
    out[:, jj, ii] = np.conj(v)
    return out


def _rng(seed):
    return np.random.default_rng(seed)


# ------------------------------------------------------------------ pins ---
def pin_decode_table(o):
    b = np.arange(256, dtype=np.uint8).reshape(1, 1, 256)
    re, im = o.decode(b)
    vals = code_values()
    assert np.array_equal(re.ravel(), vals[np.arange(256) >> 4]), "real part must be the high nibble"
    assert np.array_equal(im.ravel(), vals[np.arange(256) & 15]), "imag part must be the low nibble"


def pin_library_matmul(o):
    rng = _rng(11)
    for (T, F, N) in [(37, 3, 7), (1, 2, 5), (64, 2, 16), (5, 1, 1)]:
        volt = rng.integers(0, 256, (T, F, N), dtype=np.uint8)
        tri = o.xmac(volt)
        x = numpy_decode(volt)                               # [T][F][N]
        for f in range(F):
            X = x[:, f, :].T                                 # [N][T]
            V = X @ X.conj().T                               # library complex GEMM
            got = tri_to_full(tri[f:f + 1], N)[0]
            assert np.array_equal(got, V), f"oracle != X X^H for shape {(T, F, N)}"


def pin_hermitian(o):
    rng = _rng(12)
    volt = rng.integers(0, 256, (23, 2, 9), dtype=np.uint8)
    full = o.xmac_full(volt)
    v = full[..., 0] + 1j * full[..., 1]
    assert np.array_equal(v, np.conj(np.swapaxes(v, 1, 2))), "V_ij != conj(V_ji)"
    tri = o.xmac(volt)
    n = volt.shape[2]
    for i in range(n):
        for j in range(i + 1):
            assert tuple(tri[:, tri_index(i, j)].tolist()[0]) == tuple(full[0, i, j]), \
                "packed triangle entry differs from the full matrix"


def pin_autos(o):
    rng = _rng(13)
    volt = rng.integers(0, 256, (41, 3, 6), dtype=np.uint8)
    tri = o.xmac(volt)
    x = numpy_decode(volt)
    for i in range(volt.shape[2]):
        p = tri_index(i, i)
        assert np.all(tri[:, p, 1] == 0), "autocorrelation must be real"
        want = np.sum(np.abs(x[:, :, i]) ** 2, axis=0)
        assert np.array_equal(tri[:, p, 0].astype(np.float64), want), "auto != sum |x|^2"


def pin_constant_closed_form(o):
    vals = code_values()
    rng = _rng(14)
    N, T = 6, 97
    codes = rng.integers(0, 256, N, dtype=np.uint8)
    volt = np.broadcast_to(codes, (T, 1, N)).copy()
    tri = o.xmac(volt)
    c = [complex(int(vals[b >> 4]), int(vals[b & 15])) for b in codes]
    for i in range(N):
        for j in range(i + 1):
            want = T * c[i] * c[j].conjugate()
            got = tri[0, tri_index(i, j)]
            assert (int(got[0]), int(got[1])) == (int(want.real), int(want.imag)), \
                "constant input does not give T c_i conj(c_j)"


def pin_rank_one(o):
    rng = _rng(15)
    volt = rng.integers(0, 256, (1, 4, 8), dtype=np.uint8)
    V = tri_to_full(o.xmac(volt), 8)
    for f in range(4):
        d = np.real(np.diag(V[f]))
        mag2 = V[f].real ** 2 + V[f].imag ** 2          # exact for these integers
        assert np.array_equal(mag2, np.outer(d, d)), "T=1 matrix is not rank one"


def pin_additivity(o):
    rng = _rng(16)
    a = rng.integers(0, 256, (30, 2, 7), dtype=np.uint8)
    b = rng.integers(0, 256, (19, 2, 7), dtype=np.uint8)
    whole = o.xmac(np.concatenate([a, b], axis=0))
    assert np.array_equal(whole, o.xmac(a) + o.xmac(b)), "integration is not additive in time"
    acc = o.xmac(a)
    o.xmac(b, vis=acc)
    assert np.array_equal(whole, acc), "accumulate-into differs from one call"


def pin_permutation(o):
    rng = _rng(17)
    N = 9
    volt = rng.integers(0, 256, (25, 2, N), dtype=np.uint8)
    perm = rng.permutation(N)
    V = tri_to_full(o.xmac(volt), N)
    W = tri_to_full(o.xmac(volt[:, :, perm]), N)
    assert np.array_equal(W, V[:, perm][:, :, perm]), "not permutation equivariant"


def pin_tone_phase(o):
    """x_k(t) = round(A exp(i(w t + phi_k))): arg V_ij within 2 asin(sqrt2/(2A)) of phi_i - phi_j."""
    A, T, N = 7.0, 400, 8
    w = 2 * math.pi * 0.0371
    phi = 2 * math.pi * np.arange(N) / N + 0.3
    t = np.arange(T)[:, None]
    z = A * np.exp(1j * (w * t + phi[None, :]))
    r = np.clip(np.round(z.real), -7, 7).astype(np.int64)
    m = np.clip(np.round(z.imag), -7, 7).astype(np.int64)
    volt = (((r & 0xF) << 4) | (m & 0xF)).astype(np.uint8)[:, None, :]
    V = tri_to_full(o.xmac(volt), N)[0]
    delta = math.sqrt(2) / 2
    ang_bound = 2 * math.asin(delta / A)
    for i in range(N):
        for j in range(N):
            d = (np.angle(V[i, j]) - (phi[i] - phi[j]) + math.pi) % (2 * math.pi) - math.pi
            assert abs(d) <= ang_bound + 1e-12, f"phase of V_{i}{j} off by {d}"
            mag = abs(V[i, j])
            assert T * (A - delta) ** 2 * math.cos(ang_bound) - 1e-9 <= mag <= T * (A + delta) ** 2, \
                f"|V_{i}{j}| = {mag} outside the rounding bounds"


def pin_invalid_reading(o):
    rng = _rng(18)
    volt = rng.integers(0, 256, (33, 2, 5), dtype=np.uint8)
    volt[3, 0, 1] = 0x80
    volt[4, 1, 2] = 0x08
    volt[5, 0, 0] = 0x88
    volt[6, 1, 4] = 0x83
    bad = (((volt >> 4) & 0xF) == 8) | ((volt & 0xF) == 8)
    clean = np.where(bad, np.uint8(0), volt)
    assert np.array_equal(o.xmac(volt, zero_invalid=True), o.xmac(clean)), \
        "zero_invalid must zero every sample with a nibble equal to 8"
    assert not np.array_equal(o.xmac(volt), o.xmac(clean)), "default must decode code 8 as -8"
    x = numpy_decode(volt)
    X = x[:, 0, :].T
    assert np.array_equal(tri_to_full(o.xmac(volt)[0:1], 5)[0], X @ X.conj().T)


def pin_paper_sizes(o):
    d = {k: float(v) for k, v in read_table("paper_sizes.txt")}
    n = int(d["inputs"])
    S, Pp = int(d["stations"]), int(d["pols"])
    assert n == S * Pp
    volt = np.zeros((1, 1, n), np.uint8)
    P = o.xmac(volt).shape[1]
    assert P == n * (n + 1) // 2
    # station-pair products (s1 >= s2, p1, p2) of Appendix C map onto the flat
    # input triangle (n = 2 s + p); the paper's count includes both cross-pol
    # products of each station with itself, one of which is the conjugate of
    # the other: 33024 = N(N+1)/2 + stations.
    hits = np.zeros(P, np.int64)
    for s1 in range(S):
        for s2 in range(s1 + 1):
            for p1 in range(Pp):
                for p2 in range(Pp):
                    a, b = Pp * s1 + p1, Pp * s2 + p2
                    hits[tri_index(max(a, b), min(a, b))] += 1
    assert hits.sum() == int(d["visibilities_per_channel"])
    assert np.all(hits >= 1) and np.count_nonzero(hits == 2) == S
    total = d["visibilities_per_channel"] * d["channels"] * d["bytes_per_visibility"]
    assert abs(total - d["approx_bytes_per_time_unit"]) / d["approx_bytes_per_time_unit"] < 0.05


def pin_brute_force(o):
    rng = _rng(19)
    vals = code_values()
    volt = rng.integers(0, 256, (6, 2, 4), dtype=np.uint8)
    tri = o.xmac(volt)
    for f in range(2):
        for i in range(4):
            for j in range(i + 1):
                s = 0j
                for t in range(6):
                    bi, bj = int(volt[t, f, i]), int(volt[t, f, j])
                    xi = complex(int(vals[bi >> 4]), int(vals[bi & 15]))
                    xj = complex(int(vals[bj >> 4]), int(vals[bj & 15]))
                    s += xi * xj.conjugate()
                got = tri[f, tri_index(i, j)]
                assert (int(got[0]), int(got[1])) == (int(s.real), int(s.imag))


def pin_beam_autos(o):
    """Summed over time, the incoherent beam is the sum of the autocorrelations
    (the triangle's diagonal), for both readings of the invalid code."""
    rng = _rng(23)
    volt = rng.integers(0, 256, (12, 3, 7), dtype=np.uint8)
    volt[3, 1, 2] = 0x88
    for zi in (False, True):
        beam = o.beam(volt, 1, zi)
        tri = o.xmac(volt, zi)
        autos = np.stack([tri[:, tri_index(n, n), 0] for n in range(7)], axis=1).sum(axis=1)
        assert np.array_equal(beam.sum(axis=0), autos)
        assert np.array_equal(o.beam(volt, 12, zi)[0], autos)
        assert np.all(beam >= 0)


def pin_beam_brute_force(o):
    rng = _rng(29)
    volt = rng.integers(0, 256, (6, 2, 5), dtype=np.uint8)
    x = numpy_decode(volt)
    want = (np.abs(x.real) ** 2 + np.abs(x.imag) ** 2).sum(axis=2)        # [T][F], exact in float64
    want = want.reshape(2, 3, 2).sum(axis=1)                              # n_avg = 3
    assert np.array_equal(o.beam(volt, 3), want.astype(np.int64))


def pin_pfb_order_printed(o):
    order = __import__("oracle").pfb_order(128)
    for k, a in read_table("pfb_antenna_order.txt"):
        assert order[int(k)] == int(a) and order[64 + int(k)] == 64 + int(a)
    assert sorted(order.tolist()) == list(range(128))


def _natural_products(x_nat):
    """V_AB(f) for every natural pair by numpy's complex matrix product."""
    T, F, N = x_nat.shape
    out = np.zeros((F, N, N), np.complex128)
    for f in range(F):
        X = x_nat[:, f, :].T                                             # N x T
        out[f] = X @ X.conj().T
    return out


def pin_remap_natural_order(o):
    """Correlating in PFB order and remapping equals correlating in natural
    order (numpy), station pair by station pair, conjugates included; also
    after averaging over channel pairs and over two dumps."""
    rng = _rng(31)
    N, F, T = 8, 4, 10
    x_nat = rng.integers(0, 256, (T, F, N), dtype=np.uint8)
    perm = rng.permutation(N).astype(np.int32)                # nat_of_pfb
    x_pfb = x_nat[:, :, perm]
    full = _natural_products(numpy_decode(x_nat))
    S = N // 2
    out = o.remap(o.xmac(x_pfb), perm)
    out2 = o.remap(np.stack([o.xmac(x_pfb[:4]), o.xmac(x_pfb[4:])]), perm, f_avg=2)
    for s1 in range(S):
        for s2 in range(s1 + 1):
            for p1 in range(2):
                for p2 in range(2):
                    q = s1 * (s1 + 1) // 2 + s2
                    v = full[:, 2 * s1 + p1, 2 * s2 + p2]
                    assert np.array_equal(out[:, q, p1, p2, 0], v.real.astype(np.int64))
                    assert np.array_equal(out[:, q, p1, p2, 1], v.imag.astype(np.int64))
                    w = v.reshape(F // 2, 2).sum(axis=1)
                    assert np.array_equal(out2[:, q, p1, p2, 0], w.real.astype(np.int64))
                    assert np.array_equal(out2[:, q, p1, p2, 1], w.imag.astype(np.int64))


def pin_remap_paper_count(o):
    d = {k: float(v) for k, v in read_table("paper_sizes.txt")}
    n = int(d["inputs"])
    out = o.remap(np.zeros((1, n * (n + 1) // 2, 2), np.int64), np.arange(n, dtype=np.int32))
    assert out[0].size // 2 == int(d["visibilities_per_channel"])


def _golden_packet():
    pk = np.zeros(264, np.uint8)
    bank, samples = None, []
    for row in read_table("pfb_packet_example.txt"):
        if row[0] == "bank":
            bank = int(row[1])
        elif row[0] == "bytes":
            pk[int(row[1])] = int(row[2], 16)
        elif row[0] == "sample":
            samples.append((int(row[1]), int(row[2]), int(row[3]), int(row[4], 16)))
    return pk, bank, samples


def pin_ingest_golden_packet(o):
    """A packet written out by hand from Appendix A lands where the appendix
    says; every slot no packet filled is marked invalid (0x88)."""
    pk, bank, samples = _golden_packet()
    volt, cnt = o.ingest(pk[None], bank)
    for t, f, n, v in samples:
        assert volt[t, f, n] == v
    assert cnt[0] == 1 and cnt[1:5].sum() == 0 and cnt[5] == 500 * 768 * 4 - 1
    slot = volt[421, 2524:2528, 128:192]
    assert np.count_nonzero(slot) == 4
    assert volt[421, 2524, 127] == 0x88 and volt[421, 2528, 128] == 0x88 and volt[0, 0, 0] == 0x88
    # the same packet for another bank is rejected as out of range
    _, cnt = o.ingest(pk[None], bank + 1)
    assert cnt[3] == 1 and cnt[0] == 0


def pin_ingest_rejections(o):
    pk, bank, _ = _golden_packet()
    bad = np.stack([pk.copy() for _ in range(5)])
    bad[0, 0] = 0x09                      # header
    bad[1, 100] ^= 0x01                   # data byte: checksum mismatch
    bad[2, 263] ^= 0x10                   # checksum byte
    bad[3, 3] |= 0x01                     # sec_tick on a packet that is not the second's first
    w3 = (int(bad[4, 4]) << 8 | int(bad[4, 5])) & ~0x1FF | 500          # frame 500
    bad[4, 4], bad[4, 5] = w3 >> 8, w3 & 0xFF
    _, cnt = o.ingest(bad, bank)
    assert cnt.tolist() == [0, 1, 2, 2, 0, 500 * 768 * 4]
    volt, cnt = o.ingest(np.stack([pk, pk]), bank)          # a repeated packet
    assert cnt[0] == 2 and cnt[4] == 1 and volt[421, 2524, 128] == 0x12


def pin_ingest_round_trip(o):
    """Packets built from a block by the numpy packetiser (a separate
    implementation of the same format) ingest back to that block."""
    from synth import packets as pkts
    d = {r[0]: r[1:] for r in read_table("paper_packets.txt")}
    block = _rng(37).integers(0, 256, (500, 3072, 256), dtype=np.uint8)
    lanes = [(0, 0), (1, 3), (3, 7)]
    stream = np.concatenate([pkts.lane_packets(block, p, m, 5) for p, m in lanes])
    per_lane = int(d["packets_per_lane_per_bank"][0])
    assert stream.shape == (len(lanes) * per_lane, int(d["packet_bytes"][0]))
    assert int(d["packets_per_lane_per_second"][0]) == 20 * per_lane
    volt, cnt = o.ingest(stream[::-1], 5)                   # arrival order does not matter
    assert cnt.tolist() == [stream.shape[0], 0, 0, 0, 0, 500 * 768 * 4 - stream.shape[0]]
    for p, m in lanes:
        chans = (128 * np.arange(24)[:, None] + 16 * m + np.arange(16)[None, :]).reshape(-1)
        assert np.array_equal(volt[:, chans, 64 * p:64 * p + 64], block[:, chans, 64 * p:64 * p + 64])
    untouched = volt[:, :, 128:192].copy()                  # pfb 2 sent nothing
    assert (untouched == 0x88).all()
    # the channel groups a lane carries are the printed ones: lane (pfb 0, mgt 0)
    lane = pkts.lane_packets(block, 0, 0, 5)
    v0, c0 = o.ingest(lane, 5)
    filled = np.flatnonzero((v0[:, :, :64] != 0x88).any(axis=(0, 2)))
    starts = filled[::4]
    assert starts[:8].tolist() == [int(x) for x in d["lane0_group_starts"]]
    assert starts[-4:].tolist() == [int(x) for x in d["lane0_group_ends"]]
    assert len(starts) == int(d["channel_groups_per_lane"][0])


def _pfb_x(rng, Q, N, S):
    return rng.integers(-8, 8, (Q, N, S, 2)).astype(np.int8)


def pin_fpfb_single_tap_is_library_fft(o):
    """One tap of ones: every frame is the plain DFT of 128 samples, which
    numpy's FFT computes; channel c holds bin (c + 64) mod 128."""
    rng = _rng(41)
    Q, N, M = 2, 3, 5
    x = _pfb_x(rng, Q, N, 128 * M)
    spec, _ = o.fine_pfb(x, np.ones(128), 1.0)
    z = x[..., 0].astype(np.float64) + 1j * x[..., 1]
    Y = np.fft.fft(z.reshape(Q, N, M, 128), axis=-1)          # [Q][N][M][k]
    Y = np.roll(Y, 64, axis=-1)                                # index c = (k + 64) mod 128
    want = Y.transpose(2, 0, 3, 1).reshape(M, Q * 128, N)
    assert spec.shape == want.shape, "frame or channel count"
    assert np.allclose(spec, want, rtol=0, atol=1e-9), "single-tap filterbank must be the forward DFT"


def pin_fpfb_impulse_response(o):
    """An impulse at sample s0 of one input: frame m sees it through tap
    p = (s0 - 128 m) div 128 at point n0 = s0 mod 128, so channel c of that
    frame is h[s0 - 128 m] exp(-2 pi i k n0 / 128) with k = (c + 64) mod 128,
    and every other input, coarse channel and frame is zero."""
    rng = _rng(42)
    Q, N, taps = 2, 3, 12
    S = 128 * (taps + 3)
    h = rng.standard_normal(taps * 128)
    q0, i0, s0 = 1, 2, 128 * 7 + 37
    x = np.zeros((Q, N, S, 2), np.int8)
    x[q0, i0, s0, 0] = 3
    spec, _ = o.fine_pfb(x, h, 1.0)
    M = S // 128 - taps + 1
    want = np.zeros((M, Q * 128, N), np.complex128)
    k = (np.arange(128) + 64) % 128
    for m in range(M):
        d = s0 - 128 * m
        if 0 <= d < taps * 128:
            want[m, q0 * 128:(q0 + 1) * 128, i0] = 3 * h[d] * np.exp(-2j * np.pi * k * (s0 % 128) / 128)
    assert np.allclose(spec, want, rtol=0, atol=1e-9), "impulse response of the filterbank"


def pin_fpfb_tones(o):
    """With the window 1 / n_taps every point's taps sum to 1, so a tone at
    bin k0 (x = A exp(2 pi i k0 s / 128), integer for k0 = 0, +-32, 64) puts
    128 A into channel (k0 + 64) mod 128 of every frame and nothing
    elsewhere: the sign of the exponent and the channel order."""
    taps = 12
    S = 128 * (taps + 2)
    s = np.arange(S)
    h = np.full(taps * 128, 1.0 / taps)
    for k0, unit in ((0, np.ones(S, complex)), (32, 1j ** s), (-32, (-1j) ** s),
                     (64, (-1.0) ** s + 0j)):
        z = 5 * unit
        x = np.zeros((1, 2, S, 2), np.int8)
        x[0, 1, :, 0] = np.rint(z.real)
        x[0, 1, :, 1] = np.rint(z.imag)
        spec, _ = o.fine_pfb(x, h, 1.0)
        want = np.zeros_like(spec)
        want[:, (k0 + 64) % 128, 1] = 128 * 5
        assert np.allclose(spec, want, rtol=0, atol=1e-9), f"tone at bin {k0}"


def pin_fpfb_frame_shift(o):
    """Dropping the first 128 samples drops the first frame: frames advance
    by one block of 128 samples (critical sampling)."""
    rng = _rng(43)
    x = _pfb_x(rng, 1, 2, 128 * 15)
    h = rng.standard_normal(12 * 128)
    a, _ = o.fine_pfb(x, h, 1.0)
    b, _ = o.fine_pfb(x[:, :, 128:], h, 1.0)
    assert np.allclose(a[1:], b, rtol=0, atol=1e-9), "frame hop must be 128 samples"


def pin_fpfb_quantiser(o):
    """With one tap of ones and an impulse a + ib at the first point, every
    channel of the frame equals a + ib exactly, so the 4+4-bit codes can be
    checked against rounding half to even, saturation at +-7 and the nibble
    order of Appendix A (real part high)."""
    vals = code_values()
    for a, b, sc, want_r, want_i in ((5, -5, 0.5, 2, -2), (7, -7, 0.5, 4, -4), (3, 1, 0.5, 2, 0),
                                     (100, -100, 1.0, 7, -7), (9, 0, 1.0, 7, 0), (-9, 3, 1.0, -7, 3)):
        x = np.zeros((1, 1, 128, 2), np.int8)
        x[0, 0, 0] = (a, b)
        spec, volt = o.fine_pfb(x, np.ones(128), sc)
        assert np.allclose(spec, a + 1j * b), "flat spectrum of an impulse"
        codes = volt[0, :, 0]
        assert np.all(vals[codes >> 4] == want_r), f"real code of {a * sc}"
        assert np.all(vals[codes & 15] == want_i), f"imaginary code of {b * sc}"


def pin_fpfb_paper_structure(o):
    """The printed structure: 327.68 MHz in 256 coarse subbands of 1.28 MHz,
    12 taps x 128 points, fine channels of 10 kHz; a 12-tap filterbank over S
    samples gives S / 128 - 11 frames of 128 channels per coarse channel."""
    d = {k: int(v) for k, v in read_table("fine_pfb.txt")}
    assert d["coarse_input_bandwidth_hz"] // d["coarse_subbands"] == d["coarse_channel_hz"]
    assert d["coarse_channel_hz"] // d["fine_points"] == d["fine_channel_hz"]
    taps, L = d["fine_taps"], d["fine_points"]
    rng = _rng(44)
    x = _pfb_x(rng, 2, 1, L * (taps + 4))
    spec, volt = o.fine_pfb(x, np.ones(taps * L) / taps, 1.0)
    assert spec.shape == volt.shape == (5, 2 * L, 1), "frames and channels of a 12-tap, 128-point bank"


def pin_fpfb_feeds_xmac(o):
    """F then X: inputs carrying integer tones at bin 32 with complex
    amplitudes A_n, through the flat 12-tap window and scale 1/128, become the
    codes A_n in channel 96 of every frame (0 elsewhere), so correlating the M
    frames gives V_ij = M A_i conj(A_j) in channel 96 and zero in every other
    channel: the filterbank's output layout is the correlator's input layout."""
    taps, M, N = 12, 6, 4
    S = 128 * (M + taps - 1)
    s = np.arange(S)
    amps = [3 + 1j, -2 + 2j, 1 - 3j, -1 - 1j]
    x = np.zeros((1, N, S, 2), np.int8)
    for n, a in enumerate(amps):
        z = a * (1j ** s)
        x[0, n, :, 0] = np.rint(z.real)
        x[0, n, :, 1] = np.rint(z.imag)
    _, codes = o.fine_pfb(x, np.full(taps * 128, 1.0 / taps), 1.0 / 128)
    vis = o.xmac(codes)                                     # [128][P][2]
    want = np.zeros_like(vis)
    for i in range(N):
        for j in range(i + 1):
            v = M * amps[i] * np.conj(amps[j])
            want[96, tri_index(i, j)] = (round(v.real), round(v.imag))
    assert np.array_equal(vis, want), "filterbank codes must feed the correlator in its input layout"


ALL_PINS = [pin_decode_table, pin_library_matmul, pin_hermitian, pin_autos,
            pin_constant_closed_form, pin_rank_one, pin_additivity, pin_permutation,
            pin_tone_phase, pin_invalid_reading, pin_paper_sizes, pin_brute_force,
            pin_beam_autos, pin_beam_brute_force, pin_pfb_order_printed,
            pin_remap_natural_order, pin_remap_paper_count, pin_ingest_golden_packet,
            pin_ingest_rejections, pin_ingest_round_trip, pin_fpfb_single_tap_is_library_fft,
            pin_fpfb_impulse_response, pin_fpfb_tones, pin_fpfb_frame_shift, pin_fpfb_quantiser,
            pin_fpfb_paper_structure, pin_fpfb_feeds_xmac]
